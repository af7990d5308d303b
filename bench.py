#!/usr/bin/env python
"""Benchmark of the QTB-MD hot path on GB300 (one JSON line on stdout).

Workload (default): MgO rock salt 10x10x10 conventional cells (8000 ions),
QTB-MD at 100 K, dt = 1 fs, gamma = 1/ps, 2049-tap noise filter with
w_max = 3e14 rad/s, mixed precision (fixed-point positions, FP32 forces and
integration, FP64 energy accumulation), synthetic seeded input.

One bench "step" = one 256-step noise block: the white-noise block, the
coloured-noise filter and 256 BAOAB steps (one cooperative launch per step:
pair force from Verlet neighbour lists with the next step's B-A-O-A fused in,
preceded inside the launch by a list rebuild whenever some ion has moved half
the skin), replayed as one CUDA graph.  Metric:
atom*bead-steps/s.

--impl reference times the FP64 CPU oracle (the plain reference program of
this repository) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "atom*bead-steps/s on 1 GB300 (QTB-MD, mixed precision)"
UNIT = "atom*bead-steps/s"
BLOCK = 256

# algorithmic FP32 operations per in-range ordered pair of the force kernel
# (Buckingham + DSF Coulomb, force + energy + virial; see the design notes)
PAIR_FLOPS = 64


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ncell", type=int, default=10)
    ap.add_argument("--filter", default="auto", choices=["auto", "fp32", "bf16"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # direct launches (two 128-step calls per block) instead of the captured
    # graph: for profilers that cannot see kernels of graphs with conditional nodes
    ap.add_argument("--direct", action="store_true")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(base, rank):
    """Every rank simulates an independent replica (weak scaling, no exchange)."""
    return base + rank


def max_over_ranks(t_ms, device="cpu"):
    """Slowest rank's time (the job's time); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(t_ms)
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_units_per_rank, steps, world_size, t_ms):
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    return world_size * n_units_per_rank * steps / (t_ms / 1e3)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.samples.append([x.strip() for x in out.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def start(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()

    def stop(self):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if len(s) > 4 + k and "Active" in s[4 + k]
                          and "Not" not in s[4 + k]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def workload(ncell, precision, filt):
    from paper_1905_02521_gb300 import qtb, workloads as W
    s, pot = W.mgo_system(ncell, 100.0, gamma=1e-3)
    prec = qtb.MIXED if precision == "mixed" else qtb.FP64
    fp = qtb.FILTER_BF16 if filt == "bf16" else qtb.FILTER_FP32
    params = {k: pot[k] for k in ("mass", "charge", "buck_A", "buck_rho", "buck_C")}
    params.update(dsf_alpha=pot["dsf_alpha"], r_cut=pot["r_cut"], dt=1.0, precision=prec, filter_prec=fp,
                  seed=12345, obs_stride=BLOCK, max_records=64)
    return s, pot, params


def count_pairs(pos, box, rc):
    """In-range ordered pairs (all images) of one configuration (host, numpy)."""
    pos = np.asarray(pos)
    n = len(pos)
    tot = 0
    nmax = [int(np.ceil(rc / b)) for b in box]
    shifts = np.array([[i, j, k] for i in range(-nmax[0], nmax[0] + 1) for j in range(-nmax[1], nmax[1] + 1)
                       for k in range(-nmax[2], nmax[2] + 1)], np.float64) * box
    for a in range(0, n, 256):
        d = pos[a:a + 256, None, :] - pos[None, :, :]
        d -= box * np.round(d / box)
        for sh in shifts:
            r2 = ((d + sh) ** 2).sum(-1)
            tot += int(((r2 < rc * rc) & (r2 > 1e-12)).sum())
    return tot


def l2_flush_buffer(torch):
    return torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")


def run_ours(args):
    import torch
    from paper_1905_02521_gb300 import qtb

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    filt = args.filter
    if filt == "auto":
        filt = "bf16" if _tc_filter_available() else "fp32"
    s, pot, params = workload(args.ncell, args.precision, filt)
    params["seed"] = replica_seed(12345, rank)
    N = len(s["types"])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = qtb.qtb_init([s], params, stream=stream.cuda_stream)
    qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 2049, 0.3)
    qtb.qtb_set_profiling(ctx, not args.direct)
    flush = l2_flush_buffer(torch)

    def block():
        if args.direct:
            qtb.qtb_step_n(ctx, BLOCK // 2)
            qtb.qtb_step_n(ctx, BLOCK // 2)
        else:
            qtb.qtb_step_n(ctx, BLOCK)

    for _ in range(args.warmup):
        block()
    qtb.qtb_sync(ctx)
    rebuilds0 = qtb.qtb_list_rebuilds(ctx)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    t_wall = time.perf_counter()
    kernel_ms = {k: 0.0 for k in qtb.KERNEL_CLASSES}
    kernel_n = {k: 0 for k in qtb.KERNEL_CLASSES}
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))           # L2 flush between timed steps (outside the event pair)
            starts[i].record(stream)
        block()
        stops[i].record(stream)
        if args.direct:
            continue
        kt = qtb.qtb_kernel_times(ctx)      # per-kernel events of this block (synchronises)
        for k, (ms, n) in kt.items():
            kernel_ms[k] += ms * n
            kernel_n[k] += n
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, stops)]
    t_ms = max_over_ranks(float(np.sum(step_ms)), device="cuda")
    value = job_throughput(N * BLOCK, args.steps, ws, t_ms)
    obs = qtb.qtb_observables(ctx, 0)
    rebuilds = (qtb.qtb_list_rebuilds(ctx) - rebuilds0) / args.steps

    # roofline of the dominant kernel (pair force): algorithmic flops / mean launch time
    x, _ = qtb.qtb_get_state(ctx, 0, 1, N)
    pairs = count_pairs(x[0], s["box"], pot["r_cut"])
    force_ms = kernel_ms["force"] / max(kernel_n["force"], 1)
    achieved = PAIR_FLOPS * pairs / (force_ms * 1e-3) / 1e12 if force_ms > 0 else None
    peak = alu_peak_tflops()
    step_breakdown = {k: round(kernel_ms[k] / max(args.steps, 1), 4) for k in kernel_ms}

    # end to end through the C ABI with host buffers: H2D state, 256 steps, D2H observables
    pos_h, vel_h = qtb.qtb_get_state(ctx, 0, 1, N)
    e2e_ms = []
    for i in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        qtb.qtb_set_state(ctx, 0, pos_h, vel_h)
        qtb.qtb_step_n(ctx, BLOCK)
        rec = qtb.qtb_observables(ctx, 0)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_value = ws * N * BLOCK * args.steps / (np.sum(e2e_ms) / 1e3)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+fixed30+f64acc" if args.precision == "mixed" else "f64",
        "data": "synthetic: seeded rock-salt MgO, sigma 0.02 A, Maxwell-Boltzmann velocities",
        "config": {"workload": f"MgO rock salt {args.ncell}x{args.ncell}x{args.ncell} cells ({N} ions), QTB-MD 100 K, "
                               f"dt 1 fs, 2049-tap {filt} noise filter, 256-step blocks",
                   "n_ions": N, "n_beads": 1, "md_steps_per_bench_step": BLOCK, "precision": args.precision,
                   "filter": filt, "parallelism": f"replicas x{ws}",
                   "launch": "direct (2 x 128-step calls per block)" if args.direct else "CUDA graph per 256-step block",
                   "l2": "256 MB buffer written between timed steps (flush)"},
        "roofline": {"bound": "alu", "kernel": "k_force_list", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if achieved else None, "traffic": measured_traffic("k_force_list"),
                     "peak_source": "152 SM x 128 FP32 lanes x 2 flop x sm_max_mhz of MEASURED_PEAKS.json",
                     "flops_per_launch": PAIR_FLOPS * pairs, "pairs_per_launch": pairs, "mean_launch_ms": force_ms},
        "kernel_ms_per_bench_step": step_breakdown,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(2 * N * 3 * 8),
                "d2h_bytes_per_step": int(qtb.NREC * 8)},
        # per block: white, filter, one integrator launch, 256 step launches (a list
        # rebuild runs inside the step launch that needs it), the block clock
        "gpu_launches": 2 + 1 + BLOCK + 1,
        "list_rebuilds_per_bench_step": rebuilds,
        "wall_s": wall,
        "observables": {"K_eV": float(obs[1]), "V_eV": float(obs[2]), "step": int(obs[0])},
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sample_atoms=64)
    qtb.qtb_destroy(ctx)
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def measured_traffic(kernel):
    """DRAM bytes per launch from the committed ncu capture, or None when the
    kernel's source has changed since the counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != rec["source_sha1"]:
                return None
        return rec["dram_bytes_per_launch"]
    except Exception:
        return None


def alu_peak_tflops():
    """FP32 peak: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x max SM clock."""
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return 152 * 128 * 2 * mhz * 1e6 / 1e12


def _tc_filter_available():
    try:
        from paper_1905_02521_gb300 import qtb
        return bool(getattr(qtb, "TC_FILTER", False))
    except Exception:
        return False


def cpu_baseline(sample_atoms=64, steps=1):
    """The FP64 oracle on a bounded sample of the workload: forces on
    `sample_atoms` ions of the 8000-ion crystal (brute force over all ions and
    images) plus the coloured noise of their 3 dofs, per MD step."""
    import oracle
    from oracle import spectra as S
    from paper_1905_02521_gb300 import workloads as W
    s, pot = W.mgo_system(10, 100.0)
    h = S.taps(2049, 1.0, 100.0, 0.3)
    sel = np.arange(0, len(s["types"]), len(s["types"]) // sample_atoms)[:sample_atoms]
    oracle.build()
    t0 = time.perf_counter()
    for n in range(steps):
        oracle.pair_forces(s["pos"][0], s["types"], s["box"], pot, sel=sel)
        oracle.colored_block(12345, 0, 3 * sample_atoms, n, 1, h)
    dt = time.perf_counter() - t0
    return {"value": sample_atoms * steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{sample_atoms} of 8000 ions x {steps} step(s): brute-force periodic forces + "
                      f"2049-tap direct noise convolution, single thread, {dt:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from oracle import spectra as S
    from paper_1905_02521_gb300 import workloads as W
    oracle.build()
    s, pot = W.mgo_system(args.ncell, 100.0)
    h = S.taps(2049, 1.0, 100.0, 0.3)
    n_sample = 32
    sel = np.arange(0, len(s["types"]), max(1, len(s["types"]) // n_sample))[:n_sample]

    def one(n):
        oracle.pair_forces(s["pos"][0], s["types"], s["box"], pot, sel=sel)
        oracle.colored_block(12345, 0, 3 * len(sel), n, 1, h)

    for i in range(args.warmup):
        one(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        one(args.warmup + i)
    dt = time.perf_counter() - t0
    value = len(sel) * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"MgO rock salt {args.ncell}^3 cells, QTB-MD, 2049-tap filter (oracle sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{len(sel)} ions per step: forces + noise of the FP64 oracle"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
