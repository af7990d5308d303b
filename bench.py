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

METRIC = "atom*bead-steps/s on 1 GB300 (QTB / QTB-PIMD step, mixed precision)"
UNIT = "atom*bead-steps/s"
BLOCK = 256

# algorithmic FP32 operations per in-range ordered pair of the force kernel
# (Buckingham + DSF Coulomb, force + energy + virial; see the design notes)
PAIR_FLOPS = 64


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=48)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--equilibrate", type=int, default=32,
                    help="untimed 256-step blocks before the warm-up, after which every neighbour list is "
                         "rebuilt on the thermalised configuration (0: keep the lists of the initial lattice)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mgo8000", choices=WORKLOADS)
    ap.add_argument("--ncell", type=int, default=10, help="cells per side of the mgo8000 workload")
    ap.add_argument("--skin", type=float, default=0.0, help="neighbour-list skin, A (0: library default)")
    ap.add_argument("--rebuild-scope", type=int, default=0, choices=[0, 1],
                    help="0: a list rebuild covers the requesting systems; 1: all systems of the context")
    ap.add_argument("--generator", default="filter", choices=["filter", "fourier"],
                    help="coloured noise: time-domain filter, or Fourier segments (Eq. 9)")
    ap.add_argument("--segment-blocks", type=int, default=8, help="256-step blocks per Fourier segment")
    ap.add_argument("--autotune", action="store_true",
                    help="choose skin, lanes per bead-atom, integrator layout and rebuild scope with qtb_autotune "
                         "first (untimed)")
    ap.add_argument("--filter", default="auto", choices=["auto", "fp32", "bf16"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-blocks", type=int, default=3,
                    help="timed 256-step blocks of the FP64 form of the same workload (0: skip that leg)")
    ap.add_argument("--matched-blocks", type=int, default=8,
                    help="256-step blocks of the matched-error run of both forms (0: skip it)")
    # direct launches (two 128-step calls per block) instead of the captured
    # graph (for tools that profile launches outside graphs)
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
        # one long-lived nvidia-smi in loop mode (a sample every 50 ms), read line by line
        try:
            self._p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                        "--format=csv,noheader,nounits", "-lms", "50"],
                                       stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            return
        for line in self._p.stdout:
            if self._stop.is_set():
                break
            if line.strip():
                self.samples.append([x.strip() for x in line.strip().split(",")])

    def start(self):
        self._p = None
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()

    def stop(self):
        self._stop.set()
        if self._p is not None:
            self._p.terminate()      # the child this sampler started
            try:
                self._p.wait(timeout=5)
            except Exception:
                self._p.kill()
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


WORKLOADS = ("mgo8000", "lih_qtbpimd_p8", "lih_pimd_p32", "sweep64", "lih_pimd_p32_big", "lih_qtb_npt",
             "lih_qtbpimd_p8_npt")

# algorithmic bytes per bead-atom of one launch of the ring-polymer integrator
# (k_integrate_nm): read x, v, f, xref and the coloured noise, write x, v and the
# packed copy of the positions, 3 components each (4-byte values in the mixed
# form, 8-byte in the FP64 form)
INTEGRATOR_BYTES = {"mixed": 3 * (5 + 3) * 4, "fp64": 3 * (5 + 3) * 8}


def workload(name, ncell, precision, filt):
    """Systems, potential, context parameters, filter set-up and a description.

    mgo8000: MgO 10^3 cells (8000 ions), QTB-MD 100 K, dt 1 fs, 2049 taps, w_max 0.3 rad/fs.
    lih_qtbpimd_p8: LiH 6^3 cells (1728 ions), QTB-PIMD P = 8 (kappa_P from the solver), 50 K,
        dt 0.25 fs, 2049 taps, w_max 0.6 rad/fs.
    lih_pimd_p32: the same crystal, standard PIMD P = 32 with a white Langevin bath.
    lih_pimd_p32_big: LiH 20^3 cells (64000 ions) x 32 beads, white PIMD: the
        integrator's stream (~200 MB per step) exceeds the 129 MB L2.
    sweep64: 64 MgO systems of 3..8 cells per side (216-4096 ions) at T_i = 10 150^(i/63) K,
        QTB-MD, one context (batched), dt 1 fs, 2049 taps, w_max 0.3 rad/fs.
    lih_qtb_npt: LiH 6^3 cells (1728 ions), QTB-MD 50 K at zero pressure with the isotropic
        Langevin cell (cell period ~300 fs, friction 4e-3/fs), dt 0.25 fs, 2049 taps, w_max 0.6 rad/fs.
    lih_qtbpimd_p8_npt: lih_qtbpimd_p8 at zero pressure, the same cell acting on the centroids.
    """
    from paper_1905_02521_gb300 import qtb, workloads as W
    prec = qtb.MIXED if precision == "mixed" else qtb.FP64
    fp = qtb.FILTER_BF16 if filt == "bf16" else qtb.FILTER_FP32
    dt, setup = 1.0, None
    if name == "mgo8000":
        s, pot = W.mgo_system(ncell, 100.0, gamma=1e-3)
        systems = [s]
        setup = (qtb.NOISE_QTB, 2049, 0.3)
        desc = (f"MgO rock salt {ncell}x{ncell}x{ncell} cells ({len(s['types'])} ions), QTB-MD 100 K, dt 1 fs, "
                f"2049-tap {filt} noise filter, 256-step blocks")
    elif name in ("lih_qtbpimd_p8", "lih_pimd_p32", "lih_pimd_p32_big", "lih_qtbpimd_p8_npt"):
        P = 8 if name.startswith("lih_qtbpimd_p8") else 32
        nc = 20 if name == "lih_pimd_p32_big" else 6
        s, pot = W.lih_system(nc, 50.0, gamma=1e-3, n_beads=P)
        systems = [s]
        dt = 0.25
        if P == 8:
            setup = (qtb.NOISE_QTB_PIMD, 2049, 0.6)
            desc = f"LiH rock salt 6x6x6 cells (1728 ions) x 8 beads, QTB-PIMD (kappa_P solver) 50 K, dt 0.25 fs, 2049-tap {filt} filter"
            if name.endswith("_npt"):
                desc += ", zero pressure, isotropic Langevin cell on the centroids"
        else:
            desc = (f"LiH rock salt {nc}x{nc}x{nc} cells ({len(s['types'])} ions) x 32 beads, PIMD with white "
                    f"Langevin bath 50 K, dt 0.25 fs")
    elif name == "lih_qtb_npt":
        s, pot = W.lih_system(6, 50.0, gamma=1e-3)
        systems = [s]
        dt = 0.25
        setup = (qtb.NOISE_QTB, 2049, 0.6)
        desc = (f"LiH rock salt 6x6x6 cells (1728 ions), QTB-MD 50 K at zero pressure, isotropic Langevin cell, "
                f"dt 0.25 fs, 2049-tap {filt} filter")
    elif name == "sweep64":
        systems, pot = W.sweep_systems(64, gamma=1e-3)
        setup = (qtb.NOISE_QTB, 2049, 0.3)
        desc = (f"batched heat-capacity sweep: 64 MgO systems of 3..8 cells per side "
                f"({sum(len(x['types']) for x in systems)} ions), T = 10-1500 K (log grid), QTB-MD, dt 1 fs, "
                f"2049-tap {filt} filter, one context")
    else:
        raise ValueError(name)
    params = {k: pot[k] for k in ("mass", "charge", "buck_A", "buck_rho", "buck_C")}
    params.update(dsf_alpha=pot["dsf_alpha"], r_cut=pot["r_cut"], dt=dt, precision=prec, filter_prec=fp,
                  seed=12345, obs_stride=BLOCK, max_records=64)
    if name.endswith("_npt"):   # cell mass for a ~300 fs volume period at a bulk modulus of ~1 eV/A^3
        V = float(np.prod(systems[0]["box"]))
        params.update(npt=1, pressure=0.0, cell_mass=9.0 * 1.0 * V / (2 * np.pi / 300.0) ** 2, cell_gamma=4e-3)
    return systems, pot, params, setup, desc


def count_pairs(pos, box, rc):
    """In-range ordered pairs (all periodic images) of one configuration (host, k-d tree)."""
    from scipy.spatial import cKDTree
    box = np.asarray(box, np.float64)
    pos = np.mod(np.asarray(pos, np.float64), box)
    n = len(pos)
    if box.min() >= 2.0 * rc:
        tree = cKDTree(pos, boxsize=box)
    else:
        nmax = [int(np.ceil(rc / b)) for b in box]
        shifts = np.array([[i, j, k] for i in range(-nmax[0], nmax[0] + 1) for j in range(-nmax[1], nmax[1] + 1)
                           for k in range(-nmax[2], nmax[2] + 1)], np.float64) * box
        tree = cKDTree((pos[None, :, :] + shifts[:, None, :]).reshape(-1, 3))
    return int(tree.query_ball_point(pos, rc, return_length=True).sum()) - n


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
    systems, pot, params, setup, desc = workload(args.workload, args.ncell, args.precision, filt)
    params["seed"] = replica_seed(12345, rank)
    params["skin"] = args.skin
    params["rebuild_scope"] = args.rebuild_scope
    tuning = None
    if args.autotune:
        mode, n_taps, wmax = setup if setup is not None else (qtb.NOISE_WHITE, 1, 0.0)
        # candidates timed from the steady state the bench itself measures
        params, tuning = qtb.qtb_autotune(systems, params, mode, n_taps, wmax, n_blocks=3,
                                          equil_blocks=max(args.equilibrate, 0))
    sizes = [(len(x["types"]), int(x["pos"].shape[0])) for x in systems]   # (N, P)
    units = sum(n * p for n, p in sizes)                                    # atom*bead per MD step
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = qtb.qtb_init(systems, params, stream=stream.cuda_stream)
    if setup is not None:
        qtb.qtb_set_filter(ctx, -1, *setup)
    if args.generator == "fourier":
        qtb.qtb_set_generator(ctx, qtb.GEN_FOURIER, args.segment_blocks)
    qtb.qtb_set_profiling(ctx, not args.direct)
    # untimed equilibration: the bath brings the crystal to its steady state (the
    # QTB adds the zero-point energy within a few 1/gamma); then the lists are
    # rebuilt on that configuration, as they are in a long run after its first
    # rebuild (lists built on the initial, nearly perfect lattice give every ion the
    # same number of entries and are traversed faster than any later lists)
    for _ in range(args.equilibrate):
        qtb.qtb_step_n(ctx, BLOCK)
    if args.equilibrate > 0:
        qtb.qtb_rebuild_lists(ctx)
    qtb.qtb_sync(ctx)
    # the roofline's denominator: this GPU's FP32 FMA throughput, measured by the
    # library's own FMA-chain kernel (after the equilibration has warmed the GPU)
    fp32_peak, fp32_peak_ms = qtb.qtb_fp32_peak()
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
    value = job_throughput(units * BLOCK, args.steps, ws, t_ms)
    obs = qtb.qtb_observables(ctx, 0)
    rebuilds = (qtb.qtb_list_rebuilds(ctx) - rebuilds0) / args.steps

    # roofline of the dominant kernel (pair force): algorithmic flops / mean launch time
    pairs = 0
    states = []
    npt = bool(params.get("npt"))
    cells = [qtb.qtb_get_cell(ctx, k) if npt else None for k in range(len(sizes))]   # (edges, momentum)
    for k, (n, p) in enumerate(sizes):
        x, v = qtb.qtb_get_state(ctx, k, p, n)
        states.append((pinned(torch, x), pinned(torch, v)))   # the end-to-end leg uploads from pinned memory
        # every bead of small systems; 4 evenly spaced beads of large ones, scaled to P
        beads = range(p) if n * p <= 100000 else range(0, p, max(1, p // 4))
        box = cells[k][0] if npt else systems[k]["box"]
        pairs += int(round(sum(count_pairs(x[b], box, pot["r_cut"]) for b in beads) * p / len(beads)))
    sampled = {k: kernel_ms[k] / kernel_n[k] for k in kernel_ms if kernel_n[k]}
    launch_ms = in_graph_launch_ms(sampled, kernel_n, np.mean(step_ms), args.steps, sizes)
    force_ms = launch_ms.get("force", 0.0)
    fused = all(p == 1 for _, p in sizes)
    flops_per_launch = PAIR_FLOPS * pairs
    achieved = flops_per_launch / (force_ms * 1e-3) / 1e12 if force_ms > 0 else None
    peak = fp32_peak
    step_breakdown = {k: round(kernel_ms[k] / max(args.steps, 1), 4) for k in kernel_ms}

    # end to end through the C ABI with host buffers: H2D state, 256 steps, D2H
    # observables and the state reached
    e2e_ms = []
    rebuilds_e2e0 = qtb.qtb_list_rebuilds(ctx)
    outs = [(pinned(torch, np.zeros_like(xt.numpy())), pinned(torch, np.zeros_like(vt.numpy())))
            for xt, vt in states]
    for i in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k, (xt, vt) in enumerate(states):
            x, v = xt.numpy(), vt.numpy()
            if npt:     # the cell first: positions are taken in the cell current at the upload
                qtb.qtb_set_cell(ctx, k, *cells[k])
            qtb.qtb_set_state(ctx, k, x, v)
        qtb.qtb_step_n(ctx, BLOCK)
        for k, (n, p) in enumerate(sizes):
            qtb.qtb_observables(ctx, k)
            qtb.qtb_get_state_into(ctx, k, outs[k][0].numpy(), outs[k][1].numpy())
            if npt:
                qtb.qtb_get_cell(ctx, k)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_value = ws * units * BLOCK * args.steps / (np.sum(e2e_ms) / 1e3)
    rebuilds_e2e = (qtb.qtb_list_rebuilds(ctx) - rebuilds_e2e0) / args.steps
    integ = 1 if fused else BLOCK * len({p for _, p in sizes})
    # centroid estimators: recorded step only, every step at constant pressure
    cen = (BLOCK if npt else 1) if any(p > 1 for _, p in sizes) else 0
    cell_launches = (1 if fused else BLOCK) if npt else 0

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+fixed30+f64acc" if args.precision == "mixed" else "f64",
        "data": "synthetic: seeded rock-salt crystals, sigma 0.02 A, Maxwell-Boltzmann velocities",
        "config": {"workload": desc, "name": args.workload, "systems": len(systems),
                   "atom_beads_per_md_step": units, "md_steps_per_bench_step": BLOCK, "precision": args.precision,
                   "filter": filt if setup is not None else "none (white noise)", "parallelism": f"replicas x{ws}",
                   "skin_A": params["skin"] if params["skin"] else "default: per system min(r_cut/4, 0.8 max(1, sqrt(T/300 K)))",
                   "list_lanes": params.get("list_lanes") or "default (16)",
                   "rebuild_scope": "all systems" if params.get("rebuild_scope") else "requesting systems",
                   "autotune": tuning,
                   "noise_generator": args.generator if args.generator == "filter" else
                   f"fourier segments of {256 * args.segment_blocks} steps (Eq. 9)",
                   "launch": "direct (2 x 128-step calls per block)" if args.direct else "CUDA graph per 256-step block",
                   "equilibration": f"{args.equilibrate} untimed blocks, then every list rebuilt on that "
                                    "configuration" if args.equilibrate > 0 else "none (lists of the initial lattice)",
                   "l2": "256 MB buffer written between timed steps (flush)"},
        "roofline": {"bound": "alu", "kernel": "k_step", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if achieved else None,
                     "traffic": measured_traffic("k_step", args.workload),
                     "peak_source": "measured: FP32 FMA chains filling every SM, best of 5 launches of "
                                    f"{fp32_peak_ms:.2f} ms (qtb_fp32_peak), just before the timed region",
                     "peak_nominal": alu_peak_tflops(),
                     "frac_of_nominal": achieved / alu_peak_tflops() if achieved else None,
                     "flops_per_launch": flops_per_launch, "pairs_per_launch": pairs, "mean_launch_ms": force_ms,
                     "duration_method": "in-graph: event-timed block minus its once-per-block kernels, "
                                        "shared between the per-step kernels in the ratio of their event-timed "
                                        "samples (every 64th step)",
                     "sampled_launch_ms": sampled.get("force")},
        "roofline_integrator": integrator_roofline(launch_ms, units, sizes, args.precision, args.workload),
        "kernel_ms_per_bench_step": step_breakdown,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(2 * units * 3 * 8 + npt * len(systems) * 32),
                "d2h_bytes_per_step": int(len(systems) * (qtb.NREC * 8 + npt * 32) + 2 * units * 3 * 8),
                "list_rebuilds_per_step": rebuilds_e2e,
                "per_step": "state (and cell, at constant pressure) uploaded from pinned host memory, 256 steps, "
                            "observables, state and cell read back"},
        # per block: white, filter, the integrator (once for one-bead systems, else every
        # step per distinct bead count), 256 step launches (a list rebuild runs inside the
        # step launch that needs it), the centroid estimators of the recorded step (ring
        # polymers), the block clock
        # (+ the cell kernel: before each block's first step at constant pressure, every
        # step for ring polymers)
        "gpu_launches": 2 + integ + BLOCK + cen + 1 + cell_launches,
        "list_rebuilds_per_bench_step": rebuilds,
        "wall_s": wall,
        "observables": {"K_eV": float(obs[1]), "V_eV": float(obs[2]), "step": int(obs[0])},
    }
    qtb.qtb_destroy(ctx)
    del flush
    if args.precision == "mixed" and setup is not None and args.fp64_blocks > 0:
        # the metric compares the mixed form with the FP64 form at matched error:
        # the FP64 form of the same workload, timed from the same steady state
        fp64 = fp64_form_leg(qtb, torch, systems, params, setup, states, units, args.fp64_blocks, cells)
        fp64["mixed_over_fp64"] = value / fp64["value"]
        line["fp64_form"] = fp64
    if args.precision == "mixed" and setup is not None and args.matched_blocks > 0 and len(systems) == 1:
        line["matched_error"] = matched_error(qtb, systems, params, setup, states[0], args.matched_blocks, cells[0])
    if ws == 1 and not args.no_cpu_baseline:   # the host baseline belongs to the one-GPU line only
        line["cpu_baseline"] = cpu_baseline(args.workload, sample_atoms=64)
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def fp64_form_leg(qtb, torch, systems, params, setup, states, units, n_blocks, cells):
    """The FP64 form (every step in FP64, FP64 filter) of the same workload: the
    mixed form's steady state uploaded, lists rebuilt on it, one warm-up block,
    then n_blocks device-timed 256-step blocks with an L2 flush between them."""
    p64 = dict(params, precision=qtb.FP64, filter_prec=qtb.FILTER_FP64)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = qtb.qtb_init(systems, p64, stream=stream.cuda_stream)
    try:
        qtb.qtb_set_filter(ctx, -1, *setup)
        for k, (xt, vt) in enumerate(states):
            if cells[k] is not None:
                qtb.qtb_set_cell(ctx, k, *cells[k])
            qtb.qtb_set_state(ctx, k, xt.numpy(), vt.numpy())
        qtb.qtb_rebuild_lists(ctx)
        qtb.qtb_step_n(ctx, BLOCK)
        qtb.qtb_sync(ctx)
        flush = l2_flush_buffer(torch)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_blocks)]
        torch.cuda.synchronize()
        for i, (a, b) in enumerate(ev):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
                a.record(stream)
            qtb.qtb_step_n(ctx, BLOCK)
            b.record(stream)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
    finally:
        qtb.qtb_destroy(ctx)
    t = float(np.sum(ms))
    return {"value": units * BLOCK * n_blocks / (t / 1e3), "unit": UNIT, "ms_per_step": t / n_blocks,
            "steps": n_blocks, "dtype": "f64", "filter": "fp64 (direct convolution)",
            "start": "the mixed form's steady state, lists rebuilt, one warm-up block"}


# record slots: K, V, E = K + V, virial trace
MATCHED_OBS = (("K_eV", lambda r: r[:, 1]), ("V_eV", lambda r: r[:, 2]), ("E_eV", lambda r: r[:, 1] + r[:, 2]),
               ("virial_trace_eV", lambda r: r[:, 5] + r[:, 9] + r[:, 13]))


def block_sigma(x, n_blocks=16):
    """Standard error of the mean of a correlated series by block averaging."""
    x = np.asarray(x, np.float64)
    m = len(x) // n_blocks
    b = x[:m * n_blocks].reshape(n_blocks, m).mean(1)
    return float(b.std(ddof=1) / np.sqrt(n_blocks))


def matched_error(qtb, systems, params, setup, state, n_blocks, cell, stride=4):
    """Error of the mixed form against the FP64 form at the bench's own size.

    Both forms start from the same steady state (the mixed form's, uploaded to
    both) at step 0 with the same seed, so they draw the same Philox stream,
    and run n_blocks 256-step blocks recording every `stride` steps.  The FP64
    form stands in for the FP64 oracle, to which it is parity-pinned at 1e-12
    on the configurations the oracle can run.  For each observable: the mean of
    each form, the FP64 form's block-averaged standard error sigma, and the
    mixed form's deviation in units of sigma."""
    nrec = n_blocks * BLOCK // stride
    x, v = state[0].numpy(), state[1].numpy()
    series = {}
    for form, prec, fp in (("fp64", qtb.FP64, qtb.FILTER_FP64), ("mixed", qtb.MIXED, params["filter_prec"])):
        p = dict(params, precision=prec, filter_prec=fp, obs_stride=stride, max_records=nrec)
        ctx = qtb.qtb_init(systems, p)
        try:
            qtb.qtb_set_filter(ctx, -1, *setup)
            if cell is not None:
                qtb.qtb_set_cell(ctx, 0, *cell)
            qtb.qtb_set_state(ctx, 0, x, v)
            qtb.qtb_step_n(ctx, n_blocks * BLOCK)
            series[form] = qtb.qtb_get_series(ctx, 0, nrec)
        finally:
            qtb.qtb_destroy(ctx)
    out = {"steps": n_blocks * BLOCK, "record_stride": stride, "reference": "FP64 GPU form (parity-pinned to the "
           "FP64 oracle at 1e-12)", "sigma": "block average, 16 blocks", "observables": {}}
    worst = 0.0
    obs = MATCHED_OBS + ((("volume_A3", lambda r: r[:, 20]),) if cell is not None else ())
    for name, get in obs:
        a, b = get(series["fp64"]), get(series["mixed"])
        sig = block_sigma(a)
        dev = (b.mean() - a.mean()) / sig if sig > 0 else 0.0
        worst = max(worst, abs(dev))
        out["observables"][name] = {"fp64": float(a.mean()), "mixed": float(b.mean()), "sigma": sig,
                                    "mixed_minus_fp64_in_sigma": float(dev)}
    out["max_abs_deviation_in_sigma"] = worst
    out["matched"] = bool(worst <= 2.0)
    return out


def measured_traffic(kernel, workload_name):
    """DRAM bytes per launch from the committed ncu capture of this kernel on
    this workload, or None when there is none or the kernel's source has
    changed since the counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[f"{kernel}/{workload_name}"]
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != rec["source_sha1"]:
                return None
        return rec["dram_bytes_per_launch"]
    except Exception:
        return None


def hbm_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, "fallback"


def pinned(torch, a):
    """A page-locked host copy of array a (a torch tensor; .numpy() views its memory)."""
    t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
    t.numpy()[...] = a
    return t


def in_graph_launch_ms(sampled, kernel_n, block_ms, nblocks, sizes):
    """Mean duration of one launch of each kernel class inside the captured block.

    An event pair around a launch exposes that launch's dispatch latency (the
    graph can no longer overlap it with the previous kernel), so the sampled
    durations overstate the in-graph ones.  The event-timed block length minus
    the kernels launched once per block (white noise, filter, and the
    integrator when it is fused into the step kernel) is the time of the
    per-step launches; it is shared between them in the ratio of their
    samples."""
    if "force" not in sampled:
        return dict(sampled)
    fused = all(p == 1 for _, p in sizes)
    n_p = len({p for _, p in sizes})
    per_step = {"force": 1}
    if not fused:
        per_step["integrate"] = n_p
    once = sum(sampled[k] * kernel_n[k] / nblocks for k in sampled if k not in per_step)
    rest = (block_ms - once) / BLOCK
    w = sum(sampled[k] * c for k, c in per_step.items() if k in sampled)
    out = dict(sampled)
    for k, c in per_step.items():
        if k in sampled:
            out[k] = rest * sampled[k] / w
    return out


def integrator_roofline(launch_ms, units, sizes, precision, workload_name=None):
    """HBM roofline of the ring-polymer integrator (systems with P > 1; for
    one-bead systems it is fused into the step kernel)."""
    if all(p == 1 for _, p in sizes) or "integrate" not in launch_ms:
        return None
    ms = launch_ms["integrate"]
    nbytes = INTEGRATOR_BYTES[precision] * units
    peak, src = hbm_peak_gbs()
    achieved = nbytes / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "k_integrate_nm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": src, "bytes_per_launch": nbytes, "mean_launch_ms": ms,
            "traffic": measured_traffic("k_integrate_nm", workload_name) if workload_name else None}


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


def oracle_sample(name, ncell, n_sample, part=0, parts=1):
    """A bounded sample of one MD step of the workload for the FP64 oracle:
    forces on `n_sample` bead-atoms of bead 0 of the first system (brute force
    over all ions and images) and the random force of their 3 dofs (2049-tap
    direct convolution; white noise for standard PIMD).  With `parts` workers,
    worker `part` takes its own n_sample of n_sample * parts evenly spaced
    bead-atoms.  Returns a callable one(n) for step n, the number of
    bead-atoms it covers and the system size."""
    import oracle
    from oracle import spectra as S
    systems, pot, params, setup, desc = workload(name, ncell, "fp64", "fp32")
    s = systems[-1] if name == "sweep64" else systems[0]
    T, dt = s["T"], params["dt"]
    if setup is None:
        h = np.array([np.sqrt(8.617333262e-5 * T)])
    else:
        mode, L, wmax = setup
        P = int(s["pos"].shape[0]) if mode == 2 else 1
        h = S.taps(L, dt, T, wmax, P=P, sol=S.kappa_solve(P) if P > 1 else None)
    n = len(s["types"])
    tot = min(n, n_sample * parts)
    sel = np.arange(0, n, max(1, n // tot))[:tot][part::parts]
    oracle.build()

    def one(step):
        oracle.pair_forces(s["pos"][0], s["types"], s["box"], pot, sel=sel)
        oracle.colored_block(12345, 0, 3 * len(sel), step, 1, h)

    return one, len(sel), n


def _oracle_worker(task):
    """One process of the host-core pool: its slice of the sample, either for at
    least `seconds` of host time or for `warmup` untimed then `steps` timed steps.
    Returns (bead-atoms per step, timed steps, seconds, system size)."""
    name, ncell, n_sample, part, parts, seconds, warmup, steps = task
    one, k, n = oracle_sample(name, ncell, n_sample, part, parts)
    for i in range(warmup):
        one(i)
    t0 = time.perf_counter()
    done = 0
    while (seconds is not None and (done == 0 or time.perf_counter() - t0 < seconds)) or \
            (seconds is None and done < steps):
        one(warmup + done)
        done += 1
    return k, done, time.perf_counter() - t0, n


def oracle_pool_run(name, ncell, n_sample, seconds=None, warmup=0, steps=0):
    """The oracle on every host core: one spawned process per core (spawn, so that
    no process inherits a CUDA context), each on its own slice of the sample.
    Returns (bead-atom-steps per second over the slowest worker's time, workers,
    bead-atoms per step, seconds, system size)."""
    import multiprocessing as mp
    workers = max(1, os.cpu_count() or 1)
    tasks = [(name, ncell, n_sample, w, workers, seconds, warmup, steps) for w in range(workers)]
    with mp.get_context("spawn").Pool(workers) as pool:
        res = pool.map(_oracle_worker, tasks)
    units = sum(k * d for k, d, _, _ in res)
    t = max(dt for _, _, dt, _ in res)
    return units / t, workers, sum(k for k, _, _, _ in res), t, res[0][3], res[0][1]


def cpu_baseline(name, sample_atoms=64, min_seconds=10.0):
    """The FP64 oracle, as it stands, on every host core (see oracle_pool_run):
    each process runs its slice for about min_seconds."""
    value, workers, k, dt, n, steps = oracle_pool_run(name, 10, sample_atoms, seconds=min_seconds)
    return {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{k} of {n} bead-atoms ({sample_atoms} per process, {workers} processes), "
                      f"~{steps} step(s) each: brute-force periodic forces + random force of their dofs, "
                      f"{dt:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    # every host core, 64 bead-atoms per process and step (~50 ms of host time per step)
    value, workers, k, dt, n, _ = oracle_pool_run(args.workload, args.ncell, 64, warmup=args.warmup,
                                                  steps=args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: FP64 oracle on {k} of {n} bead-atoms per step",
                       "name": args.workload},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                             "sample": f"{k} bead-atoms per step over {workers} processes: forces + random "
                                       f"force of the FP64 oracle"},
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
