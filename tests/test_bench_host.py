"""Host-side arithmetic of bench.py (no GPU): the pair count behind the
roofline's algorithmic flops, the split of an event-timed block into in-graph
launch durations, the integrator's bytes per launch and the job throughput.

The pair count is checked against a brute-force sum over atom pairs and periodic
images, in a box smaller than 2 r_cut (several images per pair) and a larger one.
"""
import numpy as np
import pytest

import bench
from paper_1905_02521_gb300 import workloads as W


def brute_pairs(pos, box, rc):
    pos = np.mod(pos, box)
    nmax = [int(np.ceil(rc / b)) for b in box]
    n = 0
    for i in range(len(pos)):
        d = pos - pos[i]                                   # [N, 3]
        for a in range(-nmax[0], nmax[0] + 1):
            for b in range(-nmax[1], nmax[1] + 1):
                for c in range(-nmax[2], nmax[2] + 1):
                    r = np.linalg.norm(d + np.array([a, b, c]) * box, axis=1)
                    n += int((r < rc).sum())
    return n - len(pos)                                     # not the ion itself


@pytest.mark.parametrize("ncell,a,rc", [(2, 4.21, 8.0), (3, 4.21, 6.0)])
def test_count_pairs_matches_brute_force(ncell, a, rc):
    pos, _, box = W.rocksalt(ncell, a, sigma=0.05, seed=3)
    assert bench.count_pairs(pos, box, rc) == brute_pairs(pos, box, rc)


def test_in_graph_launch_split():
    nb = 16
    # one-bead systems: white and filter once per block, the rest is the step launches
    sampled = {"white": 0.04, "filter": 0.10, "force": 0.015}
    kernel_n = {"white": nb, "filter": nb, "force": 4 * nb}
    out = bench.in_graph_launch_ms(sampled, kernel_n, 3.5, nb, [(8000, 1)])
    assert out["force"] == pytest.approx((3.5 - 0.04 - 0.10) / 256)
    # ring polymers: integrator and step share the per-step time in the ratio of their samples
    sampled = {"white": 0.05, "filter": 0.2, "integrate": 0.01, "force": 0.03}
    kernel_n = {"white": nb, "filter": nb, "integrate": 4 * nb, "force": 4 * nb}
    out = bench.in_graph_launch_ms(sampled, kernel_n, 12.0, nb, [(1728, 32)])
    rest = (12.0 - 0.25) / 256
    assert out["integrate"] == pytest.approx(rest * 0.01 / 0.04)
    assert out["force"] == pytest.approx(rest * 0.03 / 0.04)
    assert out["integrate"] + out["force"] == pytest.approx(rest)


def test_integrator_roofline_and_throughput():
    assert bench.integrator_roofline({"integrate": 0.01}, 8000, [(8000, 1)], "mixed") is None
    r = bench.integrator_roofline({"integrate": 0.02}, 55296, [(1728, 32)], "mixed")
    nbytes = 96 * 55296                       # x, v, f, xref, noise read; x, v, packed x written
    assert r["bytes_per_launch"] == nbytes
    assert r["achieved"] == pytest.approx(nbytes / 0.02e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert bench.job_throughput(8000 * 256, 48, 2, 170.0) == pytest.approx(2 * 8000 * 256 * 48 / 0.170)
