"""Parity at the benchmark's full sizes, in the configuration bench.py times
(mixed form, its filters and its context parameters), on sampled outputs the
oracle can compute one by one: after 300 steps (a list rebuild, a block of the
captured graph and a partial block), the GPU forces of sampled bead-atoms
against the oracle's brute force on the GPU's own configuration, FP32 criteria
of tests/tolerances.py.

* LiH 6^3 x 8 beads, QTB-PIMD (13824 bead-atoms);
* LiH 6^3 x 32 beads, PIMD (55296 bead-atoms);
* the 64-system sweep, 216-4096 ions at 10-1500 K in one context (106416 ions):
  the smallest, a middle and the largest system.
(The 8000-ion MgO workload: tests/test_gpu_parity.py.)
"""
import os
import sys

import numpy as np
import pytest

from helpers import rel_inf, rel_l2
from tolerances import F32_INF, F32_L2

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def qtb():
    import torch
    assert torch.cuda.is_available()
    from paper_1905_02521_gb300 import build
    build.build()
    from paper_1905_02521_gb300 import qtb as q
    return q


def _bench():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    return bench


@pytest.mark.parametrize("name,picks", [("lih_qtbpimd_p8", [0]), ("lih_pimd_p32", [0]), ("sweep64", [0, 31, 63])])
def test_sampled_forces_at_full_size(qtb, oracle, name, picks):
    systems, pot, params, setup, _ = _bench().workload(name, 10, "mixed", "fp32")
    ctx = qtb.qtb_init(systems, params)
    try:
        if setup is not None:
            qtb.qtb_set_filter(ctx, -1, *setup)
        qtb.qtb_step_n(ctx, 300)
        rng = np.random.default_rng(3)
        for k in picks:
            s = systems[k]
            P, N = s["pos"].shape[0], len(s["types"])
            x, _ = qtb.qtb_get_state(ctx, k, P, N)
            f = qtb.qtb_get_forces(ctx, k, P, N) * P          # undo the 1/P of Eq. 4
            fg, fo = [], []
            for b in sorted(set(rng.choice(P, min(P, 3), replace=False).tolist())):
                sel = rng.choice(N, min(N, 24), replace=False)
                fo.append(oracle.pair_forces(x[b], s["types"], s["box"], pot, sel=sel)[0])
                fg.append(f[b, sel])
            fg, fo = np.concatenate(fg), np.concatenate(fo)
            assert rel_l2(fg, fo) < F32_L2 and rel_inf(fg, fo) < F32_INF, (name, k, rel_l2(fg, fo), rel_inf(fg, fo))
    finally:
        qtb.qtb_destroy(ctx)
