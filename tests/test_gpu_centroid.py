"""GPU parity of the centroid-virial kinetic estimators (record slots 18, 19)
against the oracle evaluated on the GPU's own state (positions, velocities of a
recorded step; the oracle recomputes the forces in FP64).

* FP64 form: within 1e-11 of the scale |r - rbar| |f| (Cauchy-Schwarz bound of
  the virial term) and of the kinetic energy;
* mixed form: the forces carry the FP32 error (relative L2 <= 1e-5), so the
  virial term is compared within 3e-5 of the same scale;
* pair potential (periodic, beads wrapped independently on download: minimum
  image), external potential, P = 4, 16 (two beads per warp of the kernel), a
  batch of systems with P = 4, 2, 1, the first record of a context (forces
  refreshed, no step), and the series row of the recorded step.
"""
import numpy as np
import pytest

from helpers import gpu_ctx, minimg, oracle_sim

from paper_1905_02521_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KB = 8.617333262e-5


@pytest.fixture(scope="module")
def qtb():
    import torch
    assert torch.cuda.is_available()
    from paper_1905_02521_gb300 import build
    build.build()
    from paper_1905_02521_gb300 import qtb as q
    return q


def _system(case):
    rng = np.random.default_rng(21)
    if case == "mgo_p4":
        s, pot = W.mgo_system(2, 300.0, n_beads=4)
    elif case == "mgo_p2":
        s, pot = W.mgo_system(2, 300.0, n_beads=2, seed=778)
    elif case == "mgo_p1":
        s, pot = W.mgo_system(2, 300.0, n_beads=1, seed=779)
    elif case == "lih_p16":
        s, pot = W.lih_system(2, 100.0, n_beads=16)
    else:
        s, pot = W.oscillators(37, 100.0, 1e-2, n_beads=4, x0=0.3, spread=0.05)
        return s, pot, 1, {"omega": 0.1}
    s["pos"] = s["pos"] + rng.normal(0, 0.03, s["pos"].shape) * (s["pos"].shape[0] > 1)
    return s, pot, 0, None


def _check(obs, s, pot, oracle, x, v, step, potential, ext, tol):
    sim = oracle_sim(oracle, s, pot, 0.5, potential=potential, ext=ext)
    sim.set_state(x, v, step)
    oo = sim.observe()
    _, _, f, _ = sim.state()
    d = x - x[:1]
    if potential == 0:
        d = minimg(d, s["box"])
    d = d - d.mean(0)
    scale = np.sqrt((d ** 2).sum() * (f ** 2).sum()) + 1e-300
    P, N = x.shape[0], x.shape[1]
    if P == 1:
        assert obs[18] == pytest.approx(1.5 * N * KB * s["T"], rel=1e-14)
        assert obs[19] == obs[1]
    assert abs(obs[18] - oo[18]) < tol * scale + 1e-13 * abs(oo[18])
    # K_0 of slot 19: FP64 in the FP64 form; the FP32 form forms each atom's
    # centroid kinetic energy in FP32 (float-float sums over atoms): ~1e-7 relative
    k0_rel = 1e-12 if tol < 1e-6 else 1e-6
    assert abs(obs[19] - oo[19]) < tol * scale + k0_rel * abs(oo[1])
    return oo


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 3e-5)])
@pytest.mark.parametrize("case", ["mgo_p4", "lih_p16", "harm_p4"])
def test_centroid_estimators_on_gpu_state(qtb, oracle, case, precision, tol):
    s, pot, potential, ext = _system(case)
    P, N = s["pos"].shape[0], s["pos"].shape[1]
    ctx = gpu_ctx(qtb, [s], pot, 0.5, precision=precision, seed=17, potential=potential, ext=ext,
                  obs_stride=8, max_records=64)
    try:
        # the first record: forces refreshed at the initial positions
        x0, v0 = qtb.qtb_get_state(ctx, 0, P, N)
        _check(qtb.qtb_observables(ctx, 0), s, pot, oracle, x0, v0, 0, potential, ext, tol)
        qtb.qtb_step_n(ctx, 40)
        obs = qtb.qtb_observables(ctx, 0)
        assert obs[0] == 40
        x, v = qtb.qtb_get_state(ctx, 0, P, N)
        oo = _check(obs, s, pot, oracle, x, v, 40, potential, ext, tol)
        ser = qtb.qtb_get_series(ctx, 0, 64)
        last = ser[np.flatnonzero(ser[:, 0] == 40)[0]]
        assert np.array_equal(last[18:20], obs[18:20])
        # a ring polymer at 100-300 K: the virial term is not negligible
        assert abs(oo[18] - 1.5 * N * KB * s["T"]) > 1e-3 * abs(oo[18])
    finally:
        qtb.qtb_destroy(ctx)


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 3e-5)])
def test_centroid_estimators_batched_bead_counts(qtb, oracle, precision, tol):
    cases = [_system(c) for c in ("mgo_p4", "mgo_p2", "mgo_p1")]
    pot = cases[0][1]
    ctx = gpu_ctx(qtb, [c[0] for c in cases], pot, 0.5, precision=precision, seed=23, obs_stride=4)
    try:
        qtb.qtb_step_n(ctx, 24)
        for k, (s, _, _, _) in enumerate(cases):
            P, N = s["pos"].shape[0], s["pos"].shape[1]
            obs = qtb.qtb_observables(ctx, k)
            assert obs[0] == 24
            x, v = qtb.qtb_get_state(ctx, k, P, N)
            _check(obs, s, pot, oracle, x, v, 24, 0, None, tol)
    finally:
        qtb.qtb_destroy(ctx)
