"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Tolerances:

* FP64 form: 1e-12 norm-wise (max |diff| / RMS) on forces, states and noise;
* mixed form: forces within 1e-5 norm-wise of the oracle evaluated on the GPU's
  own configuration (per step, first 100 steps); FP32 noise within 1e-5;
* kappa_P: the GPU solves the same least-squares problem (Eq. 10 on the
  collocation grid) by normal equations + Cholesky followed by one step of
  corrected semi-normal-equation refinement, the oracle by LAPACK; both reach
  cond(A) eps (cond <= 7e3 for P <= 32), so 1e-10 relative is required per
  node and for the taps.
"""
import numpy as np
import pytest

from helpers import gpu_ctx, minimg, oracle_sim, rel_inf, rel_l2

from oracle import spectra as S
from paper_1905_02521_gb300 import workloads as W
from tolerances import F32_INF, F32_L2  # FP32 criterion and its max-norm guard (see tolerances.py)

pytestmark = pytest.mark.gpu


def assert_force_parity(f, fo, tol):
    if tol >= 1e-6:   # FP32 form
        assert rel_l2(f, fo) < F32_L2, (rel_l2(f, fo), rel_inf(f, fo))
        assert rel_inf(f, fo) < F32_INF, (rel_l2(f, fo), rel_inf(f, fo))
    else:
        assert rel_inf(f, fo) < tol


@pytest.fixture(scope="module")
def qtb():
    import torch
    assert torch.cuda.is_available()
    from paper_1905_02521_gb300 import build
    build.build()
    from paper_1905_02521_gb300 import qtb as q
    return q


@pytest.mark.parametrize("P", [2, 4, 8, 32])
def test_kappa_solve_matches_oracle(qtb, P):
    Fg = qtb.qtb_kappa_solve(P, n=1024, y_max=1000.0, y0=1.0)
    sol = S.kappa_solve(P, n=1024, ymax=1000.0, y0=1.0)
    assert np.allclose(Fg, sol.F, rtol=1e-10, atol=0), np.abs(Fg / sol.F - 1).max()


def test_taps_match_oracle(qtb):
    s, pot = W.mgo_system(2, 300.0)
    ctx = gpu_ctx(qtb, [s], pot, 1.0)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 513, 0.3)
        h = qtb.qtb_get_taps(ctx, 0)
        ho = S.taps(513, 1.0, 300.0, 0.3)
        assert len(h) == 257
        assert rel_inf(h, ho) < 1e-12
    finally:
        qtb.qtb_destroy(ctx)


def test_kappa_taps_match_oracle(qtb):
    s, pot = W.lih_system(2, 50.0, n_beads=4, gamma=1e-3)
    s["box"] = np.array([8.16] * 3)
    pot = dict(pot, r_cut=8.0)
    ctx = gpu_ctx(qtb, [s], pot, 0.25)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB_PIMD, 257, 0.6)
        h = qtb.qtb_get_taps(ctx, 0)
        ho = S.taps(257, 0.25, 50.0, 0.6, P=4, sol=S.kappa_solve(4))
        assert rel_inf(h, ho) < 1e-10
    finally:
        qtb.qtb_destroy(ctx)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_colored_noise_block_matches_oracle(qtb, oracle, precision, tol):
    s, pot = W.mgo_system(2, 300.0)
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=precision, filter_prec=1, seed=777)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 513, 0.3)
        qtb.qtb_step_n(ctx, 300)                     # move into block 1
        eta, blk = qtb.qtb_get_noise(ctx, 0, 192)
        assert blk == 1
        h = S.taps(513, 1.0, 300.0, 0.3)
        sel = np.array([0, 1, 63, 64, 127, 128, 191])
        ref = oracle.colored_block(777, 0, 192, 256, 256, h)   # [dof][step]
        assert rel_inf(eta[:, sel], ref[sel].T) < tol
    finally:
        qtb.qtb_destroy(ctx)


@pytest.mark.parametrize("precision,tol", [(0, 1e-14), (1, 1e-5)])
def test_white_noise_block_matches_oracle(qtb, oracle, precision, tol):
    # white Langevin bath: eta = sqrt(k_B T) xi, the Philox + Box-Muller stream of every
    # dof, all dofs of a ring-polymer system, blocks 0 and 2.  FP64 form: the normals to
    # a few ulp (library log/sin/cos on either side); mixed form: Box-Muller in FP32
    # (measured 2.7e-6 norm-wise), within the FP32 noise criterion
    s, pot = W.mgo_system(2, 250.0, n_beads=2)
    D = 3 * len(s["types"]) * 2
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=precision, filter_prec=1, seed=4242)
    try:
        for blk_want, n0 in ((0, 0), (2, 512)):
            qtb.qtb_step_n(ctx, n0 - qtb.qtb_get_step(ctx))
            eta, blk = qtb.qtb_get_noise(ctx, 0, D)
            assert blk == blk_want
            ref = np.sqrt(8.617333262e-5 * 250.0) * oracle.white_block(4242, 0, D, n0, 256)   # [dof][step]
            assert rel_inf(eta, ref.T) < tol, (blk, rel_inf(eta, ref.T))
    finally:
        qtb.qtb_destroy(ctx)


@pytest.mark.parametrize("ncell", [2, 3, 4])
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_forces_match_oracle(qtb, oracle, ncell, precision, tol):
    s, pot = W.mgo_system(ncell, 300.0, sigma=0.05, seed=100 + ncell)
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=precision)
    try:
        x, _ = qtb.qtb_get_state(ctx, 0, 1, len(s["types"]))
        f = qtb.qtb_get_forces(ctx, 0, 1, len(s["types"]))[0]
        fo, eo, vo = oracle.pair_forces(x[0], s["types"], s["box"], pot)
        assert_force_parity(f, fo, tol)
        obs = qtb.qtb_observables(ctx, 0)
        assert obs[2] == pytest.approx(eo, rel=10 * tol, abs=10 * tol)
        assert np.allclose(obs[5:14].reshape(3, 3), vo, rtol=10 * tol, atol=10 * tol * np.abs(vo).max())
    finally:
        qtb.qtb_destroy(ctx)


def _oracle_taps(qtb, mode, n_taps, dt, T, omega_max, P):
    """The oracle's taps of a noise mode: theta (Eq. 7) or kappa_P (Eqs. 10, 12)."""
    if mode == qtb.NOISE_QTB:
        return S.taps(n_taps, dt, T, omega_max)
    if mode == qtb.NOISE_QTB_PIMD:
        return S.taps(n_taps, dt, T, omega_max, P=P, sol=S.kappa_solve(P))
    return None


def _traj_compare(qtb, oracle, s, pot, dt, mode, n_taps, omega_max, nsteps, check_every, tol, P=1):
    ctx = gpu_ctx(qtb, [s], pot, dt, precision=0, seed=4321)
    try:
        taps = _oracle_taps(qtb, mode, n_taps, dt, s["T"], omega_max, P)
        if taps is not None:
            qtb.qtb_set_filter(ctx, 0, mode, n_taps, omega_max)
        sim = oracle_sim(oracle, s, pot, dt, seed=4321, taps=taps)
        N = len(s["types"])
        done = 0
        while done < nsteps:
            qtb.qtb_step_n(ctx, check_every)
            sim.step(check_every, record=False)
            done += check_every
            xg, vg = qtb.qtb_get_state(ctx, 0, P, N)
            fg = qtb.qtb_get_forces(ctx, 0, P, N)
            xo, vo, fo, st = sim.state()
            assert st == done == qtb.qtb_get_step(ctx)
            assert np.abs(minimg(xg - xo, s["box"])).max() < tol * 10.0
            assert rel_inf(vg, vo) < tol
            assert rel_inf(fg, fo) < tol
        obs = qtb.qtb_observables(ctx, 0)
        oo = sim.observe()
        assert obs[1] == pytest.approx(oo[1], rel=tol)
        assert obs[2] == pytest.approx(oo[2], rel=tol)
    finally:
        qtb.qtb_destroy(ctx)


def test_fp64_qtb_trajectory_matches_oracle(qtb, oracle):
    # 64-ion MgO, QTB-MD, 513 taps: state and forces after every one of the
    # first 100 steps
    s, pot = W.mgo_system(2, 300.0)
    _traj_compare(qtb, oracle, s, pot, 1.0, qtb.NOISE_QTB, 513, 0.3, 100, 1, 1e-12)


@pytest.mark.parametrize("P", [4, 8])
def test_fp64_qtb_pimd_trajectory_matches_oracle(qtb, oracle, P):
    # QTB-PIMD (Sec. 2.3): kappa_P of Eq. 10 in the taps (Eq. 12), the time-domain
    # filter over all 3 N P normal-mode dofs (dof = (k 3 + c) N + i), the O step
    # in mode space, per-bead forces with the 1/P of Eq. 4.  64-ion LiH at 50 K,
    # dt 0.25 fs, gamma 0.01/fs (so that the coloured force moves the state
    # visibly each step), 257 taps; state, velocities and forces after every one
    # of the first 100 steps.  (Rounding-order differences grow along the stiff
    # ring-polymer trajectory as in the white PIMD test: 1e-11.)
    s, pot = W.lih_system(2, 50.0, gamma=1e-2, n_beads=P)
    s["box"] = np.array([8.16] * 3)
    rng = np.random.default_rng(11)
    s["pos"] = s["pos"] + rng.normal(0, 0.01, s["pos"].shape)
    _traj_compare(qtb, oracle, s, pot, 0.25, qtb.NOISE_QTB_PIMD, 257, 0.6, 100, 1, 1e-11, P=P)


@pytest.mark.parametrize("P", [4, 16])
def test_fp64_pimd_trajectory_matches_oracle(qtb, oracle, P):
    # white-noise PIMD: normal-mode integrator (P = 16: register-tiled transforms)
    # and per-bead forces
    s, pot = W.mgo_system(2, 300.0, n_beads=P)
    rng = np.random.default_rng(5)
    s["pos"] = s["pos"] + rng.normal(0, 0.01, s["pos"].shape)
    # (rounding-order differences of 1e-16 grow along the stiff ring-polymer
    # trajectory to ~1e-12 after 60 steps: state compared at 1e-11)
    _traj_compare(qtb, oracle, s, pot, 0.5, qtb.NOISE_WHITE, 1, 0.0, 60, 20, 1e-11, P=P)


def test_mixed_forces_on_own_configuration_first_100_steps(qtb, oracle):
    s, pot = W.mgo_system(3, 300.0)
    N = len(s["types"])
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=1, filter_prec=1)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 513, 0.3)
        for _ in range(100):   # after every one of the first 100 steps
            qtb.qtb_step_n(ctx, 1)
            x, _ = qtb.qtb_get_state(ctx, 0, 1, N)
            f = qtb.qtb_get_forces(ctx, 0, 1, N)[0]
            fo, _, _ = oracle.pair_forces(x[0], s["types"], s["box"], pot)
            assert_force_parity(f, fo, 1e-5)
    finally:
        qtb.qtb_destroy(ctx)


def test_mixed_single_step_matches_oracle_step(qtb, oracle):
    # one BAOAB step from the GPU's state, FP32 vs the oracle's FP64 step
    s, pot = W.mgo_system(2, 300.0)
    N = len(s["types"])
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=1, filter_prec=1, seed=99)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 513, 0.3)
        qtb.qtb_step_n(ctx, 37)
        x0, v0 = qtb.qtb_get_state(ctx, 0, 1, N)
        sim = oracle_sim(oracle, s, pot, 1.0, seed=99, taps=S.taps(513, 1.0, 300.0, 0.3))
        sim.set_state(x0, v0, 37)
        qtb.qtb_step_n(ctx, 1)
        sim.step(1, record=False)
        x1, v1 = qtb.qtb_get_state(ctx, 0, 1, N)
        xo, vo, _, _ = sim.state()
        assert np.abs(minimg(x1 - xo, s["box"])).max() < 1e-5
        assert rel_inf(v1, vo) < 1e-5
    finally:
        qtb.qtb_destroy(ctx)


@pytest.mark.parametrize("filter_prec", [1, 2])
def test_mixed_qtb_pimd_single_step_matches_oracle_step(qtb, oracle, filter_prec):
    # one QTB-PIMD step (P = 8, kappa_P taps) of the mixed form from the GPU's own
    # state, against the oracle's FP64 step from the same state.  FP32 filter:
    # positions within 1e-5 A, velocities within 1e-5 norm-wise.  BF16
    # tensor-core filter: the noise itself differs from the FP64 convolution by
    # up to RMS 4 * 2^-8 of RMS(eta) (the filter's bound, tests/test_gpu_filter_tc.py),
    # which the O step passes on as sqrt((1 - c1^2)/m) times that; the velocity
    # error may use that much on top of the 1e-5 of the deterministic part.
    P, L, dt, T, gamma, wmax = 8, 257, 0.25, 50.0, 1e-2, 0.6
    s, pot = W.lih_system(2, T, gamma=gamma, n_beads=P)
    s["box"] = np.array([8.16] * 3)
    s["pos"] = s["pos"] + np.random.default_rng(12).normal(0, 0.01, s["pos"].shape)
    N = len(s["types"])
    ctx = gpu_ctx(qtb, [s], pot, dt, precision=1, filter_prec=filter_prec, seed=99)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB_PIMD, L, wmax)
        qtb.qtb_step_n(ctx, 37)
        x0, v0 = qtb.qtb_get_state(ctx, 0, P, N)
        # qtb_get_state wraps every bead into the box; the normal-mode transform
        # needs the beads of an atom in one periodic image (each as the copy
        # nearest bead 0)
        x0 = x0[0][None] + minimg(x0 - x0[0][None], s["box"])
        h = S.taps(L, dt, T, wmax, P=P, sol=S.kappa_solve(P))
        sim = oracle_sim(oracle, s, pot, dt, seed=99, taps=h)
        sim.set_state(x0, v0, 37)
        qtb.qtb_step_n(ctx, 1)
        sim.step(1, record=False)
        x1, v1 = qtb.qtb_get_state(ctx, 0, P, N)
        xo, vo, _, _ = sim.state()
        assert np.abs(minimg(x1 - xo, s["box"])).max() < 1e-5
        if filter_prec == 1:
            assert rel_inf(v1, vo) < 1e-5
        else:
            m = pot["mass"][s["types"]] * W.MVV2E
            c1 = np.exp(-gamma * dt)
            kick = np.sqrt((1.0 - c1 * c1) * (h[0] ** 2 + 2.0 * (h[1:] ** 2).sum()) / m)   # RMS noise kick per atom
            kick_rms = np.sqrt((kick ** 2).mean())
            err = np.sqrt(((v1 - vo) ** 2).mean())
            assert err < 1e-5 * np.sqrt((vo ** 2).mean()) + 4 * 2.0 ** -8 * kick_rms, (err, kick_rms)
    finally:
        qtb.qtb_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_stepping_is_deterministic_and_split_invariant(qtb, precision):
    s, pot = W.mgo_system(2, 300.0)
    N = len(s["types"])
    out = []
    for split in ([600], [100, 156, 300, 44], [1] * 7 + [593]):
        ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=precision, seed=8)
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 513, 0.3)
        for n in split:
            qtb.qtb_step_n(ctx, n)
        out.append(qtb.qtb_get_state(ctx, 0, 1, N))
        qtb.qtb_destroy(ctx)
    for x, v in out[1:]:
        assert np.array_equal(x, out[0][0]) and np.array_equal(v, out[0][1])


@pytest.mark.parametrize("precision,scope", [(0, 0), (1, 0), (0, 1)])
def test_batched_uneven_systems_match_single_runs(qtb, precision, scope):
    # three systems of different size, temperature and bead count in one context.
    # Rebuild scope 0: each system rebuilds its lists on its own schedule (the hot
    # one often, the cold one rarely), so every system of the batch runs bit for
    # bit as alone.  Scope 1: all rebuild together (list order, hence rounding,
    # differs from the single runs; FP64 within 1e-12 over 300 steps).
    sa, pot = W.mgo_system(2, 100.0, seed=1)
    sb, _ = W.mgo_system(3, 700.0, seed=2)
    sc, _ = W.mgo_system(2, 300.0, seed=3, n_beads=2)
    ctx = gpu_ctx(qtb, [sa, sb, sc], pot, 1.0, precision=precision, seed=5, rebuild_scope=scope)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 257, 0.3)
        qtb.qtb_set_filter(ctx, 1, qtb.NOISE_QTB, 513, 0.3)
        qtb.qtb_step_n(ctx, 300)
        batched = [qtb.qtb_get_state(ctx, k, P, len(s["types"]))[0]
                   for k, (s, P) in enumerate([(sa, 1), (sb, 1), (sc, 2)])]
    finally:
        qtb.qtb_destroy(ctx)
    # system k of a batch uses Philox key (seed, k): a single-system context
    # reproduces it when its own seed carries the same key
    for k, (s, L, P) in enumerate([(sa, 257, 1), (sb, 513, 1), (sc, 1, 2)]):
        seed = 5 ^ (k << 32)
        c1 = gpu_ctx(qtb, [s], pot, 1.0, precision=precision, seed=seed)
        try:
            if L > 1:
                qtb.qtb_set_filter(c1, 0, qtb.NOISE_QTB, L, 0.3)
            qtb.qtb_step_n(c1, 300)
            x = qtb.qtb_get_state(c1, 0, P, len(s["types"]))[0]
            if scope == 0:
                assert np.array_equal(x, batched[k]), (k, rel_inf(x, batched[k]))
            else:
                assert rel_inf(x, batched[k]) < 1e-12
        finally:
            qtb.qtb_destroy(c1)


def test_sampled_forces_at_full_size_mixed(qtb, oracle):
    # 8000-ion MgO (the benchmark workload), mixed form: forces of 64 sampled
    # atoms against the oracle's per-atom brute force
    s, pot = W.mgo_system(10, 100.0)
    N = len(s["types"])
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=1, filter_prec=1)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 2049, 0.3)
        qtb.qtb_step_n(ctx, 20)
        x, _ = qtb.qtb_get_state(ctx, 0, 1, N)
        f = qtb.qtb_get_forces(ctx, 0, 1, N)[0]
        sel = np.random.default_rng(1).choice(N, 64, replace=False)
        fo, _, _ = oracle.pair_forces(x[0], s["types"], s["box"], pot, sel=sel)
        assert_force_parity(f[sel], fo, 1e-5)
    finally:
        qtb.qtb_destroy(ctx)


@pytest.mark.parametrize("potential,ext", [(2, {"V0": 0.1, "a": 0.5}), (1, {"omega": 0.1})])
def test_fp64_external_potential_pimd_trajectory(qtb, oracle, potential, ext):
    # separable external potentials (double well / harmonic), P = 4, white noise
    s, pot = W.oscillators(37, 100.0, 1e-2, n_beads=4, x0=0.45, spread=0.05)
    ctx = gpu_ctx(qtb, [s], pot, 0.5, precision=0, seed=31, potential=potential, ext=ext)
    try:
        sim = oracle_sim(oracle, s, pot, 0.5, seed=31, potential=potential, ext=ext)
        qtb.qtb_step_n(ctx, 300)
        sim.step(300, record=False)
        xg, vg = qtb.qtb_get_state(ctx, 0, 4, 37)
        xo, vo, fo, _ = sim.state()
        assert rel_inf(xg, xo) < 1e-12 and rel_inf(vg, vo) < 1e-12
        obs, oo = qtb.qtb_observables(ctx, 0), sim.observe()
        for k in (1, 2, 3, 4, 17):
            assert obs[k] == pytest.approx(oo[k], rel=1e-11)
    finally:
        qtb.qtb_destroy(ctx)
