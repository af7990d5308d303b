"""Isothermal-isobaric runs on the GPU (the Langevin barostat of qtb_params.npt;
Sec. 2.1 of the paper, refs [11, 12]) against the FP64 oracle and the
isothermal-isobaric law.

* FP64 form: positions, velocities, forces and cell after every one of the
  first 100 steps equal the oracle's (1e-11), with a QTB bath and a cell that
  contracts visibly over those steps;
* mixed form: one step from the GPU's own state and cell against the oracle's
  FP64 step (positions and cell 1e-5, velocities 1e-5 norm-wise);
* the ideal gas samples P(V) ~ V^N exp(-P V / k_B T): <V> = (N + 1) k_B T / P;
* a cold crystal's volume fluctuations give its bulk modulus: var(V) = k_B T V / B;
* ring polymers (the cell on the centroid modes): the FP64 form against the
  oracle after each of 60 QTB-PIMD steps, one mixed step against the oracle's,
  the ideal gas's volume law with P = 4 beads;
* LiH / LiD under QTB-MD and classical Langevin at zero pressure: the lattice
  parameter against temperature (Figs. 2 and 6 of the paper, with the synthetic
  potential): classically the two isotopes share one curve that grows with T;
  with the quantum bath the zero-point motion expands the lighter crystal more
  (LiH above LiD) and both lie above the classical curve at low T.
"""
import numpy as np
import pytest

from helpers import gpu_ctx, minimg, oracle_sim, rel_inf

from oracle import spectra as S
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


def _cell_mass(B, V, period):
    """Cell mass giving a volume oscillation of the given period (fs) for bulk modulus B."""
    return 9.0 * B * V / (2 * np.pi / period) ** 2


# static bulk modulus of the MgO model at its E(V) minimum (tests/test_oracle_npt.py): ~2.56 eV/A^3
B_MGO = 2.56


def test_fp64_npt_trajectory_matches_oracle(qtb, oracle):
    # 64-ion MgO at 300 K from the 4.21 A lattice, zero pressure: the model's static
    # minimum is at 4.128 A, so the cell contracts over the first steps; QTB bath,
    # 513 taps; cell period ~200 fs
    s, pot = W.mgo_system(2, 300.0, gamma=2e-3)
    N = len(s["types"])
    V = np.prod(s["box"])
    npt = {"pressure": 0.0, "mass": _cell_mass(B_MGO, V, 200.0), "gamma": 5e-3}
    taps = S.taps(513, 1.0, 300.0, 0.3)
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=0, seed=4321, npt=npt)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 513, 0.3)
        sim = oracle_sim(oracle, s, pot, 1.0, seed=4321, taps=taps, npt=npt)
        for step in range(1, 101):
            qtb.qtb_step_n(ctx, 1)
            sim.step(1, record=False)
            box_g, pe_g = qtb.qtb_get_cell(ctx, 0)
            box_o, pe_o = sim.cell()
            assert np.abs(box_g / box_o - 1).max() < 1e-12, (step, box_g, box_o)
            assert pe_g == pytest.approx(pe_o, rel=1e-10, abs=1e-10 * abs(pe_o) + 1e-12)
            xg, vg = qtb.qtb_get_state(ctx, 0, 1, N)
            fg = qtb.qtb_get_forces(ctx, 0, 1, N)
            xo, vo, fo, _ = sim.state()
            assert np.abs(minimg(xg - xo, box_o)).max() < 1e-10
            assert rel_inf(vg, vo) < 1e-11 and rel_inf(fg, fo) < 1e-11
        assert box_o[0] < 0.995 * s["box"][0]        # the cell did move
        obs = qtb.qtb_observables(ctx, 0)
        assert obs[20] == pytest.approx(np.prod(box_o), rel=1e-12)
    finally:
        qtb.qtb_destroy(ctx)


def test_fp64_npt_fused_steps_match_oracle(qtb, oracle):
    # 300 steps in one call (a CUDA-graph block of 256 and 44 direct steps): every
    # step but the last of a call updates the cell inside the step kernel and
    # runs the next step's first half there; the oracle steps one at a time
    s, pot = W.mgo_system(2, 300.0, gamma=2e-3)
    N = len(s["types"])
    npt = {"pressure": 0.001, "mass": _cell_mass(B_MGO, np.prod(s["box"]), 200.0), "gamma": 5e-3}
    taps = S.taps(513, 1.0, 300.0, 0.3)
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=0, seed=4242, npt=npt)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 513, 0.3)
        sim = oracle_sim(oracle, s, pot, 1.0, seed=4242, taps=taps, npt=npt)
        qtb.qtb_step_n(ctx, 300)
        sim.step(300, record=False)
        box_g, pe_g = qtb.qtb_get_cell(ctx, 0)
        box_o, pe_o = sim.cell()
        assert np.abs(box_g / box_o - 1).max() < 1e-11
        assert pe_g == pytest.approx(pe_o, rel=1e-9, abs=1e-12)
        xg, vg = qtb.qtb_get_state(ctx, 0, 1, N)
        xo, vo, _, _ = sim.state()
        assert np.abs(minimg(xg - xo, box_o)).max() < 1e-9 and rel_inf(vg, vo) < 1e-9
        assert abs(box_o[0] / s["box"][0] - 1) > 2e-3   # the cell did move
    finally:
        qtb.qtb_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_fused_npt_steps_equal_single_steps(qtb, precision):
    # the fused step (cell update and the next step's first half in the step
    # kernel) does the arithmetic of the cell kernel and integrator launches that
    # single-step calls make: the two runs agree bit for bit, lists rebuilt alike
    s, pot = W.lih_system(3, 50.0, gamma=1e-3)
    N = len(s["types"])
    npt = {"pressure": 0.0, "mass": _cell_mass(1.0, np.prod(s["box"]), 300.0), "gamma": 4e-3}
    out = []
    for calls in ([300], [1] * 300):
        ctx = gpu_ctx(qtb, [s], pot, 0.25, precision=precision, filter_prec=1, seed=8, npt=npt)
        try:
            qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 1025, 0.6)
            for n in calls:
                qtb.qtb_step_n(ctx, n)
            out.append((qtb.qtb_get_state(ctx, 0, 1, N), qtb.qtb_get_cell(ctx, 0), qtb.qtb_list_rebuilds(ctx)))
        finally:
            qtb.qtb_destroy(ctx)
    (xa, va), (ba, pa), ra = out[0]
    (xb, vb), (bb, pb), rb = out[1]
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(ba, bb) and pa == pb
    assert ra == rb and ra > 0


def test_mixed_npt_single_step_matches_oracle_step(qtb, oracle):
    s, pot = W.mgo_system(2, 300.0, gamma=2e-3)
    N = len(s["types"])
    V = np.prod(s["box"])
    npt = {"pressure": 0.0, "mass": _cell_mass(B_MGO, V, 200.0), "gamma": 5e-3}
    taps = S.taps(513, 1.0, 300.0, 0.3)
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=1, filter_prec=1, seed=99, npt=npt)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 513, 0.3)
        qtb.qtb_step_n(ctx, 37)
        x0, v0 = qtb.qtb_get_state(ctx, 0, 1, N)
        box0, pe0 = qtb.qtb_get_cell(ctx, 0)
        sim = oracle_sim(oracle, s, pot, 1.0, seed=99, taps=taps, npt=npt)
        sim.set_cell(box0, pe0, 1)
        sim.set_state(x0, v0, 37)
        qtb.qtb_step_n(ctx, 1)
        sim.step(1, record=False)
        x1, v1 = qtb.qtb_get_state(ctx, 0, 1, N)
        box1, _ = qtb.qtb_get_cell(ctx, 0)
        xo, vo, _, _ = sim.state()
        boxo, _ = sim.cell()
        assert np.abs(box1 / boxo - 1).max() < 1e-5
        assert np.abs(minimg(x1 - xo, boxo)).max() < 1e-5
        assert rel_inf(v1, vo) < 1e-5
    finally:
        qtb.qtb_destroy(ctx)


def _unwrap_beads(x, box):
    """Beads of each atom in bead 0's image (the GPU wraps each bead into the box)."""
    return x[:1] + minimg(x - x[:1], box)


@pytest.mark.parametrize("P", [4, 8])
def test_fp64_npt_pimd_trajectory_matches_oracle(qtb, oracle, P):
    # 64-ion MgO ring polymers at 300 K from the 4.21 A lattice, zero pressure,
    # QTB-PIMD (kappa_P taps of the solver, 513 taps), FP64 form against the
    # oracle after each step: the cell acts on the centroids, the integrator's
    # internal modes keep their physical length, the centroid kernel ends the
    # closing kick of the centroid with the cell's friction
    s, pot = W.mgo_system(2, 300.0, gamma=2e-3, n_beads=P, seed=91)
    rng = np.random.default_rng(4)
    s["pos"] = s["pos"] + rng.normal(0, 0.02, s["pos"].shape)
    N = len(s["types"])
    npt = {"pressure": 0.0, "mass": _cell_mass(B_MGO, np.prod(s["box"]), 200.0), "gamma": 5e-3}
    taps = S.taps(513, 1.0, 300.0, 0.3, P=P, sol=S.kappa_solve(P))
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=0, seed=515, npt=npt)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB_PIMD, 513, 0.3)
        sim = oracle_sim(oracle, s, pot, 1.0, seed=515, taps=taps, npt=npt)
        for step in range(1, 61):
            qtb.qtb_step_n(ctx, 1)
            sim.step(1, record=False)
            box_g, pe_g = qtb.qtb_get_cell(ctx, 0)
            box_o, pe_o = sim.cell()
            assert np.abs(box_g / box_o - 1).max() < 1e-12, (step, box_g, box_o)
            assert pe_g == pytest.approx(pe_o, rel=1e-9, abs=1e-12)
            xg, vg = qtb.qtb_get_state(ctx, 0, P, N)
            fg = qtb.qtb_get_forces(ctx, 0, P, N)
            xo, vo, fo, _ = sim.state()
            assert np.abs(minimg(xg - xo, box_o)).max() < 1e-10, step
            assert rel_inf(vg, vo) < 1e-10 and rel_inf(fg, fo) < 1e-10, step
        obs, oo = qtb.qtb_observables(ctx, 0), sim.observe()
        for k in (1, 2, 3, 4, 14, 15, 16, 18, 19, 20, 21, 22):
            assert obs[k] == pytest.approx(oo[k], rel=1e-9, abs=1e-9), k
        assert box_o[0] < 0.997 * s["box"][0]        # the cell did move
    finally:
        qtb.qtb_destroy(ctx)


def test_mixed_npt_pimd_single_step_matches_oracle_step(qtb, oracle):
    P = 8
    s, pot = W.mgo_system(2, 300.0, gamma=2e-3, n_beads=P, seed=92)
    N = len(s["types"])
    npt = {"pressure": 0.0, "mass": _cell_mass(B_MGO, np.prod(s["box"]), 200.0), "gamma": 5e-3}
    taps = S.taps(513, 1.0, 300.0, 0.3, P=P, sol=S.kappa_solve(P))
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=1, filter_prec=1, seed=77, npt=npt)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB_PIMD, 513, 0.3)
        qtb.qtb_step_n(ctx, 37)
        x0, v0 = qtb.qtb_get_state(ctx, 0, P, N)
        box0, pe0 = qtb.qtb_get_cell(ctx, 0)
        sim = oracle_sim(oracle, s, pot, 1.0, seed=77, taps=taps, npt=npt)
        sim.set_cell(box0, pe0, 1)
        sim.set_state(_unwrap_beads(x0, box0), v0, 37)
        qtb.qtb_step_n(ctx, 1)
        sim.step(1, record=False)
        x1, v1 = qtb.qtb_get_state(ctx, 0, P, N)
        box1, _ = qtb.qtb_get_cell(ctx, 0)
        xo, vo, _, _ = sim.state()
        boxo, _ = sim.cell()
        assert np.abs(box1 / boxo - 1).max() < 1e-5
        assert np.abs(minimg(x1 - xo, boxo)).max() < 1e-5
        assert rel_inf(v1, vo) < 1e-5
    finally:
        qtb.qtb_destroy(ctx)


def test_ring_polymer_ideal_gas_volume_on_gpu(qtb):
    # 256 non-interacting ring polymers of 4 beads at 300 K (mixed form): the
    # internal modes do not feel the cell, so <V> = (N + 1) k_B T / P_ext again
    N, Pb, T, m = 256, 4, 300.0, 40.0
    kT = KB * T
    V_exact = 10000.0
    Pext = (N + 1) * kT / V_exact
    pot = {"mass": np.array([m]), "charge": np.zeros(1), "buck_A": np.zeros((1, 1)),
           "buck_rho": np.ones((1, 1)), "buck_C": np.zeros((1, 1)), "dsf_alpha": 0.2, "r_cut": 1.0}
    rng = np.random.default_rng(9)
    L = V_exact ** (1 / 3)
    pos = np.repeat(rng.uniform(0, L, (1, N, 3)), Pb, axis=0) + rng.normal(0, 0.01, (Pb, N, 3))
    s = {"pos": pos, "vel": rng.normal(0, np.sqrt(kT / (m * W.MVV2E)), (Pb, N, 3)),
         "types": np.zeros(N, np.int32), "box": np.array([L] * 3), "T": T, "gamma": 0.01}
    npt = {"pressure": Pext, "mass": 9 * (N + 1) * kT / (2 * np.pi / 400.0) ** 2, "gamma": 0.005}
    ctx = gpu_ctx(qtb, [s], pot, 2.0, precision=1, seed=19, npt=npt, obs_stride=16, max_records=16384)
    try:
        qtb.qtb_step_n(ctx, 8192)
        qtb.qtb_step_n(ctx, 16 * 12288)
        ser = qtb.qtb_get_series(ctx, 0, 12288)
    finally:
        qtb.qtb_destroy(ctx)
    V = ser[:, 20]
    nb = 24
    sem = V[: len(V) // nb * nb].reshape(nb, -1).mean(1).std(ddof=1) / np.sqrt(nb)
    print(f"ring-polymer ideal gas: <V> {V.mean():.1f} +- {sem:.1f}, exact {V_exact:.1f}; "
          f"var/<V>^2 {V.var() / V.mean()**2:.5f} exact {1 / (N + 1):.5f}")
    assert abs(V.mean() - V_exact) < 3 * sem + 1e-3 * V_exact
    assert V.var() / V.mean() ** 2 == pytest.approx(1 / (N + 1), rel=0.15)
    assert ser[:, 21].mean() == pytest.approx(1.5 * N * kT, rel=0.03)   # centroids at k_B T


def test_ideal_gas_volume_on_gpu(qtb):
    # 512 non-interacting particles (zero pair tables) at 300 K: <V> = (N + 1) k_B T / P
    # (volume fluctuations of 4 %: the cell stays far above 0.9 of its edges)
    N, T, m = 512, 300.0, 40.0
    kT = KB * T
    V_exact = 20000.0
    P = (N + 1) * kT / V_exact
    pot = {"mass": np.array([m]), "charge": np.zeros(1), "buck_A": np.zeros((1, 1)),
           "buck_rho": np.ones((1, 1)), "buck_C": np.zeros((1, 1)), "dsf_alpha": 0.2, "r_cut": 1.0}
    rng = np.random.default_rng(8)
    L = V_exact ** (1 / 3)
    s = {"pos": rng.uniform(0, L, (1, N, 3)), "vel": rng.normal(0, np.sqrt(kT / (m * W.MVV2E)), (1, N, 3)),
         "types": np.zeros(N, np.int32), "box": np.array([L] * 3), "T": T, "gamma": 0.01}
    npt = {"pressure": P, "mass": 9 * (N + 1) * kT / (2 * np.pi / 400.0) ** 2, "gamma": 0.005}
    ctx = gpu_ctx(qtb, [s], pot, 2.0, precision=1, seed=17, npt=npt, obs_stride=16, max_records=16384)
    try:
        qtb.qtb_step_n(ctx, 8192)
        qtb.qtb_step_n(ctx, 16 * 12288)
        V = qtb.qtb_get_series(ctx, 0, 12288)[:, 20]
    finally:
        qtb.qtb_destroy(ctx)
    nb = 24
    sem = V[: len(V) // nb * nb].reshape(nb, -1).mean(1).std(ddof=1) / np.sqrt(nb)
    print(f"ideal gas: <V> {V.mean():.1f} +- {sem:.1f}, exact {V_exact:.1f}; var/<V>^2 {V.var() / V.mean()**2:.5f} "
          f"exact {1 / (N + 1):.5f}")
    assert abs(V.mean() - V_exact) < 3 * sem + 1e-3 * V_exact
    assert V.var() / V.mean() ** 2 == pytest.approx(1 / (N + 1), rel=0.15)


def _lattice_parameter(qtb, isotope, T, quantum, ncell=3, steps=24576, neq=8192, P=1):
    s, pot = W.lih_system(ncell, T, gamma=2e-3, isotope=isotope, seed=31, n_beads=P)
    V = np.prod(s["box"])
    npt = {"pressure": 0.0, "mass": _cell_mass(1.0, V, 300.0), "gamma": 4e-3}
    ctx = gpu_ctx(qtb, [s], pot, 0.25, precision=1, filter_prec=1, seed=23, npt=npt, obs_stride=16,
                  max_records=4096)
    try:
        if quantum:
            qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB if P == 1 else qtb.NOISE_QTB_PIMD, 2049, 0.6)
        qtb.qtb_step_n(ctx, neq)
        qtb.qtb_step_n(ctx, steps)
        V = qtb.qtb_get_series(ctx, 0, steps // 16)[:, 20]
    finally:
        qtb.qtb_destroy(ctx)
    a = (V / ncell ** 3) ** (1 / 3)
    nb = 16
    sem = a[: len(a) // nb * nb].reshape(nb, -1).mean(1).std(ddof=1) / np.sqrt(nb)
    return a.mean(), sem


def test_lih_lid_lattice_parameter_against_temperature(qtb):
    res = {}
    for T in (20.0, 150.0, 300.0):
        for iso in ("H", "D"):
            for q in (False, True):
                res[(T, iso, q)] = _lattice_parameter(qtb, iso, T, q)
    for T in (20.0, 150.0, 300.0):
        print("T %5.0f K: classical LiH %.5f(%.0e) LiD %.5f(%.0e) | QTB LiH %.5f(%.0e) LiD %.5f(%.0e)" % (
            T, *res[(T, "H", False)], *res[(T, "D", False)], *res[(T, "H", True)], *res[(T, "D", True)]))
    sig = lambda *k: np.sqrt(sum(res[x][1] ** 2 for x in k))  # noqa: E731
    # classical: no isotope effect; thermal expansion
    for T in (20.0, 150.0, 300.0):
        d = res[(T, "H", False)][0] - res[(T, "D", False)][0]
        assert abs(d) < 4 * sig((T, "H", False), (T, "D", False)) + 2e-5
    assert res[(300.0, "H", False)][0] > res[(20.0, "H", False)][0]
    # quantum bath: zero-point expansion, larger for the lighter isotope
    for T in (20.0, 150.0):
        assert res[(T, "H", True)][0] - res[(T, "D", True)][0] > 4 * sig((T, "H", True), (T, "D", True))
        assert res[(T, "D", True)][0] - res[(T, "D", False)][0] > 4 * sig((T, "D", True), (T, "D", False))
    # at low T the quantum lattice parameter saturates: it moves less from 20 to 150 K
    # than the classical one does
    dq = res[(150.0, "H", True)][0] - res[(20.0, "H", True)][0]
    dc = res[(150.0, "H", False)][0] - res[(20.0, "H", False)][0]
    assert dq < dc


def test_lih_lattice_parameter_qtb_pimd_converges_faster_than_pimd(qtb):
    # LiH 3^3 at zero pressure (the comparison of Figs. 2 and 6 of the paper,
    # with the synthetic potential): PIMD with 32 beads is the converged
    # quantum lattice parameter at 150 and 300 K; QTB-PIMD with 8 beads lands
    # on it where PIMD with 8 beads has not yet converged (150 K), and QTB-MD
    # alone overestimates the expansion (zero-point energy leaking into the
    # anharmonic modes)
    res = {}
    for T in (150.0, 300.0):
        for key, P, q in (("qtb_md", 1, True), ("qtb_pimd8", 8, True), ("pimd8", 8, False), ("pimd32", 32, False)):
            res[(T, key)] = _lattice_parameter(qtb, "H", T, q, P=P)
    res[(150.0, "pimd32_D")] = _lattice_parameter(qtb, "D", 150.0, False, P=32)
    for k, (a, e) in sorted(res.items()):
        print(f"T {k[0]:5.0f} K {k[1]:10s} a = {a:.5f} +- {e:.5f}")
    sig = lambda *k: np.sqrt(sum(res[x][1] ** 2 for x in k))  # noqa: E731
    for T in (150.0, 300.0):
        ref = res[(T, "pimd32")][0]
        assert abs(res[(T, "qtb_pimd8")][0] - ref) < 4 * sig((T, "qtb_pimd8"), (T, "pimd32"))
        assert res[(T, "qtb_md")][0] - ref > 4 * sig((T, "qtb_md"), (T, "pimd32"))
    assert abs(res[(300.0, "pimd8")][0] - res[(300.0, "pimd32")][0]) < 4 * sig((300.0, "pimd8"), (300.0, "pimd32"))
    assert abs(res[(150.0, "qtb_pimd8")][0] - res[(150.0, "pimd32")][0]) < \
        abs(res[(150.0, "pimd8")][0] - res[(150.0, "pimd32")][0])
    assert res[(150.0, "pimd32")][0] - res[(150.0, "pimd32_D")][0] > 4 * sig((150.0, "pimd32"), (150.0, "pimd32_D"))


def test_crystal_volume_fluctuations_match_bulk_modulus_on_gpu(qtb, oracle):
    # 216-ion MgO at 20 K (white bath, zero pressure, mixed form): the volume
    # fluctuates about the static minimum with var(V) = k_B T V / B, B = V d^2E/dV^2
    # of the perfect lattice from the oracle's own energies (the compressibility
    # of the harmonic crystal, which the cell equations must reproduce)
    from scipy.optimize import minimize_scalar
    pot = W.mgo_potential()

    def E(a):
        p, t, b = W.rocksalt(1, a, sigma=0.0)
        return oracle.pair_forces(p, t, b, pot)[1]
    a0 = minimize_scalar(E, bracket=(4.1, 4.13, 4.16), tol=1e-10).x
    h = 1e-3 * a0 ** 3
    EV = lambda V: E(V ** (1.0 / 3.0))  # noqa: E731
    B = a0 ** 3 * (EV(a0 ** 3 + h) - 2 * EV(a0 ** 3) + EV(a0 ** 3 - h)) / h ** 2
    T = 20.0
    s, _ = W.mgo_system(3, T, gamma=1e-2, sigma=0.0, seed=5)
    s["pos"] = W.rocksalt(3, a0, sigma=0.0)[0][None]
    s["box"] = np.array([3 * a0] * 3)
    V0 = np.prod(s["box"])
    npt = {"pressure": 0.0, "mass": _cell_mass(B, V0, 200.0), "gamma": 0.01}
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=1, seed=13, npt=npt, obs_stride=16, max_records=8192)
    try:
        qtb.qtb_step_n(ctx, 4096)
        qtb.qtb_step_n(ctx, 16 * 6144)
        V = qtb.qtb_get_series(ctx, 0, 6144)[:, 20]
    finally:
        qtb.qtb_destroy(ctx)
    ratio = V.var() / (KB * T * V0 / B)
    print(f"B = {B:.3f} eV/A^3, <V>/V0 - 1 = {V.mean() / V0 - 1:.2e}, var(V) / (k_B T V / B) = {ratio:.3f}")
    assert V.mean() == pytest.approx(V0, rel=2e-3)
    assert ratio == pytest.approx(1.0, abs=0.2)


def test_constant_volume_cell_and_volume_slot(qtb):
    # without the barostat the cell is the given one, its momentum 0, and record
    # slot 20 the constant volume
    s, pot = W.mgo_system(2, 300.0)
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=1)
    try:
        qtb.qtb_step_n(ctx, 10)
        box, pe = qtb.qtb_get_cell(ctx, 0)
        assert np.array_equal(box, s["box"]) and pe == 0.0
        assert qtb.qtb_observables(ctx, 0)[20] == pytest.approx(np.prod(s["box"]), rel=1e-15)
    finally:
        qtb.qtb_destroy(ctx)


def test_collapsing_cell_is_reported(qtb):
    # a pressure far beyond the crystal's bulk modulus drives the cell below 0.9 of
    # its edges, the margin its cell lists are built for: the run must stop with an
    # error (the cell bit, or the overflow or non-finite check it triggers), not go
    # on with missing pairs
    s, pot = W.mgo_system(2, 300.0, gamma=2e-3)
    V = np.prod(s["box"])
    npt = {"pressure": 50.0, "mass": _cell_mass(B_MGO, V, 100.0), "gamma": 1e-3}
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=1, npt=npt)
    try:
        with pytest.raises(qtb.QtbError) as e:
            for _ in range(40):
                qtb.qtb_step_n(ctx, 50)
                qtb.qtb_sync(ctx)
        assert e.value.code in (qtb.ERR_STATE, qtb.ERR_OVERFLOW, qtb.ERR_NONFINITE)
    finally:
        qtb.qtb_destroy(ctx)


def test_npt_arguments_are_checked(qtb):
    s1, pot = W.mgo_system(2, 300.0)
    with pytest.raises(qtb.QtbError) as e:   # the cell needs a mass
        gpu_ctx(qtb, [s1], pot, 1.0, npt={"pressure": 0.0, "mass": 0.0, "gamma": 1e-3})
    assert e.value.code == qtb.ERR_ARG


def test_set_cell_then_state_continues_like_the_oracle(qtb, oracle):
    # a cell and state set mid-run (edges 0.4 % larger, another cell momentum): the
    # positions scale with the cell, and the FP64 run from there follows the oracle
    # started from the same cell, state and step for 40 steps
    s, pot = W.mgo_system(2, 300.0, gamma=2e-3)
    N = len(s["types"])
    npt = {"pressure": 0.002, "mass": _cell_mass(B_MGO, np.prod(s["box"]), 200.0), "gamma": 5e-3}
    taps = S.taps(513, 1.0, 300.0, 0.3)
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=0, seed=77, npt=npt)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 513, 0.3)
        qtb.qtb_step_n(ctx, 30)
        x0, v0 = qtb.qtb_get_state(ctx, 0, 1, N)
        box0, pe0 = qtb.qtb_get_cell(ctx, 0)
        box1, pe1 = box0 * 1.004, -0.5 * pe0 + 0.01
        qtb.qtb_set_cell(ctx, 0, box1, pe1)
        box_g, pe_g = qtb.qtb_get_cell(ctx, 0)
        assert np.abs(box_g / box1 - 1).max() < 1e-15 and pe_g == pe1
        xs, vs = qtb.qtb_get_state(ctx, 0, 1, N)
        assert np.abs(minimg(xs - x0 * 1.004, box1)).max() < 1e-12 and np.array_equal(vs, v0)
        x1 = x0 * 1.004 + 0.01 * np.sin(np.arange(3 * N)).reshape(1, N, 3)
        qtb.qtb_set_state(ctx, 0, x1, v0)
        sim = oracle_sim(oracle, s, pot, 1.0, seed=77, taps=taps, npt=npt)
        sim.set_cell(box1, pe1, 1)
        sim.set_state(x1, v0, 30)
        for step in range(40):
            qtb.qtb_step_n(ctx, 1)
            sim.step(1, record=False)
            box_g, pe_g = qtb.qtb_get_cell(ctx, 0)
            box_o, pe_o = sim.cell()
            assert np.abs(box_g / box_o - 1).max() < 1e-12, (step, box_g, box_o)
            assert pe_g == pytest.approx(pe_o, rel=1e-10, abs=1e-12)
            xg, vg = qtb.qtb_get_state(ctx, 0, 1, N)
            xo, vo, _, _ = sim.state()
            assert np.abs(minimg(xg - xo, box_o)).max() < 1e-10 and rel_inf(vg, vo) < 1e-10
    finally:
        qtb.qtb_destroy(ctx)


def test_set_cell_arguments_are_checked(qtb):
    s, pot = W.mgo_system(2, 300.0)
    npt = {"pressure": 0.0, "mass": _cell_mass(B_MGO, np.prod(s["box"]), 200.0), "gamma": 5e-3}
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=1, npt=npt)
    try:
        box = np.asarray(s["box"], np.float64)
        for bad_box, bad_pe in ((box * [1.0, 1.0, 1.01], 0.0),   # anisotropic
                                (box * 0.85, 0.0),                # below the lists' margin
                                (box * np.nan, 0.0), (box, np.inf)):
            with pytest.raises(qtb.QtbError) as e:
                qtb.qtb_set_cell(ctx, 0, bad_box, bad_pe)
            assert e.value.code == qtb.ERR_ARG
        with pytest.raises(qtb.QtbError) as e:
            qtb.qtb_set_cell(ctx, 1, box, 0.0)
        assert e.value.code == qtb.ERR_ARG
        qtb.qtb_step_n(ctx, 5)    # the context is still usable
        qtb.qtb_sync(ctx)
    finally:
        qtb.qtb_destroy(ctx)
    c2 = gpu_ctx(qtb, [s], pot, 1.0, precision=1)
    try:
        with pytest.raises(qtb.QtbError) as e:   # constant volume
            qtb.qtb_set_cell(c2, 0, s["box"], 0.0)
        assert e.value.code == qtb.ERR_ARG
    finally:
        qtb.qtb_destroy(c2)


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_cells_match_single_runs(qtb, precision):
    # two crystals of different size and temperature in one isothermal-isobaric
    # context: each has its own cell (and its own rebuild schedule), so each runs bit
    # for bit as alone, where system k of a batch uses Philox key (seed, k)
    sa, pot = W.mgo_system(2, 150.0, gamma=2e-3, seed=51)
    sb, _ = W.mgo_system(3, 600.0, gamma=2e-3, seed=52)
    npt = {"pressure": 0.003, "mass": _cell_mass(B_MGO, np.prod(sb["box"]), 200.0), "gamma": 5e-3}
    ctx = gpu_ctx(qtb, [sa, sb], pot, 1.0, precision=precision, seed=5, npt=npt)
    try:
        qtb.qtb_set_filter(ctx, 1, qtb.NOISE_QTB, 513, 0.3)
        qtb.qtb_step_n(ctx, 300)
        batched = [(qtb.qtb_get_state(ctx, k, 1, len(s["types"]))[0], qtb.qtb_get_cell(ctx, k))
                   for k, s in enumerate((sa, sb))]
    finally:
        qtb.qtb_destroy(ctx)
    for k, s in enumerate((sa, sb)):
        c1 = gpu_ctx(qtb, [s], pot, 1.0, precision=precision, seed=5 ^ (k << 32), npt=npt)
        try:
            if k == 1:
                qtb.qtb_set_filter(c1, 0, qtb.NOISE_QTB, 513, 0.3)
            qtb.qtb_step_n(c1, 300)
            x = qtb.qtb_get_state(c1, 0, 1, len(s["types"]))[0]
            box, pe = qtb.qtb_get_cell(c1, 0)
            assert np.array_equal(x, batched[k][0])
            assert np.array_equal(box, batched[k][1][0]) and pe == batched[k][1][1]
        finally:
            qtb.qtb_destroy(c1)


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_ring_polymer_cells_match_single_runs(qtb, precision):
    # two ring-polymer crystals (P = 4 and 2) in one isothermal-isobaric context:
    # each system's record is reduced in groups of its own force units and its
    # centroid kernel CTAs are its own, so each runs bit for bit as alone
    sa, pot = W.mgo_system(2, 200.0, gamma=2e-3, seed=61, n_beads=4)
    sb, _ = W.mgo_system(3, 500.0, gamma=2e-3, seed=62, n_beads=2)
    npt = {"pressure": 0.002, "mass": _cell_mass(B_MGO, np.prod(sb["box"]), 200.0), "gamma": 5e-3}
    ctx = gpu_ctx(qtb, [sa, sb], pot, 1.0, precision=precision, seed=7, npt=npt)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB_PIMD, 513, 0.3)
        qtb.qtb_step_n(ctx, 300)
        batched = [(qtb.qtb_get_state(ctx, k, s["pos"].shape[0], len(s["types"])), qtb.qtb_get_cell(ctx, k))
                   for k, s in enumerate((sa, sb))]
    finally:
        qtb.qtb_destroy(ctx)
    for k, s in enumerate((sa, sb)):
        c1 = gpu_ctx(qtb, [s], pot, 1.0, precision=precision, seed=7 ^ (k << 32), npt=npt)
        try:
            if k == 0:
                qtb.qtb_set_filter(c1, 0, qtb.NOISE_QTB_PIMD, 513, 0.3)
            qtb.qtb_step_n(c1, 300)
            x, v = qtb.qtb_get_state(c1, 0, s["pos"].shape[0], len(s["types"]))
            box, pe = qtb.qtb_get_cell(c1, 0)
            assert np.array_equal(x, batched[k][0][0]) and np.array_equal(v, batched[k][0][1])
            assert np.array_equal(box, batched[k][1][0]) and pe == batched[k][1][1]
        finally:
            qtb.qtb_destroy(c1)


def test_ring_polymer_set_cell_then_state_continues_like_the_oracle(qtb, oracle):
    # P = 4 FP64: a cell and state set mid-run, then 30 steps against the oracle
    # started from the same cell, state and step (the internal modes rescale with
    # the cell from the set scale on)
    P = 4
    s, pot = W.mgo_system(2, 300.0, gamma=2e-3, n_beads=P, seed=93)
    N = len(s["types"])
    npt = {"pressure": 0.001, "mass": _cell_mass(B_MGO, np.prod(s["box"]), 200.0), "gamma": 5e-3}
    taps = S.taps(513, 1.0, 300.0, 0.3, P=P, sol=S.kappa_solve(P))
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=0, seed=31, npt=npt)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB_PIMD, 513, 0.3)
        qtb.qtb_step_n(ctx, 20)
        x0, v0 = qtb.qtb_get_state(ctx, 0, P, N)
        box0, pe0 = qtb.qtb_get_cell(ctx, 0)
        box1, pe1 = box0 * 0.997, 0.5 * pe0 - 0.02
        x1 = _unwrap_beads(x0, box0) * 0.997
        qtb.qtb_set_cell(ctx, 0, box1, pe1)
        qtb.qtb_set_state(ctx, 0, x1, v0)
        sim = oracle_sim(oracle, s, pot, 1.0, seed=31, taps=taps, npt=npt)
        sim.set_cell(box1, pe1, 1)
        sim.set_state(x1, v0, 20)
        for step in range(30):
            qtb.qtb_step_n(ctx, 1)
            sim.step(1, record=False)
            box_g, pe_g = qtb.qtb_get_cell(ctx, 0)
            box_o, pe_o = sim.cell()
            assert np.abs(box_g / box_o - 1).max() < 1e-12, (step, box_g, box_o)
            assert pe_g == pytest.approx(pe_o, rel=1e-9, abs=1e-12)
            xg, vg = qtb.qtb_get_state(ctx, 0, P, N)
            xo, vo, _, _ = sim.state()
            assert np.abs(minimg(xg - xo, box_o)).max() < 1e-10 and rel_inf(vg, vo) < 1e-10
    finally:
        qtb.qtb_destroy(ctx)
