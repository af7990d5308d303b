"""Physics pins of the oracle's integrator: what the paper fixes about the dynamics.

* thermostat off (gamma = 0): energy conservation, time reversibility and
  momentum conservation of the Langevin/BAOAB integrator (Eq. 8 without bath,
  Eq. 4 for the ring polymer);
* white bath on harmonic oscillators at a large step: the stationary covariance
  of the B A O A B splitting, solved exactly as a discrete Lyapunov equation,
  for one bead and per normal mode of a ring polymer (exact free rotation);
* QTB on harmonic oscillators reproduces theta(w0, T) of Eq. 1 up to the
  friction correction, computed independently by quadrature of the Langevin
  response with the filter's own spectral density (Eqs. 6-8);
* PIMD on harmonic oscillators reproduces the finite-P closed form of the
  primitive estimator (Eqs. 3, 5, 11);
* QTB-PIMD on harmonic oscillators gives the bead-averaged <x^2> = theta/(m w^2)
  that Eq. 10 demands, again with the friction correction by quadrature;
* the centroid-virial kinetic estimators (slots 18, 19) match the same closed
  forms: E_P/2 for PIMD, and for QTB-PIMD the centroid-mode estimator gives the
  quantum theta/2 while the classical-centroid one does not.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import spectra as S
from paper_1905_02521_gb300 import workloads as W

HBAR, KB, MVV2E = 0.6582119569, 8.617333262e-5, 103.64269652680505


def _block_sigma(x, nblk=20):
    b = np.array_split(np.asarray(x), nblk)
    m = np.array([bb.mean() for bb in b])
    return m.std(ddof=1) / np.sqrt(nblk)


def test_nve_conservation_and_reversibility(oracle):
    sysd, pot = W.mgo_system(2, T=300.0, gamma=0.0)
    sim = oracle.Sim(sysd["pos"], sysd["vel"], sysd["types"], pot, sysd["box"], 300.0, 0.0, 1.0, seed=1)
    rec0 = sim.observe()
    rec = sim.step(400)
    E = rec[:, 1] + rec[:, 2]
    E0 = rec0[1] + rec0[2]
    assert np.abs(E - E0).max() < 2e-3 * rec0[1]
    assert np.abs(rec[:, 14:17] - rec0[14:17]).max() < 1e-10
    # reverse the velocities and integrate back to the start
    x, v, f, st = sim.state()
    sim.set_state(x, -v, st)
    sim.step(400, record=False)
    xb, vb, _, _ = sim.state()
    assert np.abs(xb - sysd["pos"]).max() < 1e-7
    assert np.abs(vb + sysd["vel"]).max() < 1e-9


def test_ring_polymer_nve_conserves_effective_hamiltonian(oracle):
    sysd, pot = W.mgo_system(2, T=300.0, gamma=0.0, n_beads=4)
    rng = np.random.default_rng(2)
    pos = sysd["pos"] + rng.normal(0, 0.01, sysd["pos"].shape)
    sim = oracle.Sim(pos, sysd["vel"], sysd["types"], pot, sysd["box"], 300.0, 0.0, 0.5, seed=1)
    r0 = sim.observe()
    rec = sim.step(300)
    H = rec[:, 1] + rec[:, 3] + rec[:, 2]
    assert np.abs(H - (r0[1] + r0[3] + r0[2])).max() < 2e-3 * r0[1]


@pytest.mark.slow
def test_baoab_harmonic_stationary_covariance(oracle):
    # White bath at omega dt = 0.5, far from the continuous-time limit.  One step
    # B A O A B is a linear map of (x, v) plus Gaussian noise injected at O, so its
    # stationary covariance solves a discrete Lyapunov equation.  For this splitting
    # it is k_B T/(m w^2) in x at any stable step (Leimkuhler & Matthews 2013) and
    # (k_B T/m)(1 - (w dt/2)^2) in v at the full step; another order of the same
    # steps (A B O B A: 1/(1 - (w dt/2)^2)) or a wrong noise amplitude misses it by
    # percents, against a statistical error of ~0.2 % here.
    from scipy.linalg import solve_discrete_lyapunov
    w0, T, gamma, dt, m = 0.1, 300.0, 0.02, 5.0, 1.008
    mk, kT = m * MVV2E, KB * T
    c = np.exp(-gamma * dt)
    Bk = np.array([[1.0, 0.0], [-0.5 * dt * w0 ** 2, 1.0]])
    Ad = np.array([[1.0, 0.5 * dt], [0.0, 1.0]])
    Ou = np.array([[1.0, 0.0], [0.0, c]])
    M = Bk @ Ad @ Ou @ Ad @ Bk
    n = Bk @ Ad @ np.array([0.0, np.sqrt((1.0 - c * c) * kT / mk)])
    cov = solve_discrete_lyapunov(M, np.outer(n, n))
    assert cov[0, 0] == pytest.approx(kT / (mk * w0 ** 2), rel=1e-12)
    assert cov[1, 1] == pytest.approx(kT / mk * (1.0 - (0.5 * w0 * dt) ** 2), rel=1e-12)
    sysd, pot = W.oscillators(100, T, gamma, mass=m)           # 300 independent oscillators
    sim = oracle.Sim(sysd["pos"], sysd["vel"], sysd["types"], pot, None, T, gamma, dt, seed=11,
                     potential=oracle.POT_HARMONIC, ext={"omega": w0})
    sim.step(500, record=False)
    rec = sim.step(20000)
    K, V = rec[:, 1] / 300.0, rec[:, 2] / 300.0                # per oscillator
    assert abs(K.mean() - 0.5 * mk * cov[1, 1]) < 4 * _block_sigma(K)
    assert abs(V.mean() - 0.5 * mk * w0 ** 2 * cov[0, 0]) < 4 * _block_sigma(V)
    assert K.mean() < 0.5 * kT * 0.97                          # the splitting's kinetic bias is resolved


def _rp_mode_covariances(w0, P, T, gamma, dt, m, wk):
    """Stationary (q, v) covariance of each ring-polymer normal mode under one step
    B(dt/2) A(dt/2) O(dt) A(dt/2) B(dt/2): B kicks with the external force
    -(m w0^2/P) q (Eq. 4), A is the exact free rotation at w_k (Eq. 11), O the white
    bath at k_B T; the noise enters at O."""
    from scipy.linalg import solve_discrete_lyapunov
    mk, kT, c = m * MVV2E, KB * T, np.exp(-gamma * dt)
    out = []
    for w in wk:
        Bk = np.array([[1.0, 0.0], [-0.5 * dt * w0 ** 2 / P, 1.0]])
        if w == 0.0:
            Ar = np.array([[1.0, 0.5 * dt], [0.0, 1.0]])
        else:
            cs, sn = np.cos(0.5 * dt * w), np.sin(0.5 * dt * w)
            Ar = np.array([[cs, sn / w], [-w * sn, cs]])
        Ou = np.array([[1.0, 0.0], [0.0, c]])
        n = Bk @ Ar @ np.array([0.0, np.sqrt((1.0 - c * c) * kT / mk)])
        out.append(solve_discrete_lyapunov(Bk @ Ar @ Ou @ Ar @ Bk, np.outer(n, n)))
    return out


@pytest.mark.slow
def test_ring_polymer_baoab_stationary_covariance(oracle):
    # P = 4 ring polymers in a harmonic well at beta hbar w0 = 3 with a 5 fs step:
    # every normal mode is a linear system, so the exact stationary averages of the
    # discrete scheme follow from one Lyapunov solve per mode.  The bead-averaged
    # <x^2>, the kinetic energy and the spring energy of the oracle's trajectory must
    # match them; a drift in place of the exact free rotation, a missing 1/P on the
    # external force or a mode transform that is not orthogonal would not.
    w0, gamma, dt, m, P = 0.1, 0.02, 5.0, 1.008, 4
    T = HBAR * w0 / (3.0 * KB)
    mk, kT = m * MVV2E, KB * T
    wP = np.sqrt(P) * KB * T / HBAR
    wk = 2 * wP * np.sin(np.arange(P) * np.pi / P)
    # the construction itself: at a small step the continuous-time ring polymer
    for w, cov in zip(wk, _rp_mode_covariances(w0, P, T, gamma, 0.01, m, wk)):
        assert cov[0, 0] == pytest.approx(kT / (mk * (w0 ** 2 / P + w ** 2)), rel=1e-4)
        assert cov[1, 1] == pytest.approx(kT / mk, rel=1e-4)
    covs = _rp_mode_covariances(w0, P, T, gamma, dt, m, wk)
    x2_ex = np.mean([cv[0, 0] for cv in covs])                      # (1/P) sum_k <q_k^2>
    K_ex = 0.5 * mk * sum(cv[1, 1] for cv in covs)
    spring_ex = 0.5 * mk * sum(w * w * cv[0, 0] for w, cv in zip(wk, covs))
    sysd, pot = W.oscillators(100, T, gamma, n_beads=P, mass=m)
    sim = oracle.Sim(sysd["pos"], sysd["vel"], sysd["types"], pot, None, T, gamma, dt, seed=17,
                     potential=oracle.POT_HARMONIC, ext={"omega": w0})
    sim.step(1000, record=False)
    rec = sim.step(20000)
    for q, ex in ((17, x2_ex), (1, K_ex), (3, spring_ex)):
        y = rec[:, q] / 300.0                                         # per 1-D oscillator
        assert abs(y.mean() - ex) < 4 * _block_sigma(y), (q, y.mean(), ex)
    # the step is large enough for the discrete scheme to differ from the continuous
    # limit (kinetic energy P k_B T/2 per oscillator) by more than the tolerance above
    y = rec[:, 1] / 300.0
    assert P * kT / 2 - K_ex > 4 * _block_sigma(y) + abs(y.mean() - K_ex)


def _quad_x2_v2(wgrid_S, w0, gamma, m, wmax):
    """<x^2>, <v^2> of a Langevin oscillator driven by noise of density 2 m gamma S(w)."""
    def resp(w):
        return 2 * gamma / (m * MVV2E * ((w0 ** 2 - w ** 2) ** 2 + (gamma * w) ** 2)) / np.pi
    pts = [w0]
    x2 = integrate.quad(lambda w: resp(w) * wgrid_S(w), 0, wmax, points=pts, limit=2000)[0]
    v2 = integrate.quad(lambda w: resp(w) * w * w * wgrid_S(w), 0, wmax, points=pts, limit=2000)[0]
    return x2, v2


def _filter_density(h, dt):
    k = np.arange(1, len(h))
    return lambda w: (h[0] + 2 * np.cos(w * dt * k) @ h[1:]) ** 2


@pytest.mark.slow
def test_qtb_harmonic_oscillator_energy(oracle):
    w0, T, gamma, dt, L, m = 0.1, 100.0, 0.01, 0.5, 513, 1.008
    h = S.taps(L, dt, T, 0.5)
    sysd, pot = W.oscillators(100, T, gamma, mass=m)
    sim = oracle.Sim(sysd["pos"], sysd["vel"], sysd["types"], pot, None, T, gamma, dt, seed=7, taps=h,
                     potential=oracle.POT_HARMONIC, ext={"omega": w0})
    sim.step(2000, record=False)
    rec = sim.step(20000)
    E = (rec[:, 1] + rec[:, 2]) / 300.0
    x2, v2 = _quad_x2_v2(_filter_density(h, dt), w0, gamma, m, np.pi / dt)
    E_q = 0.5 * m * MVV2E * (v2 + w0 ** 2 * x2)
    sig = _block_sigma(E)
    assert abs(E.mean() - E_q) < 4 * sig + 5e-3 * E_q
    # and the friction-free target of Eq. 1 is close (gamma/w0 = 0.1)
    assert E_q == pytest.approx(S.theta(w0, T), rel=0.03)
    # quantum, not classical: theta is ~4x k_B T here
    assert E.mean() > 3 * KB * T


@pytest.mark.slow
def test_pimd_harmonic_primitive_energy_closed_form(oracle):
    w0, gamma, dt, m = 0.1, 0.01, 0.5, 1.008
    T = HBAR * w0 / (3.0 * KB)                       # beta hbar w0 = 3
    for P in (1, 4):
        sysd, pot = W.oscillators(100, T, gamma, n_beads=P, mass=m)
        sim = oracle.Sim(sysd["pos"], sysd["vel"], sysd["types"], pot, None, T, gamma, dt, seed=11,
                         potential=oracle.POT_HARMONIC, ext={"omega": w0})
        sim.step(3000, record=False)
        rec = sim.step(20000)
        E = rec[:, 4] / 300.0
        k = np.arange(P)
        E_P = KB * T * np.sum(1.0 / (1.0 + (2 * P / 3.0) ** 2 * np.sin(k * np.pi / P) ** 2))
        sig = _block_sigma(E)
        assert abs(E.mean() - E_P) < 4 * sig + 3e-3 * E_P, (P, E.mean(), E_P, sig)
        # centroid-virial estimators: <K_cv> = <V> = E_P/2 for a harmonic potential,
        # with a variance that, unlike the primitive one, does not grow with P
        for q in (18, 19):
            Ecv = (rec[:, q] + rec[:, 2]) / 300.0
            assert abs(Ecv.mean() - E_P) < 4 * _block_sigma(Ecv) + 3e-3 * E_P, (P, q, Ecv.mean(), E_P)
        if P > 1:
            assert rec[:, 18].std() < 0.5 * (rec[:, 4] - rec[:, 2]).std()


@pytest.mark.slow
def test_qtb_pimd_harmonic_position_variance(oracle):
    w0, T, gamma, dt, L, m, P = 0.1, 100.0, 0.01, 0.5, 513, 1.008, 4
    sol = S.kappa_solve(P)
    h = S.taps(L, dt, T, 0.5, P=P, sol=sol)
    sysd, pot = W.oscillators(50, T, gamma, n_beads=P, mass=m)
    sim = oracle.Sim(sysd["pos"], sysd["vel"], sysd["types"], pot, None, T, gamma, dt, seed=13, taps=h,
                     potential=oracle.POT_HARMONIC, ext={"omega": w0})
    sim.step(2000, record=False)
    rec = sim.step(16000)
    x2 = rec[:, 17] / 150.0                          # bead-averaged <x^2> per 1-D oscillator
    dens = _filter_density(h, dt)
    wk = oracle.nm_freqs(P, T)
    q2 = [_quad_x2_v2(dens, np.sqrt(w0 ** 2 / P + wk[k] ** 2), gamma, m, np.pi / dt)[0] for k in range(P)]
    x2_q = np.mean(q2)
    sig = _block_sigma(x2)
    assert abs(x2.mean() - x2_q) < 4 * sig + 5e-3 * x2_q
    # Eq. 10: without friction the bead average is the quantum theta/(m w0^2)
    assert x2_q == pytest.approx(S.theta(w0, T) / (m * MVV2E * w0 ** 2), rel=0.05)
    # kinetic energy per oscillator: the centroid-mode kinetic energy plus the
    # virial term (m w0^2/2P) sum_{k>0} <q_k^2>, each mode by quadrature; without
    # friction theta/2.  The classical-centroid K_cv (k_B T/2 for the centroid)
    # misses the centroid's quantum part.
    v2_0 = _quad_x2_v2(dens, w0 / np.sqrt(P), gamma, m, np.pi / dt)[1]
    vir = 0.5 * m * MVV2E * w0 ** 2 / P * np.sum(q2[1:])
    K_q = 0.5 * m * MVV2E * v2_0 + vir
    Kcv0 = rec[:, 19] / 150.0
    assert abs(Kcv0.mean() - K_q) < 4 * _block_sigma(Kcv0) + 5e-3 * K_q
    assert K_q == pytest.approx(0.5 * S.theta(w0, T), rel=0.05)
    Kcv = rec[:, 18] / 150.0
    assert abs(Kcv.mean() - (0.5 * KB * T + vir)) < 4 * _block_sigma(Kcv) + 5e-3 * K_q
    assert Kcv.mean() < 0.9 * K_q
