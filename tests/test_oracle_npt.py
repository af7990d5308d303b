"""Pins of the oracle's isothermal-isobaric (Langevin barostat) integrator.

Sec. 2.1 of the paper runs its isothermal-isobaric simulations with Quigley and
Probert's Langevin extension of the constant-pressure equations (refs [11, 12])
and prints no equations; the oracle integrates the isotropic
Martyna-Tobias-Klein equations with Langevin friction and noise on the particles
and on the cell (qtb_oracle.c).  What fixes it independently of its own code:

* the ideal gas: the isothermal-isobaric law P(V) ~ V^N exp(-P V / k_B T) gives
  <V> = (N + 1) k_B T / P and var(V) / <V>^2 = 1 / (N + 1) exactly (a dropped
  kinetic term or alpha = 1 instead of 1 + 3/N_f shifts <V> by 1/(N + 1));
* the pressure: the virial trace / 3V of the perfect lattice is -dE/dV of its
  static energy (finite differences of the oracle's own energies);
* the harmonic crystal: at low T the volume fluctuates with
  var(V) = k_B T V / B, B = V d^2E/dV^2 at the static minimum, around that
  minimum;
* a frozen cell (infinite cell mass) reduces the step to the constant-volume
  BAOAB step.

Ring polymers (P > 1), whose cell acts on the centroid modes:

* the ideal gas again: the internal modes do not feel the cell, so the
  volume law is the classical one, <V> = (N + 1) k_B T / P;
* the centroid virial W_cv (record slot 22) is -dPhi/dlog(lam) of the bead-
  averaged energy when the centroids scale with the cell and the bead offsets
  stay fixed (finite differences of the oracle's own energies);
* a frozen cell reduces the step to the constant-volume ring-polymer step.
"""
import numpy as np
import pytest

from paper_1905_02521_gb300 import workloads as W

KB = 8.617333262e-5


def _block_sem(x, nb=40):
    b = np.asarray(x)[: len(x) // nb * nb].reshape(nb, -1).mean(1)
    return b.std(ddof=1) / np.sqrt(nb)


def _ideal_gas(oracle, N=8, T=300.0, m=40.0, gamma_e=0.01, nsteps=400000):
    kT = KB * T
    P = (N + 1) * kT / 1000.0
    pot = {"mass": np.array([m]), "charge": np.zeros(1), "buck_A": np.zeros((1, 1)),
           "buck_rho": np.ones((1, 1)), "buck_C": np.zeros((1, 1)), "dsf_alpha": 0.2, "r_cut": 1.0}
    rng = np.random.default_rng(3)
    L = 10.0
    pos = rng.uniform(0, L, (1, N, 3))
    vel = rng.normal(0, np.sqrt(kT / (m * W.MVV2E)), (1, N, 3))
    Wm = 9 * (N + 1) * kT / (2 * np.pi / 200.0) ** 2   # cell period ~200 fs
    sim = oracle.Sim(pos, vel, np.zeros(N, np.int32), pot, np.array([L] * 3), T, 0.01, 1.0, seed=5,
                     npt={"pressure": P, "mass": Wm, "gamma": gamma_e})
    sim.step(5000, record=False)
    rec = sim.step(nsteps)
    return rec, (N + 1) * kT / P, N


def test_ideal_gas_volume_distribution(oracle):
    rec, Vexact, N = _ideal_gas(oracle)
    V = rec[:, 20]
    sem = _block_sem(V)
    assert abs(V.mean() - Vexact) < 3 * sem, (V.mean(), Vexact, sem)
    assert V.var() / V.mean() ** 2 == pytest.approx(1.0 / (N + 1), rel=0.08)
    # the particles stay canonical at T
    assert rec[:, 1].mean() == pytest.approx(1.5 * N * KB * 300.0, rel=0.02)


def _lattice(a):
    return W.rocksalt(1, a, sigma=0.0)


def test_virial_pressure_is_minus_dE_dV(oracle):
    # lattice constants with no neighbour shell within the finite-difference step
    # of r_cut = 8 A (the energy-shifted Buckingham term has a small force step
    # there, so a shell crossing it would spoil the derivative)
    pot = W.mgo_potential()
    for a in (4.05, 4.128, 4.3):
        k = np.arange(1, 400)
        assert np.min(np.abs(0.5 * a * np.sqrt(k) - 8.0)) > 4e-3
        pos, types, box = _lattice(a)
        _, e, vir = oracle.pair_forces(pos, types, box, pot)
        V = a ** 3
        h = 1e-5 * a

        def E(aa):
            p, t, b = _lattice(aa)
            return oracle.pair_forces(p, t, b, pot)[1]
        dEdV = (E(a + h) - E(a - h)) / ((a + h) ** 3 - (a - h) ** 3)
        assert np.trace(vir) / (3 * V) == pytest.approx(-dEdV, rel=1e-6, abs=1e-8)


@pytest.mark.slow
def test_crystal_volume_fluctuations_match_bulk_modulus(oracle):
    from scipy.optimize import minimize_scalar
    pot = W.mgo_potential()

    def E(a):
        p, t, b = _lattice(a)
        return oracle.pair_forces(p, t, b, pot)[1]
    a0 = minimize_scalar(E, bracket=(4.1, 4.13, 4.16), tol=1e-10).x
    V0 = a0 ** 3
    h = 1e-3 * V0
    EV = lambda V: E(V ** (1.0 / 3.0))  # noqa: E731
    B = V0 * (EV(V0 + h) - 2 * EV(V0) + EV(V0 - h)) / h ** 2
    T = 20.0
    pos, types, box = _lattice(a0)
    vel = W.maxwell_boltzmann(pot["mass"][types], T, 7)
    Wm = 9 * B * V0 / (2 * np.pi / 200.0) ** 2
    sim = oracle.Sim(pos[None], vel, types, pot, box, T, 0.01, 1.0, seed=9,
                     npt={"pressure": 0.0, "mass": Wm, "gamma": 0.01})
    sim.step(2000, record=False)
    V = sim.step(60000)[:, 20]
    assert V.mean() == pytest.approx(V0, rel=2e-3)
    assert V.var() / (KB * T * V0 / B) == pytest.approx(1.0, abs=0.2)


def test_frozen_cell_reduces_to_constant_volume_step(oracle):
    pot = W.mgo_potential()
    pos, types, box = W.rocksalt(1, 4.128, sigma=0.03, seed=11)
    vel = W.maxwell_boltzmann(pot["mass"][types], 300.0, 4)
    a = oracle.Sim(pos[None], vel, types, pot, box, 300.0, 0.01, 1.0, seed=3)
    b = oracle.Sim(pos[None], vel, types, pot, box, 300.0, 0.01, 1.0, seed=3,
                   npt={"pressure": 0.0, "mass": 1e300, "gamma": 0.01})
    a.step(50, record=False)
    b.step(50, record=False)
    xa, va, _, _ = a.state()
    xb, vb, _, _ = b.state()
    assert np.abs(xa - xb).max() < 1e-12 and np.abs(va - vb).max() < 1e-12
    assert np.allclose(b.cell()[0], box, rtol=1e-14)


def _ideal_gas_rp(oracle, N=8, P=4, T=300.0, m=40.0, nsteps=300000):
    kT = KB * T
    Pext = (N + 1) * kT / 1000.0
    pot = {"mass": np.array([m]), "charge": np.zeros(1), "buck_A": np.zeros((1, 1)),
           "buck_rho": np.ones((1, 1)), "buck_C": np.zeros((1, 1)), "dsf_alpha": 0.2, "r_cut": 1.0}
    rng = np.random.default_rng(8)
    L = 10.0
    pos = np.repeat(rng.uniform(0, L, (1, N, 3)), P, axis=0) + rng.normal(0, 0.01, (P, N, 3))
    vel = rng.normal(0, np.sqrt(kT / (m * W.MVV2E)), (P, N, 3))
    Wm = 9 * (N + 1) * kT / (2 * np.pi / 200.0) ** 2
    sim = oracle.Sim(pos, vel, np.zeros(N, np.int32), pot, np.array([L] * 3), T, 0.01, 1.0, seed=15,
                     npt={"pressure": Pext, "mass": Wm, "gamma": 0.01})
    sim.step(5000, record=False)
    rec = sim.step(nsteps)
    return rec, (N + 1) * kT / Pext, N


def test_ring_polymer_ideal_gas_volume_distribution(oracle):
    rec, Vexact, N = _ideal_gas_rp(oracle)
    V = rec[:, 20]
    sem = _block_sem(V)
    assert abs(V.mean() - Vexact) < 3 * sem, (V.mean(), Vexact, sem)
    assert V.var() / V.mean() ** 2 == pytest.approx(1.0 / (N + 1), rel=0.1)
    # the centroid modes stay canonical at T (3N/2 k_B T), the centroid virial is 0
    assert rec[:, 21].mean() == pytest.approx(1.5 * N * KB * 300.0, rel=0.03)
    assert np.abs(rec[:, 22]).max() == 0.0


@pytest.mark.parametrize("P", [1, 3])
def test_centroid_virial_is_minus_dPhi_dlog_lam(oracle, P):
    pot = W.mgo_potential()
    a = 4.2
    pos, types, box = W.rocksalt(1, a, sigma=0.05, seed=31)
    rng = np.random.default_rng(5)
    off = rng.normal(0, 0.04, (P, len(types), 3))
    off -= off.mean(0)                                   # offsets about the centroid
    beads = pos[None] + off

    def phi(lam):
        return sum(oracle.pair_forces(lam * pos + off[b], types, lam * box, pot)[1] for b in range(P)) / P

    # the lattice constant keeps every neighbour shell away from r_cut over the step
    k = np.arange(1, 400)
    assert np.min(np.abs(0.5 * a * np.sqrt(k) - 8.0)) > 0.05
    h = 1e-5
    dphi = (phi(1 + h) - phi(1 - h)) / (2 * h)
    sim = oracle.Sim(beads, None, types, pot, box, 300.0, 0.01, 1.0, seed=1)
    rec = sim.observe()
    assert rec[22] == pytest.approx(-dphi, rel=1e-6, abs=1e-7)
    if P == 1:
        assert rec[22] == rec[5] + rec[9] + rec[13]
    else:
        assert abs(rec[22] - (rec[5] + rec[9] + rec[13])) > 1e-3   # the offsets matter


def test_ring_polymer_frozen_cell_reduces_to_constant_volume_step(oracle):
    pot = W.mgo_potential()
    pos, types, box = W.rocksalt(1, 4.128, sigma=0.03, seed=12)
    P = 4
    rng = np.random.default_rng(2)
    beads = pos[None] + rng.normal(0, 0.03, (P, len(types), 3))
    vel = W.maxwell_boltzmann(pot["mass"][types], 300.0, 6, n_beads=P)
    a = oracle.Sim(beads, vel, types, pot, box, 300.0, 0.01, 0.5, seed=9)
    b = oracle.Sim(beads, vel, types, pot, box, 300.0, 0.01, 0.5, seed=9,
                   npt={"pressure": 0.0, "mass": 1e300, "gamma": 0.01})
    a.step(40, record=False)
    b.step(40, record=False)
    xa, va, _, _ = a.state()
    xb, vb, _, _ = b.state()
    assert np.abs(xa - xb).max() < 1e-11 and np.abs(va - vb).max() < 1e-11
    assert np.allclose(b.cell()[0], box, rtol=1e-14)
