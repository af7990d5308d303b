"""Pins of the harmonic-lattice reference (oracle/lattice.py).

* the finite-difference Hessian of harmonic oscillators (the oracle's own
  external-potential forces) gives every mode at w0: units and mass weighting;
* 64-ion MgO at the perfect rock-salt sites: forces vanish, the Hessian is
  symmetric, the three translations are zero modes (acoustic sum rule), all
  other modes are real;
* an independent route to one optical mode: the force constant of a rigid
  displacement of the cation sublattice against the anion sublattice gives
  w^2 = k (1/m_Mg + 1/m_O), which must be an eigenvalue;
* the Langevin kinetic-energy density integrates to k_B T/2 per mode for a
  white bath whatever gamma (equipartition), and to theta(w_m)/2 as gamma -> 0
  for the quantum density S = theta (Eq. 1);
* harmonic_energy: zero-point limit and classical limit.
"""
import numpy as np
import pytest

from oracle import lattice as L
from oracle import spectra as S
from paper_1905_02521_gb300 import workloads as W

KB, MVV2E, HBAR = 8.617333262e-5, 103.64269652680505, 0.6582119569


@pytest.fixture(scope="module")
def mgo(oracle):
    pot = W.mgo_potential()
    x, t, box = W.rocksalt(2, 4.21, 0.0)
    H = L.hessian(lambda y: oracle.pair_forces(y, t, box, pot)[0], x)
    return pot, x, t, box, H


def test_harmonic_oscillators_give_w0(oracle):
    w0, m = 0.08, 1.008
    s, pot = W.oscillators(5, 100.0, 0.0, mass=m, spread=0.3)
    sim = oracle.Sim(s["pos"], None, s["types"], pot, None, 100.0, 0.0, 1.0, seed=1,
                     potential=oracle.POT_HARMONIC, ext={"omega": w0})

    def forces(y):
        sim.set_state(y[None], np.zeros((1,) + y.shape), 0)
        return sim.state()[2][0]
    H = L.hessian(forces, s["pos"][0])
    w, _ = L.modes(H, pot["mass"][s["types"]])
    assert np.allclose(w, w0, rtol=1e-8)


def test_mgo_hessian_structure(oracle, mgo):
    pot, x, t, box, H = mgo
    f, _, _ = oracle.pair_forces(x, t, box, pot)
    assert np.abs(f).max() < 1e-10
    assert np.abs(H - H.T).max() < 1e-9 * np.abs(H).max()
    w, U = L.modes(H, pot["mass"][t])
    assert np.all(np.abs(w[:3]) < 1e-5) and np.all(w[3:] > 0.04)
    # the translations: H times a uniform displacement vanishes
    for c in range(3):
        u = np.zeros_like(x)
        u[:, c] = 1.0
        assert np.abs(H @ u.reshape(-1)).max() < 1e-8 * np.abs(H).max()


def test_rigid_sublattice_mode_is_an_eigenvalue(oracle, mgo):
    pot, x, t, box, H = mgo
    w, _ = L.modes(H, pot["mass"][t])
    cat = t == 0
    h = 1e-4

    def fcat(u):
        y = x.copy()
        y[cat, 0] += u
        return oracle.pair_forces(y, t, box, pot)[0][cat, 0].sum()
    k = -(fcat(h) - fcat(-h)) / (2 * h) / cat.sum()      # eV/A^2 per cation
    mu = 1.0 / (1.0 / pot["mass"][0] + 1.0 / pot["mass"][1])
    wt = np.sqrt(k / (mu * MVV2E))
    assert np.abs(w - wt).min() < 1e-6 * wt
    assert 0.05 < wt < 0.2


def test_langevin_density_normalisation():
    T, wm = 150.0, 0.1
    kT = KB * T
    for gamma in (0.002, 0.02, 0.1):
        e = L.mode_kinetic_energy(wm, gamma, lambda om: np.full_like(om, kT), 60.0, npts=600001)
        # the exact integral to infinity is k_B T/2; the tail beyond 60 is gamma k_B T/(pi 60)
        assert e == pytest.approx(0.5 * kT - gamma * kT / (np.pi * 60.0), rel=2e-4)
    e = L.mode_kinetic_energy(wm, 1e-4, lambda om: S.theta(om, T), 0.5, npts=600001)
    assert e == pytest.approx(0.5 * float(S.theta(wm, T)), rel=2e-3)


def test_harmonic_energy_limits():
    w = np.array([0.0, 0.0, 0.0, 0.05, 0.1, 0.15])
    zp = -1.0 + 0.5 * HBAR * w.sum() + 1.5 * KB * 1e-3      # zero point + free translations
    assert L.harmonic_energy(-1.0, w, 1e-3) == pytest.approx(zp, rel=1e-12)
    hot = L.harmonic_energy(-1.0, w, 1e5)
    assert hot == pytest.approx(-1.0 + 3 * KB * 1e5 + 1.5 * KB * 1e5, rel=1e-4)
