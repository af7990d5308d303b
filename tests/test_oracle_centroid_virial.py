"""Pins of the oracle's centroid-virial kinetic estimators (record slots 18, 19).

The paper gives only the primitive estimator (Eq. 5); the ring polymer of
Eqs. 3-4 also admits the centroid-virial form
    K_cv = 3N k_B T/2 + (1/2) sum_s sum_i (r_i,s - rbar_i) . grad_i V(r_s)/P,
and, for a bath that does not hold the centroid at k_B T (QTB-PIMD, Eq. 12),
K_cv,0 = the same virial term plus the centroid-mode kinetic energy
K_0 = sum_i m_i P |vbar_i|^2/2.  Pinned here against what does not go through
the estimator's own formula:

* one bead: K_cv is the equipartition value and K_cv,0 the kinetic energy;
* the virial term is half the derivative of the bead-averaged potential
  (1/P) sum_s V(rbar + lam (r_s - rbar)) at lam = 1 (central differences of
  the oracle's energies), in a periodic crystal with a bead moved by a box
  vector (minimum image);
* harmonic beads: the virial term is (m w^2/2P) sum (r - rbar)^2 from the
  positions alone; equal bead velocities give K_0 = K, opposite ones K_0 = 0.
"""
import numpy as np
import pytest

from paper_1905_02521_gb300 import workloads as W

KB, MVV2E = 8.617333262e-5, 103.64269652680505


def _sim(oracle, pos, vel, sysd, pot, T=300.0, **kw):
    return oracle.Sim(pos, vel, sysd["types"], pot, sysd.get("box"), T, 0.0, 1.0, seed=1, **kw)


def test_one_bead_is_equipartition_and_kinetic_energy(oracle):
    sysd, pot = W.mgo_system(2, T=300.0)
    rec = _sim(oracle, sysd["pos"], sysd["vel"], sysd, pot).observe()
    N = sysd["pos"].shape[1]
    assert rec[18] == pytest.approx(1.5 * N * KB * 300.0, rel=1e-14)
    assert rec[19] == pytest.approx(rec[1], rel=1e-14)


def test_virial_term_is_the_scaling_derivative_of_the_bead_potential(oracle):
    sysd, pot = W.mgo_system(2, T=300.0, n_beads=4)
    rng = np.random.default_rng(5)
    pos = sysd["pos"] + rng.normal(0, 0.05, sysd["pos"].shape)
    box = np.asarray(sysd["box"], np.float64)
    cen = pos.mean(0)
    # bead 2 of atom 3 one box vector away: the same physical ring polymer
    moved = pos.copy()
    moved[2, 3] += box * np.array([1.0, -1.0, 0.0])
    rec = _sim(oracle, moved, None, sysd, pot).observe()
    N = pos.shape[1]
    term = rec[18] - 1.5 * N * KB * 300.0
    h = 1e-4
    Vp = _sim(oracle, cen + (1 + h) * (pos - cen), None, sysd, pot).observe()[2]
    Vm = _sim(oracle, cen + (1 - h) * (pos - cen), None, sysd, pot).observe()[2]
    dV = (Vp - Vm) / (2 * h)
    assert abs(term) > 0.05                      # a non-trivial configuration
    assert term == pytest.approx(0.5 * dV, rel=1e-6)
    assert rec[19] == pytest.approx(term, rel=1e-12)   # no velocities: K_0 = 0


def test_harmonic_beads_closed_forms(oracle):
    w0, m, P, N, T = 0.1, 1.008, 4, 20, 100.0
    sysd, pot = W.oscillators(N, T, 0.0, n_beads=P, mass=m)
    rng = np.random.default_rng(6)
    pos = rng.normal(0, 0.2, (P, N, 3))
    v1 = rng.normal(0, 0.01, (1, N, 3))
    kw = dict(potential=oracle.POT_HARMONIC, ext={"omega": w0})
    same = _sim(oracle, pos, np.repeat(v1, P, 0), sysd, pot, T=T, **kw).observe()
    opp = _sim(oracle, pos, np.concatenate([v1, -v1, v1, -v1]), sysd, pot, T=T, **kw).observe()
    term = 0.5 * m * MVV2E * w0 ** 2 / P * ((pos - pos.mean(0)) ** 2).sum()
    assert same[18] == pytest.approx(1.5 * N * KB * T + term, rel=1e-12)
    assert same[19] == pytest.approx(same[1] + term, rel=1e-12)
    assert opp[19] == pytest.approx(term, rel=1e-12)
    assert opp[18] == pytest.approx(same[18], rel=1e-14)
