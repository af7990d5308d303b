"""The oracle's physical constants against CODATA 2018 (tests/golden/codata2018_si.txt).

The unit system of the method is eV, A, fs, u, e, K: hbar (Eq. 1), k_B (Eqs. 1, 3),
the kinetic-energy factor u A^2/fs^2 -> eV and the Coulomb constant of the pair
potential follow from the SI values.  A mistyped digit in any of the oracle's
copies (Python modules and the C half) fails here: the C half is read through
what it computes (ring-polymer frequencies, kinetic energy, Coulomb energy).
"""
import numpy as np
import pytest

from golden_values import units
from oracle import lattice as L
from oracle import spectra as S
from oracle import wells as Wl

U = units()
REL = 1e-10   # the oracle carries 10-12 significant digits


def test_python_constants():
    assert S.HBAR == pytest.approx(U["hbar"], rel=REL)
    assert S.KB == pytest.approx(U["k_B"], rel=REL)
    assert L.MVV2E == pytest.approx(U["mvv2e"], rel=REL)
    assert Wl.MVV2E == pytest.approx(U["mvv2e"], rel=REL)


@pytest.mark.parametrize("P,T", [(4, 50.0), (32, 300.0)])
def test_c_ring_polymer_frequencies(oracle, P, T):
    # free ring-polymer frequencies 2 w_P sin(k pi / P), w_P = sqrt(P) k_B T / hbar (Eqs. 3, 11)
    wP = np.sqrt(P) * U["k_B"] * T / U["hbar"]
    expect = np.sort(2 * wP * np.sin(np.arange(P) * np.pi / P))
    assert np.allclose(np.sort(oracle.nm_freqs(P, T)), expect, rtol=REL, atol=0)


def test_c_kinetic_energy_and_coulomb(oracle):
    # two unlike ions 3 A apart, Coulomb only with a plain 1/r inside r_cut (alpha = 0):
    # the energy is k_e q_i q_j (1/r - 1/r_c + (r - r_c)/r_c^2), the kinetic energy sum m v^2 / 2
    pot = {"mass": np.array([24.305, 15.999]), "charge": np.array([2.0, -2.0]),
           "buck_A": np.zeros((2, 2)), "buck_rho": np.ones((2, 2)), "buck_C": np.zeros((2, 2)),
           "dsf_alpha": 0.0, "r_cut": 8.0}
    box = np.array([40.0, 40.0, 40.0])
    x = np.array([[[10.0, 10.0, 10.0], [13.0, 10.0, 10.0]]])
    v = np.array([[[0.01, -0.02, 0.005], [-0.003, 0.004, 0.02]]])
    types = np.array([0, 1], np.int32)
    sim = oracle.Sim(x, v, types, pot, box, 300.0, 0.0, 1.0, seed=1)
    rec = sim.observe()
    K = 0.5 * U["mvv2e"] * (pot["mass"][:, None] * v[0] ** 2).sum()
    r, rc = 3.0, 8.0
    V = U["k_e"] * (-4.0) * (1 / r - 1 / rc + (r - rc) / rc ** 2)
    assert rec[1] == pytest.approx(K, rel=REL)
    assert rec[2] == pytest.approx(V, rel=REL)
