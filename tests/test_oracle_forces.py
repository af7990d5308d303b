"""Pins of the oracle's pair forces (the grad V of Eqs. 4 and 8).

Checked against: central finite differences of the energy, Newton's third law,
the symmetry of the ideal crystal, the rock-salt Madelung constant, the
strain derivative of the energy (virial) and the periodic-image invariance of
a replicated supercell (the multi-image case r_c > L/2).
"""
import numpy as np
import pytest
from scipy.special import erfc

from golden_values import units, values
from paper_1905_02521_gb300 import workloads as W

MADELUNG_ROCKSALT = values("lattice_sums.txt")["madelung_rocksalt"]   # Borwein, Borwein & Taylor 1985
KE = units()["k_e"]                                                   # CODATA 2018


@pytest.fixture(scope="module")
def mgo():
    return W.mgo_potential()


@pytest.mark.parametrize("ncell", [2, 3])
def test_forces_are_minus_energy_gradient(oracle, mgo, ncell):
    pos, t, box = W.rocksalt(ncell, 4.21, sigma=0.05, seed=11)
    f, e, _ = oracle.pair_forces(pos, t, box, mgo)
    rng = np.random.default_rng(3)
    h = 1e-5
    frms = np.sqrt((f ** 2).mean())
    for _ in range(12):
        i, c = rng.integers(len(pos)), rng.integers(3)
        xp, xm = pos.copy(), pos.copy()
        xp[i, c] += h
        xm[i, c] -= h
        dE = (oracle.pair_forces(xp, t, box, mgo)[1] - oracle.pair_forces(xm, t, box, mgo)[1]) / (2 * h)
        assert -dE == pytest.approx(f[i, c], abs=2e-6 * frms)


def test_newton_third_law_and_ideal_lattice(oracle, mgo):
    pos, t, box = W.rocksalt(3, 4.21, sigma=0.05, seed=5)
    f, _, _ = oracle.pair_forces(pos, t, box, mgo)
    assert np.abs(f.sum(0)).max() < 1e-10
    pos0, t0, box0 = W.rocksalt(3, 4.21, sigma=0.0)
    f0, _, _ = oracle.pair_forces(pos0, t0, box0, mgo)
    assert np.abs(f0).max() < 1e-10


@pytest.mark.parametrize("alpha,rc,ncell,tol", [(0.3, 12.0, 6, 2e-5), (0.2, 8.0, 4, 0.03)])
def test_dsf_coulomb_reproduces_madelung(oracle, mgo, alpha, rc, ncell, tol):
    # DSF energy plus its constant self term -(erfc(a rc)/(2 rc) + a/sqrt(pi)) sum q^2
    pos, t, box = W.rocksalt(ncell, 4.21, sigma=0.0)
    p = dict(mgo, buck_A=np.zeros((2, 2)), buck_C=np.zeros((2, 2)), dsf_alpha=alpha, r_cut=rc)
    _, e, _ = oracle.pair_forces(pos, t, box, p)
    N = len(pos)
    e_self = -(erfc(alpha * rc) / (2 * rc) + alpha / np.sqrt(np.pi)) * KE * 4.0 * N
    r0 = 4.21 / 2
    M = -(e + e_self) / (N / 2) / (KE * 4.0 / r0)
    assert M == pytest.approx(MADELUNG_ROCKSALT, rel=tol)


def test_virial_is_strain_derivative(oracle, mgo):
    pos, t, box = W.rocksalt(3, 4.21, sigma=0.05, seed=8)
    _, _, vir = oracle.pair_forces(pos, t, box, mgo)
    assert np.allclose(vir, vir.T, atol=1e-9)
    eps = 1e-6
    for a in range(3):
        s = np.ones(3)
        s[a] = 1 + eps
        ep = oracle.pair_forces(pos * s, t, box * s, mgo)[1]
        s[a] = 1 - eps
        em = oracle.pair_forces(pos * s, t, box * s, mgo)[1]
        assert vir[a, a] == pytest.approx(-(ep - em) / (2 * eps), rel=1e-6, abs=1e-6)


def test_multi_image_cell_equals_replicated_supercell(oracle, mgo):
    # 2x2x2 MgO has L = 8.42 A < 2 r_c: every atom sees several images of each
    # neighbour.  The 2x2x2x(2^3) replica of the same configuration is the same
    # infinite crystal, so forces and energy per atom must agree.
    pos, t, box = W.rocksalt(2, 4.21, sigma=0.05, seed=21)
    f, e, vir = oracle.pair_forces(pos, t, box, mgo)
    shifts = np.array([[i, j, k] for i in range(2) for j in range(2) for k in range(2)]) * box
    big = np.concatenate([pos + s for s in shifts])
    bt = np.concatenate([t] * 8)
    fb, eb, vb = oracle.pair_forces(big, bt, 2 * box, mgo)
    assert eb / len(big) == pytest.approx(e / len(pos), rel=1e-12)
    for r in range(8):
        assert np.allclose(fb[r * len(pos):(r + 1) * len(pos)], f, atol=1e-11)
    assert np.allclose(vb / 8, vir, atol=1e-9)
    # sampled-atom mode equals the full evaluation
    fs, _, _ = oracle.pair_forces(pos, t, box, mgo, sel=[3, 17, 40])
    assert np.allclose(fs, f[[3, 17, 40]], atol=0, rtol=0)
