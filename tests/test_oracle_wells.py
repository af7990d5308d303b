"""Pins of the exact 1-D thermal reference (oracle/wells.py).

* harmonic potential: E_n = hbar w (n + 1/2); <E> = theta(w, T) of Eq. 1 and
  <x^2> = theta/(m w^2) at low and high temperature;
* the double well's averages are converged in the grid (4000 vs 8000 points);
* at high temperature the double well tends to the classical averages, at low
  temperature its energy lies well above the classical one (zero point);
* the double well of the study (V0 = 0.1 eV, a = 0.5 A, m = 1.008 u) has its
  ground state below the barrier, and its anharmonicity parameter of Eq. 13,
  hbar^2/(2 m V0 a^2) = 0.083, lies below the double-well critical value the
  paper prints in Sec. 3 (tests/golden/paper_values.txt): weakly anharmonic.
"""
import numpy as np
import pytest

from golden_values import values
from oracle import spectra as S
from oracle import wells as Wl

M, W0 = 1.008, 0.1


def test_harmonic_levels_and_theta():
    E, _ = Wl.levels(Wl.harmonic(M, W0), M, 2.5, npts=6000, nlev=20)
    n = np.arange(20)
    assert np.allclose(E, S.HBAR * W0 * (n + 0.5), rtol=2e-5)
    for T in (50.0, 300.0, 1000.0):
        e, x2 = Wl.thermal(Wl.harmonic(M, W0), M, T, 3.0, npts=6000, nlev=80)
        th = float(S.theta(W0, T))
        assert e == pytest.approx(th, rel=3e-5)
        assert x2 == pytest.approx(th / (M * Wl.MVV2E * W0 ** 2), rel=3e-5)


def test_double_well_grid_converged():
    V = Wl.double_well(0.1, 0.5)
    a = Wl.thermal(V, M, 100.0, 1.6, npts=4000)
    b = Wl.thermal(V, M, 100.0, 1.6, npts=8000)
    assert a[0] == pytest.approx(b[0], rel=1e-5) and a[1] == pytest.approx(b[1], rel=1e-5)


def test_double_well_limits():
    V = Wl.double_well(0.1, 0.5)
    hot = Wl.thermal(V, M, 3000.0, 2.0, npts=6000, nlev=200)
    hot_c = Wl.classical(V, M, 3000.0, 2.0)
    assert hot[0] == pytest.approx(hot_c[0], rel=0.03) and hot[1] == pytest.approx(hot_c[1], rel=0.03)
    hv = Wl.thermal(V, M, 3000.0, 2.0, npts=6000, nlev=200, with_v=True)[2]
    assert hv == pytest.approx(hot_c[2], rel=0.05)
    cold = Wl.thermal(V, M, 50.0, 1.6, with_v=True)
    cold_c = Wl.classical(V, M, 50.0, 1.6)
    assert cold[0] > cold_c[0] + 0.03            # zero-point energy ~ hbar w_min / 2 ~ 0.06 eV
    # <E> = <K> + <V> with <K> > 0 and V >= 0
    assert 0.0 < cold[2] < cold[0]
    E, _ = Wl.levels(V, M, 1.6)
    assert E[0] < 0.1                             # ground state below the barrier
    C = S.HBAR ** 2 / (2 * M * Wl.MVV2E * 0.1 * 0.25)   # Eq. 13 with V0 = 0.1 eV, d = a = 0.5 A
    assert C == pytest.approx(0.083, abs=0.002)
    assert C < values("paper_values.txt")["C_crit_double_well"]
