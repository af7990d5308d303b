"""Pins of the Fourier-segment generator of the oracle (oracle/fourier.py, Eq. 9).

* the generator equals Eq. 9 written out as printed (direct summation, no FFT):
  R = sqrt(2 m gamma/dt) eta for the same normals;
* with a constant spectrum the map from the segment's normals to eta is
  orthogonal (every eta_t a unit-norm combination, distinct t orthogonal), so
  the white bath is recovered exactly, and Parseval holds sample by sample;
* the averaged periodogram of the generated noise reproduces S = theta W at
  every grid frequency (chi-square bands) and the variance is (1/n) sum_j S_j;
* consecutive segments are uncorrelated across their boundary, while inside a
  segment the lag-1 correlation is the one of S (the segment artefact).
"""
import numpy as np
import pytest

from oracle import fourier as F
from oracle import spectra as S


def test_generator_is_eq9_as_printed():
    n, dt, T, wmax = 64, 1.0, 300.0, 0.3
    m, gamma = 15.999, 1e-3
    Sj = F.segment_spectrum(n, dt, T, wmax)
    rng = np.random.default_rng(3)
    a, b = rng.normal(size=n // 2 + 1), rng.normal(size=n // 2 + 1)
    xi = np.zeros(n)
    xi[0], xi[1] = a[0], a[n // 2]
    xi[2:n:2], xi[3:n:2] = a[1:n // 2], b[1:n // 2]
    mvv = 103.64269652680505
    I_R = 2.0 * m * mvv * gamma * Sj            # eV^2 fs / A^2 ... in the units of m in eV fs^2/A^2
    R = F.eq9_literal(a, b, I_R, n, dt)
    eta = F.eq9_from_normals(xi[None, :], Sj)[0]
    ref = np.sqrt(2.0 * m * mvv * gamma / dt) * eta
    assert np.abs(R - ref).max() < 1e-12 * np.abs(ref).max()


def test_constant_spectrum_gives_an_orthogonal_map():
    n = 16
    M = F.eq9_from_normals(np.eye(n), np.ones(n // 2 + 1))  # row k: eta for xi = e_k
    assert np.abs(M @ M.T - np.eye(n)).max() < 1e-13
    kT = S.KB * 250.0
    xi = np.random.default_rng(4).normal(size=(50, 256))
    eta = F.eq9_from_normals(xi, np.full(129, kT))
    assert np.allclose((eta ** 2).sum(1), kT * (xi ** 2).sum(1), rtol=1e-12)


def test_periodogram_and_variance_reproduce_the_spectrum():
    n, dt, T, wmax, M = 256, 1.0, 100.0, 0.3, 4000
    Sj = F.segment_spectrum(n, dt, T, wmax)
    eta = F.eq9_segment(12345, 0, M, 3, n, Sj)
    per = (np.abs(np.fft.rfft(eta, axis=1)) ** 2 / n).mean(0)
    rel = per / Sj
    sig = np.full_like(Sj, 1.0 / np.sqrt(M))
    sig[0] = sig[-1] = np.sqrt(2.0 / M)      # real bins: chi-square with one degree of freedom
    live = Sj > 1e-8 * Sj.max()               # beyond the cutoff S is ~e^-100: rounding level
    assert live.sum() >= 12                   # the grid bins below w_max = 0.3 rad/fs
    assert np.all(np.abs(rel - 1.0)[live] < 5.0 * sig[live])
    assert np.all(per[~live] < 2.0 * Sj[~live] + 1e-28)  # tiny bins: their own level or rounding
    full = Sj[0] + Sj[-1] + 2.0 * Sj[1:-1].sum()
    var = (eta ** 2).mean()
    assert var == pytest.approx(full / n, rel=5.0 * np.sqrt(2.0 / (M * n)) * 4)


def test_segments_are_uncorrelated_across_the_boundary():
    n, dt, T, wmax, M = 128, 1.0, 100.0, 0.3, 20000
    Sj = F.segment_spectrum(n, dt, T, wmax)
    e0 = F.eq9_segment(7, 1, M, 0, n, Sj)
    e1 = F.eq9_segment(7, 1, M, 1, n, Sj)
    var = (e0 ** 2).mean()
    across = (e0[:, -1] * e1[:, 0]).mean() / var
    inside = (e0[:, :-1] * e0[:, 1:]).mean() / var
    w = F.segment_omegas(n, dt)
    target = (Sj[0] + Sj[-1] * np.cos(w[-1] * dt) + 2.0 * (Sj[1:-1] * np.cos(w[1:-1] * dt)).sum()) / \
             (Sj[0] + Sj[-1] + 2.0 * Sj[1:-1].sum())
    assert abs(across) < 5.0 / np.sqrt(M)
    assert abs(inside - target) < 5.0 / np.sqrt(M * (n - 1))
    assert target > 0.5                      # strongly correlated inside a segment at 100 K
