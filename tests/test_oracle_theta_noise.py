"""Pins of the oracle's theta (Eq. 1), white noise and coloured-noise filter.

Each check compares the oracle with something other than itself: a textbook
thermal average, published Philox known-answer vectors, numpy's FFT, Parseval's
identity, and the sampled periodogram against the target spectral density
(Eqs. 6-7).
"""
import numpy as np
import pytest
from scipy import stats

from golden_values import philox_kat
from oracle import spectra as S

HBAR, KB = 0.6582119569, 8.617333262e-5


def test_theta_is_thermal_average_of_levels():
    # Eq. 1 is the mean energy of a quantum oscillator: sum_n (n+1/2) hbar w p_n.
    for w, T in [(0.01, 300.0), (0.1, 100.0), (0.2, 1000.0), (0.05, 10.0)]:
        x = HBAR * w / (KB * T)
        n = np.arange(0, 20000)
        p = np.exp(-n * x)
        E = (HBAR * w * (n + 0.5) * p).sum() / p.sum()
        assert S.theta(w, T) == pytest.approx(E, rel=1e-12)


def test_theta_limits_and_fig3_shape():
    w = 0.1
    hw = HBAR * w
    # zero-point limit hbar w / 2 and classical limit k_B T (Fig. 3)
    assert S.theta(w, 1.0) == pytest.approx(hw / 2, rel=1e-12)
    assert S.theta(w, 1e6) == pytest.approx(KB * 1e6, rel=1e-6)
    assert S.theta(0.0, 300.0) == pytest.approx(KB * 300.0, rel=1e-15)
    # normalized energy vs reduced temperature: increasing, above both limits
    t = np.linspace(0.01, 3.0, 300)          # k_B T / (hbar w)
    e = np.array([S.theta(w, ti * hw / KB) for ti in t]) / hw
    assert np.all(np.diff(e) >= 0) and np.all(np.diff(e[t > 0.1]) > 0)
    assert np.all(e >= 0.5 - 1e-12) and np.all(e >= t - 1e-12)
    # high-T expansion of (x/2) coth(x/2): theta/(hbar w) - t = 1/(12 t) - 1/(720 t^3) + ...
    assert e[-1] - t[-1] == pytest.approx(1.0 / (12 * t[-1]) - 1.0 / (720 * t[-1] ** 3), rel=1e-4)


# Published known-answer vectors of Philox4x32-10 (Salmon et al., SC'11), tests/golden/.
KAT = philox_kat()


@pytest.mark.parametrize("ctr,key,expect", KAT)
def test_philox_known_answers(oracle, ctr, key, expect):
    assert list(oracle.philox(ctr, key)) == expect


def test_white_noise_is_standard_normal(oracle):
    xi = oracle.white_block(12345, 3, 64, -37, 4096)   # includes negative steps
    flat = xi.ravel()
    assert abs(flat.mean()) < 5.0 / np.sqrt(flat.size)
    assert abs(flat.var() - 1.0) < 6.0 * np.sqrt(2.0 / flat.size)
    assert stats.kstest(flat, "norm").pvalue > 1e-4
    # uncorrelated across steps (lag 1..3 share a Philox call) and across dofs
    for lag in (1, 2, 3, 4):
        c = (xi[:, lag:] * xi[:, :-lag]).mean()
        assert abs(c) < 5.0 / np.sqrt(xi[:, lag:].size)
    c = (xi[1:] * xi[:-1]).mean()
    assert abs(c) < 5.0 / np.sqrt(xi[1:].size)
    # block form equals the pointwise definition; distinct systems differ
    assert xi[5, 100] == oracle.white(12345, 3, 5, -37 + 100)
    assert oracle.white(12345, 4, 5, 63) != oracle.white(12345, 3, 5, 63)


def test_taps_reproduce_spectrum_by_fft():
    L, dt = 257, 1.0
    Sj = S.spectrum(L, dt, 150.0, 0.3)
    h = S.taps_from_spectrum(Sj)
    K = (L - 1) // 2
    circ = np.concatenate([h, h[1:][::-1]])          # h_0..h_K, h_{-K}..h_{-1}
    H = np.fft.fft(circ)
    assert np.max(np.abs(H.imag)) < 1e-13 * np.abs(H.real).max()
    assert np.allclose(H.real[:K + 1], np.sqrt(Sj), rtol=0, atol=1e-13 * np.sqrt(Sj).max())
    # Parseval: sum_k h_k^2 = (1/L) sum_j S_j
    e_time = h[0] ** 2 + 2 * (h[1:] ** 2).sum()
    e_freq = (Sj[0] + 2 * Sj[1:].sum()) / L
    assert e_time == pytest.approx(e_freq, rel=1e-12)


def test_white_limit_gives_delta_taps():
    # theta -> k_B T (no cutoff) must give the plain Langevin noise sqrt(kT) xi
    K = 100
    kT = KB * 300.0
    h = S.taps_from_spectrum(np.full(K + 1, kT))
    assert h[0] == pytest.approx(np.sqrt(kT), rel=1e-13)
    assert np.max(np.abs(h[1:])) < 1e-14


def test_colored_noise_periodogram_matches_target(oracle):
    # Eqs. 6-7 in discrete time: eta has autocovariance c_m = sum_k h_k h_{k+m}
    # and spectral density |H(w)|^2, equal to S = theta W at the tap grid.  The
    # expected periodogram of an Ns-step record is sum_m (1 - |m|/Ns) c_m cos(w m dt).
    L, dt, T = 65, 1.0, 80.0
    h = S.taps(L, dt, T, 0.6)
    M, Ns = 600, 65 * 16
    eta = oracle.colored_block(777, 0, M, 5, Ns, h)
    I = np.abs(np.fft.rfft(eta, axis=1)) ** 2 / Ns
    Ihat = I.mean(0)[1:-1]
    w = 2 * np.pi * np.arange(Ns // 2 + 1) / (Ns * dt)
    hf = np.concatenate([h[1:][::-1], h])
    c = np.convolve(hf, hf[::-1])                        # lags -(L-1)..(L-1)
    m = np.arange(-(L - 1), L)
    expect = (np.cos(np.outer(w, m) * dt) @ (c * (1 - np.abs(m) / Ns)))[1:-1]
    band = expect > 1e-2 * expect.max()
    assert band.sum() > 100
    z = (Ihat[band] / expect[band] - 1.0) * np.sqrt(M)
    assert np.max(np.abs(z)) < 5.0
    assert abs(z.mean()) < 5.0 / np.sqrt(band.sum())
    # |H(w)|^2 at the tap grid frequencies is the target spectrum itself
    k = np.arange(1, len(h))
    Sg = S.spectrum(L, dt, T, 0.6)
    wg = 2 * np.pi * np.arange(len(Sg)) / (L * dt)
    Hg = h[0] + 2 * np.cos(np.outer(wg, k) * dt) @ h[1:]
    assert np.allclose(Hg ** 2, Sg, rtol=1e-10, atol=1e-14)
    # variance of eta is c_0 = sum h^2
    assert eta.var() == pytest.approx(c[L - 1], rel=0.02)
