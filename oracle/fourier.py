"""Fourier-segment generator of the random force (Eq. 9), FP64 reference.

TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU baseline
of the benchmark import this module.  It shares no code with the CUDA path.

Eq. 9 (Sec. 2.2): over a segment of n MD steps the random force is drawn in
Fourier space, each frequency w_j = 2 pi j/(n dt) getting (a_j + i b_j)
sqrt(I_R(w_j) n dt / 2) with a_j, b_j standard normal, and the time series is
its inverse Fourier transform.  I_R = 2 m gamma theta (Eq. 7), or 2 m gamma
kappa_P for QTB-PIMD (Eq. 12).

Readings where the paper is silent:

* Normalisation of the inverse transform: R(t_l) = (1/(n dt)) sum_j R~_j
  exp(i w_j t_l), sum over j = 0..n-1 with R~_{n-j} = conj(R~_j) (a real force).
  Then <R^2> = (1/(n dt)) sum_j I_R(w_j), the discrete form of
  (1/2 pi) int I_R dw.
* The bins j = 0 and j = n/2 are their own conjugates, hence real: there
  R~_j = a_j sqrt(I_R n dt) (the same mean square as the complex bins).
* The generator produces the sequence eta of discrete spectral density S(w) on
  the segment grid (S = theta W, or kappa_P W, W the cutoff of spectra.py), so
  that R = sqrt(2 m gamma / dt) eta, exactly as for the time-domain filter.
  In this form eta_t = (1/sqrt(n)) sum_j c_j exp(2 pi i j t/n) with
  c_0 = sqrt(S_0) a_0, c_{n/2} = sqrt(S_{n/2}) a_{n/2},
  c_j = sqrt(S_j/2) (a_j + i b_j) for 0 < j < n/2, c_{n-j} = conj(c_j).
* Normals: the n normals of a segment are the white-noise sequence xi of the
  same seed, system and dof over the segment's steps t = seg n .. seg n + n - 1
  (the Philox stream of the time-domain filter), assigned as
  a_0 = xi_0, a_{n/2} = xi_1, a_j = xi_{2j}, b_j = xi_{2j+1} (0 < j < n/2).
* Segments are independent: the sequence is stationary within a segment (in
  fact periodic with period n) and uncorrelated across segment boundaries.
"""
import numpy as np

from . import white_block
from . import spectra as S


def segment_omegas(n, dt):
    """w_j = 2 pi j/(n dt), j = 0..n/2 (rad/fs)."""
    return 2.0 * np.pi * np.arange(n // 2 + 1) / (n * dt)


def segment_spectrum(n, dt, T, omega_max, P=1, sol=None, white=False):
    """S_j on the segment grid: k_B T (white), theta W (P = 1) or kappa_P W."""
    w = segment_omegas(n, dt)
    if white:
        return np.full_like(w, S.KB * T)
    if P == 1 and sol is None:
        base = S.theta(w, T)
    else:
        if sol is None:
            sol = S.kappa_solve(P)
        base = S.kappa(w, T, sol)
    return base * S.cutoff(w, omega_max)


def eq9_from_normals(xi, Sj):
    """eta [ndof][n] from the segment's normals xi [ndof][n] and S_j (j = 0..n/2)."""
    xi = np.atleast_2d(np.asarray(xi, np.float64))
    n = xi.shape[1]
    h = n // 2
    c = np.zeros((xi.shape[0], h + 1), np.complex128)
    c[:, 0] = np.sqrt(Sj[0]) * xi[:, 0]
    c[:, h] = np.sqrt(Sj[h]) * xi[:, 1]
    j = np.arange(1, h)
    c[:, j] = np.sqrt(Sj[j] / 2.0) * (xi[:, 2 * j] + 1j * xi[:, 2 * j + 1])
    # numpy's inverse real transform: (1/n) sum_j c_j e^{+2 pi i j t/n}, Hermitian-extended
    return np.fft.irfft(c, n, axis=1) * np.sqrt(n)


def eq9_segment(seed, sys, ndof, seg, n, Sj):
    """eta of dofs 0..ndof-1 of system `sys` over segment `seg` (steps seg n .. seg n + n - 1)."""
    return eq9_from_normals(white_block(seed, sys, ndof, seg * n, n), Sj)


def eq9_literal(a, b, I_R, n, dt):
    """Eq. 9 written out as printed, with the readings above: R~_j = (a_j + i b_j)
    sqrt(I_R(w_j) n dt / 2) for 0 < j < n/2, the real bins 0 and n/2, then
    R(t_l) = (1/(n dt)) sum_{j=0}^{n-1} R~_j exp(i w_j t_l) by direct summation.
    a, b: [n/2 + 1] normals (b_0, b_{n/2} unused); I_R: [n/2 + 1].  Returns R [n]."""
    h = n // 2
    Rt = np.zeros(n, np.complex128)
    Rt[0] = a[0] * np.sqrt(I_R[0] * n * dt)
    Rt[h] = a[h] * np.sqrt(I_R[h] * n * dt)
    for j in range(1, h):
        Rt[j] = (a[j] + 1j * b[j]) * np.sqrt(I_R[j] * n * dt / 2.0)
        Rt[n - j] = np.conj(Rt[j])
    t = np.arange(n) * dt
    w = 2.0 * np.pi * np.arange(n) / (n * dt)
    R = (Rt[None, :] * np.exp(1j * w[None, :] * t[:, None])).sum(axis=1) / (n * dt)
    return R.real
