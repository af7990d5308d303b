"""Spectral half of the FP64 oracle: theta, kappa_P, the cutoff and the filter taps.

TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU baseline
of the benchmark import this module.  It shares no code with the CUDA path.

Method (Dammak, Hayoun, Brieuc, Geneste, "Nuclear quantum effects in molecular
dynamics simulations"):

* Eq. 1   theta(w, T) = hbar w [1/2 + 1/(exp(beta hbar w) - 1)].
* Eqs. 6-7  the random force has power spectral density I_R = 2 m gamma theta.
* Eq. 10  kappa_P solves (1/P) sum_k kappa_P(w_k)/(m w_k^2) = theta(w)/(m w^2),
* Eq. 11  with w_k^2 = w^2/P + 4 w_P^2 sin^2(k pi / P), w_P = sqrt(P)/(beta hbar).
* Eq. 12  QTB-PIMD replaces theta by kappa_P in the spectral density.

Readings where the paper is silent:

* Discrete spectrum.  The coloured sequence eta_n has discrete-time spectral
  density S(w) = theta(w) W(w) for |w| <= pi/dt, so that sqrt(2 m gamma/dt) eta
  has the density 2 m gamma theta W of Eq. 7; W is a Fermi cutoff
  1/(1 + exp((|w| - w_max)/(w_max/50))) (no cutoff when w_max <= 0).
* Taps.  Zero-phase filter of odd length L = 2K+1 on the grid w_j = 2 pi j/(L dt):
  h_k = (1/L) sum_{j=-K..K} sqrt(S(w_j)) cos(w_j k dt), so that the filter's
  frequency response equals sqrt(S) at every grid frequency.
* kappa_P solver.  kappa_P/(k_B T) = F_P(y), y = beta hbar w, a function of
  (y, P) only.  With y_k^2 = y^2 + 4 P sin^2(k pi/P) (Eq. 11 in these units,
  the k = 0 mode at y = w/sqrt(P) scaled) Eq. 10 reads
      sum_k (y^2/y_k^2) F_P(y_k) = f(sqrt(P) y),   f(x) = x (1/2 + 1/(e^x - 1)).
  The plain fixed-point (Picard or damped Jacobi) iteration of this equation
  diverges for P >= 4 (oscillatory near-null components), so F_P is taken as
  the least-squares solution of the overdetermined collocation system: F_P on
  n nodes y_i = y0 sinh(i dt_), linear interpolation in y between nodes, the
  equation imposed at the nodes and at the midpoints (2n-1 rows, each row
  divided by f(sqrt(P) y)), and above y_max the asymptotic tail
      F_P(y) ~ f(sqrt(P) y)/P + sqrt(P)/(2 y)          (P >= 2).
  The least-squares solve is numpy's (LAPACK) routine.
"""
from __future__ import annotations

import numpy as np

HBAR = 0.6582119569        # eV fs
KB = 8.617333262e-5        # eV / K

# default collocation grid of the kappa_P solve (dimensionless)
KAPPA_N = 1024
KAPPA_YMAX = 1000.0
KAPPA_Y0 = 1.0


def f_theta(x):
    """theta / (k_B T) as a function of x = beta hbar w (Eq. 1); f(0) = 1."""
    x = np.abs(np.asarray(x, dtype=np.float64))
    out = np.empty_like(x)
    small = x < 1e-6
    out[small] = 1.0 + x[small] ** 2 / 12.0
    xs = x[~small]
    with np.errstate(over="ignore"):
        out[~small] = xs * (0.5 + 1.0 / np.expm1(xs))
    return out


def theta(omega, T):
    """Eq. 1, omega in rad/fs, T in K, result in eV."""
    omega = np.asarray(omega, dtype=np.float64)
    if T <= 0:
        return 0.5 * HBAR * np.abs(omega)
    kT = KB * T
    return kT * f_theta(HBAR * omega / kT)


def cutoff(omega, omega_max):
    """Fermi roll-off W(omega) applied to the spectral density."""
    omega = np.abs(np.asarray(omega, dtype=np.float64))
    if omega_max is None or omega_max <= 0:
        return np.ones_like(omega)
    width = omega_max / 50.0
    with np.errstate(over="ignore"):
        return 1.0 / (1.0 + np.exp((omega - omega_max) / width))


def grid_omegas(L, dt):
    """Non-negative filter grid frequencies w_j = 2 pi j/(L dt), j = 0..K."""
    K = (L - 1) // 2
    return 2.0 * np.pi * np.arange(K + 1) / (L * dt)


def taps_from_spectrum(S):
    """Zero-phase taps h_0..h_K from S_0..S_K (S_{-j} = S_j), length L = 2K+1."""
    S = np.asarray(S, dtype=np.float64)
    K = len(S) - 1
    L = 2 * K + 1
    a = np.sqrt(S)
    j = np.arange(1, K + 1)
    k = np.arange(K + 1)
    # cos(2 pi j k / L) with the exact integer phase (j k mod L)
    ph = (np.outer(k, j) % L).astype(np.float64)
    h = (a[0] + 2.0 * (np.cos(2.0 * np.pi * ph / L) @ a[1:])) / L
    return h


# ---------------------------------------------------------------------------
# kappa_P (Eq. 10)

def _mode_shifts(P):
    return 4.0 * P * np.sin(np.arange(P) * np.pi / P) ** 2


def kappa_tail(P, y):
    y = np.asarray(y, dtype=np.float64)
    if P == 1:
        return f_theta(y)
    return f_theta(np.sqrt(P) * y) / P + np.sqrt(P) / (2.0 * y)


class KappaSolution:
    """F_P on the collocation grid, evaluable at any y >= 0."""

    def __init__(self, P, F, n, ymax, y0):
        self.P, self.F, self.n, self.ymax, self.y0 = P, np.asarray(F), n, ymax, y0
        self.dts = np.arcsinh(ymax / y0) / (n - 1)
        self.y = y0 * np.sinh(np.arange(n) * self.dts)

    def __call__(self, y):
        y = np.abs(np.asarray(y, dtype=np.float64))
        if self.P == 1:
            return f_theta(y)
        out = np.empty_like(y)
        inside = y <= self.ymax
        yi = y[inside]
        i = np.minimum((np.arcsinh(yi / self.y0) / self.dts).astype(np.int64), self.n - 2)
        lam = (yi - self.y[i]) / (self.y[i + 1] - self.y[i])
        out[inside] = self.F[i] * (1.0 - lam) + self.F[i + 1] * lam
        out[~inside] = kappa_tail(self.P, y[~inside])
        return out


def kappa_system(P, n=KAPPA_N, ymax=KAPPA_YMAX, y0=KAPPA_Y0):
    """Collocation matrix A ((2n-1) x n) and right-hand side b of Eq. 10."""
    dts = np.arcsinh(ymax / y0) / (n - 1)
    y = y0 * np.sinh(np.arange(n) * dts)
    ym = y0 * np.sinh(np.arange(2 * n - 1) * dts / 2.0)
    c = _mode_shifts(P)
    A = np.zeros((len(ym), n))
    b = f_theta(np.sqrt(P) * ym).copy()
    for k in range(P):
        yk = np.sqrt(ym ** 2 + c[k])
        w = np.ones_like(ym) if k == 0 else ym ** 2 / (ym ** 2 + c[k])
        inside = yk <= ymax
        rows = np.nonzero(inside)[0]
        i = np.minimum((np.arcsinh(yk[inside] / y0) / dts).astype(np.int64), n - 2)
        lam = (yk[inside] - y[i]) / (y[i + 1] - y[i])
        np.add.at(A, (rows, i), w[inside] * (1.0 - lam))
        np.add.at(A, (rows, i + 1), w[inside] * lam)
        b[~inside] -= w[~inside] * kappa_tail(P, yk[~inside])
    scale = 1.0 / f_theta(np.sqrt(P) * ym)
    return A * scale[:, None], b * scale


def kappa_solve(P, n=KAPPA_N, ymax=KAPPA_YMAX, y0=KAPPA_Y0):
    """Solve Eq. 10 for F_P = kappa_P/(k_B T) (see the module docstring)."""
    if P == 1:
        return KappaSolution(1, f_theta(y0 * np.sinh(np.arange(n) * np.arcsinh(ymax / y0) / (n - 1))),
                             n, ymax, y0)
    A, b = kappa_system(P, n, ymax, y0)
    F, *_ = np.linalg.lstsq(A, b, rcond=None)
    return KappaSolution(P, F, n, ymax, y0)


def kappa(omega, T, sol):
    """kappa_P(omega, T) in eV from a dimensionless solution."""
    kT = KB * T
    return kT * sol(HBAR * np.asarray(omega, dtype=np.float64) / kT)


def eq10_residual(sol, y):
    """Relative residual of Eq. 10 at arbitrary y (dimensionless form)."""
    P = sol.P
    y = np.asarray(y, dtype=np.float64)
    c = _mode_shifts(P)
    tot = np.zeros_like(y)
    for k in range(P):
        yk = np.sqrt(y ** 2 + c[k])
        w = np.ones_like(y) if k == 0 else y ** 2 / yk ** 2
        tot += w * sol(yk)
    rhs = f_theta(np.sqrt(P) * y)
    return (tot - rhs) / rhs


# ---------------------------------------------------------------------------
# spectra and taps for a system

def spectrum(L, dt, T, omega_max, P=1, sol=None):
    """S_j = theta W (P = 1 / QTB-MD) or kappa_P W (QTB-PIMD) on the tap grid."""
    w = grid_omegas(L, dt)
    if P == 1 and sol is None:
        base = theta(w, T)
    else:
        if sol is None:
            sol = kappa_solve(P)
        base = kappa(w, T, sol)
    return base * cutoff(w, omega_max)


def taps(L, dt, T, omega_max, P=1, sol=None):
    return taps_from_spectrum(spectrum(L, dt, T, omega_max, P, sol))
