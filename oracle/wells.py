"""Exact quantum thermal averages of a particle in a 1-D potential, FP64.

TEST INFRASTRUCTURE.  Only the test-suite imports this module.  It shares no
code with the CUDA path.

Reference for the zero-point-energy-leakage study (Sec. 2.2: QTB can transfer
energy from high- to low-frequency modes; Sec. 2.3: QTB-PIMD, Eqs. 10-12, is
exact for any P in a harmonic system and converges with P otherwise).  The
Hamiltonian H = -hbar^2/(2 m) d^2/dx^2 + V(x) is discretised by second-order
finite differences on a uniform grid of `npts` points in [-xmax, xmax] (wave
functions vanish at the ends); its lowest `nlev` eigenpairs (a library
tridiagonal eigensolver) give the canonical averages
<O> = sum_n exp(-E_n/k_B T) <n|O|n> / sum_n exp(-E_n/k_B T).
Units: x in A, m in u, energies in eV.
"""
import numpy as np
from scipy.linalg import eigh_tridiagonal

from .spectra import HBAR, KB

MVV2E = 103.64269652680505  # eV per u A^2 / fs^2


def double_well(V0, a):
    """V(x) = V0 (x^2/a^2 - 1)^2 (the external potential DOUBLEWELL)."""
    return lambda x: V0 * (x * x / (a * a) - 1.0) ** 2


def harmonic(m, omega):
    """V(x) = m omega^2 x^2 / 2 (omega in rad/fs)."""
    return lambda x: 0.5 * m * MVV2E * omega * omega * x * x


def levels(V, m, xmax, npts=4000, nlev=60, with_v=False):
    """Lowest eigenvalues E_n (eV), the expectation of x^2 in each state (and of V)."""
    x = np.linspace(-xmax, xmax, npts + 2)[1:-1]
    dx = x[1] - x[0]
    t = HBAR * HBAR / (2.0 * m * MVV2E * dx * dx)      # hbar^2/(2 m dx^2), eV
    diag = 2.0 * t + V(x)
    off = np.full(npts - 1, -t)
    E, psi = eigh_tridiagonal(diag, off, select="i", select_range=(0, nlev - 1))
    nrm = (psi * psi).sum(0)
    x2 = (psi * psi * (x * x)[:, None]).sum(0) / nrm
    if with_v:
        return E, x2, (psi * psi * V(x)[:, None]).sum(0) / nrm
    return E, x2


def thermal(V, m, T, xmax, npts=4000, nlev=60, with_v=False):
    """Canonical <E> (eV) and <x^2> (A^2) at temperature T (K) (and <V>, eV)."""
    E, x2, v = levels(V, m, xmax, npts, nlev, with_v=True)
    w = np.exp(-(E - E[0]) / (KB * T))
    if w[-1] > 1e-12 * w.sum():
        raise ValueError("not enough levels for this temperature")
    out = (float((w * E).sum() / w.sum()), float((w * x2).sum() / w.sum()))
    return out + (float((w * v).sum() / w.sum()),) if with_v else out


def classical(V, m, T, xmax, npts=20001):
    """Classical canonical <E> = k_B T/2 + <V> and <x^2> by quadrature (and <V>)."""
    x = np.linspace(-xmax, xmax, npts)
    v = V(x)
    w = np.exp(-(v - v.min()) / (KB * T))
    Z = np.trapezoid(w, x)
    vm = np.trapezoid(w * v, x) / Z
    return 0.5 * KB * T + vm, np.trapezoid(w * x * x, x) / Z, vm
