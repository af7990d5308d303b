"""Harmonic lattice dynamics of a periodic crystal, and the Langevin velocity
spectrum it implies, FP64.

TEST INFRASTRUCTURE.  Only the test-suite imports this module.  It shares no
code with the CUDA path.

Reference for two physics checks of QTB-MD on the MgO crystal (Sec. 2.2):

* Energy.  In the harmonic approximation about a configuration x0 where the
  forces vanish, the quantum canonical energy is V(x0) + sum_m theta(w_m, T)
  (Eq. 1) over the vibrational modes, plus k_B T/2 of kinetic energy for each
  free translation (a Langevin bath at w -> 0 gives theta(0) = k_B T).  The
  modes are the eigenpairs of the mass-weighted Hessian
  D = M^-1/2 H M^-1/2 (w_m^2 = eigenvalues in (rad/fs)^2 after the u A^2/fs^2
  to eV conversion); H is built by central differences of the oracle's FP64
  forces.
* Velocity spectrum.  A mode of frequency w_m under the Langevin equation
  (Eq. 8) with a random force of density 2 m gamma S(w) (Eqs. 6-7) has the
  one-sided spectral density of its kinetic energy
      g_m(w) = (gamma/pi) w^2 S(w) / ((w_m^2 - w^2)^2 + gamma^2 w^2),
  so that int_0^inf g_m dw = <m v^2/2> of the mode (the response integral of
  the friction correction).  The sum over modes is the phonon density of
  states weighted by the bath, which the paper warns is broadened (and given
  a high-frequency tail) by a large gamma (Sec. 3).  Free translations are
  left out (g -> delta-like at w = 0).

Units: A, fs, eV, u; w in rad/fs.
"""
import numpy as np

from .spectra import theta

MVV2E = 103.64269652680505  # eV per u A^2 / fs^2


def hessian(forces, x0, h=1e-4):
    """H[3N][3N] = -dF/dx by central differences of forces(x) ([N][3] -> [N][3])."""
    x0 = np.asarray(x0, np.float64)
    n = x0.size
    H = np.zeros((n, n))
    for k in range(n):
        xp = x0.copy().reshape(-1)
        xm = x0.copy().reshape(-1)
        xp[k] += h
        xm[k] -= h
        fp = forces(xp.reshape(x0.shape)).reshape(-1)
        fm = forces(xm.reshape(x0.shape)).reshape(-1)
        H[:, k] = -(fp - fm) / (2.0 * h)
    return H


def modes(H, masses):
    """Frequencies w (rad/fs, ascending; negative for unstable modes) and the
    mass-weighted eigenvectors (columns) of the symmetrised Hessian."""
    m3 = np.repeat(np.asarray(masses, np.float64), 3)
    Hs = 0.5 * (H + H.T)
    D = Hs / np.sqrt(m3[:, None] * m3[None, :]) / MVV2E
    lam, U = np.linalg.eigh(D)
    return np.sign(lam) * np.sqrt(np.abs(lam)), U


def harmonic_energy(V0, w, T, n_free=3, tol=1e-6):
    """V0 + sum_m theta(w_m, T) over modes with w_m > tol, plus n_free k_B T/2."""
    from .spectra import KB
    wv = np.asarray(w)[np.asarray(w) > tol]
    return V0 + float(theta(wv, T).sum()) + 0.5 * n_free * KB * T


def langevin_kinetic_density(w_modes, gamma, S, omega):
    """g(omega) = sum_m (gamma/pi) omega^2 S(omega) / ((w_m^2 - omega^2)^2 + gamma^2 omega^2)
    over the given (vibrational) modes; S a callable density (eV)."""
    om = np.asarray(omega, np.float64)
    wm = np.asarray(w_modes, np.float64)
    vib = wm[wm != 0.0]
    den = (vib[None, :] ** 2 - om[:, None] ** 2) ** 2 + (gamma * om[:, None]) ** 2
    r = om ** 2 * (1.0 / den).sum(1)
    # a free mode (w_m = 0): w^2 / (w^4 + gamma^2 w^2) = 1 / (w^2 + gamma^2)
    r = r + (wm == 0.0).sum() / (om ** 2 + gamma ** 2)
    return (gamma / np.pi) * S(om) * r


def mode_kinetic_energy(w_m, gamma, S, wmax, npts=200001):
    """int_0^wmax g_m(w) dw of one mode, by the trapezoid rule on a fine grid
    refined around the resonance."""
    w_m = float(w_m)
    lo = max(w_m - 50 * gamma, 0.0)
    hi = min(w_m + 50 * gamma, wmax)
    grid = np.unique(np.concatenate([np.linspace(0.0, wmax, npts // 2), np.linspace(lo, hi, npts // 2)]))
    g = langevin_kinetic_density([w_m], gamma, S, grid)
    return float(np.trapezoid(g, grid))
