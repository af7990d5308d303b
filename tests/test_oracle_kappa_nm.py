"""Pins of the oracle's kappa_P solve (Eq. 10) and ring-polymer normal modes (Eq. 11).

kappa_P is checked against: the P = 1 identity kappa_1 = theta; an independent
closed form for P = 2 (Eq. 10 with P = 2 is G(s) + G(s + 8) = R(s), solved by an
alternating series); the residual of Eq. 10 at off-grid frequencies; the limits
kappa_P(0) = k_B T and kappa_P ~ hbar w / (2 sqrt P).  The normal-mode matrix is
checked against a finite-difference Hessian of the spring energy of Eq. 3.
"""
import numpy as np
import pytest

from oracle import spectra as S

HBAR, KB = 0.6582119569, 8.617333262e-5


@pytest.fixture(scope="module")
def sols():
    return {P: S.kappa_solve(P) for P in (1, 2, 4, 8, 32)}


def _p2_series(y):
    # G(s) + G(s+8) = R(s), G = F/s, R(s) = f(sqrt(2 s))/s  (Eq. 10, P = 2, s = y^2).
    # G = sum_n (-1)^n R(s + 8n); partial sums averaged repeatedly (Euler).
    s = y * y
    n = np.arange(400000)
    ss = s + 8.0 * n
    terms = (-1.0) ** n * S.f_theta(np.sqrt(2 * ss)) / ss
    q = np.cumsum(terms)[-80:]
    for _ in range(60):
        q = 0.5 * (q[1:] + q[:-1])
    return s * q[-1]


def test_p1_is_theta(sols):
    y = np.linspace(0, 50, 101)
    assert np.allclose(sols[1](y), S.f_theta(y), rtol=1e-15)


def test_p2_against_alternating_series(sols):
    for y in (0.3, 1.0, 2.5, 6.0, 15.0, 40.0):
        assert sols[2](np.array([y]))[0] == pytest.approx(_p2_series(y), rel=2e-6)


@pytest.mark.parametrize("P", [2, 4, 8, 32])
def test_eq10_residual_off_grid(sols, P):
    rng = np.random.default_rng(P)
    y = np.concatenate([rng.uniform(0, 5, 300), rng.uniform(5, 200, 300), rng.uniform(200, 3000, 50)])
    r = S.eq10_residual(sols[P], y)
    assert np.max(np.abs(r)) < 1e-5


@pytest.mark.parametrize("P", [2, 4, 8, 32])
def test_kappa_limits_and_shape(sols, P):
    F = sols[P]
    assert F(np.array([0.0]))[0] == pytest.approx(1.0, abs=2e-6)      # kappa_P(0) = k_B T
    yb = np.array([800.0, 5000.0])
    assert np.allclose(F(yb) / (yb / (2 * np.sqrt(P))), 1.0, rtol=2e-3)
    y = np.linspace(0.0, 300.0, 3001)
    v = F(y)
    assert np.all(v > 0)
    # below theta (the ring polymer already carries part of the quantum fluctuation)
    assert np.all(v <= S.f_theta(y) * (1 + 1e-6))


def test_kappa_independent_of_grid():
    a = S.kappa_solve(8, n=1024)
    b = S.kappa_solve(8, n=1536, ymax=1500.0)
    y = np.linspace(0, 200, 777)
    assert np.allclose(a(y), b(y), rtol=2e-4)


def test_plain_fixed_point_iteration_diverges():
    # Reading recorded with the solver: the fixed-point (row-normalised Jacobi)
    # iteration F <- F + (f - sum_k w_k F(y_k)) / sum_k w_k of Eq. 10 is unstable
    # for P >= 4, which is why the oracle solves Eq. 10 by least squares.
    P, n, Y = 8, 601, 30.0
    y = np.linspace(0.0, Y, n)
    dy = y[1] - y[0]
    c = 4 * P * np.sin(np.arange(P) * np.pi / P) ** 2
    yk = np.sqrt(y[None, :] ** 2 + c[:, None])
    wk = np.where(yk > 0, y[None, :] ** 2 / np.where(yk > 0, yk ** 2, 1.0), 1.0)
    wk[0] = 1.0
    rhs = S.f_theta(np.sqrt(P) * y)
    F = S.f_theta(np.sqrt(P) * y) / P
    F[0] = 1.0

    def at(F, q):
        out = S.kappa_tail(P, np.maximum(q, 1e-9))
        ins = q <= Y
        t = q[ins] / dy
        i = np.minimum(t.astype(int), n - 2)
        fr = t - i
        out[ins] = F[i] * (1 - fr) + F[i + 1] * fr
        return out

    res = []
    with np.errstate(all="ignore"):
        for _ in range(150):
            Fk = np.stack([F] + [at(F, yk[k]) for k in range(1, P)])
            R = rhs - (wk * Fk).sum(0)
            res.append(np.abs(R).max())
            F = F + R / wk.sum(0)
    assert res[-1] > 1e10 * res[0]


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 8, 32])
def test_normal_modes_diagonalize_spring(oracle, P):
    T, m = 50.0, 1.008
    Cm = oracle.nm_matrix(P)
    assert np.allclose(Cm.T @ Cm, np.eye(P), atol=1e-13)
    wP = np.sqrt(P) * KB * T / HBAR

    def spring(x):   # Eq. 3 spring term of one 1-D ring polymer (energy / m)
        return sum(0.5 * wP ** 2 * (x[s] - x[(s + 1) % P]) ** 2 for s in range(P))

    H = np.zeros((P, P))
    eps = 1e-3
    x0 = np.zeros(P)
    for a in range(P):
        for b in range(P):
            def e(da, db):
                x = x0.copy()
                x[a] += da
                x[b] += db
                return spring(x)
            H[a, b] = (e(eps, eps) - e(eps, -eps) - e(-eps, eps) + e(-eps, -eps)) / (4 * eps * eps)
    D = Cm.T @ H @ Cm
    wk = oracle.nm_freqs(P, T)
    assert np.allclose(D, np.diag(wk ** 2), atol=1e-8 * max(wP ** 2, 1e-30))
    # Eq. 11: adding V/P = w^2 x^2/(2P) per bead shifts every mode by w^2/P
    w = 0.07
    D2 = Cm.T @ (H + np.eye(P) * w * w / P) @ Cm
    assert np.allclose(np.diag(D2), w * w / P + 4 * wP ** 2 * np.sin(np.arange(P) * np.pi / P) ** 2,
                       rtol=1e-8, atol=1e-12)
