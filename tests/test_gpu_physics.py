"""Physics on the GPU path (through the C ABI), pinned to what the paper fixes.

* Equilibrium observables of QTB-MD on 64-ion MgO (the small benchmark
  workload, 2000 steps) within 2 sigma of the oracle's own statistical error
  (block averages), in the FP64 and the mixed form.
* QTB on harmonic oscillators reproduces theta(w0, T) of Eq. 1 up to the
  friction correction (quadrature of the Langevin response with the filter's
  own spectral density, Eqs. 6-8), in both forms and with the tensor-core filter.
* QTB-PIMD on harmonic oscillators gives the bead-averaged <x^2> that Eq. 10
  demands, theta/(m w0^2), for P = 2, 4, 8, and the centroid-mode virial
  estimator (record slot 19) gives the quantum kinetic energy theta/2;
* standard PIMD: the centroid-virial estimator (slot 18) averages to the
  finite-P closed form E_P/2 with a smaller fluctuation than the primitive one.
"""
import numpy as np
import pytest
from scipy import integrate

from helpers import gpu_ctx, oracle_sim
from oracle import spectra as S
from paper_1905_02521_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HBAR, KB, MVV2E = 0.6582119569, 8.617333262e-5, 103.64269652680505


@pytest.fixture(scope="module")
def qtb():
    import torch
    assert torch.cuda.is_available()
    from paper_1905_02521_gb300 import build
    build.build()
    from paper_1905_02521_gb300 import qtb as q
    return q


def _block_sigma(x, nblk=10):
    b = np.array_split(np.asarray(x), nblk)
    m = np.array([bb.mean() for bb in b])
    return m.std(ddof=1) / np.sqrt(nblk)


@pytest.fixture(scope="module")
def oracle_mgo_series(oracle):
    s, pot = W.mgo_system(2, 300.0)
    h = S.taps(513, 1.0, 300.0, 0.3)
    sim = oracle_sim(oracle, s, pot, 1.0, seed=2718, taps=h)
    rec = sim.step(2000)
    return s, pot, rec


@pytest.mark.parametrize("precision,filt", [(0, 0), (1, 1), (1, 2)])
def test_equilibrium_observables_within_2sigma(qtb, oracle_mgo_series, precision, filt):
    s, pot, rec = oracle_mgo_series
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=precision, filter_prec=filt, seed=2718, max_records=2000)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 513, 0.3)
        qtb.qtb_step_n(ctx, 2000)
        ser = qtb.qtb_get_series(ctx, 0, 2000)
    finally:
        qtb.qtb_destroy(ctx)
    assert len(ser) == 2000 and ser[-1, 0] == 2000
    # second half (equilibrated): kinetic and potential energy, their sum, the virial
    # trace (pressure work) and the total momentum, against the oracle's block error
    obs = {"K": lambda r: r[:, 1], "V": lambda r: r[:, 2], "E": lambda r: r[:, 1] + r[:, 2],
           "W": lambda r: r[:, 5] + r[:, 9] + r[:, 13], "|p|": lambda r: np.linalg.norm(r[:, 14:17], axis=1)}
    form = {(0, 0): "FP64", (1, 1): "mixed, FP32 filter", (1, 2): "mixed, BF16 tensor-core filter"}[(precision, filt)]
    for name, f in obs.items():
        o, g = f(rec[1000:]), f(ser[1000:])
        sig = _block_sigma(o)
        print("%-30s %-4s GPU %.6g  oracle %.6g +- %.2g  (%+.2f sigma)"
              % (form, name, g.mean(), o.mean(), sig, (g.mean() - o.mean()) / sig))
        if name in ("K", "V"):
            assert abs(g.mean() - o.mean()) <= 2 * sig, (name, g.mean(), o.mean(), sig)
        else:
            assert abs(g.mean() - o.mean()) <= 3 * sig, (name, g.mean(), o.mean(), sig)


def _quad_x2_v2(dens, w0, gamma, m, wmax):
    def resp(w):
        return 2 * gamma / (m * MVV2E * ((w0 ** 2 - w ** 2) ** 2 + (gamma * w) ** 2)) / np.pi
    x2 = integrate.quad(lambda w: resp(w) * dens(w), 0, wmax, points=[w0], limit=2000)[0]
    v2 = integrate.quad(lambda w: resp(w) * w * w * dens(w), 0, wmax, points=[w0], limit=2000)[0]
    return x2, v2


def _filter_density(h, dt):
    k = np.arange(1, len(h))
    return lambda w: (h[0] + 2 * np.cos(w * dt * k) @ h[1:]) ** 2


@pytest.mark.parametrize("precision,filt", [(0, 0), (1, 1), (1, 2)])
def test_qtb_harmonic_oscillators_reproduce_theta(qtb, precision, filt):
    w0, T, gamma, dt, L, m = 0.1, 100.0, 0.01, 0.5, 513, 1.008
    sysd, pot = W.oscillators(2000, T, gamma, mass=m)
    ctx = gpu_ctx(qtb, [sysd], pot, dt, precision=precision, filter_prec=filt, seed=31, potential=qtb.POT_HARMONIC,
                  ext={"omega": w0}, max_records=20000)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, L, 0.5)
        qtb.qtb_step_n(ctx, 2048)
        ser = qtb.qtb_get_series(ctx, 0, 20000)
        qtb.qtb_step_n(ctx, 16384)
        ser = qtb.qtb_get_series(ctx, 0, 20000)[-16384:]
    finally:
        qtb.qtb_destroy(ctx)
    E = (ser[:, 1] + ser[:, 2]) / (3 * 2000)
    h = S.taps(L, dt, T, 0.5)
    x2, v2 = _quad_x2_v2(_filter_density(h, dt), w0, gamma, m, np.pi / dt)
    E_q = 0.5 * m * MVV2E * (v2 + w0 ** 2 * x2)
    tol = 4 * _block_sigma(E, 16) + 5e-3 * E_q + (0.01 * E_q if filt == 2 else 0.0)
    assert abs(E.mean() - E_q) < tol, (E.mean(), E_q)
    assert E_q == pytest.approx(S.theta(w0, T), rel=0.03)


@pytest.mark.parametrize("P", [2, 4, 8])
def test_qtb_pimd_harmonic_bead_variance_eq10(qtb, oracle, P):
    w0, T, gamma, dt, L, m = 0.1, 100.0, 0.01, 0.5, 513, 1.008
    sysd, pot = W.oscillators(1000, T, gamma, n_beads=P, mass=m)
    ctx = gpu_ctx(qtb, [sysd], pot, dt, precision=0, seed=77, potential=qtb.POT_HARMONIC, ext={"omega": w0},
                  max_records=20000)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB_PIMD, L, 0.5)
        qtb.qtb_step_n(ctx, 2048 + 16384)
        ser = qtb.qtb_get_series(ctx, 0, 20000)[-16384:]
    finally:
        qtb.qtb_destroy(ctx)
    x2 = ser[:, 17] / (3 * 1000)
    h = S.taps(L, dt, T, 0.5, P=P, sol=S.kappa_solve(P))
    dens = _filter_density(h, dt)
    wk = oracle.nm_freqs(P, T)
    x2_q = np.mean([_quad_x2_v2(dens, np.sqrt(w0 ** 2 / P + wk[k] ** 2), gamma, m, np.pi / dt)[0]
                    for k in range(P)])
    assert abs(x2.mean() - x2_q) < 4 * _block_sigma(x2, 16) + 5e-3 * x2_q
    # Eq. 10: without friction the bead average is the quantum value theta/(m w0^2)
    assert x2_q == pytest.approx(S.theta(w0, T) / (m * MVV2E * w0 ** 2), rel=0.05)
    # centroid-mode estimator (slot 19): the centroid's kinetic energy plus the virial
    # term (m w0^2 / 2P) sum_{k>0} <q_k^2>, each mode by quadrature; ~theta/2
    q2 = [_quad_x2_v2(dens, np.sqrt(w0 ** 2 / P + wk[k] ** 2), gamma, m, np.pi / dt)[0] for k in range(P)]
    v2_0 = _quad_x2_v2(dens, w0 / np.sqrt(P), gamma, m, np.pi / dt)[1]
    K_q = 0.5 * m * MVV2E * v2_0 + 0.5 * m * MVV2E * w0 ** 2 / P * np.sum(q2[1:])
    Kcv0 = ser[:, 19] / (3 * 1000)
    assert abs(Kcv0.mean() - K_q) < 4 * _block_sigma(Kcv0, 16) + 5e-3 * K_q, (Kcv0.mean(), K_q)
    assert K_q == pytest.approx(0.5 * float(S.theta(w0, T)), rel=0.05)


@pytest.mark.parametrize("P", [4, 8])
def test_pimd_harmonic_centroid_virial_closed_form(qtb, P):
    # standard PIMD (white bath): <K_cv> = <V> = E_P / 2 per dof (Eqs. 3, 5, 11), with a
    # fluctuation well below that of the primitive estimator
    w0, gamma, dt, m = 0.1, 0.01, 0.5, 1.008
    T = HBAR * w0 / (3.0 * KB)                       # beta hbar w0 = 3
    sysd, pot = W.oscillators(1000, T, gamma, n_beads=P, mass=m)
    ctx = gpu_ctx(qtb, [sysd], pot, dt, precision=0, seed=78, potential=qtb.POT_HARMONIC, ext={"omega": w0},
                  max_records=20000)
    try:
        qtb.qtb_step_n(ctx, 4096 + 16384)
        ser = qtb.qtb_get_series(ctx, 0, 20000)[-16384:]
    finally:
        qtb.qtb_destroy(ctx)
    k = np.arange(P)
    E_P = KB * T * np.sum(1.0 / (1.0 + (2 * P / 3.0) ** 2 * np.sin(k * np.pi / P) ** 2))
    Kcv = ser[:, 18] / 3000.0
    assert abs(Kcv.mean() - 0.5 * E_P) < 4 * _block_sigma(Kcv, 16) + 3e-3 * E_P, (Kcv.mean(), 0.5 * E_P)
    assert ser[:, 18].std() < 0.5 * (ser[:, 4] - ser[:, 2]).std()
