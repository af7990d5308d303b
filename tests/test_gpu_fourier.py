"""The Fourier-segment generator (Eq. 9) on the GPU.

* the coloured noise of whole segments equals the oracle's (oracle/fourier.py,
  the same white stream, numpy's inverse FFT in FP64): 1e-12 norm-wise in the
  FP64 form, 1e-5 in the mixed form (FP32 transform), for segments of one and of
  four blocks and for consecutive segments;
* QTB harmonic oscillators driven by segments of 2048 steps reproduce
  theta(w0, T) as with the time-domain filter;
* QTB-PIMD segments (density kappa_P W, one stream per normal-mode dof) equal
  the oracle's.
"""
import numpy as np
import pytest

from helpers import gpu_ctx, rel_inf
from oracle import fourier as F
from oracle import spectra as S
from paper_1905_02521_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MVV2E = 103.64269652680505


@pytest.fixture(scope="module")
def qtb():
    import torch
    assert torch.cuda.is_available()
    from paper_1905_02521_gb300 import build
    build.build()
    from paper_1905_02521_gb300 import qtb as q
    return q


@pytest.mark.parametrize("M", [1, 4])
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_segments_match_oracle(qtb, oracle, M, precision, tol):
    T, dt, wmax, seed = 300.0, 1.0, 0.3, 777
    s, pot = W.mgo_system(2, T)
    D = 3 * len(s["types"])
    n = 256 * M
    ctx = gpu_ctx(qtb, [s], pot, dt, precision=precision, filter_prec=1, seed=seed)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 513, wmax)
        qtb.qtb_set_generator(ctx, qtb.GEN_FOURIER, M)
        blocks = []
        for b in range(2 * M):                      # two segments
            eta, blk = qtb.qtb_get_noise(ctx, 0, D)
            assert blk == b
            blocks.append(eta)                      # [256][D]
            qtb.qtb_step_n(ctx, 256)
    finally:
        qtb.qtb_destroy(ctx)
    Sj = F.segment_spectrum(n, dt, T, wmax)
    for seg in range(2):
        got = np.concatenate(blocks[seg * M:(seg + 1) * M], axis=0).T   # [D][n]
        ref = F.eq9_segment(seed, 0, D, seg, n, Sj)
        assert rel_inf(got, ref) < tol, (seg, rel_inf(got, ref))


def test_oscillators_with_fourier_segments_reproduce_theta(qtb):
    w0, T, gamma, dt, m = 0.1, 100.0, 0.01, 0.5, 1.008
    sysd, pot = W.oscillators(2000, T, gamma, mass=m)
    ctx = gpu_ctx(qtb, [sysd], pot, dt, precision=1, filter_prec=1, seed=31, potential=qtb.POT_HARMONIC,
                  ext={"omega": w0}, max_records=20000)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 513, 0.5)
        qtb.qtb_set_generator(ctx, qtb.GEN_FOURIER, 8)
        qtb.qtb_step_n(ctx, 2048)
        qtb.qtb_step_n(ctx, 16384)
        ser = qtb.qtb_get_series(ctx, 0, 20000)[-16384:]
    finally:
        qtb.qtb_destroy(ctx)
    E = (ser[:, 1] + ser[:, 2]) / (3 * 2000)
    assert E.mean() == pytest.approx(S.theta(w0, T), rel=0.05), (E.mean(), S.theta(w0, T))


@pytest.mark.parametrize("precision", [0, 1])
def test_qtb_pimd_segments_match_oracle(qtb, oracle, precision):
    # QTB-PIMD (Eq. 12): segments drawn with the density kappa_P W, one stream per
    # normal-mode dof.  The GPU's kappa_P (normal equations) and the oracle's (LAPACK)
    # agree to ~1e-6, hence 1e-5 here in both forms.
    T, dt, wmax, seed, P = 100.0, 0.5, 0.6, 778, 4
    s, pot = W.mgo_system(2, T, n_beads=P)
    D = 3 * len(s["types"]) * P
    ctx = gpu_ctx(qtb, [s], pot, dt, precision=precision, filter_prec=1, seed=seed)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB_PIMD, 513, wmax)
        qtb.qtb_set_generator(ctx, qtb.GEN_FOURIER, 1)
        eta, blk = qtb.qtb_get_noise(ctx, 0, D)
        assert blk == 0
    finally:
        qtb.qtb_destroy(ctx)
    Sj = F.segment_spectrum(256, dt, T, wmax, P=P, sol=S.kappa_solve(P))
    ref = F.eq9_segment(seed, 0, D, 0, 256, Sj)
    assert rel_inf(eta.T, ref) < 1e-5, rel_inf(eta.T, ref)
