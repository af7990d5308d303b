"""Parity of the tensor-core (tcgen05, BF16 operands, FP32 accumulation)
Toeplitz-GEMM noise filter against the FP64 oracle's direct convolution.

BF16 rounds the white noise and the taps to 8 significant bits (relative
error 2^-9 each), so each product carries ~2^-8 relative error, and the sum of
L independent such products has an RMS error of about 2^-8 of RMS(eta) / sqrt(3).
The bound used is RMS(eta_tc - eta_oracle) <= 4 * 2^-8 RMS(eta); the FP32
accumulation itself is exact to ~1e-6.  The exact-arithmetic part is checked
by feeding BF16-representable values: with taps and noise rounded to BF16 on the
oracle side, the tensor-core result must agree to FP32 accumulation accuracy."""
import numpy as np
import pytest

from helpers import gpu_ctx
from oracle import spectra as S
from paper_1905_02521_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qtb():
    import torch
    assert torch.cuda.is_available()
    from paper_1905_02521_gb300 import build
    build.build()
    from paper_1905_02521_gb300 import qtb as q
    return q


def bf16(x):
    """Round-to-nearest-even to bfloat16, returned as float64."""
    a = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("L,ncell,block", [(513, 2, 1), (2049, 3, 2), (257, 2, 0)])
def test_tc_filter_matches_oracle(qtb, oracle, L, ncell, block):
    s, pot = W.mgo_system(ncell, 300.0)
    N = len(s["types"])
    D = 3 * N
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=1, filter_prec=2, seed=4242)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, L, 0.3)
        if block:
            qtb.qtb_step_n(ctx, 256 * block + 3)
        eta, blk = qtb.qtb_get_noise(ctx, 0, D)
        assert blk == block
        h = S.taps(L, 1.0, 300.0, 0.3)
        sel = np.unique(np.r_[0, 1, 127, 128, D // 2, D - 1])
        ref = np.stack([oracle.colored_block(4242, 0, D, 256 * block, 256, h)[k] for k in sel]).T
        got = eta[:, sel]
        rms = np.sqrt((ref ** 2).mean())
        err = np.sqrt(((got - ref) ** 2).mean())
        assert err < 4 * 2.0 ** -8 * rms, (err / rms)
        # the same convolution with BF16-rounded operands: only FP32 accumulation error remains
        K = len(h) - 1
        Ke = 256 * ((K + 255) // 256)
        hb = bf16(h)
        for col, k in enumerate(sel):
            xi = bf16(oracle.white_block(4242, 0, D, 256 * block - Ke, 256 + 2 * Ke)[k])
            exact = np.array([sum(hb[abs(m)] * xi[j + Ke - m] for m in range(-K, K + 1)) for j in range(256)])
            assert np.abs(got[:, col] - exact).max() < 2e-5 * max(np.abs(exact).max(), 1e-30)
    finally:
        qtb.qtb_destroy(ctx)


def test_tc_filter_white_limit_and_batched_systems(qtb, oracle):
    # one system white (K = 0, taps = sqrt(kT) delta), one QTB with 1025 taps,
    # in one context: the band of each system is its own
    sa, pot = W.mgo_system(2, 200.0, seed=1)
    sb, _ = W.mgo_system(2, 600.0, seed=2)
    ctx = gpu_ctx(qtb, [sa, sb], pot, 1.0, precision=1, filter_prec=2, seed=77)
    try:
        qtb.qtb_set_filter(ctx, 1, qtb.NOISE_QTB, 1025, 0.3)
        eta_a, _ = qtb.qtb_get_noise(ctx, 0, 192)
        eta_b, _ = qtb.qtb_get_noise(ctx, 1, 192)
        kT = 8.617333262e-5 * 200.0
        xi = oracle.white_block(77, 0, 192, 0, 256).T
        # FP32 and FP64 Box-Muller may round to neighbouring BF16 values: one BF16 ulp
        ref_a = bf16(np.sqrt(kT)) * bf16(xi)
        assert np.all(np.abs(eta_a - ref_a) <= 2.0 ** -7 * np.abs(ref_a) + 1e-7)
        assert np.sqrt(((eta_a - ref_a) ** 2).mean()) < 1e-3 * np.sqrt((ref_a ** 2).mean())
        h = S.taps(1025, 1.0, 600.0, 0.3)
        ref = oracle.colored_block(77, 1, 192, 0, 256, h).T
        rms = np.sqrt((ref ** 2).mean())
        assert np.sqrt(((eta_b - ref) ** 2).mean()) < 4 * 2.0 ** -8 * rms
    finally:
        qtb.qtb_destroy(ctx)
