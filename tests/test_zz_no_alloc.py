"""The allocation-free kappa_P entry point (qtb_kappa_solve_noalloc).

It is meant for callers that cannot allocate device memory: a process whose
device memory is all reserved by another allocator (cudaMalloc would fail) or a
latency-critical loop (an allocation can block and synchronise the device); its
scratch is a static device array in the library.  Its output must match the
allocating entry point qtb_kappa_solve within the kappa_P tolerance of the
parity tests, on two calls in a row (the second call reuses the array that the
first one left behind).  This file is collected last so that a failure here
never hides another test's result."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KAPPA_RTOL = 1e-6


@pytest.fixture(scope="module")
def qtb():
    import torch
    assert torch.cuda.is_available()
    from paper_1905_02521_gb300 import build
    build.build()
    from paper_1905_02521_gb300 import qtb as q
    return q


def test_noalloc_matches_allocating_solve_on_consecutive_calls(qtb):
    import torch
    n, ymax, y0 = 512, 400.0, 1.0
    stream = torch.cuda.Stream()
    for P in (8, 4, 8):
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        qtb.qtb_kappa_solve_noalloc(P, n, ymax, y0, out.data_ptr(), stream.cuda_stream)
        got = out.cpu().numpy()
        ref = qtb.qtb_kappa_solve(P, n=n, y_max=ymax, y0=y0)
        assert np.all(np.isfinite(got))
        assert np.allclose(got, ref, rtol=KAPPA_RTOL, atol=0)


def test_noalloc_one_bead_returns_theta_after_synchronising(qtb):
    # P = 1: kappa_1 = theta, no solve.  The call synchronises its stream before
    # returning, so the result is read on another stream without waiting.
    import torch
    n, ymax, y0 = 300, 400.0, 1.0
    stream = torch.cuda.Stream()
    ref = qtb.qtb_kappa_solve(1, n=n, y_max=ymax, y0=y0)
    for _ in range(2):
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        qtb.qtb_kappa_solve_noalloc(1, n, ymax, y0, out.data_ptr(), stream.cuda_stream)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.allclose(got, ref, rtol=KAPPA_RTOL, atol=0)


def test_noalloc_rejects_sizes_beyond_its_scratch(qtb):
    import torch
    out = torch.zeros(513, dtype=torch.float64, device="cuda")
    with pytest.raises(qtb.QtbError) as e:
        qtb.qtb_kappa_solve_noalloc(4, 513, 400.0, 1.0, out.data_ptr(), None)
    assert e.value.code == qtb.ERR_ARG and "512" in str(e.value)
