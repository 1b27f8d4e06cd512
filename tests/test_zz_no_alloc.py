"""The allocation-free direct solve, sap_band_solve_noalloc, against the
existing entry points that allocate (sap_factor with P = 1, SaP-D, plus
sap_apply_preconditioner): the same kernels, so the results must agree to the
tolerance the apply parity tests use, on two calls in a row (the second call
reuses the scratch array the first one left behind).

It exists for callers that cannot call cudaMalloc.  This file is named so that
pytest collects it last."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
import sap_inputs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sap():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1509_07919_gb300 as S
    return S


def _noalloc(S, band, N, K, b, x, prec, timeout=None):
    """Call the C entry point directly through the C ABI."""
    fn = S._lib.sap_band_solve_noalloc
    return fn(ctypes.c_void_p(band.data_ptr()), N, K, ctypes.c_void_p(b.data_ptr()),
              ctypes.c_void_p(x.data_ptr()), prec,
              ctypes.c_void_p(timeout.data_ptr()) if timeout is not None else None,
              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _need(N, K, s):
    """Scratch bytes of one call, the formula documented in include/sap.h."""
    r = lambda v: (v + 255) // 256 * 256
    n = (N + 31) // 32 * 32
    W = 2 * K + 1
    t = 256 + r(n * W * s) + 2 * r(n * 32 * (1 + (K + 31) // 32) * s) + r((2 * N + 2 * K + 8) * 8)
    if s == 4:
        t += r(N * W * 4)
    if K > (208 if s == 4 else 128):
        M = (K + 16 + 15) // 16 * 16
        t += r(M * (M + 4) * s)
    return t


@pytest.mark.parametrize("prec,tol,N,K", [(0, 1e-11, 20011, 25), (0, 1e-11, 4000, 50), (1, 1e-4, 20011, 25),
                                          (1, 1e-4, 4000, 50), (0, 1e-11, 2500, 200), (1, 1e-4, 3000, 300)])
def test_noalloc_matches_allocating_path_twice(sap, prec, tol, N, K):
    """The last two sizes put the factor window in the scratch array (bands
    too wide for a shared-memory window)."""
    band_np = G.dense_banded(N, K, 1.0, 4242 + K)
    band = torch.from_numpy(band_np).cuda()
    h = sap.sap_factor(band, N, K, P=1, variant=sap.SAP_D, precision=prec)
    for call in range(2):
        b_np = G.adjoint_seed(N, 17 + call)
        b = torch.from_numpy(b_np).cuda()
        x = torch.full_like(b, float("nan"))
        flag = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        st = _noalloc(sap, band, N, K, b, x, prec, flag if call == 0 else None)
        assert st == sap.SAP_OK, sap.sap_status_string(st)
        if call == 0:
            assert int(flag.item()) == 0        # no bounded wait gave up
        ref = sap.sap_apply_preconditioner(h, b)
        torch.cuda.synchronize()
        xs, rs = x.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(xs))
        assert np.linalg.norm(xs - rs) / np.linalg.norm(rs) <= tol, (call, np.linalg.norm(xs - rs))
        # and it is the direct solve: P = 1 makes the preconditioner exact
        xo = O.Sap(band_np, N, K, 1, O.SAP_D).apply(b_np)
        assert np.linalg.norm(xs - xo) / np.linalg.norm(xo) <= (1e-10 if prec == 0 else 1e-3)


def test_noalloc_rejects_sizes_beyond_its_array(sap):
    N, K = 200000, 60          # (2K+1) N doubles > 32 MiB
    band = torch.zeros((2 * K + 1) * N, dtype=torch.float64, device="cuda")
    b = torch.zeros(N, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    assert _noalloc(sap, band, N, K, b, x, 0) == sap.SAP_ERR_INVALID_ARG
    assert _noalloc(sap, band, N, K, b, b, 0) == sap.SAP_ERR_INVALID_ARG


@pytest.mark.parametrize("prec,s,K,nmax", [(0, 8, 25, 23168), (1, 4, 25, 35840), (1, 4, 250, 16000)])
def test_noalloc_size_limit_is_the_documented_formula(sap, prec, s, K, nmax):
    """Sizes on both sides of the 32 MiB limit, by the header's formula (which
    counts the FP32 copy of the band and, for wide bands, the factor window):
    the largest N that fits solves, the next one is refused, and an FP32 size
    that only the factor and sweep terms would admit is refused too."""
    N = nmax
    while _need(N + 1, K, s) <= 1 << 25:
        N += 1
    while _need(N, K, s) > 1 << 25:
        N -= 1
    if nmax != 16000:
        assert N == nmax
    band_np = G.dense_banded(N, K, 1.0, 777 + K)
    band = torch.from_numpy(band_np).cuda()
    b_np = G.adjoint_seed(N, 5)
    b = torch.from_numpy(b_np).cuda()
    x = torch.full_like(b, float("nan"))
    assert _noalloc(sap, band, N, K, b, x, prec) == sap.SAP_OK
    ref = sap.sap_apply_preconditioner(sap.sap_factor(band, N, K, P=1, variant=sap.SAP_D, precision=prec), b)
    torch.cuda.synchronize()
    xs, rs = x.cpu().numpy(), ref.cpu().numpy()
    assert np.linalg.norm(xs - rs) / np.linalg.norm(rs) <= (1e-11 if prec == 0 else 1e-4)
    N2 = N + 1
    band2 = torch.zeros((2 * K + 1) * N2, dtype=torch.float64, device="cuda")
    b2 = torch.zeros(N2, dtype=torch.float64, device="cuda")
    x2 = torch.zeros_like(b2)
    assert _noalloc(sap, band2, N2, K, b2, x2, prec) == sap.SAP_ERR_INVALID_ARG
    if s == 4 and K == 25:
        N3 = 40000       # fits without the band copy (29.3 MB), not with it (37.4 MB)
        n3 = (N3 + 31) // 32 * 32
        assert n3 * 51 * 4 + 2 * n3 * 32 * 2 * 4 + (2 * N3 + 58) * 8 <= 1 << 25 < _need(N3, K, s)
        band3 = torch.zeros(51 * N3, dtype=torch.float64, device="cuda")
        b3 = torch.zeros(N3, dtype=torch.float64, device="cuda")
        assert _noalloc(sap, band3, N3, K, b3, torch.zeros_like(b3), prec) == sap.SAP_ERR_INVALID_ARG
