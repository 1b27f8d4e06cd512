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


def _noalloc(S, band, N, K, b, x, prec):
    """Call the C entry point directly through the C ABI."""
    fn = S._lib.sap_band_solve_noalloc
    return fn(ctypes.c_void_p(band.data_ptr()), N, K, ctypes.c_void_p(b.data_ptr()),
              ctypes.c_void_p(x.data_ptr()), prec, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


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
        st = _noalloc(sap, band, N, K, b, x, prec)
        assert st == sap.SAP_OK, sap.sap_status_string(st)
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
