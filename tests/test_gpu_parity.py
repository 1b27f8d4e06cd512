"""GPU parity: every step of the CUDA path (through the C ABI) against the FP64
CPU oracle on the same seeded inputs.

Tolerances (FP64 path): factors within 1e-11 relative (per block, max norm),
spike tips / Rbar within 1e-11, preconditioner output within 1e-11, final
solutions ||x - x_oracle|| / ||x_oracle|| <= 1e-8 with true relres <= 1e-10.
FP32 preconditioner: factors within 64 K u32 relative; the FP64 outer
iteration still has to reach relres <= 1e-10 and the 1e-8 solution match."""
import numpy as np
import pytest
import torch

import oracle as O
import sap_inputs as G

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def sap():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1509_07919_gb300 as S
    return S


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def make(N, K, d, seed):
    band = G.dense_banded(N, K, d, seed)
    xt = G.x_true(N, seed)
    b = O.spmv(band, N, K, xt)
    return band, xt, b


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def maxerr(a, b):
    """Largest entrywise difference relative to the largest entry of b: a wrong
    value on a few entries (a seam row, a purification term) cannot hide in a
    norm."""
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ------------------------------------------------------------------ SpMV --

@pytest.mark.parametrize("N,K", [(10007, 7), (1000, 50), (513, 1), (300, 127)])
def test_spmv_parity(sap, N, K):
    band, xt, _ = make(N, K, 1.0, 100 + K)
    # poison the padding slots: the kernel must not read them
    bp = band.reshape(2 * K + 1, N).copy()
    for c in range(2 * K + 1):
        lo, hi = max(0, K - c), min(N, N + K - c)
        bp[c, :lo] = np.nan
        bp[c, hi:] = np.nan
    bd = dev(bp.reshape(-1))
    x = dev(xt)
    for tr in (False, True):
        y = host(sap.sap_spmv(bd, N, K, x, transpose=tr))
        yo = O.spmv(band, N, K, xt, transpose=tr)
        scale = O.spmv(np.abs(band), N, K, np.abs(xt), transpose=tr)
        assert np.all(np.abs(y - yo) <= 1e-14 * scale + 1e-300), (tr, np.abs(y - yo).max())


# ------------------------------------------------------------- factors --

@pytest.mark.parametrize("N,K,P", [(2000, 10, 8), (4003, 50, 4), (997, 33, 5), (600, 1, 3), (1500, 64, 2),
                                   (700, 90, 3), (1000, 128, 2), (1200, 129, 2), (1100, 256, 2)])
def test_block_lu_parity_fp64(sap, N, K, P):
    """K <= 128: the factor window in shared memory; K > 128: in global memory."""
    band, _, _ = make(N, K, 1.0, 200 + K)
    h = sap.sap_factor(dev(band), N, K, P=P, variant=sap.SAP_D, precision=sap.SAP_FP64)
    o = O.Sap(band, N, K, P, O.SAP_D)
    assert list(sap.sap_get_partition(h)) == list(o.offsets)
    for i in range(P):
        fg, fo = sap.sap_get_block_lu(h, i), o.block(i, 0)
        assert np.abs(fg - fo).max() <= 1e-11 * np.abs(fo).max(), (i, np.abs(fg - fo).max())
    assert sap.sap_n_boosted(h) == 0 == o.n_boosted


@pytest.mark.parametrize("N,K,P", [(4003, 50, 4), (2000, 10, 8), (700, 100, 3), (1000, 127, 3), (1300, 200, 2),
                                   (900, 208, 2), (900, 209, 2), (1700, 400, 2), (1500, 512, 2)])
def test_block_lu_parity_fp32(sap, N, K, P):
    """K <= 208: the factor window in shared memory; K > 208: in global memory
    (the last case with blocks narrower than the band)."""
    band, _, _ = make(N, K, 1.0, 300 + K)
    h = sap.sap_factor(dev(band), N, K, P=P, variant=sap.SAP_D, precision=sap.SAP_FP32)
    o = O.Sap(band, N, K, P, O.SAP_D)
    for i in range(P):
        fg, fo = sap.sap_get_block_lu(h, i), o.block(i, 0)
        assert np.abs(fg - fo).max() <= 64 * K * U32 * np.abs(fo).max()


@pytest.mark.parametrize("N,K,P,prec,variant", [(4000, 10, 7, 1, 1), (8000, 50, 6, 1, 1), (8000, 50, 6, 0, 1),
                                                (6000, 100, 4, 1, 0), (4004, 1, 9, 1, 0), (6000, 64, 3, 0, 0),
                                                (7000, 120, 5, 1, 1), (4096, 33, 3, 0, 1)])
def test_lu_tma_staging_equals_cp_async_staging(sap, monkeypatch, N, K, P, prec, variant):
    """The block LU / UL with the band staged by TMA boxes (default) and with the
    per-element cp.async staging (SAP_LU_STAGING=cp_async) run the same
    arithmetic in the same order on the same values: the factors, and for
    SaP-C the spike tips built from the UL tiles, agree bit for bit."""
    band, _, _ = make(N, K, 1.0, 1300 + K)
    bd = dev(band)
    h1 = sap.sap_factor(bd, N, K, P=P, variant=variant, precision=prec)
    monkeypatch.setenv("SAP_LU_STAGING", "cp_async")
    h2 = sap.sap_factor(bd, N, K, P=P, variant=variant, precision=prec)
    monkeypatch.delenv("SAP_LU_STAGING")
    for i in range(P):
        np.testing.assert_array_equal(sap.sap_get_block_lu(h1, i), sap.sap_get_block_lu(h2, i))
    if variant == 1:
        for i in range(P - 1):
            for w in ("V", "W"):
                np.testing.assert_array_equal(sap.sap_get_interface(h1, i, w), sap.sap_get_interface(h2, i, w))
    o = O.Sap(band, N, K, P, variant)
    tol = 1e-11 if prec == 0 else 64 * K * U32
    for i in (0, P - 1):
        fo = o.block(i, 0)
        assert np.abs(sap.sap_get_block_lu(h1, i) - fo).max() <= tol * np.abs(fo).max()


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-4)])
@pytest.mark.parametrize("N,K,P", [(1200, 10, 5), (3001, 40, 6), (900, 64, 3), (2100, 99, 3), (1500, 130, 3)])
def test_spike_tips_and_rbar_parity(sap, N, K, P, prec, tol):
    """K = 99 (FP64) and K = 130 (both precisions) put the spike kernel's K x K
    matrices in its global workspace.  The coupling blocks B_i, C_{i+1} have no
    copy of their own on the GPU (the kernels read them in place from the band);
    test_apply_reads_the_coupling_blocks checks that reading."""
    band, _, _ = make(N, K, 1.0, 400 + K)
    h = sap.sap_factor(dev(band), N, K, P=P, variant=sap.SAP_C, precision=prec)
    o = O.Sap(band, N, K, P, O.SAP_C)
    bt = O.transpose_band(band, N, K)
    oa = O.Sap(bt, N, K, P, O.SAP_C)
    for i in range(P - 1):
        for w in ("V", "W", "R"):
            g, r = sap.sap_get_interface(h, i, w), o.interface(i, w)
            assert np.abs(g - r).max() <= tol * max(np.abs(r).max(), 1.0), (i, w, np.abs(g - r).max())
            ga, ra = sap.sap_get_interface(h, i, w, adjoint=True), oa.interface(i, w)
            assert np.abs(ga - ra).max() <= tol * max(np.abs(ra).max(), 1.0), ("adj", i, w)


# --------------------------------------------------------------- apply --

@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("N,K,P", [(2000, 10, 8), (4003, 50, 4), (1111, 33, 3), (777, 5, 1)])
def test_apply_parity(sap, variant, N, K, P):
    band, _, _ = make(N, K, 1.0, 500 + K)
    r = G.adjoint_seed(N, 500 + K)
    for prec, tol in ((0, 1e-11), (1, 1e-4)):
        h = sap.sap_factor(dev(band), N, K, P=P, variant=variant, precision=prec)
        o = O.Sap(band, N, K, P, variant)
        z = host(sap.sap_apply_preconditioner(h, dev(r)))
        zo = o.apply(r)
        assert maxerr(z, zo) <= tol, (prec, maxerr(z, zo))
        oa = O.Sap(O.transpose_band(band, N, K), N, K, P, variant)
        za = host(sap.sap_apply_preconditioner(h, dev(r), transpose=True))
        assert maxerr(za, oa.apply(r)) <= tol, (prec, "adjoint", maxerr(za, oa.apply(r)))


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-4)])
@pytest.mark.parametrize("N,K,P", [(1200, 10, 5), (3001, 40, 6), (2100, 99, 3), (1500, 130, 3)])
def test_apply_reads_the_coupling_blocks(sap, prec, tol, N, K, P):
    """SaP-C apply of vectors supported on the 2K rows around one interface
    (the rows that B_i and C_{i+1} couple, Eq. (2.5)), forward and transposed,
    entry by entry against the oracle, whose B_i / C_{i+1} are explicit copies:
    a wrong coupling entry read by the tip, reduced-solve or purification
    kernels changes these outputs directly."""
    band, _, _ = make(N, K, 1.0, 450 + K)
    h = sap.sap_factor(dev(band), N, K, P=P, variant=sap.SAP_C, precision=prec)
    o = O.Sap(band, N, K, P, O.SAP_C)
    oa = O.Sap(O.transpose_band(band, N, K), N, K, P, O.SAP_C)
    off = o.offsets
    rng = np.random.default_rng(K)
    for i in range(P - 1):
        sr = int(off[i + 1])
        for lo, hi in ((sr - K, sr), (sr, sr + K), (sr - K, sr + K)):
            r = np.zeros(N)
            r[lo:hi] = rng.uniform(-1, 1, hi - lo)
            z = host(sap.sap_apply_preconditioner(h, dev(r)))
            assert maxerr(z, o.apply(r)) <= tol, (i, lo, hi, maxerr(z, o.apply(r)))
            za = host(sap.sap_apply_preconditioner(h, dev(r), transpose=True))
            assert maxerr(za, oa.apply(r)) <= tol, ("adj", i, lo, hi, maxerr(za, oa.apply(r)))


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("N,K,P", [(4003, 50, 2), (3001, 100, 3), (2500, 20, 1), (1111, 33, 3), (5000, 127, 2)])
def test_segmented_sweeps_parity(sap, variant, N, K, P):
    """Sweeps split into S concurrent segments (two passes with transfer
    matrices) against the oracle's apply, forward and transposed, for explicit
    segment counts; the count in use is reported and lowered to keep every
    full segment at least max(ceil(K/32), 2) chunks of 32 rows."""
    band, xt, b = make(N, K, 1.0, 800 + K)
    r = G.adjoint_seed(N, 800 + K)
    o = O.Sap(band, N, K, P, variant)
    oa = O.Sap(O.transpose_band(band, N, K), N, K, P, variant)
    zo, zao = o.apply(r), oa.apply(r)
    nmin = N // P
    ng = -(-K // 32)
    for prec, tol in ((0, 1e-11), (1, 1e-4)):
        if K > sap.sap_max_K(prec) or (variant == 1 and K > (98 if prec == 0 else 120)):
            continue
        for S in (1, 2, 3, 7, 1000):
            h = sap.sap_factor(dev(band), N, K, P=P, variant=variant, precision=prec, segments=S)
            z = host(sap.sap_apply_preconditioner(h, dev(r)))
            assert maxerr(z, zo) <= tol, (prec, S, maxerr(z, zo))
            za = host(sap.sap_apply_preconditioner(h, dev(r), transpose=True))
            assert maxerr(za, zao) <= tol, (prec, S, "adjoint", maxerr(za, zao))
            x, info, st = sap.sap_solve(h, dev(b))
            assert st == sap.SAP_OK and info.relres <= 1e-10
            assert 1 <= info.segments <= S
            assert info.segments <= max(1, (-(-nmin // 32)) // max(ng, 2))
            if S == 1:
                assert info.segments == 1


# --------------------------------------------------------------- solve --

@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("N,K,P,d", [(10000, 10, 8, 1.2), (6007, 50, 6, 1.0), (3000, 20, 10, 0.8)])
def test_solve_parity(sap, variant, prec, N, K, P, d):
    band, xt, b = make(N, K, d, 600 + K)
    xo, io, _ = O.solve(band, N, K, b, P, variant)
    assert io.status == O.OK
    h = sap.sap_factor(dev(band), N, K, P=P, variant=variant, precision=prec)
    x, info, st = sap.sap_solve(h, dev(b))
    x = host(x)
    assert st == sap.SAP_OK
    assert info.graphed == 1                     # the iteration ran as a captured CUDA graph
    assert info.relres <= 1e-10
    assert np.linalg.norm(b - O.spmv(band, N, K, x)) / np.linalg.norm(b) <= 1e-10
    assert relerr(x, xo) <= 1e-8
    if prec == 0:
        assert abs(info.iters - io.iters) <= 0.5, (info.iters, io.iters)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_adjoint_and_grad_parity(sap, variant, prec):
    N, K, P = 5003, 30, 5
    band, xt, b = make(N, K, 1.0, 700)
    g = G.adjoint_seed(N, 700)
    lo, io, _ = O.solve_adjoint(band, N, K, g, P, variant)
    xo, _, _ = O.solve(band, N, K, b, P, variant)
    h = sap.sap_factor(dev(band), N, K, P=P, variant=variant, precision=prec)
    lam, info, st = sap.sap_solve_adjoint(h, dev(g))
    assert st == sap.SAP_OK and info.relres <= 1e-10
    assert relerr(host(lam), lo) <= 1e-8
    x, _, _ = sap.sap_solve(h, dev(b))
    gb = host(sap.sap_grad_band(h, lam, x))
    gbo = O.grad_band(N, K, lo, xo)
    assert np.abs(gb - gbo).max() <= 1e-8 * np.abs(gbo).max()
    pad = np.array([not (0 <= (k % N) + (k // N) - K < N) for k in range(band.size)])
    assert np.all(gb[pad] == 0.0)


def test_autograd_matches_oracle_and_fd(sap):
    """SapSolve.backward: dl/db = lambda, dl/dband = -lambda x^T (band), checked
    against the oracle gradient and against central differences of the GPU
    solve (tol 1e-14) on 60 sampled band entries and on every entry of b."""
    N, K, P = 1500, 8, 3
    band, xt, b = make(N, K, 1.0, 800)
    w = G.adjoint_seed(N, 800)
    bd = dev(band).requires_grad_(True)
    bb = dev(b).requires_grad_(True)
    x = sap.sap_solve_autograd(bd, bb, N, K, P=P, variant=sap.SAP_C, precision=sap.SAP_FP64, tol=1e-14)
    loss = (x * dev(w)).sum()
    loss.backward()
    lo, _, _ = O.solve_adjoint(band, N, K, w, P, O.SAP_C, tol=1e-14)
    xo, _, _ = O.solve(band, N, K, b, P, O.SAP_C, tol=1e-14)
    assert relerr(host(bb.grad), lo) <= 1e-8
    gbo = O.grad_band(N, K, lo, xo)
    assert np.abs(host(bd.grad) - gbo).max() <= 1e-8 * np.abs(gbo).max()
    # central differences of the GPU solve on sampled band entries and b entries
    rng = np.random.default_rng(1)
    valid = [k for k in range(band.size) if 0 <= (k % N) + (k // N) - K < N]

    # one handle on a private copy of the band: perturb in place and refactor
    work = dev(band)
    hh = sap.sap_factor(work, N, K, P=P, variant=sap.SAP_C, precision=sap.SAP_FP64, tol=1e-14)
    bdev = dev(b)
    wd = dev(w)

    def lossf_band(bnd):
        work.copy_(dev(bnd))
        sap.sap_refactor(hh)
        xx, _, _ = sap.sap_solve(hh, bdev)
        return float((xx * wd).sum())

    gband = host(bd.grad)
    for k in rng.choice(valid, 60, replace=False):
        hstep = 1e-5 * max(1.0, abs(band[k]))
        bp, bm = band.copy(), band.copy()
        bp[k] += hstep
        bm[k] -= hstep
        fd = (lossf_band(bp) - lossf_band(bm)) / (2 * hstep)
        assert abs(fd - gband[k]) <= 1e-6 * max(1.0, abs(gband[k])), (k, fd, gband[k])
    # every entry of b (l is linear in b, so the difference quotient is exact up to the solve)
    work.copy_(dev(band))
    sap.sap_refactor(hh)
    gb = host(bb.grad)
    for k in range(N):
        hstep = 1e-5 * max(1.0, abs(b[k]))
        bp, bm = bdev.clone(), bdev.clone()
        bp[k] += hstep
        bm[k] -= hstep
        xp, _, _ = sap.sap_solve(hh, bp)
        xm, _, _ = sap.sap_solve(hh, bm)
        fd = float(((xp - xm) * wd).sum()) / (2 * hstep)
        assert abs(fd - gb[k]) <= 1e-6 * max(1.0, abs(gb[k])), (k, fd, gb[k])


# ------------------------------------------------------------ edge cases --

def test_invalid_arguments(sap):
    N, K = 100, 10
    band = dev(G.dense_banded(N, K, 1.0, 1))
    with pytest.raises(sap.SapError) as e:
        sap.sap_factor(band, N, K, P=8, variant=sap.SAP_C)        # N_i = 12 < 2K
    assert e.value.status == sap.SAP_ERR_INVALID_ARG
    with pytest.raises(sap.SapError):
        sap.sap_factor(band, N, N, P=1)                            # K >= N
    with pytest.raises(sap.SapError):
        sap.sap_factor(band, N, K, P=-1)
    # above the shared-memory limit of the sweep ring (two chunks ahead)
    assert sap.sap_max_K(sap.SAP_FP64) == 256 and sap.sap_max_K(sap.SAP_FP32) == 512
    with pytest.raises(sap.SapError) as e:
        sap.sap_factor(dev(G.dense_banded(600, 257, 1.0, 1)), 600, 257, P=1, precision=sap.SAP_FP64)
    assert e.value.status == sap.SAP_ERR_NOT_IMPLEMENTED
    with pytest.raises(sap.SapError) as e:
        sap.sap_factor(dev(G.dense_banded(1100, 513, 1.0, 1)), 1100, 513, P=1, precision=sap.SAP_FP32)
    assert e.value.status == sap.SAP_ERR_NOT_IMPLEMENTED
    with pytest.raises(sap.SapError) as e:          # the same limit for SaP-C
        sap.sap_factor(dev(G.dense_banded(4000, 257, 1.0, 1)), 4000, 257, P=2, variant=sap.SAP_C,
                       precision=sap.SAP_FP64)
    assert e.value.status == sap.SAP_ERR_NOT_IMPLEMENTED


def test_zero_rhs_and_p1_exact(sap):
    N, K = 3000, 12
    band, xt, b = make(N, K, 1.0, 900)
    h = sap.sap_factor(dev(band), N, K, P=1, precision=sap.SAP_FP64)
    x, info, st = sap.sap_solve(h, dev(np.zeros(N)))
    assert st == sap.SAP_OK and np.all(host(x) == 0.0)
    x, info, st = sap.sap_solve(h, dev(b))
    assert st == sap.SAP_OK and info.iters == 0.25 and info.n_matvec == 1
    assert relerr(host(x), xt) <= 1e-10


def test_boosted_pivot_matches_oracle(sap):
    """A zero pivot (Sec. 2.2) is boosted to +tau on both sides."""
    N, K = 64, 2
    A = np.diag(np.full(N, 4.0)) + np.diag(np.ones(N - 1), 1) + np.diag(np.ones(N - 1), -1)
    A[3, 3] = 0.0
    A[3, 2] = A[2, 3] = 0.0
    from tests._dense import dense_to_band
    band = dense_to_band(A, K)
    eps = 1e-3 / np.abs(A).max()
    h = sap.sap_factor(dev(band), N, K, P=1, precision=sap.SAP_FP64, boost_eps=eps)
    o = O.Sap(band, N, K, 1, O.SAP_D, boost_eps=eps)
    assert sap.sap_n_boosted(h) == o.n_boosted == 1
    np.testing.assert_allclose(sap.sap_get_block_lu(h, 0), o.block(0, 0), rtol=1e-13, atol=1e-15)


def test_not_converged_status(sap):
    N, K, P = 4000, 4, 400
    band, xt, b = make(N, K, 0.3, 901)
    h = sap.sap_factor(dev(band), N, K, P=P, variant=sap.SAP_D, precision=sap.SAP_FP64, max_iters=1)
    x, info, st = sap.sap_solve(h, dev(b), raise_on_error=False)
    assert st in (sap.SAP_ERR_NOT_CONVERGED, sap.SAP_OK)
    if st == sap.SAP_ERR_NOT_CONVERGED:
        assert info.relres > 1e-10


def test_bounded_wait_reports_timeout_and_context_survives(sap):
    """Failure detection without a GPU fault: a device wait on a barrier that
    nothing completes gives up after its poll limit and the call reports
    SAP_ERR_TIMEOUT; a solve afterwards still works (the context is intact)."""
    assert sap.sap_selftest_wait_timeout(1000) == sap.SAP_ERR_TIMEOUT
    assert sap.sap_selftest_wait_timeout(0) == sap.SAP_ERR_INVALID_ARG
    N, K, P = 3000, 6, 3
    band, xt, b = make(N, K, 1.0, 905)
    h = sap.sap_factor(dev(band), N, K, P=P, variant=sap.SAP_D, precision=sap.SAP_FP32)
    x, info, st = sap.sap_solve(h, dev(b))
    assert st == sap.SAP_OK and info.relres <= 1e-10
    assert np.linalg.norm(host(x) - xt) / np.linalg.norm(xt) <= 1e-8


@pytest.mark.parametrize("N,K,P,prec", [(20000, 200, 10, 1), (12000, 128, 6, 0), (9000, 170, 5, 1),
                                        (12000, 400, 6, 1), (8000, 250, 4, 0), (9000, 300, 3, 1),
                                        (6000, 512, 3, 1), (5000, 256, 2, 0)])
def test_wide_band_solve_parity(sap, N, K, P, prec):
    """Wide bands (K > 127, SaP-D; K = 200 and 400 of the K sweep, and the
    largest K of each precision, 512 and 256): 4 + couplings per chunk,
    unsegmented sweeps; above K = 208 (FP32) / 128 (FP64) the factor window
    lives in global memory, above K = 288 (FP32) / 128 (FP64) the sweep
    prefetches two chunks ahead instead of four."""
    band, xt, b = make(N, K, 1.0, 900 + K)
    xo, io, _ = O.solve(band, N, K, b, P, O.SAP_D)
    h = sap.sap_factor(dev(band), N, K, P=P, precision=prec)
    x, info, st = sap.sap_solve(h, dev(b))
    assert st == sap.SAP_OK and info.relres <= 1e-10
    assert relerr(host(x), xo) <= 1e-8
    g = G.adjoint_seed(N, 900 + K)
    lo, _, _ = O.solve_adjoint(band, N, K, g, P, O.SAP_D)
    lam, ainfo, ast = sap.sap_solve_adjoint(h, dev(g))
    assert ast == sap.SAP_OK and relerr(host(lam), lo) <= 1e-8


@pytest.mark.parametrize("N,K,P,prec", [(8000, 250, 4, 1), (6000, 150, 3, 0), (5000, 121, 4, 1), (6000, 256, 3, 0)])
def test_wide_band_sapc_solve_parity(sap, N, K, P, prec):
    """SaP-C with wide bands: UL windows and spike workspaces in global memory
    (K > 120 in FP32, K > 98 in FP64); forward and adjoint against the oracle."""
    band, xt, b = make(N, K, 1.0, 930 + K)
    xo, io, _ = O.solve(band, N, K, b, P, O.SAP_C)
    h = sap.sap_factor(dev(band), N, K, P=P, variant=sap.SAP_C, precision=prec)
    x, info, st = sap.sap_solve(h, dev(b))
    assert st == sap.SAP_OK and info.relres <= 1e-10
    assert relerr(host(x), xo) <= 1e-8
    g = G.adjoint_seed(N, 930 + K)
    lo, _, _ = O.solve_adjoint(band, N, K, g, P, O.SAP_C)
    lam, ainfo, ast = sap.sap_solve_adjoint(h, dev(g))
    assert ast == sap.SAP_OK and ainfo.relres <= 1e-10 and relerr(host(lam), lo) <= 1e-8


@pytest.mark.parametrize("nx,ny,P,prec", [(60, 40, 4, 1), (60, 40, 4, 0), (200, 130, 8, 1)])
def test_convection_diffusion_sapc_parity(sap, nx, ny, P, prec):
    """The sparse-in-band nonsymmetric convection-diffusion operator (5-point
    upwind, Peclet 10) treated as a dense band, SaP-C, against the oracle."""
    band, N, K = G.convection_diffusion(nx, ny)
    xt = G.x_true(N, G.config_seed(4))
    b = O.spmv(band, N, K, xt)
    xo, io, _ = O.solve(band, N, K, b, P, O.SAP_C)
    assert io.status == O.OK
    h = sap.sap_factor(dev(band), N, K, P=P, variant=sap.SAP_C, precision=prec)
    x, info, st = sap.sap_solve(h, dev(b))
    assert st == sap.SAP_OK and info.relres <= 1e-10
    assert relerr(host(x), xo) <= 1e-8


def test_autotune_picks_the_fastest_measured_candidate(sap):
    """The measured autotuner times refactor + solve for each (P, segments)
    candidate and returns the fastest; the default P grid is N / {16000 .. 1000}
    and one and two blocks per SM (152, 304) where N / P >= 64."""
    N, K = 60000, 50
    band, xt, b = make(N, K, 1.0, 950)
    bd = dev(band)
    P, S, table = sap.sap_autotune(bd, N, K, precision=sap.SAP_FP32)
    assert sorted(p for p, _ in table) == sorted({max(1, min(N // 64, (N + r // 2) // r))
                                                  for r in (16000, 8000, 4000, 2000, 1000)} | {152, 304})
    assert all(v > 0 for v in table.values())
    assert table[(P, S)] == min(table.values())
    P2, S2, t2 = sap.sap_autotune(bd, N, K, P_cands=[10, 20], seg_cands=[1, 4], b=dev(b),
                                  precision=sap.SAP_FP32)
    assert set(t2) == {(10, 1), (10, 4), (20, 1), (20, 4)} and (P2, S2) in t2
    h = sap.sap_factor(bd, N, K, P=P2, segments=S2, precision=sap.SAP_FP32)
    x, info, st = sap.sap_solve(h, dev(b))
    assert st == sap.SAP_OK and info.relres <= 1e-10


# ------------------------------------------------ full-size configuration --

def test_full_size_dense_banded_n200k_k50_p50(sap):
    """The N=200000, K=50, d=1, P=50 workload: SaP-D and SaP-C, FP64 and FP32
    preconditioners, against the oracle's solution."""
    N, K, P = 200000, 50, 50
    band, xt, b = make(N, K, 1.0, G.config_seed(2))
    bd = dev(band)
    for variant in (0, 1):
        xo, io, _ = O.solve(band, N, K, b, P, variant)
        for prec in (0, 1):
            h = sap.sap_factor(bd, N, K, P=P, variant=variant, precision=prec)
            x, info, st = sap.sap_solve(h, dev(b))
            assert st == sap.SAP_OK and info.relres <= 1e-10
            assert relerr(host(x), xo) <= 1e-8


@pytest.mark.parametrize("K", [100, 400])
def test_full_size_k_sweep_autotuned_p(sap, K):
    """The K sweep's N = 200000, d = 1 workloads at the partition count the
    autotuner picks (sap_factor with P = 0), FP32 preconditioner, through the
    concurrent forward + adjoint pair as the benchmark runs them: sampled block
    factors against the oracle's (K = 400: the many-CTA LU with its factor
    windows in global memory), the forward solution against the oracle's with
    the same P, and both true residuals recomputed on the host."""
    N = 200000
    seed = G.config_seed(3)
    band, xt, b = make(N, K, 1.0, seed)
    g = G.adjoint_seed(N, seed)
    h = sap.sap_factor(dev(band), N, K, P=0, variant=sap.SAP_D, precision=sap.SAP_FP32)
    P = sap.sap_num_partitions(h)
    assert P >= 50
    x, lam, ix, il, st = sap.sap_solve_pair(h, dev(b), dev(g))
    assert st == sap.SAP_OK and ix.relres <= 1e-10 and il.relres <= 1e-10 and ix.P == P
    xh, lh = host(x), host(lam)
    assert np.linalg.norm(b - O.spmv(band, N, K, xh)) / np.linalg.norm(b) <= 1e-10
    assert np.linalg.norm(g - O.spmv(band, N, K, lh, transpose=True)) / np.linalg.norm(g) <= 1e-10
    xo, io, o = O.solve(band, N, K, b, P, O.SAP_D)
    assert io.status == O.OK and relerr(xh, xo) <= 1e-8
    for i in (0, P // 2, P - 1):
        fg, fo = sap.sap_get_block_lu(h, i), o.block(i, 0)
        assert np.abs(fg - fo).max() <= 64 * K * U32 * np.abs(fo).max(), (i, np.abs(fg - fo).max())


def test_full_size_convection_diffusion_400x250_sapc_p32(sap):
    """The 400 x 250 convection-diffusion workload (N = 100000, K = 250), SaP-C,
    P = 32, FP32 preconditioner with FP64 BiCGStab(2): the true residual
    recomputed on the host, and the solution against the oracle's."""
    band, N, K = G.convection_diffusion(400, 250)
    assert (N, K) == (100000, 250)
    xt = G.x_true(N, G.config_seed(4))
    b = O.spmv(band, N, K, xt)
    h = sap.sap_factor(dev(band), N, K, P=32, variant=sap.SAP_C, precision=sap.SAP_FP32)
    x, info, st = sap.sap_solve(h, dev(b))
    assert st == sap.SAP_OK and info.relres <= 1e-10
    xh = host(x)
    assert np.linalg.norm(b - O.spmv(band, N, K, xh)) / np.linalg.norm(b) <= 1e-10
    xo, io, _ = O.solve(band, N, K, b, 32, O.SAP_C)
    assert io.status == O.OK and relerr(xh, xo) <= 1e-8


# ---------------------------------------------- concurrent fwd + adjoint --

@pytest.mark.parametrize("variant,prec,S", [(0, 1, 0), (0, 1, 1), (1, 1, 0), (0, 0, 0), (1, 0, 0)])
def test_solve_pair_equals_sequential_solves(sap, variant, prec, S):
    """sap_solve_pair runs the forward and adjoint iterations concurrently on
    separate workspaces: the same kernels in the same order per direction, so
    x and lambda equal the sequential sap_solve / sap_solve_adjoint results bit
    for bit, and the oracle's within the solve tolerances; twice in a row."""
    N, K, P = 6007, 50, 6
    band, xt, b = make(N, K, 1.0, 2100 + 10 * variant + prec)
    g = G.adjoint_seed(N, 2100)
    h = sap.sap_factor(dev(band), N, K, P=P, variant=variant, precision=prec, segments=S)
    xs, _, _ = sap.sap_solve(h, dev(b))
    ls, _, _ = sap.sap_solve_adjoint(h, dev(g))
    xo, _, _ = O.solve(band, N, K, b, P, variant)
    lo, _, _ = O.solve_adjoint(band, N, K, g, P, variant)
    for _ in range(2):
        x, lam, ix, il, st = sap.sap_solve_pair(h, dev(b), dev(g))
        assert st == sap.SAP_OK and ix.relres <= 1e-10 and il.relres <= 1e-10
        assert ix.graphed == 1 and il.graphed == 1
        assert torch.equal(x, xs) and torch.equal(lam, ls)
        assert relerr(host(x), xo) <= 1e-8 and relerr(host(lam), lo) <= 1e-8
    sap.sap_refactor(h)
    x, lam, ix, il, st = sap.sap_solve_pair(h, dev(b), dev(g))
    assert st == sap.SAP_OK and torch.equal(x, xs) and torch.equal(lam, ls)


def test_solve_pair_invalid_arguments(sap):
    N, K = 500, 5
    band, xt, b = make(N, K, 1.0, 2200)
    h = sap.sap_factor(dev(band), N, K, P=2)
    bd = dev(b)
    x = torch.empty_like(bd)
    assert sap.sap_solve_pair(h, bd, bd, x, x, raise_on_error=False)[4] == sap.SAP_ERR_INVALID_ARG
    assert sap.sap_solve_pair(h, bd, bd, bd, x, raise_on_error=False)[4] == sap.SAP_ERR_INVALID_ARG


def test_full_size_solve_pair_n200k_k50_p50(sap):
    """The N=200000, K=50, P=50 workload through the concurrent pair, FP32
    preconditioner: both results against the oracle."""
    N, K, P = 200000, 50, 50
    seed = G.config_seed(2)
    band, xt, b = make(N, K, 1.0, seed)
    g = G.adjoint_seed(N, seed)
    h = sap.sap_factor(dev(band), N, K, P=P, precision=sap.SAP_FP32)
    x, lam, ix, il, st = sap.sap_solve_pair(h, dev(b), dev(g))
    assert st == sap.SAP_OK and ix.relres <= 1e-10 and il.relres <= 1e-10
    xo, _, _ = O.solve(band, N, K, b, P, O.SAP_D)
    lo, _, _ = O.solve_adjoint(band, N, K, g, P, O.SAP_D)
    assert relerr(host(x), xo) <= 1e-8 and relerr(host(lam), lo) <= 1e-8


@pytest.mark.parametrize("N,K,P,variant,prec", [(8000, 250, 4, 1, 1), (5000, 130, 2, 0, 2), (3000, 20, 1, 0, 0),
                                                (9000, 120, 3, 1, 0)])
def test_solve_pair_wide_tc_and_p1(sap, N, K, P, variant, prec):
    """The pair on wide-band SaP-C (multi-CTA reduced solves, separate
    transposed scratch), on the tensor-core factorisation, and with P = 1:
    bit-identical to the sequential solves."""
    band, xt, b = make(N, K, 1.0, 2300 + K)
    g = G.adjoint_seed(N, 2300 + K)
    h = sap.sap_factor(dev(band), N, K, P=P, variant=variant, precision=prec)
    xs, ix0, _ = sap.sap_solve(h, dev(b))
    ls, il0, _ = sap.sap_solve_adjoint(h, dev(g))
    x, lam, ix, il, st = sap.sap_solve_pair(h, dev(b), dev(g))
    assert st == sap.SAP_OK and ix.relres <= 1e-10 and il.relres <= 1e-10
    assert torch.equal(x, xs) and torch.equal(lam, ls)
    assert ix.iters == ix0.iters and il.iters == il0.iters
    assert ix.tc_update == int(prec == 2 and 64 <= K <= 192)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("prec,N,K,P", [(1, 9000, 160, 3), (1, 12000, 250, 4), (1, 8000, 280, 2),
                                        (1, 12000, 400, 4), (0, 12000, 250, 4)])
def test_segmented_sweeps_wide_bands(sap, variant, prec, N, K, P):
    """Segmented sweeps with more than 4 couplings per chunk (on request; FP32
    up to K = 512, FP64 up to 256): the sweep kernel with 2 or 4 preparation
    warps, the transfer matrices and history responses of the wide kernel
    (history columns in tiles of 32), the chain with its matrices read from L2
    where one exceeds shared memory (K >= 250) and histories longer than its
    thread count (K = 280, 400), forward and transposed applies against the
    oracle entry by entry, and a solve."""
    band, xt, b = make(N, K, 1.0, 900 + K)
    r = G.adjoint_seed(N, 900 + K)
    zo = O.Sap(band, N, K, P, variant).apply(r)
    zao = O.Sap(O.transpose_band(band, N, K), N, K, P, variant).apply(r)
    tol = 1e-11 if prec == 0 else 1e-4
    for S in (2, 3, 6):
        h = sap.sap_factor(dev(band), N, K, P=P, variant=variant, precision=prec, segments=S)
        z = host(sap.sap_apply_preconditioner(h, dev(r)))
        assert maxerr(z, zo) <= tol, (S, maxerr(z, zo))
        za = host(sap.sap_apply_preconditioner(h, dev(r), transpose=True))
        assert maxerr(za, zao) <= tol, (S, "adjoint", maxerr(za, zao))
        x, info, st = sap.sap_solve(h, dev(b))
        assert st == sap.SAP_OK and info.relres <= 1e-10
        assert info.segments == S
