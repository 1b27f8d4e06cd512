"""GPU parity of the batched path (independent systems of their own N_i, K_i,
factored and solved together) against the FP64 CPU oracle, system by system:
every x_i to relres <= 1e-10 and within 1e-8 of the oracle's solution with the
same partition count, the adjoint lambda_i and the band gradient, the autograd
backward against central differences, and the uneven 64-system batch of
N ~ U{10^4..10^5}, K ~ U{8..64}."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def make_batch(specs, d):
    bands, xts, bs = [], [], []
    for N, K, seed in specs:
        band = G.dense_banded(N, K, d, seed)
        xt = G.x_true(N, seed)
        bands.append(band)
        xts.append(xt)
        bs.append(O.spmv(band, N, K, xt))
    return bands, xts, bs


SMALL = [(1500, 5, 11), (4003, 40, 12), (2500, 17, 13), (6000, 33, 14), (1999, 8, 15), (3200, 26, 16)]


@pytest.mark.parametrize("variant,prec", [(0, 1), (1, 0), (0, 0), (1, 1)])
def test_batched_solve_adjoint_grad_parity(sap, variant, prec):
    bands, xts, bs = make_batch(SMALL, 1.0)
    Ns = [s[0] for s in SMALL]
    Ks = [s[1] for s in SMALL]
    gs = [G.adjoint_seed(N, sd) for N, _, sd in SMALL]
    bds = [dev(b) for b in bands]
    bh = sap.sap_factor_batched(bds, Ns, Ks, variant=variant, precision=prec)
    Ps = sap.sap_batch_partitions(bh)
    assert len(Ps) == len(SMALL) and all(p >= 1 for p in Ps)
    xs, infos, stats, st = sap.sap_solve_batched(bh, [dev(b) for b in bs])
    assert st == sap.SAP_OK and all(v == sap.SAP_OK for v in stats)
    lams, ainfos, astats, ast = sap.sap_solve_adjoint_batched(bh, [dev(g) for g in gs])
    assert ast == sap.SAP_OK
    grads = sap.sap_grad_band_batched(bh, lams, xs)
    for i, (N, K, _) in enumerate(SMALL):
        x = host(xs[i])
        assert infos[i].relres <= 1e-10 and infos[i].graphed == 1
        assert np.linalg.norm(bs[i] - O.spmv(bands[i], N, K, x)) / np.linalg.norm(bs[i]) <= 1e-10
        xo, io, _ = O.solve(bands[i], N, K, bs[i], Ps[i], variant)
        assert io.status == O.OK
        assert relerr(x, xo) <= 1e-8, (i, relerr(x, xo))
        lo, _, _ = O.solve_adjoint(bands[i], N, K, gs[i], Ps[i], variant)
        assert ainfos[i].relres <= 1e-10
        assert relerr(host(lams[i]), lo) <= 1e-8, (i, "adjoint")
        gbo = O.grad_band(N, K, lo, xo)
        assert np.abs(host(grads[i]) - gbo).max() <= 1e-8 * np.abs(gbo).max()


def test_batched_refactor_and_explicit_partitions(sap):
    """Refactor after the band values change; an explicit P applies to every system."""
    bands, xts, bs = make_batch(SMALL[:3], 1.0)
    Ns = [s[0] for s in SMALL[:3]]
    Ks = [s[1] for s in SMALL[:3]]
    bds = [dev(b) for b in bands]
    bh = sap.sap_factor_batched(bds, Ns, Ks, P=2, precision=sap.SAP_FP64)
    assert sap.sap_batch_partitions(bh) == [2, 2, 2]
    bands2, _, bs2 = make_batch([(N, K, sd + 100) for N, K, sd in SMALL[:3]], 1.1)
    for bd, b2 in zip(bds, bands2):
        bd.copy_(dev(b2))
    sap.sap_refactor_batched(bh)
    xs, infos, _, st = sap.sap_solve_batched(bh, [dev(b) for b in bs2])
    assert st == sap.SAP_OK
    for i, (N, K, _) in enumerate(SMALL[:3]):
        xo, _, _ = O.solve(bands2[i], N, K, bs2[i], 2, O.SAP_D)
        assert relerr(host(xs[i]), xo) <= 1e-8


def test_batched_autograd_matches_oracle_and_fd(sap):
    specs = [(400, 3, 21), (650, 6, 22), (520, 4, 23)]
    bands, xts, bs = make_batch(specs, 1.0)
    Ns = [s[0] for s in specs]
    Ks = [s[1] for s in specs]
    ws = [G.adjoint_seed(N, sd) for N, _, sd in specs]
    bds = [dev(b).requires_grad_(True) for b in bands]
    bbs = [dev(b).requires_grad_(True) for b in bs]
    opts = dict(P=2, variant=sap.SAP_C, precision=sap.SAP_FP64, tol=1e-14)
    xs = sap.sap_solve_batched_autograd(bds, bbs, Ns, Ks, **opts)
    loss = sum((x * dev(w)).sum() for x, w in zip(xs, ws))
    loss.backward()
    rng = np.random.default_rng(3)
    for i, (N, K, _) in enumerate(specs):
        lo, _, _ = O.solve_adjoint(bands[i], N, K, ws[i], 2, O.SAP_C, tol=1e-14)
        xo, _, _ = O.solve(bands[i], N, K, bs[i], 2, O.SAP_C, tol=1e-14)
        assert relerr(host(bbs[i].grad), lo) <= 1e-8
        gbo = O.grad_band(N, K, lo, xo)
        assert np.abs(host(bds[i].grad) - gbo).max() <= 1e-8 * np.abs(gbo).max()
        # central differences on a few band entries of this system
        valid = [k for k in range(bands[i].size) if 0 <= (k % N) + (k // N) - K < N]

        def lossf(bnd):
            h = sap.sap_factor(dev(bnd), N, K, **opts)
            xx, _, _ = sap.sap_solve(h, dev(bs[i]))
            return float(host(xx) @ ws[i])

        gband = host(bds[i].grad)
        for k in rng.choice(valid, 4, replace=False):
            hstep = 1e-5 * max(1.0, abs(bands[i][k]))
            bp, bm = bands[i].copy(), bands[i].copy()
            bp[k] += hstep
            bm[k] -= hstep
            fd = (lossf(bp) - lossf(bm)) / (2 * hstep)
            assert abs(fd - gband[k]) <= 1e-6 * max(1.0, abs(gband[k])), (i, k, fd, gband[k])


def test_batch_of_64_uneven_systems(sap):
    """The 64-system batch, N ~ U{10^4..10^5}, K ~ U{8..64}, d = 1, FP32
    preconditioner with FP64 BiCGStab(2): every system to relres <= 1e-10 and
    within 1e-8 of the oracle's solution with the same partition count."""
    specs = G.batch_specs(64)
    bands, xts, bs = make_batch(specs, 1.0)
    Ns = [s[0] for s in specs]
    Ks = [s[1] for s in specs]
    bh = sap.sap_factor_batched([dev(b) for b in bands], Ns, Ks, precision=sap.SAP_FP32)
    Ps = sap.sap_batch_partitions(bh)
    xs, infos, stats, st = sap.sap_solve_batched(bh, [dev(b) for b in bs])
    assert st == sap.SAP_OK
    for i, (N, K, _) in enumerate(specs):
        assert infos[i].relres <= 1e-10, (i, infos[i].relres)
        x = host(xs[i])
        assert np.linalg.norm(bs[i] - O.spmv(bands[i], N, K, x)) / np.linalg.norm(bs[i]) <= 1e-10
        xo, io, _ = O.solve(bands[i], N, K, bs[i], Ps[i], O.SAP_D)
        assert io.status == O.OK
        assert relerr(x, xo) <= 1e-8, (i, relerr(x, xo))


def test_batch_with_a_wide_band_system(sap):
    """One system's window exceeds shared memory (K = 300): the persistent LU
    keeps every CTA's window in global memory."""
    specs = [(3000, 300, 41), (2500, 20, 42), (5000, 64, 43)]
    bands, xts, bs = make_batch(specs, 1.0)
    Ns = [s[0] for s in specs]
    Ks = [s[1] for s in specs]
    bh = sap.sap_factor_batched([dev(b) for b in bands], Ns, Ks, P=2, precision=sap.SAP_FP32)
    xs, infos, stats, st = sap.sap_solve_batched(bh, [dev(b) for b in bs])
    assert st == sap.SAP_OK
    for i, (N, K, _) in enumerate(specs):
        assert infos[i].relres <= 1e-10
        xo, _, _ = O.solve(bands[i], N, K, bs[i], 2, O.SAP_D)
        assert relerr(host(xs[i]), xo) <= 1e-8, (i, relerr(host(xs[i]), xo))


def test_batched_invalid_arguments(sap):
    band = dev(G.dense_banded(100, 3, 1.0, 5))
    with pytest.raises(sap.SapError):
        sap.sap_factor_batched([band], [100], [100])       # K >= N
    with pytest.raises(ValueError):
        sap.sap_factor_batched([band], [100, 50], [3])


def test_batched_pair_equals_sequential_batched_solves(sap):
    """sap_solve_pair_batched: every system's forward and adjoint iterations in
    the same lockstep rounds give what the separate batched calls give, bit
    for bit (FP32 preconditioner; SaP-D and SaP-C)."""
    for variant in (0, 1):
        bands, xts, bs = make_batch(SMALL[:4], 1.0)
        Ns = [s[0] for s in SMALL[:4]]
        Ks = [s[1] for s in SMALL[:4]]
        gs = [G.adjoint_seed(N, sd) for N, _, sd in SMALL[:4]]
        bh = sap.sap_factor_batched([dev(b) for b in bands], Ns, Ks, variant=variant, precision=sap.SAP_FP32)
        xs, _, _, st = sap.sap_solve_batched(bh, [dev(b) for b in bs])
        ls, _, _, ast = sap.sap_solve_adjoint_batched(bh, [dev(g) for g in gs])
        assert st == ast == sap.SAP_OK
        xp, lp, ix, il, stats, pst = sap.sap_solve_pair_batched(bh, [dev(b) for b in bs], [dev(g) for g in gs])
        assert pst == sap.SAP_OK and len(stats) == 8 and all(v == sap.SAP_OK for v in stats)
        for i in range(4):
            assert ix[i].relres <= 1e-10 and il[i].relres <= 1e-10
            assert torch.equal(xp[i], xs[i]) and torch.equal(lp[i], ls[i])
