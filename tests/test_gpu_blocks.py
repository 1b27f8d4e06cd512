"""GPU tests of SaP with a bandwidth of its own per block (include/sap_blocks.h;
Sec. 2.2 third-stage reordering, Sec. 3.1 entire spikes) against the oracle
(oracle/blocks.py): the per-block Cuthill-McKee order (one deterministic rule
on both sides, so the permutations agree exactly), the blocks' half-bandwidths,
the spike tips and reduced matrices, the preconditioner apply entry by entry
(SaP-D and SaP-C, FP64 and FP32 factors, CM and random block numberings, a
global K above sap_max_K), solves, refactoring and the errors of the
operations the handle does not offer; the preconditioner of A^T (adjoint and pair
solves) against the oracle built on the transposed band with the same block
numbering."""
import numpy as np
import pytest
import torch

import oracle as O
import oracle.blocks as OB
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


def maxerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def system(N, K, P, d, seed):
    off = O.partition(N, P)
    return off, G.block_scrambled(N, K, off, d, seed)


def random_perm(off, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.permutation(int(off[i + 1] - off[i])) for i in range(len(off) - 1)])


TOL = {0: 1e-11, 1: 1e-4}


@pytest.mark.parametrize("N,K,P", [(24000, 24, 12), (6000, 40, 4), (600, 10, 4)])
def test_block_cm_is_the_oracles(sap, N, K, P):
    off, S = system(N, K, P, 1.0, 20 + K)
    perm, Ki = sap.sap_block_cm_reorder(dev(S.band), N, K, P)
    po, Ko = OB.block_cm(S.band, N, K, P)
    assert np.array_equal(host(perm).astype(np.int64), po)
    assert Ki == Ko.tolist()
    assert np.array_equal(Ko, S.k0)          # the hidden bandwidths are found again


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("N,K,P,order", [(24000, 24, 12, "cm"), (6000, 40, 4, "cm"), (600, 10, 4, "random"),
                                         (4000, 16, 1, "cm")])
def test_apply_parity(sap, prec, variant, N, K, P, order):
    off, S = system(N, K, P, 0.8, 30 + K)
    perm = OB.block_cm(S.band, N, K, P)[0] if order == "cm" else random_perm(off, K)
    band = dev(S.band)
    h = sap.sap_factor_blocks(band, N, K, dev(perm.astype(np.int32)), P=P, variant=variant, precision=prec)
    o = OB.BlockSap(S.band, N, K, P, perm, variant)
    assert sap.sap_get_block_bandwidths(h) == o.Ki.tolist()
    assert sap.sap_num_partitions(h) == P
    r = G.adjoint_seed(N, 31 + K)
    z = host(sap.sap_apply_preconditioner(h, dev(r)))
    assert maxerr(z, o.apply(r)) <= TOL[prec], maxerr(z, o.apply(r))
    # vectors on the 2K rows around one interface reach the tips and couplings directly
    rng = np.random.default_rng(K)
    for i in range(P - 1):
        sr = int(off[i + 1])
        r2 = np.zeros(N)
        r2[sr - K:sr + K] = rng.uniform(-1, 1, 2 * K)
        z2 = host(sap.sap_apply_preconditioner(h, dev(r2)))
        assert maxerr(z2, o.apply(r2)) <= TOL[prec], (i, maxerr(z2, o.apply(r2)))


@pytest.mark.parametrize("prec", [0, 1])
def test_tips_and_reduced_matrices(sap, prec):
    N, K, P = 24000, 24, 12
    off, S = system(N, K, P, 0.8, 40)
    perm = OB.block_cm(S.band, N, K, P)[0]
    h = sap.sap_factor_blocks(dev(S.band), N, K, dev(perm.astype(np.int32)), P=P, variant=1, precision=prec)
    o = OB.BlockSap(S.band, N, K, P, perm, O.SAP_C)
    tol = 1e-12 if prec == 0 else 2e-5
    for i in range(P - 1):
        for which, ref in (("V", o.Vb[i]), ("W", o.Wt[i]), ("R", o.R[i][0]), ("B", o.B[i]), ("C", o.C[i])):
            m = sap.sap_get_interface(h, i, which)
            assert np.abs(m - ref).max() <= tol * max(1.0, np.abs(ref).max()), (i, which)


@pytest.mark.parametrize("prec", [0, 1])
def test_global_bandwidth_above_the_limit(sap, prec):
    """K = 300 exceeds the FP64 limit of sap_factor; the reordered blocks'
    K_i <= 150 do not, so the per-block handle factors and solves it."""
    N, K, P = 20000, 300, 10
    off, S = system(N, K, P, 1.0, 50)
    if prec == 0:
        assert K > sap.sap_max_K(0)
        with pytest.raises(sap.SapError):
            sap.sap_factor(dev(S.band), N, K, P=P, variant=1, precision=0)
    perm, Ki = sap.sap_block_cm_reorder(dev(S.band), N, K, P)
    po, Ko = OB.block_cm(S.band, N, K, P)
    assert np.array_equal(host(perm).astype(np.int64), po) and max(Ko) <= 150
    h = sap.sap_factor_blocks(dev(S.band), N, K, dev(po.astype(np.int32)), P=P, variant=1, precision=prec)
    o = OB.BlockSap(S.band, N, K, P, po, O.SAP_C)
    r = G.adjoint_seed(N, 51)
    z = host(sap.sap_apply_preconditioner(h, dev(r)))
    assert maxerr(z, o.apply(r)) <= TOL[prec]
    xt = G.x_true(N, 52)
    b = O.spmv(S.band, N, K, xt)
    x, info, st = sap.sap_solve(h, dev(b))
    assert st == 0 and info.relres <= 1e-10
    assert np.abs(host(x) - xt).max() <= 1e-7


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("variant", [0, 1])
def test_solve_matches_the_unreordered_solver(sap, prec, variant):
    """Same preconditioner in exact arithmetic: the solution and (up to a
    quarter of an iteration from rounding) the iteration count of sap_factor's
    handle on the same matrix; the graph-driven iteration runs."""
    N, K, P = 24000, 24, 12
    off, S = system(N, K, P, 0.6, 60 + variant)
    band = dev(S.band)
    xt = G.x_true(N, 61)
    b = dev(O.spmv(S.band, N, K, xt))
    perm, _ = sap.sap_block_cm_reorder(band, N, K, P)
    hb = sap.sap_factor_blocks(band, N, K, perm, P=P, variant=variant, precision=prec)
    hp = sap.sap_factor(band, N, K, P=P, variant=variant, precision=prec)
    x, info, st = sap.sap_solve(hb, b)
    xp, infop, stp = sap.sap_solve(hp, b)
    assert st == 0 and stp == 0
    assert info.relres <= 1e-10 and info.graphed == 1
    assert abs(info.iters - infop.iters) <= 0.5, (info.iters, infop.iters)
    assert np.abs(host(x) - xt).max() <= 1e-8 * np.abs(xt).max() * 100
    # the host-buffer entry runs the same path
    xh = torch.empty(N, dtype=torch.float64)
    sap.sap_solve_host(hb, torch.from_numpy(O.spmv(S.band, N, K, xt)), xh)
    assert np.abs(xh.numpy() - host(x)).max() <= 1e-12 * np.abs(host(x)).max()


def test_refactor_and_pattern_change(sap):
    N, K, P = 6000, 40, 4
    off, S = system(N, K, P, 0.8, 70)
    band = dev(S.band)
    po, _ = OB.block_cm(S.band, N, K, P)
    perm = dev(po.astype(np.int32))
    h = sap.sap_factor_blocks(band, N, K, perm, P=P, variant=1, precision=0)
    b2 = S.band.copy()
    b2 *= np.linspace(0.5, 2.0, b2.size)                  # new values, same pattern
    band.copy_(torch.from_numpy(b2))
    sap.sap_refactor(h)
    o = OB.BlockSap(b2, N, K, P, po, O.SAP_C)
    r = G.adjoint_seed(N, 71)
    assert maxerr(host(sap.sap_apply_preconditioner(h, dev(r))), o.apply(r)) <= 1e-11
    # an entry inside the global band but outside its block's reordered band
    Ki = sap.sap_get_block_bandwidths(h)
    p0 = po[:int(off[1])]
    a, c = next((a, c) for a in range(int(off[1])) for c in range(max(0, a - K), min(int(off[1]), a + K + 1))
                if abs(int(p0[a]) - int(p0[c])) > Ki[0])
    b3 = b2.copy()
    b3[(K + a - c) * N + c] = 0.5
    band.copy_(torch.from_numpy(b3))
    with pytest.raises(sap.SapError) as e:
        sap.sap_refactor(h)
    assert e.value.status == sap.SAP_ERR_INVALID_ARG


def test_operations_not_offered(sap):
    N, K, P = 6000, 40, 4
    off, S = system(N, K, P, 0.8, 80)
    band = dev(S.band)
    perm, _ = sap.sap_block_cm_reorder(band, N, K, P)
    h = sap.sap_factor_blocks(band, N, K, perm, P=P, variant=1, precision=1)
    with pytest.raises(sap.SapError):
        sap.sap_get_block_lu(h, 0)
    with pytest.raises(sap.SapError):
        sap.sap_get_block_bandwidths(sap.sap_factor(band, N, K, P=P))
    bad = host(perm).copy()
    bad[1] = bad[0]                                       # not a permutation of block 0
    with pytest.raises(sap.SapError) as e:
        sap.sap_factor_blocks(band, N, K, dev(bad), P=P)
    assert e.value.status == sap.SAP_ERR_INVALID_ARG
    with pytest.raises(sap.SapError):
        sap.sap_factor_blocks(band, N, K, perm, P=0)


def test_full_size_bench_workload(sap):
    """The bench's workload (N = 200000, K = 100, P = 50, FP32 factors): the
    permutations and bandwidths equal the oracle's, and the SaP-C and SaP-D
    applies match it entry by entry."""
    N, K, P = 200000, 100, 50
    off, S = system(N, K, P, 1.0, 90)
    band = dev(S.band)
    perm, Ki = sap.sap_block_cm_reorder(band, N, K, P)
    po, Ko = OB.block_cm(S.band, N, K, P)
    assert np.array_equal(host(perm).astype(np.int64), po) and Ki == Ko.tolist()
    r = G.adjoint_seed(N, 91)
    for variant in (1, 0):
        h = sap.sap_factor_blocks(band, N, K, perm, P=P, variant=variant, precision=1)
        o = OB.BlockSap(S.band, N, K, P, po, variant)
        z = host(sap.sap_apply_preconditioner(h, dev(r)))
        assert maxerr(z, o.apply(r)) <= 1e-4


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("variant", [0, 1])
def test_transposed_preconditioner_and_adjoint_solves(sap, prec, variant):
    """The preconditioner of A^T (the blocks of A^T renumbered by the same
    permutations are the transposes of the reordered blocks; couplings
    B'_i = C_{i+1}^T, C'_{i+1} = B_i^T): its apply entry by entry, its tips and
    reduced matrices, the adjoint solve by its residual, the pair solve against
    the separate solves, and both directions again after a refactor."""
    N, K, P = 24000, 24, 12
    off, S = system(N, K, P, 0.8, 100 + variant)
    po, _ = OB.block_cm(S.band, N, K, P)
    band = dev(S.band)
    h = sap.sap_factor_blocks(band, N, K, dev(po.astype(np.int32)), P=P, variant=variant, precision=prec)
    bt = O.transpose_band(S.band, N, K)
    oa = OB.BlockSap(bt, N, K, P, po, variant)
    of = OB.BlockSap(S.band, N, K, P, po, variant)
    r = G.adjoint_seed(N, 101)
    za = host(sap.sap_apply_preconditioner(h, dev(r), transpose=True))
    assert maxerr(za, oa.apply(r)) <= TOL[prec]
    assert maxerr(host(sap.sap_apply_preconditioner(h, dev(r))), of.apply(r)) <= TOL[prec]
    if variant == 1:
        tol = 1e-12 if prec == 0 else 2e-5
        for i in range(P - 1):
            for which, ref in (("V", oa.Vb[i]), ("W", oa.Wt[i]), ("R", oa.R[i][0]), ("B", oa.B[i]), ("C", oa.C[i])):
                m = sap.sap_get_interface(h, i, which, adjoint=True)
                assert np.abs(m - ref).max() <= tol * max(1.0, np.abs(ref).max()), (i, which)
    g = G.adjoint_seed(N, 102)
    lam, info, st = sap.sap_solve_adjoint(h, dev(g))
    assert st == 0 and info.relres <= 1e-10 and info.graphed == 1
    res = g - O.spmv(S.band, N, K, host(lam), transpose=True)
    assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(g)
    xt = G.x_true(N, 103)
    b = O.spmv(S.band, N, K, xt)
    x1, _, _ = sap.sap_solve(h, dev(b))
    x2, l2, ix, il, st2 = sap.sap_solve_pair(h, dev(b), dev(g))
    assert st2 == 0
    assert np.abs(host(x2) - host(x1)).max() <= 1e-12 * np.abs(host(x1)).max()
    assert np.abs(host(l2) - host(lam)).max() <= 1e-12 * np.abs(host(lam)).max()
    # new values, same pattern: both directions follow
    b2 = S.band * np.linspace(0.7, 1.3, S.band.size)
    band.copy_(torch.from_numpy(b2))
    sap.sap_refactor(h)
    oa2 = OB.BlockSap(O.transpose_band(b2, N, K), N, K, P, po, variant)
    za2 = host(sap.sap_apply_preconditioner(h, dev(r), transpose=True))
    assert maxerr(za2, oa2.apply(r)) <= TOL[prec]


@pytest.mark.parametrize("prec,N,K", [(1, 4800, 800), (0, 3000, 480)])
def test_wide_blocks_take_the_narrow_spike_tiles(sap, prec, N, K):
    """Blocks so wide that the entire-spike kernel narrows its column tiles to
    fit shared memory (FP32: K_b > 352, 32 columns per CTA; FP64: K_b > 224,
    16 columns), with the reduced matrices of a global K of 800 / 480: the
    apply and the tips against the oracle, and a solve."""
    P = 2
    off = O.partition(N, P)
    S = G.block_scrambled(N, K, off, 1.0, 110, k0_lo=0.95)
    po, Ko = OB.block_cm(S.band, N, K, P)
    assert min(Ko) > (352 if prec == 1 else 224)
    h = sap.sap_factor_blocks(dev(S.band), N, K, dev(po.astype(np.int32)), P=P, variant=1, precision=prec)
    o = OB.BlockSap(S.band, N, K, P, po, O.SAP_C)
    r = G.adjoint_seed(N, 111)
    assert maxerr(host(sap.sap_apply_preconditioner(h, dev(r))), o.apply(r)) <= TOL[prec]
    tol = 1e-12 if prec == 0 else 2e-5
    for which, ref in (("V", o.Vb[0]), ("W", o.Wt[0])):
        m = sap.sap_get_interface(h, 0, which)
        assert np.abs(m - ref).max() <= tol * max(1.0, np.abs(ref).max()), which
    xt = G.x_true(N, 112)
    x, info, st = sap.sap_solve(h, dev(O.spmv(S.band, N, K, xt)))
    assert st == 0 and info.relres <= 1e-10
