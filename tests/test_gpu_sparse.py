"""GPU tests of the sparse front end (include/sap_sparse.h; Sec. 2.2, 3.2, 3.3)
against the oracle (oracle/sparse.py): the matching's objective (the optimum is
unique in value, not always in the permutation), the scale factors' I-matrix
property, the Cuthill-McKee order (one deterministic rule on both sides, so
the permutations agree exactly), the bandwidth, the band element by element,
the permutations of right-hand side and solution, and the whole path into
sap_factor / sap_solve against a dense solve."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import oracle.sparse as OS
import sap_inputs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sap():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1509_07919_gb300 as S
    return S


def to_dev(S, sysm):
    return S.Csr(sysm.n, torch.from_numpy(sysm.rowptr).cuda(), torch.from_numpy(sysm.col).cuda(),
                 torch.from_numpy(sysm.val).cuda())


def host(t):
    return t.detach().cpu().numpy()


def matching_cost(sysm, sigma):
    a, c = OS.db_costs(sysm.n, sysm.rowptr, sysm.col, sysm.val)
    tot = 0.0
    for i in range(sysm.n):
        lo, hi = sysm.rowptr[i], sysm.rowptr[i + 1]
        p = lo + np.searchsorted(sysm.col[lo:hi], sigma[i])
        assert p < hi and sysm.col[p] == sigma[i], "the matching uses an entry that is not stored"
        tot += c[p]
    return tot


@pytest.mark.parametrize("d,seed", [(1.5, 21), (0.3, 22), (0.05, 23)])
def test_db_matches_the_oracle_optimum(sap, d, seed):
    sysm = G.sparse_scrambled(160, 4, 0.5, d, seed)
    A = to_dev(sap, sysm)
    rownew, r, s, lp = sap.sap_db_reorder(A, scale=True)
    sigma = host(rownew).astype(np.int64)
    assert sorted(sigma.tolist()) == list(range(sysm.n))
    db = OS.db_match(sysm.n, sysm.rowptr, sysm.col, sysm.val)
    assert matching_cost(sysm, sigma) == pytest.approx(db.cost, abs=1e-10 * sysm.n)
    assert lp == pytest.approx(db.logprod, rel=1e-12, abs=1e-10)
    # I-matrix: |r_i a_ij s_j| <= 1, = 1 on the matching
    Ad = OS.csr_to_dense(sysm.n, sysm.rowptr, sysm.col, sysm.val)
    B = np.abs(host(r)[:, None] * Ad * host(s)[None, :])
    assert B.max() <= 1.0 + 1e-12
    assert np.allclose(B[np.arange(sysm.n), sigma], 1.0, rtol=0, atol=1e-12)


def test_db_recovers_the_hidden_rows_at_size(sap):
    """A strictly diagonally dominant matrix with shuffled rows has a unique
    optimal matching, the hidden one (n = 100000)."""
    sysm = G.sparse_scrambled(100000, 12, 0.3, 1.5, 24)
    rownew, _, _, _ = sap.sap_db_reorder(to_dev(sap, sysm), scale=False)
    assert np.array_equal(host(rownew), sysm.sym[sysm.rowsrc])


def test_db_reports_a_structurally_singular_matrix(sap):
    n = 4
    rowptr = np.array([0, 2, 4, 6, 8], dtype=np.int64)
    col = np.array([0, 1, 0, 1, 0, 1, 2, 3], dtype=np.int32)   # rows 0-2 only reach columns 0, 1
    val = np.ones(8)
    sysm = G.SparseSystem(n, rowptr, col, val, 0, np.arange(n), np.arange(n))
    with pytest.raises(sap.SapError) as e:
        sap.sap_db_reorder(to_dev(sap, sysm))
    assert e.value.status == sap.SAP_ERR_SINGULAR


@pytest.mark.parametrize("n,K0,seed", [(500, 3, 25), (3000, 10, 26), (2000, 2, 27)])
def test_cm_order_is_the_oracle_order(sap, n, K0, seed):
    sysm = G.sparse_scrambled(n, K0, 0.4, 1.2, seed)
    A = to_dev(sap, sysm)
    rownew, _, _, _ = sap.sap_db_reorder(A, scale=False)
    perm, K = sap.sap_cm_reorder(A, rownew)
    sigma = host(rownew).astype(np.int64)
    perm_o = OS.cm_order(n, OS.sym_pattern(n, sysm.rowptr, sysm.col, sigma))
    assert np.array_equal(host(perm), perm_o)
    K_o = OS.bandwidth(n, sysm.rowptr, sysm.col, perm_o[sigma], perm_o)
    assert K == K_o <= 2 * K0
    rn = sap.sap_perm_compose(perm, rownew)
    assert np.array_equal(host(rn), perm_o[sigma])
    assert sap.sap_sparse_bandwidth(A, rn, perm) == K_o


def test_cm_handles_several_components_and_no_rownew(sap):
    """Two disjoint scrambled bands (a block-diagonal matrix) and the identity
    row map."""
    s1 = G.sparse_scrambled(300, 3, 0.5, 1.5, 28)
    s2 = G.sparse_scrambled(200, 2, 0.5, 1.5, 29)
    n = 500
    rowptr = np.concatenate([s1.rowptr, s1.rowptr[-1] + s2.rowptr[1:]])
    col = np.concatenate([s1.col, s2.col + 300]).astype(np.int32)
    val = np.concatenate([s1.val, s2.val])
    sysm = G.SparseSystem(n, rowptr, col, val, 3, np.arange(n), np.arange(n))
    A = to_dev(sap, sysm)
    perm, K = sap.sap_cm_reorder(A, None)
    perm_o = OS.cm_order(n, OS.sym_pattern(n, rowptr, col, None))
    assert np.array_equal(host(perm), perm_o)
    assert K == OS.bandwidth(n, rowptr, col, perm_o, perm_o)


@pytest.mark.parametrize("scaled", [False, True])
def test_band_is_the_oracle_band(sap, scaled):
    sysm = G.sparse_scrambled(700, 5, 0.5, 0.8, 30)
    A = to_dev(sap, sysm)
    rownew, r, s, _ = sap.sap_db_reorder(A, scale=scaled)
    perm, K = sap.sap_cm_reorder(A, rownew)
    rn = sap.sap_perm_compose(perm, rownew)
    band = sap.sap_sparse_to_band(A, rn, perm, K, r, s)
    band_o = OS.to_band(sysm.n, sysm.rowptr, sysm.col, sysm.val, host(rn), host(perm), K,
                        host(r) if scaled else None, host(s) if scaled else None)
    np.testing.assert_array_equal(host(band), band_o)
    with pytest.raises(sap.SapError) as e:                   # an entry outside a too narrow band
        sap.sap_sparse_to_band(A, rn, perm, K - 1, r, s)
    assert e.value.status == sap.SAP_ERR_INVALID_ARG


def test_rhs_and_solution_permutations(sap):
    n = 1000
    rng = np.random.default_rng(5)
    p = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
    q = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
    r = torch.from_numpy(rng.uniform(0.5, 2, n)).cuda()
    b = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
    out = host(sap.sap_sparse_permute_rhs(b, p, r))
    exp = np.empty(n)
    exp[host(p)] = host(r) * host(b)
    np.testing.assert_array_equal(out, exp)
    x = host(sap.sap_sparse_unpermute_solution(b, q, r))
    np.testing.assert_array_equal(x, host(r) * host(b)[host(q)])


@pytest.mark.parametrize("scaled,variant", [(False, 0), (True, 0), (True, 1)])
def test_front_end_into_the_banded_solver(sap, scaled, variant):
    """DB, CM, band assembly, SaP (FP32 preconditioner, FP64 BiCGStab(2)) on
    the reordered band, the solution mapped back: the dense solve of A_s."""
    n = 3000
    sysm = G.sparse_scrambled(n, 8, 0.4, 1.0, 31)
    A = to_dev(sap, sysm)
    rownew, r, s, _ = sap.sap_db_reorder(A, scale=scaled)
    perm, K = sap.sap_cm_reorder(A, rownew)
    rn = sap.sap_perm_compose(perm, rownew)
    band = sap.sap_sparse_to_band(A, rn, perm, K, r, s)
    b_np = G.x_true(n, 31)
    bb = sap.sap_sparse_permute_rhs(torch.from_numpy(b_np).cuda(), rn, r)
    h = sap.sap_factor(band, n, K, P=4, variant=variant, precision=sap.SAP_FP32)
    y, info, st = sap.sap_solve(h, bb)
    assert st == sap.SAP_OK and info.relres <= 1e-10
    x = host(sap.sap_sparse_unpermute_solution(y, perm, s))
    xd = np.linalg.solve(OS.csr_to_dense(n, sysm.rowptr, sysm.col, sysm.val), b_np)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-8


def reordered(sap, sysm, scaled=True):
    A = to_dev(sap, sysm)
    rownew, r, s, _ = sap.sap_db_reorder(A, scale=scaled)
    perm, K = sap.sap_cm_reorder(A, rownew)
    rn = sap.sap_perm_compose(perm, rownew)
    return A, rn, perm, r, s, K


@pytest.mark.parametrize("frac", [0.0, 1e-3, 3e-2, 0.3, 2.0])
def test_drop_bandwidth_meets_its_definition(sap, frac):
    """K' satisfies the drop rule computed by the oracle from the same entries
    (the GPU sums the weights in another order: within rounding)."""
    sysm = G.sparse_scrambled(900, 6, 0.5, 1.0, 32)
    A, rn, perm, r, s, K = reordered(sap, sysm)
    Kp = sap.sap_sparse_drop_bandwidth(A, rn, perm, K, frac, r, s)
    w = OS.dist_weights(sysm.n, sysm.rowptr, sysm.col, sysm.val, host(rn), host(perm), K, host(r), host(s))
    tot = w.sum()
    assert 0 <= Kp <= K
    assert w[Kp + 1:].sum() <= frac * tot * (1 + 1e-12)
    assert Kp == 0 or w[Kp:].sum() > frac * tot * (1 - 1e-12)
    if frac == 0.0:
        assert Kp == K
    if frac >= 1.0:
        assert Kp == 0


def test_dropped_band_is_the_oracle_band(sap):
    sysm = G.sparse_scrambled(700, 5, 0.5, 1.0, 33)
    A, rn, perm, r, s, K = reordered(sap, sysm)
    Kp = max(1, K // 2)
    band = sap.sap_sparse_to_band(A, rn, perm, Kp, r, s, drop=True)
    band_o = OS.to_band(sysm.n, sysm.rowptr, sysm.col, sysm.val, host(rn), host(perm), Kp, host(r), host(s),
                        drop=True)
    np.testing.assert_array_equal(host(band), band_o)


@pytest.mark.parametrize("frac,variant", [(1e-3, 0), (2e-2, 0), (1e-3, 1)])
def test_sparse_operator_with_a_dropped_band_preconditioner(sap, frac, variant):
    """Sec. 2.2's sparse solve: the outer BiCGStab(2) on the reordered sparse
    matrix (sap_set_operator_csr), SaP of its dropped band (K' < K) as the
    preconditioner; the solution of the original system against a sparse
    direct solve, and its true residual."""
    sp = pytest.importorskip("scipy.sparse")
    spl = pytest.importorskip("scipy.sparse.linalg")
    n = 20000
    sysm = G.sparse_scrambled(n, 16, 0.3, 1.0, 34)
    A, rn, perm, r, s, K = reordered(sap, sysm)
    Kp = sap.sap_sparse_drop_bandwidth(A, rn, perm, K, frac, r, s)
    assert Kp < K
    band = sap.sap_sparse_to_band(A, rn, perm, Kp, r, s, drop=True)
    b_np = G.x_true(n, 34)
    bb = sap.sap_sparse_permute_rhs(torch.from_numpy(b_np).cuda(), rn, r)
    h = sap.sap_factor(band, n, Kp, P=8, variant=variant, precision=sap.SAP_FP32)
    sap.sap_set_operator_csr(h, A, rn, perm, r, s)
    y, info, st = sap.sap_solve(h, bb)
    assert st == sap.SAP_OK and info.relres <= 1e-10
    x = host(sap.sap_sparse_unpermute_solution(y, perm, s))
    As = sp.csr_matrix((sysm.val, sysm.col, sysm.rowptr), shape=(n, n))
    assert np.linalg.norm(b_np - As @ x) / np.linalg.norm(b_np) <= 1e-9
    xd = spl.spsolve(As.tocsc(), b_np)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-8
    # transposed solves are not defined for a sparse operator
    _, _, st2 = sap.sap_solve_adjoint(h, bb, raise_on_error=False)
    assert st2 == sap.SAP_ERR_NOT_IMPLEMENTED


def test_sparse_operator_without_drop_is_the_band_solve(sap):
    """No drop-off: the sparse operator is the band's matrix, so the solve
    reaches the band-operator solution (to the iteration's tolerance); then
    the band restored as the operator."""
    n = 6000
    sysm = G.sparse_scrambled(n, 8, 0.4, 1.0, 35)
    A, rn, perm, r, s, K = reordered(sap, sysm)
    band = sap.sap_sparse_to_band(A, rn, perm, K, r, s)
    bb = sap.sap_sparse_permute_rhs(torch.from_numpy(G.x_true(n, 35)).cuda(), rn, r)
    h = sap.sap_factor(band, n, K, P=4, variant=sap.SAP_D, precision=sap.SAP_FP32)
    y1, i1, st1 = sap.sap_solve(h, bb)
    sap.sap_set_operator_csr(h, A, rn, perm, r, s)
    y2, i2, st2 = sap.sap_solve(h, bb)
    assert st1 == st2 == sap.SAP_OK
    assert np.linalg.norm(host(y2) - host(y1)) / np.linalg.norm(host(y1)) <= 1e-9
    sap.sap_set_operator_csr(h, None)
    y3, _, st3 = sap.sap_solve(h, bb)
    assert st3 == sap.SAP_OK and torch.equal(y3, y1)
