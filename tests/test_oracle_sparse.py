"""Pins of the sparse front-end oracle (oracle/sparse.py, Sec. 2.2): each
check compares it with something other than itself - brute force over all
permutations, a library assignment solver, linear-programming duality,
the hidden structure the synthetic input was built from, a dense
construction, a dense solve."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
import oracle.sparse as OS
import sap_inputs as G


def rand_costs(n, seed, p_inf=0.25):
    rng = np.random.default_rng(seed)
    C = rng.uniform(0, 5, (n, n))
    C[rng.uniform(size=(n, n)) < p_inf] = math.inf
    for i in range(n):                       # keep a perfect assignment possible
        C[i, (i * 3 + seed) % n] = rng.uniform(0, 5)
    return C


def brute_min(C):
    n = len(C)
    return min(sum(C[i][p[i]] for i in range(n)) for p in itertools.permutations(range(n)))


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (5, 3), (6, 4), (7, 5), (7, 6)])
def test_hungarian_is_the_brute_force_optimum(n, seed):
    C = rand_costs(n, seed)
    a, u, v = OS.hungarian(C.tolist())
    assert sorted(a.tolist()) == list(range(n))
    assert sum(C[i][a[i]] for i in range(n)) == pytest.approx(brute_min(C), abs=1e-12)


def test_hungarian_matches_a_library_assignment_solver():
    opt = pytest.importorskip("scipy.optimize")
    for seed in range(3):
        C = np.random.default_rng(seed).uniform(0, 10, (40, 40))
        a, u, v = OS.hungarian(C.tolist())
        r, c = opt.linear_sum_assignment(C)
        assert C[np.arange(40), a].sum() == pytest.approx(C[r, c].sum(), rel=1e-13)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_hungarian_duals_certify_optimality(seed):
    """LP duality: feasible potentials (reduced costs >= 0 on every edge)
    whose sum equals the assignment's cost prove the assignment optimal."""
    C = rand_costs(12, seed)
    a, u, v = OS.hungarian(C.tolist())
    fin = np.isfinite(C)
    red = C - u[:, None] - v[None, :]
    assert np.all(red[fin] >= -1e-12)
    assert np.all(np.abs(red[np.arange(12), a]) <= 1e-12)
    assert C[np.arange(12), a].sum() == pytest.approx(u.sum() + v.sum(), abs=1e-11)


def test_hungarian_rejects_a_structurally_singular_matrix():
    C = [[1.0, math.inf], [2.0, math.inf]]
    with pytest.raises(ValueError):
        OS.hungarian(C)


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_db_restores_the_hidden_diagonal(seed):
    """On a row-shuffled strictly diagonally dominant matrix the product of
    the diagonal is the unique maximum over permutations (any other cycle of
    entries is smaller entry by entry), so the matching puts every row back on
    the column of its old diagonal entry, and c = 0 there (row maxima)."""
    S = G.sparse_scrambled(80, 4, 0.4, 1.5, seed)
    db = OS.db_match(S.n, S.rowptr, S.col, S.val)
    assert np.array_equal(db.sigma, S.sym[S.rowsrc])
    assert db.cost == pytest.approx(0.0, abs=1e-12)
    A = OS.csr_to_dense(S.n, S.rowptr, S.col, S.val)
    assert db.logprod == pytest.approx(np.log(np.abs(A[np.arange(S.n), db.sigma])).sum(), rel=1e-14)


def test_db_scaling_gives_an_i_matrix():
    """|r_i a_ij s_j| <= 1 for every entry and = 1 on the matching."""
    S = G.sparse_scrambled(70, 3, 0.6, 0.3, 7)        # weak diagonal: the scaling has work to do
    db = OS.db_match(S.n, S.rowptr, S.col, S.val)
    r, s = OS.db_scaling(db.a, db.u, db.v)
    A = OS.csr_to_dense(S.n, S.rowptr, S.col, S.val)
    Bs = np.abs(r[:, None] * A * s[None, :])
    assert Bs.max() <= 1.0 + 1e-12
    assert np.allclose(Bs[np.arange(S.n), db.sigma], 1.0, rtol=0, atol=1e-12)


def min_bandwidth_brute(nb):
    n = len(nb)
    best = n
    for p in itertools.permutations(range(n)):
        best = min(best, max((abs(p[x] - p[y]) for x in range(n) for y in nb[x]), default=0))
    return best


def perm_bandwidth(nb, perm):
    return max((abs(int(perm[x]) - int(perm[y])) for x in range(len(nb)) for y in nb[x]), default=0)


@pytest.mark.parametrize("shape", ["path", "cycle", "two_paths"])
def test_cm_reaches_the_optimal_bandwidth_on_paths_and_cycles(shape):
    n = 9
    rng = np.random.default_rng(1)
    lab = rng.permutation(n)                 # scrambled labels
    edges = [(i, i + 1) for i in range(n - 1)]
    if shape == "cycle":
        edges.append((n - 1, 0))
    if shape == "two_paths":
        edges = [(i, i + 1) for i in range(3)] + [(i, i + 1) for i in range(4, n - 1)]
    nb = [set() for _ in range(n)]
    for a, b in edges:
        nb[lab[a]].add(int(lab[b]))
        nb[lab[b]].add(int(lab[a]))
    nb = [sorted(x) for x in nb]
    perm = OS.cm_order(n, nb)
    assert sorted(perm.tolist()) == list(range(n))
    assert perm_bandwidth(nb, perm) == min_bandwidth_brute(nb) == (2 if shape == "cycle" else 1)


def test_cm_is_never_below_the_optimum_on_small_random_graphs():
    rng = np.random.default_rng(2)
    for _ in range(6):
        n = 7
        nb = [set() for _ in range(n)]
        for a in range(n):
            for b in range(a + 1, n):
                if rng.uniform() < 0.35:
                    nb[a].add(b)
                    nb[b].add(a)
        nb = [sorted(x) for x in nb]
        perm = OS.cm_order(n, nb)
        assert sorted(perm.tolist()) == list(range(n))
        assert perm_bandwidth(nb, perm) >= min_bandwidth_brute(nb)


@pytest.mark.parametrize("seed,K0", [(8, 3), (9, 5), (10, 8)])
def test_db_cm_recovers_a_narrow_band(seed, K0):
    """After the matching and CM of B + B^T, the bandwidth of the scrambled
    band is back within twice the hidden one (from about n)."""
    S = G.sparse_scrambled(300, K0, 0.5, 1.5, seed)
    db = OS.db_match(S.n, S.rowptr, S.col, S.val)
    perm = OS.cm_order(S.n, OS.sym_pattern(S.n, S.rowptr, S.col, db.sigma))
    K = OS.bandwidth(S.n, S.rowptr, S.col, perm[db.sigma], perm)
    K_before = OS.bandwidth(S.n, S.rowptr, S.col, np.arange(S.n), np.arange(S.n))
    assert K <= 2 * K0 < K_before // 10


def test_bandwidth_and_band_agree_with_a_dense_construction():
    S = G.sparse_scrambled(50, 3, 0.5, 0.8, 11)
    rng = np.random.default_rng(3)
    rn, cn = rng.permutation(S.n), rng.permutation(S.n)
    r, s = rng.uniform(0.5, 2, S.n), rng.uniform(0.5, 2, S.n)
    A = OS.csr_to_dense(S.n, S.rowptr, S.col, S.val)
    B = np.zeros_like(A)
    B[np.ix_(rn, cn)] = (r[:, None] * A) * s[None, :]
    I, J = np.nonzero(B)
    K = OS.bandwidth(S.n, S.rowptr, S.col, rn, cn)
    assert K == np.abs(I - J).max()
    band = OS.to_band(S.n, S.rowptr, S.col, S.val, rn, cn, K, r, s).reshape(2 * K + 1, S.n)
    for I in range(S.n):
        for J in range(max(0, I - K), min(S.n, I + K + 1)):
            assert band[K + I - J, J] == B[I, J]


@pytest.mark.parametrize("scale", [False, True])
def test_reordered_band_solve_is_the_dense_solve(scale):
    """The whole front end: DB (with or without scaling), CM, band assembly,
    the banded oracle solve of the reordered system, and the solution mapped
    back, against numpy's dense solve of the original sparse system."""
    S = G.sparse_scrambled(240, 4, 0.5, 1.2, 12)
    db = OS.db_match(S.n, S.rowptr, S.col, S.val)
    perm = OS.cm_order(S.n, OS.sym_pattern(S.n, S.rowptr, S.col, db.sigma))
    rn, cn = perm[db.sigma], perm
    r, s = OS.db_scaling(db.a, db.u, db.v) if scale else (np.ones(S.n), np.ones(S.n))
    K = OS.bandwidth(S.n, S.rowptr, S.col, rn, cn)
    band = OS.to_band(S.n, S.rowptr, S.col, S.val, rn, cn, K, r, s)
    b = G.x_true(S.n, 12)
    bb = np.empty(S.n)
    bb[rn] = r * b
    y, info, _ = O.solve(band, S.n, K, bb, 1, O.SAP_D)
    x = s * y[cn]
    A = OS.csr_to_dense(S.n, S.rowptr, S.col, S.val)
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-10


@pytest.mark.parametrize("frac", [0.0, 1e-4, 1e-2, 0.2, 5.0])
def test_drop_bandwidth_from_the_entry_list(frac):
    """The drop-off's K' against the tail sums taken directly over the stored
    entries: the smallest K' whose dropped entries weigh at most frac of all."""
    S = G.sparse_scrambled(120, 6, 0.5, 1.0, 13)
    db = OS.db_match(S.n, S.rowptr, S.col, S.val)
    perm = OS.cm_order(S.n, OS.sym_pattern(S.n, S.rowptr, S.col, db.sigma))
    rn, cn = perm[db.sigma], perm
    r, s = OS.db_scaling(db.a, db.u, db.v)
    K = OS.bandwidth(S.n, S.rowptr, S.col, rn, cn)
    Kp = OS.drop_bandwidth(OS.dist_weights(S.n, S.rowptr, S.col, S.val, rn, cn, K, r, s), frac)
    ent = [(abs(int(rn[i]) - int(cn[S.col[p]])), abs((r[i] * S.val[p]) * s[S.col[p]]))
           for i in range(S.n) for p in range(S.rowptr[i], S.rowptr[i + 1])]
    total = sum(e for _, e in ent)
    tail = lambda k: sum(e for d, e in ent if d > k)
    assert tail(Kp) <= frac * total * (1 + 1e-12)
    assert Kp == 0 or tail(Kp - 1) > frac * total
    if frac == 0.0:
        assert Kp == K
    if frac >= 1.0:
        assert Kp == 0
    band = OS.to_band(S.n, S.rowptr, S.col, S.val, rn, cn, Kp, r, s, drop=True)
    kept = sum(abs(x) for x in band)
    assert kept == pytest.approx(total - tail(Kp), rel=1e-12)

