"""Pins of the third-stage-reordering oracle (oracle/blocks.py, Sec. 2.2
"Third-stage reordering", Sec. 3.1): each compares it with something other
than itself - dense solves of the blocks, the unreordered SaP oracle (whose
own pins are in test_oracle_pins.py; the preconditioner does not depend on
the blocks' numbering in exact arithmetic), the hidden structure of the
synthetic input, a dense construction of the reordered blocks."""
import numpy as np
import pytest

import oracle as O
import oracle.blocks as OB
import sap_inputs as G


def system(N, K, P, d, seed):
    off = O.partition(N, P)
    return off, G.block_scrambled(N, K, off, d, seed)


def dense(band, N, K):
    B = np.asarray(band).reshape(2 * K + 1, N)
    A = np.zeros((N, N))
    for c in range(2 * K + 1):
        for j in range(N):
            i = j + c - K
            if 0 <= i < N:
                A[i, j] = B[c, j]
    return A


def identity_perm(off):
    return np.concatenate([np.arange(off[i + 1] - off[i]) for i in range(len(off) - 1)])


def random_perm(off, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.permutation(int(off[i + 1] - off[i])) for i in range(len(off) - 1)])


def test_generator_hides_narrow_bands():
    """In the hidden numbering every block is a band of half-bandwidth k0_i
    (its full band: every entry within k0_i present), and the scrambled block
    still fits the global band."""
    N, K, P = 700, 14, 4
    off, S = system(N, K, P, 1.0, 3)
    A = dense(S.band, N, K)
    for i in range(P):
        s, e = int(off[i]), int(off[i + 1])
        h = S.hid[s:e]
        assert sorted(h.tolist()) == list(range(e - s))
        Ah = np.zeros((e - s, e - s))
        Ah[np.ix_(h, h)] = A[s:e, s:e]
        I, J = np.nonzero(Ah)
        assert np.abs(I - J).max() == S.k0[i]
        k = int(S.k0[i])
        assert all(Ah[a, b] != 0 for a in range(e - s) for b in range(max(0, a - k), min(e - s, a + k + 1)))
    assert np.all(S.k0 <= (K + 1) // 2)


def test_block_bandwidth_agrees_with_a_dense_construction():
    N, K, P = 400, 10, 3
    off, S = system(N, K, P, 0.8, 4)
    A = dense(S.band, N, K)
    perm = random_perm(off, 1)
    for i in range(P):
        s, e = int(off[i]), int(off[i + 1])
        p = perm[s:e]
        Ah = np.zeros((e - s, e - s))
        Ah[np.ix_(p, p)] = A[s:e, s:e]
        I, J = np.nonzero(Ah)
        assert OB.block_bandwidth(S.band, N, K, s, e - s, p) == np.abs(I - J).max()


@pytest.mark.parametrize("seed", [5, 6])
def test_block_cm_recovers_the_hidden_bandwidths(seed):
    N, K, P = 1200, 16, 5
    off, S = system(N, K, P, 1.0, seed)
    perm, Ks = OB.block_cm(S.band, N, K, P)
    for i in range(P):
        s, e = int(off[i]), int(off[i + 1])
        assert sorted(perm[s:e].tolist()) == list(range(e - s))
        assert OB.block_bandwidth(S.band, N, K, s, e - s, np.arange(e - s)) > 2 * S.k0[i] - 2
    # CM of a scrambled full band of half-bandwidth k0 gives k0 back
    assert np.array_equal(Ks, S.k0)


def test_full_spikes_are_dense_block_solves():
    """Pi_i^T Vhat_i = A_i^{-1} [0; B_i] and Pi_{i+1}^T What_{i+1} =
    A_{i+1}^{-1} [C_{i+1}; 0] (Eq. (2.2)), from numpy's dense solves."""
    N, K, P = 900, 12, 4
    off, S = system(N, K, P, 0.7, 8)
    perm, _ = OB.block_cm(S.band, N, K, P)
    bs = OB.BlockSap(S.band, N, K, P, perm, O.SAP_C)
    A = dense(S.band, N, K)
    for i in range(P - 1):
        s0, s1, s2 = int(off[i]), int(off[i + 1]), int(off[i + 2])
        rv = np.zeros((s1 - s0, K))
        rv[-K:] = A[s1 - K:s1, s1:s1 + K]
        rw = np.zeros((s2 - s1, K))
        rw[:K] = A[s1:s1 + K, s1 - K:s1]
        V = np.linalg.solve(A[s0:s1, s0:s1], rv)
        Wd = np.linalg.solve(A[s1:s2, s1:s2], rw)
        assert np.abs(bs.Vfull[i][perm[s0:s1]] - V).max() <= 1e-13 * np.abs(V).max()
        assert np.abs(bs.Wfull[i][perm[s1:s2]] - Wd).max() <= 1e-13 * np.abs(Wd).max()


def test_tips_and_reduced_matrices_equal_the_lu_ul_ones():
    """The tips taken out of the entire spikes equal the unreordered oracle's
    bottom-LU / top-UL tips, and so do the reduced matrices Rbar_i."""
    N, K, P = 900, 12, 4
    off, S = system(N, K, P, 0.7, 9)
    perm, _ = OB.block_cm(S.band, N, K, P)
    bs = OB.BlockSap(S.band, N, K, P, perm, O.SAP_C)
    ref = O.Sap(S.band, N, K, P, O.SAP_C)
    for i in range(P - 1):
        for mine, code in ((bs.Vb[i], "V"), (bs.Wt[i], "W"), (bs.R[i][0], "R")):
            theirs = ref.interface(i, code)
            assert np.abs(mine - theirs).max() <= 1e-12 * max(1.0, np.abs(theirs).max()), code


@pytest.mark.parametrize("variant", [O.SAP_D, O.SAP_C])
@pytest.mark.parametrize("order", ["identity", "cm", "random"])
def test_apply_does_not_depend_on_the_block_numbering(variant, order):
    """M^{-1} r of the reordered preconditioner equals the unreordered
    oracle's, whatever the blocks' permutations (CM, random, none)."""
    N, K, P = 1500, 16, 5
    off, S = system(N, K, P, 0.5, 10)
    perm = {"identity": identity_perm(off), "cm": OB.block_cm(S.band, N, K, P)[0],
            "random": random_perm(off, 2)}[order]
    r = G.x_true(N, 11)
    z = OB.BlockSap(S.band, N, K, P, perm, variant).apply(r)
    zr = O.Sap(S.band, N, K, P, variant).apply(r)
    assert np.abs(z - zr).max() <= 1e-12 * np.abs(zr).max()


def test_sapd_is_the_block_diagonal_solve_and_p1_the_exact_one():
    N, K, P = 800, 10, 4
    off, S = system(N, K, P, 0.6, 12)
    perm, _ = OB.block_cm(S.band, N, K, P)
    A = dense(S.band, N, K)
    r = G.x_true(N, 13)
    z = OB.BlockSap(S.band, N, K, P, perm, O.SAP_D).apply(r)
    zd = np.concatenate([np.linalg.solve(A[off[i]:off[i + 1], off[i]:off[i + 1]], r[off[i]:off[i + 1]])
                         for i in range(P)])
    assert np.abs(z - zd).max() <= 1e-13 * np.abs(zd).max()
    one = OB.BlockSap(S.band, N, K, 1, OB.block_cm(S.band, N, K, 1)[0], O.SAP_D)
    x = np.linalg.solve(A, r)
    assert np.abs(one.apply(r) - x).max() <= 1e-12 * np.abs(x).max()


def test_boosted_pivot_uses_the_whole_band_threshold():
    """tau = boost_eps max |a_ij| over the whole band (couplings included,
    Sec. 2.2); a zero first pivot is boosted once, to +tau, and L U of the
    block is then A_0 with a_00 = tau."""
    N, K, P = 300, 6, 3
    off, S = system(N, K, P, 1.0, 14)
    band = S.band.copy()
    band[K * N + 0] = 0.0                      # a_00 = 0
    a = OB.BlockSap(band, N, K, P, identity_perm(off), O.SAP_D, boost_eps=1e-3)
    tau = 1e-3 * O.band_absmax(band, N, K)
    assert a.tau == tau and a.n_boosted == 1
    n, Ki = int(off[1]), int(a.Ki[0])
    f = a.lu[0]
    L, U = np.eye(n), np.zeros((n, n))
    for r in range(n):
        for c in range(max(0, r - Ki), min(n, r + Ki + 1)):
            (L if c < r else U)[r, c] = f[r, c - r + Ki]
    A0 = dense(band, N, K)[:n, :n]
    A0[0, 0] = tau
    assert np.abs(L @ U - A0).max() <= 1e-13 * np.abs(A0).max()


MUTATIONS = {
    "tips from the new numbering's bottom rows": ("_tip_rows_v", lambda p, n, K: np.arange(n - K, n)),
    "top tip rows from the bottom": ("_tip_rows_w", lambda p, K: p[len(p) - K:]),
    "right-hand side gathered, not scattered": ("_to_new", lambda p, v: v[p]),
}


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_planted_mutations_fail_a_pin(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(OB, attr, fn)
    N, K, P = 1500, 16, 5
    off, S = system(N, K, P, 0.5, 10)
    perm, _ = OB.block_cm(S.band, N, K, P)
    r = G.x_true(N, 11)
    z = OB.BlockSap(S.band, N, K, P, perm, O.SAP_C).apply(r)
    zr = O.Sap(S.band, N, K, P, O.SAP_C).apply(r)
    assert np.abs(z - zr).max() > 1e-6 * np.abs(zr).max()


def test_adjoint_preconditioner_of_the_transposed_band():
    """The preconditioner of A^T keeps the blocks' numbering: BlockSap of the
    transposed band with the same permutations.  SaP-D: its inverse is exactly
    the transpose of the forward one (M = D block diagonal, (D^T)^{-1} =
    (D^{-1})^T), checked on dense matrices; SaP-C: it equals the unreordered
    oracle built on A^T (truncation makes it differ from the transpose)."""
    N, K, P = 240, 6, 4
    off, S = system(N, K, P, 0.8, 15)
    perm, _ = OB.block_cm(S.band, N, K, P)
    bt = O.transpose_band(S.band, N, K)
    fwd = OB.BlockSap(S.band, N, K, P, perm, O.SAP_D)
    adj = OB.BlockSap(bt, N, K, P, perm, O.SAP_D)
    E = np.eye(N)
    Mf = np.column_stack([fwd.apply(E[:, j]) for j in range(N)])
    Ma = np.column_stack([adj.apply(E[:, j]) for j in range(N)])
    assert np.abs(Ma - Mf.T).max() <= 1e-13 * np.abs(Mf).max()
    r = G.adjoint_seed(N, 16)
    za = OB.BlockSap(bt, N, K, P, perm, O.SAP_C).apply(r)
    zr = O.Sap(bt, N, K, P, O.SAP_C).apply(r)
    assert np.abs(za - zr).max() <= 1e-12 * np.abs(zr).max()
