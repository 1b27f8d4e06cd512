"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the
mathematics, independent of the oracle itself: the paper's worked storage
example, closed forms, library routines in special cases where they reduce to
the same factorisation, exactness of the method in cases where the
truncation drops nothing, and invariants of the Krylov recurrences.

Each test names the passage it pins."""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
import sap_inputs as G
from tests._dense import band_to_dense, block_factor_to_dense, dense_to_band

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U64 = 2.0 ** -53


def rand_band(N, K, d, seed):
    return G.dense_banded(N, K, d, seed)


# ---------------------------------------------------------------- storage ---

def test_band_layout_matches_paper_picture():
    """Section 3.1 "Matrix storage": the N=8, K=2 picture.  Picture row r,
    column c holds the label a_ij; it must sit at band[c * N + r] and be
    what the oracle's SpMV reads as a_ij."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "band_layout_n8_k2.txt"))
            if ln.strip() and not ln.startswith("#")]
    N, K = 8, 2
    assert len(rows) == N and all(len(r) == 2 * K + 1 for r in rows)
    band = np.full((2 * K + 1) * N, np.nan)          # padding poisoned
    labels = {}
    rng = np.random.default_rng(0)
    for r, row in enumerate(rows):
        for c, lab in enumerate(row):
            if lab == "*":
                continue
            i, j = int(lab[1]) - 1, int(lab[2]) - 1
            v = rng.uniform(1, 2)
            band[c * N + r] = v
            labels[(i, j)] = v
    # columns of A via the oracle SpMV on unit vectors; padding must be ignored
    for j in range(N):
        e = np.zeros(N); e[j] = 1.0
        col = O.spmv(band, N, K, e)
        for i in range(N):
            expect = labels.get((i, j), 0.0)
            assert col[i] == expect, (i, j)
    # every in-band (i, j) appears exactly once in the picture
    assert set(labels) == {(i, j) for i in range(N) for j in range(N) if abs(i - j) <= K}


# -------------------------------------------------------------- partition ---

@pytest.mark.parametrize("N,P,expect", [
    (10, 3, [4, 3, 3]), (7, 7, [1] * 7), (10000, 8, [1250] * 8),
    (200000, 50, [4000] * 50), (100000, 32, [3125] * 32), (11, 4, [3, 3, 3, 2]),
])
def test_partition_closed_form(N, P, expect):
    """Section 3.1: the first P_r blocks have floor(N/P)+1 rows, the rest
    floor(N/P), N = P floor(N/P) + P_r."""
    off = O.partition(N, P)
    assert list(np.diff(off)) == expect
    assert off[0] == 0 and off[-1] == N


# ------------------------------------------------------------------ SpMV ---

def test_spmv_matches_dense():
    N, K = 37, 5
    band = rand_band(N, K, 1.0, 3)
    # poison padding: the matvec must never read it
    b2 = band.reshape(2 * K + 1, N).copy()
    for c in range(2 * K + 1):
        for j in range(N):
            if not (0 <= j + c - K < N):
                b2[c, j] = np.nan
    b2 = b2.reshape(-1)
    A = band_to_dense(band, N, K)
    x = G.x_true(N, 1)
    np.testing.assert_allclose(O.spmv(b2, N, K, x), A @ x, rtol=0, atol=1e-13)
    np.testing.assert_allclose(O.spmv(b2, N, K, x, transpose=True), A.T @ x, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(band_to_dense(O.transpose_band(band, N, K), N, K), A.T)


# -------------------------------------------------------------------- LU ---

def _block_dense(band, N, K, s, n):
    A = band_to_dense(band, N, K)
    return A[s:s + n, s:s + n]


def test_lu_reconstructs_block_and_is_banded():
    """Section 3.1 LU/UL: L_i U_i = A_i without pivoting, L unit lower, both
    confined to the band (no fill outside it)."""
    N, K, P = 90, 4, 3
    band = rand_band(N, K, 1.0, 11)
    s = O.Sap(band, N, K, P, O.SAP_D)
    off = s.offsets
    for i in range(P):
        n = off[i + 1] - off[i]
        LU = block_factor_to_dense(s.block(i, 0), K)
        L = np.tril(LU, -1) + np.eye(n)
        U = np.triu(LU)
        Ai = _block_dense(band, N, K, off[i], n)
        assert np.abs(L @ U - Ai).max() <= 10 * U64 * K * np.abs(Ai).max() * 10
        assert s.n_boosted == 0


def test_lu_equals_scipy_on_column_dominant_block():
    """Special case where partial pivoting never swaps rows: for a matrix that
    is diagonally dominant by columns, GEPP keeps the pivot on the diagonal
    (dominance by columns is inherited by every Schur complement), so
    LAPACK's getrf returns the unique no-pivot factors."""
    N, K = 64, 6
    rowdom = rand_band(N, K, 1.3, 5)
    A = band_to_dense(rowdom, N, K).T                   # column dominant
    band = dense_to_band(A, K)
    f = np.zeros((N, 2 * K + 1))
    for r in range(N):
        for d in range(-K, K + 1):
            if 0 <= r + d < N:
                f[r, d + K] = A[r, r + d]
    nb = O.block_lu(f, N, K, tau=0.0)
    assert nb == 0
    Pm, L, U = sla.lu(A)
    np.testing.assert_array_equal(Pm, np.eye(N))
    LU = block_factor_to_dense(f, K)
    np.testing.assert_allclose(np.tril(LU, -1) + np.eye(N), L, rtol=0, atol=1e-13)
    np.testing.assert_allclose(np.triu(LU), U, rtol=1e-13, atol=1e-13)
    del band


def test_lu_pivots_are_ratios_of_leading_minors():
    """Closed form of the no-pivot LU: u_kk = det(A[:k+1,:k+1]) / det(A[:k,:k])."""
    N, K = 12, 3
    band = rand_band(N, K, 1.0, 21)
    A = band_to_dense(band, N, K)
    s = O.Sap(band, N, K, 1, O.SAP_D)
    u = np.diag(block_factor_to_dense(s.block(0, 0), K))
    dets = [1.0] + [np.linalg.det(A[:k, :k]) for k in range(1, N + 1)]
    np.testing.assert_allclose(u, np.array(dets[1:]) / np.array(dets[:-1]), rtol=1e-11)


def test_boost_replaces_small_pivot():
    """Section 2.2: a pivot below the threshold is replaced by the boosting
    value (here sign(0) -> +tau) and counted."""
    N, K = 10, 2
    A = np.diag(np.full(N, 4.0)) + np.diag(np.ones(N - 1), 1) + np.diag(np.ones(N - 1), -1)
    A[3, 3] = 0.0
    A[3, 2] = 0.0                      # keeps the Schur update of pivot 3 at exactly 0
    A[2, 3] = 0.0
    band = dense_to_band(A, K)
    tau = 1e-3
    s = O.Sap(band, N, K, 1, O.SAP_D, tau=tau)
    assert s.n_boosted == 1
    LU = block_factor_to_dense(s.block(0, 0), K)
    assert LU[3, 3] == tau


# -------------------------------------------------------------------- UL ---

def test_ul_reconstructs_and_is_flip_of_lu():
    """Section 2.1: A_i = U'_i L'_i with unit upper U'; it is the LU of the
    reversed block J A_i J read backwards (J = exchange matrix)."""
    N, K = 40, 5
    band = rand_band(N, K, 1.0, 8)
    A = band_to_dense(band, N, K)
    f = np.zeros((N, 2 * K + 1))
    for r in range(N):
        for d in range(-K, K + 1):
            if 0 <= r + d < N:
                f[r, d + K] = A[r, r + d]
    g = f.copy()
    O.block_ul(f, N, K, 0.0)
    UL = block_factor_to_dense(f, K)
    Up = np.triu(UL, 1) + np.eye(N)
    Lp = np.tril(UL)
    assert np.abs(Up @ Lp - A).max() < 1e-12 * np.abs(A).max()
    J = np.eye(N)[::-1]
    AJ = J @ A @ J
    for r in range(N):
        for d in range(-K, K + 1):
            g[r, d + K] = AJ[r, r + d] if 0 <= r + d < N else 0.0
    O.block_lu(g, N, K, 0.0)
    LUJ = block_factor_to_dense(g, K)
    np.testing.assert_allclose(J @ (np.tril(LUJ, -1) + np.eye(N)) @ J, Up, atol=1e-13)
    np.testing.assert_allclose(J @ np.triu(LUJ) @ J, Lp, atol=1e-13)


# ------------------------------------------------------------ spike tips ---

@pytest.mark.parametrize("N,K,P", [(60, 4, 3), (50, 5, 2), (120, 6, 5)])
def test_spike_tips_equal_full_spike_ends(N, K, P):
    """Eq. (2.2): A_i V_i = [0; 0; B_i], A_{i+1} W_{i+1} = [C_{i+1}; 0; 0].
    The tips from the bottom LU blocks / top UL blocks (Section 2.1,
    computational savings) are the bottom / top K rows of the full spikes,
    computed here by dense solves.  Also pins the triangular shapes of B, C."""
    band = rand_band(N, K, 1.0, 17)
    A = band_to_dense(band, N, K)
    s = O.Sap(band, N, K, P, O.SAP_C)
    off = s.offsets
    for i in range(P - 1):
        a0, a1, a2 = off[i], off[i + 1], off[i + 2]
        B = s.interface(i, "B")
        C = s.interface(i, "C")
        np.testing.assert_array_equal(B, A[a1 - K:a1, a1:a1 + K])
        np.testing.assert_array_equal(C, A[a1:a1 + K, a1 - K:a1])
        np.testing.assert_array_equal(np.triu(B, 1), 0)   # lower triangular
        np.testing.assert_array_equal(np.tril(C, -1), 0)  # upper triangular
        Ai, Aj = A[a0:a1, a0:a1], A[a1:a2, a1:a2]
        rhsV = np.zeros((a1 - a0, K)); rhsV[-K:] = B
        rhsW = np.zeros((a2 - a1, K)); rhsW[:K] = C
        Vfull = np.linalg.solve(Ai, rhsV)
        Wfull = np.linalg.solve(Aj, rhsW)
        np.testing.assert_allclose(s.interface(i, "V"), Vfull[-K:], rtol=0, atol=1e-12)
        np.testing.assert_allclose(s.interface(i, "W"), Wfull[:K], rtol=0, atol=1e-12)
        # Rbar = I - W^(t) V^(b), Eq. (2.5a)
        np.testing.assert_allclose(s.interface(i, "R"), np.eye(K) - Wfull[:K] @ Vfull[-K:],
                                   rtol=0, atol=1e-12)


def test_reduced_solve_solves_R_i():
    """Eq. (2.4)-(2.5): the three steps solve R_i [xb; xt] = [gb; gt] with
    R_i = [[I, V^(b)_i], [W^(t)_{i+1}, I]] exactly (the truncation only drops
    M_i and N_i, not anything inside R_i)."""
    N, K, P = 80, 5, 4
    band = rand_band(N, K, 0.8, 2)
    s = O.Sap(band, N, K, P, O.SAP_C)
    rng = np.random.default_rng(1)
    for i in range(P - 1):
        V, W = s.interface(i, "V"), s.interface(i, "W")
        R = np.block([[np.eye(K), V], [W, np.eye(K)]])
        g = rng.standard_normal(2 * K)
        xb, xt = s.reduced_solve(i, g[:K], g[K:])
        np.testing.assert_allclose(np.concatenate([xb, xt]), np.linalg.solve(R, g), atol=1e-12)


def test_dense_getrf_matches_lapack():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((9, 9))
    st, lu, piv = O.dense_getrf(a)
    assert st == 0
    lu2, piv2 = sla.lu_factor(a)
    np.testing.assert_array_equal(piv, piv2)
    np.testing.assert_allclose(lu, lu2, atol=1e-14)
    b = rng.standard_normal(9)
    np.testing.assert_allclose(O.dense_getrs(lu, piv, b), np.linalg.solve(a, b), atol=1e-12)


# ---------------------------------------------------------------- apply ---

def test_apply_P1_is_exact():
    """P = 1: M = A, so one apply is the banded solve."""
    N, K = 70, 4
    band = rand_band(N, K, 1.0, 4)
    A = band_to_dense(band, N, K)
    r = G.x_true(N, 9)
    for var in (O.SAP_D, O.SAP_C):
        z = O.Sap(band, N, K, 1, var).apply(r)
        np.testing.assert_allclose(z, np.linalg.solve(A, r), rtol=0, atol=1e-12 * np.abs(z).max())


def test_sapd_apply_is_block_diagonal_solve():
    """SaP-D (Section 2.1.1): x ~ g = D^{-1} b, D = diag(A_1..A_P)."""
    N, K, P = 75, 3, 4
    band = rand_band(N, K, 1.0, 6)
    A = band_to_dense(band, N, K)
    s = O.Sap(band, N, K, P, O.SAP_D)
    off = s.offsets
    r = G.x_true(N, 2)
    z = s.apply(r)
    for i in range(P):
        a, b = off[i], off[i + 1]
        np.testing.assert_allclose(z[a:b], np.linalg.solve(A[a:b, a:b], r[a:b]), atol=1e-12)


def test_sapc_P2_is_exact():
    """With P = 2 the reduced system is the single block R_1 (there are no
    M_i or N_i to drop), so SaP-C is a direct solver."""
    N, K = 64, 6
    band = rand_band(N, K, 0.9, 12)
    A = band_to_dense(band, N, K)
    r = G.x_true(N, 3)
    z = O.Sap(band, N, K, 2, O.SAP_C).apply(r)
    np.testing.assert_allclose(z, np.linalg.solve(A, r), atol=1e-11 * np.abs(z).max())


def test_sapc_exact_when_middle_spikes_decouple():
    """If the middle block A_2 (P = 3) splits into two decoupled halves, W_2
    vanishes in its bottom K rows and V_2 in its top K rows, so M_1 = N_2 = 0
    in Eq. (2.4) and the truncated reduction is exact: SaP-C = A^{-1}.  This
    pins both purification terms (C_i and B_i) of a middle block."""
    N, K, P = 90, 4, 3
    A = band_to_dense(rand_band(N, K, 1.0, 13), N, K)
    off = O.partition(N, P)
    mid = (off[1] + off[2]) // 2
    A[mid:mid + K, mid - K:mid] = 0.0
    A[mid - K:mid, mid:mid + K] = 0.0
    band = dense_to_band(A, K)
    r = G.x_true(N, 4)
    s = O.Sap(band, N, K, P, O.SAP_C)
    np.testing.assert_allclose(s.apply(r), np.linalg.solve(A, r), atol=1e-11)
    # and SaP-D is not exact on the same matrix (the coupling is real)
    assert np.abs(O.Sap(band, N, K, P, O.SAP_D).apply(r) - np.linalg.solve(A, r)).max() > 1e-3


def test_sapc_equals_sapd_without_coupling():
    """B_i = C_i = 0: the spikes vanish, Rbar_i = I, and SaP-C reduces to
    SaP-D bit for bit (Section 2.1.1)."""
    N, K, P = 60, 3, 3
    A = band_to_dense(rand_band(N, K, 1.0, 14), N, K)
    off = O.partition(N, P)
    for s_ in off[1:-1]:
        A[s_:s_ + K, s_ - K:s_] = 0.0
        A[s_ - K:s_, s_:s_ + K] = 0.0
    band = dense_to_band(A, K)
    r = G.x_true(N, 5)
    zc = O.Sap(band, N, K, P, O.SAP_C).apply(r)
    zd = O.Sap(band, N, K, P, O.SAP_D).apply(r)
    np.testing.assert_array_equal(zc, zd)
    np.testing.assert_allclose(zd, np.linalg.solve(A, r), atol=1e-12)


def test_sapc_truncation_error_decays_with_dominance():
    """Section 2.1: for d > 1 the spikes decay away from their source, so the
    dropped M_i, N_i shrink and SaP-C approaches A^{-1} as d grows; SaP-C is
    a better preconditioner than SaP-D."""
    N, K, P = 200, 4, 8
    r = G.x_true(N, 6)
    errs_c, errs_d = [], []
    for d in (1.0, 2.0, 8.0):
        band = rand_band(N, K, d, 15)
        x = np.linalg.solve(band_to_dense(band, N, K), r)
        errs_c.append(np.linalg.norm(O.Sap(band, N, K, P, O.SAP_C).apply(r) - x) / np.linalg.norm(x))
        errs_d.append(np.linalg.norm(O.Sap(band, N, K, P, O.SAP_D).apply(r) - x) / np.linalg.norm(x))
    assert errs_c[0] > errs_c[1] > errs_c[2]
    assert errs_c[2] < 1e-8
    assert all(c < d for c, d in zip(errs_c, errs_d))


# ----------------------------------------------------------- BiCGStab(2) ---

@pytest.mark.parametrize("N,K,P,var,d", [
    (150, 4, 5, O.SAP_D, 1.0), (200, 6, 4, O.SAP_C, 1.0), (180, 3, 6, O.SAP_C, 0.6),
    (120, 10, 3, O.SAP_D, 1.2),
])
def test_bicgstab2_solution_matches_dense_solve(N, K, P, var, d):
    """The outer Krylov solve converges to A^{-1} b: true residual <= 1e-10
    and agreement with LAPACK's dense solve."""
    band = rand_band(N, K, d, 30 + N)
    A = band_to_dense(band, N, K)
    xt = G.x_true(N, 30)
    b = A @ xt
    x, info = O.Sap(band, N, K, P, var).solve(b, tol=1e-10)
    assert info.status == O.OK
    assert info.relres <= 1e-10
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-10
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-8
    assert (info.iters * 4) % 1 == 0           # quarters


def test_bicgstab2_exact_preconditioner_exits_at_first_quarter():
    """M = A (P = 1): A~ = I, so alpha = 1 and the first BiCG update zeroes
    the residual: exit at 1/4 iteration (Section 4.1.1 quarters)."""
    N, K = 100, 5
    band = rand_band(N, K, 1.0, 41)
    b = O.spmv(band, N, K, G.x_true(N, 41))
    _, info = O.Sap(band, N, K, 1, O.SAP_D).solve(b)
    assert info.status == O.OK and info.iters == 0.25 and info.n_matvec == 1


def test_bicgstab2_nilpotent_coupling_exits_at_three_quarters():
    """Block upper-triangular A (C_2 = 0) with SaP-D, P = 2: D^{-1} A = I + E
    with E^2 = 0, so the minimal polynomial of A~ has degree 2 and the BiCG
    part terminates after its second step (matvec 3): exit at 3/4."""
    N, K = 80, 4
    A = band_to_dense(rand_band(N, K, 1.0, 42), N, K)
    off = O.partition(N, 2)
    s_ = off[1]
    A[s_:, :s_] = 0.0
    band = dense_to_band(A, K)
    b = A @ G.x_true(N, 42)
    x, info = O.Sap(band, N, K, 2, O.SAP_D).solve(b)
    assert info.status == O.OK and info.iters == 0.75
    np.testing.assert_allclose(x, np.linalg.solve(A, b), atol=1e-10)


def test_bicgstab2_recursive_residual_tracks_true_residual():
    """Invariant of the BiCGStab(l) recurrences: the updated r^0 equals the
    preconditioned residual M^{-1}(b - A x) of the updated iterate at every
    exit point (a dropped or mis-signed term in the x, r or u updates breaks
    it immediately)."""
    N, K, P = 300, 5, 10
    band = rand_band(N, K, 0.7, 43)
    b = O.spmv(band, N, K, G.x_true(N, 43))
    x, info = O.Sap(band, N, K, P, O.SAP_D).solve(b, tol=1e-12, trace=True)
    assert info.status == O.OK
    tr = info.trace
    assert len(tr) >= 6
    scale = tr[0, 1] + 1.0
    for mv, rn, pn, rel in tr:
        assert abs(rn - pn) <= 1e-9 * max(scale, 1.0), (mv, rn, pn)
    # exits happen at matvecs 1, 3, 4 (mod 4)
    assert set((tr[:, 0] % 4).astype(int)) <= {1, 3, 0}


def test_sapc_needs_fewer_iterations_than_sapd():
    """Section 4.1.1: the coupled preconditioner is of better quality."""
    N, K, P = 2000, 8, 10
    band = rand_band(N, K, 1.0, 44)
    b = O.spmv(band, N, K, G.x_true(N, 44))
    _, ic = O.Sap(band, N, K, P, O.SAP_C).solve(b)
    _, id_ = O.Sap(band, N, K, P, O.SAP_D).solve(b)
    assert ic.status == id_.status == O.OK
    assert ic.iters <= id_.iters


def test_not_converged_reports_status():
    N, K, P = 400, 4, 40
    band = rand_band(N, K, 0.3, 45)
    b = O.spmv(band, N, K, G.x_true(N, 45))
    x, info = O.Sap(band, N, K, P, O.SAP_D).solve(b, max_iters=1)
    assert info.status in (O.NOT_CONVERGED, O.OK)
    if info.status == O.NOT_CONVERGED:
        assert info.relres > 1e-10


# -------------------------------------------------------------- adjoint ---

def test_adjoint_solve_matches_dense_transpose_solve():
    N, K, P = 160, 5, 4
    band = rand_band(N, K, 1.0, 50)
    A = band_to_dense(band, N, K)
    g = G.adjoint_seed(N, 50)
    for var in (O.SAP_D, O.SAP_C):
        lam, info, _ = O.solve_adjoint(band, N, K, g, P, var)
        assert info.status == O.OK
        np.testing.assert_allclose(lam, np.linalg.solve(A.T, g), atol=1e-8 * np.abs(lam).max())


def test_grad_band_matches_central_differences():
    """d(w^T x)/d a_ij = -lambda_i x_j on the band, lambda = A^{-T} w;
    d(w^T x)/d b = lambda.  Central differences of oracle solves at tol 1e-14."""
    N, K, P = 40, 3, 2
    band = rand_band(N, K, 1.0, 51)
    b = O.spmv(band, N, K, G.x_true(N, 51))
    w = G.adjoint_seed(N, 51)

    def loss(bd, bb):
        x, info, _ = O.solve(bd, N, K, bb, P, O.SAP_C, tol=1e-14)
        assert info.status == O.OK
        return w @ x

    x, _, _ = O.solve(band, N, K, b, P, O.SAP_C, tol=1e-14)
    lam, _, _ = O.solve_adjoint(band, N, K, w, P, O.SAP_C, tol=1e-14)
    gb = O.grad_band(N, K, lam, x)
    rng = np.random.default_rng(0)
    valid = [k for k in range(band.size) if 0 <= (k % N) + (k // N) - K < N]
    for k in rng.choice(valid, 25, replace=False):
        h = 1e-5 * max(1.0, abs(band[k]))
        bp, bm = band.copy(), band.copy()
        bp[k] += h; bm[k] -= h
        fd = (loss(bp, b) - loss(bm, b)) / (2 * h)
        assert abs(fd - gb[k]) <= 1e-6 * max(1.0, abs(gb[k])), (k, fd, gb[k])
    for k in rng.choice(N, 8, replace=False):
        h = 1e-5 * max(1.0, abs(b[k]))
        bp, bm = b.copy(), b.copy()
        bp[k] += h; bm[k] -= h
        fd = (loss(band, bp) - loss(band, bm)) / (2 * h)
        assert abs(fd - lam[k]) <= 1e-6 * max(1.0, abs(lam[k]))
    # padding of the band storage gets a zero gradient
    pad = [k for k in range(band.size) if not (0 <= (k % N) + (k // N) - K < N)]
    assert np.all(gb[pad] == 0.0)


# ------------------------------------------------------------ generators ---

def test_generator_dominance_and_determinism():
    """Eq. (2.6) with equality: |a_ii| = d * sum_{j != i} |a_ij|."""
    N, K, d = 500, 7, 1.2
    band = G.dense_banded(N, K, d, 99)
    A = band_to_dense(band, N, K)
    off = np.abs(A).sum(1) - np.abs(np.diag(A))
    np.testing.assert_allclose(np.diag(A), d * off, rtol=1e-14)
    np.testing.assert_array_equal(band, G.dense_banded(N, K, d, 99))
    assert not np.array_equal(band, G.dense_banded(N, K, d, 98))


def test_convection_diffusion_is_weakly_dominant_m_matrix():
    band, N, K = G.convection_diffusion(12, 9, seed=7)
    A = band_to_dense(band, N, K)
    off = A - np.diag(np.diag(A))
    assert np.all(off <= 0) and np.all(np.diag(A) > 0)
    assert np.all(np.diag(A) >= np.abs(off).sum(1) - 1e-12)
    assert K == 9 and N == 108
    assert not np.allclose(A, A.T)


# ------------------------------------------- BF16 trailing-update LU (oracle) ---

def test_bf16_round_matches_hand_computed_ties():
    """Round to nearest bfloat16, ties to even: the spacing at 1 is 2^-7."""
    from oracle.bf16tu import bf16_round
    x = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 3 * 2.0 ** -8), 1 + 2.0 ** -8 + 2.0 ** -20,
                  3.0, 0.0, 2.0 ** -130, 1 + 2.0 ** -9])
    want = np.array([1.0, 1.0, 1 + 2.0 ** -6, -(1 + 2.0 ** -6), 1 + 2.0 ** -7, 3.0, 0.0, 2.0 ** -130, 1.0])
    assert np.array_equal(bf16_round(x), want)
    # every result has at most 8 significant bits; the error is at most half a spacing
    y = np.random.default_rng(1).uniform(-4, 4, 10000)
    r = bf16_round(y)
    m, e = np.frexp(r)
    assert np.all(np.abs(m * 256 - np.round(m * 256)) == 0)
    assert np.all(np.abs(r - y) <= 2.0 ** -8 * np.abs(y) + 1e-300)


def test_blocked_lu_without_rounding_equals_plain_lu():
    """The panel organisation of the BF16 trailing-update LU is the plain
    Doolittle LU of Sec. 3.1 when the operand rounding is the identity."""
    from oracle.bf16tu import block_factors
    N, K = 300, 37
    band = rand_band(N, K, 1.0, 77)
    f = np.zeros((N, 2 * K + 1))
    b2 = band.reshape(2 * K + 1, N)
    for r in range(N):
        for d in range(-K, K + 1):
            if 0 <= r + d < N:
                f[r, d + K] = b2[K - d, r + d]
    O.block_lu(f, N, K, 0.0)
    g, nb = block_factors(band, N, K, 0, N, 0.0, rnd=lambda a: a)
    assert nb == 0
    assert np.abs(g - f).max() <= 1e-12 * np.abs(f).max()


def test_bf16_trailing_update_error_is_at_bf16_level():
    """With BF16 operands the factors reproduce the block to a BF16-level
    residual (neither exact nor garbage)."""
    from oracle.bf16tu import block_lu_panels, dense_block
    N, K = 400, 64
    band = rand_band(N, K, 1.0, 78)
    A = dense_block(band, N, K, 0, N)
    F, _ = block_lu_panels(A, K, 0.0)
    L = np.tril(F, -1) + np.eye(N)
    U = np.triu(F)
    rel = np.linalg.norm(L @ U - A) / np.linalg.norm(A)
    assert 1e-5 < rel < 1e-2, rel


# ------------------------------------------------- conjugate gradient ---
# Section 3: for a symmetric positive definite A the outer iteration is CG,
# preconditioned by the SaP factorisation (Saad, Algorithm 9.1).

def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_spd_generator_is_symmetric_positive_definite():
    N, K, d = 120, 5, 1.05
    band = G.dense_banded_spd(N, K, d, 61)
    A = band_to_dense(band, N, K)
    assert np.array_equal(A, A.T)
    off = np.abs(A).sum(1) - np.abs(np.diag(A))
    np.testing.assert_allclose(np.diag(A), d * off, rtol=1e-14)
    assert np.linalg.eigvalsh(A).min() > 0
    np.testing.assert_array_equal(band, G.dense_banded_spd(N, K, d, 61))


def test_pcg_exact_preconditioner_converges_in_one_step():
    """P = 1: M = A, so z_0 = A^{-1} b, alpha_0 = (b, A^{-1} b) / (A^{-1} b, b) = 1 and
    x_1 = A^{-1} b."""
    N, K = 300, 4
    band = G.dense_banded_spd(N, K, 1.1, 62)
    b = O.spmv(band, N, K, G.x_true(N, 62))
    x, info = O.Sap(band, N, K, 1, O.SAP_D).solve_cg(b)
    assert info.status == O.OK and info.iters == 1 and info.n_matvec == 1
    xd = np.linalg.solve(band_to_dense(band, N, K), b)
    assert _rel(x, xd) <= 1e-12


@pytest.mark.parametrize("N,K,P", [(60, 2, 3), (96, 3, 4)])
def test_pcg_finite_termination_block_jacobi(N, K, P):
    """SaP-D: M = blockdiag(A_i) and A - M is the coupling (two K x K blocks per interface),
    so M^{-1} A = I + (rank <= 2K(P-1)) has at most m = 2K(P-1)+1 distinct eigenvalues and
    CG, in exact arithmetic, ends within m steps; half as many do not suffice here."""
    band = G.dense_banded_spd(N, K, 1.0, 63 + N)
    b = O.spmv(band, N, K, G.x_true(N, 63))
    s = O.Sap(band, N, K, P, O.SAP_D)
    m = 2 * K * (P - 1) + 1
    _, full = s.solve_cg(b, tol=0.0, max_iters=m)
    _, half = s.solve_cg(b, tol=0.0, max_iters=m // 2)
    assert full.relres <= 1e-12, full.relres
    assert half.relres >= 1e-6, half.relres


@pytest.mark.parametrize("N,var,steps", [(400, O.SAP_D, (1, 2, 4, 7)), (48, O.SAP_C, (1, 2, 3))])
def test_pcg_iterates_match_scipy_cg(N, var, steps):
    """SciPy's independent preconditioned CG, given the oracle's M^{-1} as its preconditioner,
    produces the same iterate after every step count (SaP-C on short blocks, 12 = 2K rows,
    where its truncated spikes leave something to iterate on)."""
    from scipy.sparse.linalg import LinearOperator, cg
    K, P = 6, 4
    band = G.dense_banded_spd(N, K, 1.0, 64)
    A = band_to_dense(band, N, K)
    b = O.spmv(band, N, K, G.x_true(N, 64))
    s = O.Sap(band, N, K, P, var)
    Minv = LinearOperator((N, N), matvec=s.apply, dtype=np.float64)
    for k in steps:
        x, info = s.solve_cg(b, tol=0.0, max_iters=k)
        assert info.iters == k and info.n_matvec == k
        xs, _ = cg(A, b, x0=np.zeros(N), rtol=0.0, atol=0.0, maxiter=k, M=Minv)
        assert _rel(x, xs) <= 1e-11, (k, _rel(x, xs))
        assert info.relres > 1e-13          # still iterating: a meaningful comparison


@pytest.mark.parametrize("var", [O.SAP_D, O.SAP_C])
def test_pcg_solution_matches_cholesky_solve(var):
    N, K, P = 2000, 8, 5
    band = G.dense_banded_spd(N, K, 1.0, 65)
    xt = G.x_true(N, 65)
    b = O.spmv(band, N, K, xt)
    x, info, _ = O.solve_cg(band, N, K, b, P, var)
    assert info.status == O.OK and info.relres <= 1e-10
    xd = sla.solve(band_to_dense(band, N, K), b, assume_a="pos")
    assert _rel(x, xd) <= 1e-9
    xb, ib, _ = O.solve(band, N, K, b, P, var)
    assert _rel(x, xb) <= 1e-9


def test_pcg_recursive_residual_and_restart():
    """The recursive residual r_j = b - A x_j (unpreconditioned) matches the true residual
    where the exit test passes; asking for less than rounding allows makes the confirmation
    fail, which restarts the method from the true residual without losing accuracy."""
    N, K, P = 1500, 6, 6
    band = G.dense_banded_spd(N, K, 1.0, 66)
    b = O.spmv(band, N, K, G.x_true(N, 66))
    s = O.Sap(band, N, K, P, O.SAP_D)
    x, info = s.solve_cg(b, tol=1e-10, trace=True)
    t = info.trace
    assert info.status == O.OK and t[-1, 3] >= 0
    bn = np.linalg.norm(b)
    assert abs(t[-1, 1] / bn - t[-1, 3]) <= 1e-3 * t[-1, 3] + 1e-15
    np.testing.assert_array_equal(t[:, 0], np.arange(1, len(t) + 1))
    _, tight = s.solve_cg(b, tol=1e-18, max_iters=120, trace=True)
    assert tight.status == O.NOT_CONVERGED and tight.n_restarts >= 1
    assert tight.relres <= 1e-14
    # the step after the first restart is a fresh CG step from the true residual
    # r = b - A x (p = z = M^{-1} r): recompute (r, z) and ||r - alpha A z|| from x
    t = tight.trace
    row = int(np.nonzero(t[:, 3] >= 0)[0][0])
    assert row + 1 < len(t)
    xj, _ = s.solve_cg(b, tol=1e-18, max_iters=int(t[row, 0]))
    r = b - O.spmv(band, N, K, xj)
    z = s.apply(r)
    q = O.spmv(band, N, K, z)
    rz = float(r @ z)
    rn = np.linalg.norm(r - rz / float(z @ q) * q)
    assert abs(t[row + 1, 2] - rz) <= 1e-8 * abs(rz)
    assert abs(t[row + 1, 1] - rn) <= 1e-6 * rn


def test_bicgstab2_restart_equals_fresh_solve_from_current_x():
    """Both convergence-failure branches of the BiCGStab(2) exit test (reading of
    Section 4.1.1's exit points; Sleijpen-Fokkema print no residual replacement).

    Asking for 1e-18 makes the recursive residual pass its test while the true
    residual (rounding level, ~1e-16) fails the confirmation.  After matvec 4 the
    method restarts from the current x_R: r^0 = M^{-1}(b - A x_R), r~0 = r^0, with
    alpha = 0 (so the first beta is 0, which makes the u^0 = 0 and omega = 1 resets
    implied).  That is exactly a fresh solve of A y = b - A x_R from y = 0, so the
    recursive residual norms after the restart must equal the fresh solve's, row by
    row (the vectors r^j, u^j are the same arithmetic on the same data).  After
    matvec 1 or 3 a failed confirmation changes nothing, so the window between two
    restarts, which contains such a carry-on, matches as well.  b is scaled by 2^50
    (exact, so every iterate scales exactly) to put the restart at residual norms of
    order one: there a kept alpha would show, since beta = alpha rho_1 / rho_0 is not
    scale-invariant once rho_0 is reset to 1."""
    N, K, P = 300, 5, 10
    band = rand_band(N, K, 0.7, 43)
    b = O.spmv(band, N, K, G.x_true(N, 43)) * 2.0 ** 50
    s = O.Sap(band, N, K, P, O.SAP_D)
    tol = 1e-18
    x, info = s.solve(b, tol=tol, max_iters=40, trace=True)
    assert info.status == O.NOT_CONVERGED and info.n_restarts >= 2
    assert info.relres <= 1e-15                       # restarts keep the accuracy
    t = info.trace
    btn = np.linalg.norm(s.apply(b))
    passed = t[:, 1] <= tol * btn
    mv = t[:, 0].astype(int)
    restarts = np.nonzero(passed & (mv % 4 == 0))[0]
    assert len(restarts) >= 2
    r0, r1 = int(restarts[0]), int(restarts[1])
    carry_on = [k for k in range(r0 + 1, r1) if passed[k] and mv[k] % 4 in (1, 3)]
    assert carry_on, "the window must contain a failed confirmation after matvec 1 or 3"
    # x_R: the iterate at the first restart (the restart does not move x)
    xr, ir = s.solve(b, tol=tol, max_iters=mv[r0] // 4)
    assert ir.n_restarts == 1
    bp = b - O.spmv(band, N, K, xr)
    _, fresh = s.solve(bp, tol=tol, max_iters=(mv[r1] - mv[r0]) // 4 + 1, trace=True)
    tf = fresh.trace
    window = t[r0 + 1:r1 + 1]
    np.testing.assert_array_equal(window[:, 0] - mv[r0], tf[:len(window), 0])
    np.testing.assert_allclose(window[:, 1], tf[:len(window), 1], rtol=1e-12, atol=0)
    # and the true residual keeps tracking: the restarted iterate is x_R + y
    assert abs(t[r0, 2] - np.linalg.norm(s.apply(bp))) <= 1e-12 * t[r0, 2]


@pytest.mark.parametrize("var", [O.SAP_D, O.SAP_C])
def test_openmp_build_is_bit_identical(var):
    """The CPU baseline's multi-core leg: the oracle built with -fopenmp runs
    the independent blocks in parallel (factor, tips, applies) with every
    block's arithmetic unchanged, so factors, applies and the whole solve
    equal the single-threaded build's bit for bit."""
    N, K, P = 6000, 12, 12
    band = rand_band(N, K, 1.0, 91)
    b = O.spmv(band, N, K, G.x_true(N, 91))
    s1 = O.Sap(band, N, K, P, var)
    s2 = O.Sap(band, N, K, P, var, omp=True)
    for i in (0, 5, P - 1):
        np.testing.assert_array_equal(s1.block(i), s2.block(i))
    r = G.adjoint_seed(N, 91)
    np.testing.assert_array_equal(s1.apply(r), s2.apply(r))
    x1, i1 = s1.solve(b)
    x2, i2 = s2.solve(b)
    np.testing.assert_array_equal(x1, x2)
    assert (i1.iters, i1.n_matvec, i1.n_restarts) == (i2.iters, i2.n_matvec, i2.n_restarts)
    assert O.omp_threads() >= 1
