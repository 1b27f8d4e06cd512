"""Third-stage reordering and SaP with a bandwidth of its own per block
(Sec. 2.2, "Third-stage reordering"; Sec. 3.1, "Use of registers and shared
memory").

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU leg of ``bench.py`` may use this module; the library never imports it.
It shares no code with the CUDA path.  Plain FP64 numpy, row loops.

After the DB and CM reorderings the band of A (half-bandwidth K) is split
into the blocks A_i of the partition, and a third CM pass reorders every
block on its own: Ahat_i = Pi_i A_i Pi_i^T, with the half-bandwidth K_i of
Ahat_i.  The blocks are factored Ahat_i = L_i U_i (no pivoting, boosted
pivots).  The coupling blocks B_i, C_{i+1} keep their places in the global
numbering, so in the new numbering of a block the rows they touch are spread
over the whole block: SaP-C computes the entire spikes A_i^{-1}[0; B_i] and
A_{i+1}^{-1}[C_{i+1}; 0] by multi-right-hand-side solves with the factors of
Ahat_i, and takes the tips V^(b)_i, W^(t)_{i+1} (the spike rows at the
interface, in the old numbering) out of them; no UL factorisation is used.
The preconditioner is then the one of Eq. (2.3)-(2.5) on A: in exact
arithmetic it does not depend on how the blocks are ordered or factored.

Permutations are "new index of old index": perm[s_i + a] = new local index
of local row/column a of block i (s_i its first row).
"""
from __future__ import annotations

import numpy as np

from . import FP64_EPS, SAP_C, SAP_D, band_absmax, block_lu, dense_getrf, dense_getrs, partition
from . import sparse as _sparse


def _bands(band, N, K):
    return np.asarray(band, dtype=np.float64).reshape(2 * K + 1, N)


def block_entries(band, N, K, s, n):
    """Stored entries (a, b, value) of block [s, s+n) of the band, local
    indices, zeros left out (Sec. 3.1 storage: a_ij at band[(K+i-j) N + j])."""
    B = _bands(band, N, K)
    rows, cols, vals = [], [], []
    for c in range(2 * K + 1):
        off = c - K                       # i = j + off
        j0, j1 = max(s, s - off), min(s + n, s + n - off)
        if j1 <= j0:
            continue
        j = np.arange(j0, j1)
        v = B[c, j0:j1]
        nz = v != 0.0
        rows.append(j[nz] + off - s)
        cols.append(j[nz] - s)
        vals.append(v[nz])
    if not rows:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0)
    return np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)


def block_pattern(band, N, K, s, n):
    """Neighbour lists of the pattern of A_i + A_i^T (off-diagonal nonzeros)."""
    a, b, _ = block_entries(band, N, K, s, n)
    nb = [set() for _ in range(n)]
    for x, y in zip(a.tolist(), b.tolist()):
        if x != y:
            nb[x].add(y)
            nb[y].add(x)
    return [sorted(t) for t in nb]


def block_bandwidth(band, N, K, s, n, p):
    """Half-bandwidth of Pi A_i Pi^T: max |p(a) - p(b)| over the nonzeros."""
    a, b, _ = block_entries(band, N, K, s, n)
    return int(np.abs(p[a] - p[b]).max()) if len(a) else 0


def block_cm(band, N, K, P):
    """The third-stage reordering: Cuthill-McKee (the multi-start rule of
    Sec. 3.3) of every block's A_i + A_i^T on its own.  Returns (perm, K_i)."""
    off = partition(N, P)
    perm = np.zeros(N, dtype=np.int64)
    Ks = np.zeros(P, dtype=np.int64)
    for i in range(P):
        s, n = int(off[i]), int(off[i + 1] - off[i])
        p = np.asarray(_sparse.cm_order(n, block_pattern(band, N, K, s, n)), dtype=np.int64)
        perm[s:s + n] = p
        Ks[i] = block_bandwidth(band, N, K, s, n, p)
    return perm, Ks


def _tip_rows_v(p, n, K):
    """New-numbering rows of the old bottom K rows of a block (V^(b))."""
    return p[n - K:]


def _tip_rows_w(p, K):
    """New-numbering rows of the old top K rows of a block (W^(t))."""
    return p[:K]


def _to_new(p, v):
    """Pi v: the entry of old row a moves to row p(a)."""
    u = np.zeros_like(v)
    u[p] = v
    return u


def _to_old(p, u):
    """Pi^T u."""
    return u[p]


class BlockSap:
    """The SaP preconditioner of A with every block A_i factored after its
    own symmetric reordering Pi_i (half-bandwidth K_i >= 1 of Ahat_i).

    ``boost_eps`` is relative: tau = boost_eps * max |a_ij| over the band of
    A (default: FP64 unit roundoff), as for the unreordered preconditioner."""

    def __init__(self, band, N, K, P, perm, variant=SAP_D, boost_eps=None, tau=None):
        self.band = np.ascontiguousarray(band, dtype=np.float64)
        self.N, self.K, self.P, self.variant = int(N), int(K), int(P), int(variant)
        self.off = partition(N, P)
        perm = np.asarray(perm, dtype=np.int64)
        if tau is None:
            tau = (FP64_EPS if boost_eps is None else boost_eps) * band_absmax(self.band, N, K)
        self.tau = float(tau)
        self.perm, self.Ki, self.lu = [], [], []
        self.n_boosted = 0
        for i in range(P):
            s, n = int(self.off[i]), int(self.off[i + 1] - self.off[i])
            p = perm[s:s + n]
            if sorted(p.tolist()) != list(range(n)):
                raise ValueError(f"block {i}: not a permutation")
            a, b, v = block_entries(self.band, N, K, s, n)
            Ki = max(1, int(np.abs(p[a] - p[b]).max()) if len(a) else 0)
            W = 2 * Ki + 1
            f = np.zeros(n * W)                    # row-major dense band of Ahat_i
            f[p[a] * W + (p[b] - p[a] + Ki)] = v
            self.n_boosted += block_lu(f, n, Ki, self.tau)
            self.perm.append(p)
            self.Ki.append(Ki)
            self.lu.append(f.reshape(n, W))
        self.Ki = np.array(self.Ki)
        self.B, self.C, self.Vfull, self.Wfull = [], [], [], []
        self.Vb, self.Wt, self.R = [], [], []
        if self.variant == SAP_C and P > 1:
            self._spikes()

    # ---- blocks ----
    def block_solve(self, i, y):
        """Ahat_i^{-1} y (y: n_i x m, or n_i), forward with the unit-lower L_i,
        backward with U_i, in the block's new numbering."""
        f, Ki = self.lu[i], int(self.Ki[i])
        n = f.shape[0]
        y = np.array(y, dtype=np.float64, copy=True)
        for r in range(n):
            lo = max(0, r - Ki)
            if r > lo:
                y[r] -= f[r, Ki - (r - lo):Ki] @ y[lo:r]
        for r in range(n - 1, -1, -1):
            hi = min(n, r + Ki + 1)
            if hi > r + 1:
                y[r] -= f[r, Ki + 1:Ki + (hi - r)] @ y[r + 1:hi]
            y[r] /= f[r, Ki]
        return y

    def block_apply(self, i, v):
        """A_i^{-1} v in the old numbering: Pi_i^T Ahat_i^{-1} Pi_i v."""
        p = self.perm[i]
        return _to_old(p, self.block_solve(i, _to_new(p, v)))

    # ---- SaP-C factor phase ----
    def coupling(self, i):
        """B_i and C_{i+1} of interface i (K x K, Sec. 2.1): B_i(r, q) =
        a(s-K+r, s+q), C_{i+1}(r, q) = a(s+r, s-K+q), s = first row of block i+1."""
        Bd = _bands(self.band, self.N, self.K)
        K, s = self.K, int(self.off[i + 1])
        Bm, Cm = np.zeros((K, K)), np.zeros((K, K))
        for r in range(K):
            for q in range(K):
                if q <= r:
                    Bm[r, q] = Bd[K + (s - K + r) - (s + q), s + q]
                if q >= r:
                    Cm[r, q] = Bd[K + (s + r) - (s - K + q), s - K + q]
        return Bm, Cm

    def _spikes(self):
        K = self.K
        for i in range(self.P - 1):
            n0 = int(self.off[i + 1] - self.off[i])
            n1 = int(self.off[i + 2] - self.off[i + 1])
            Bm, Cm = self.coupling(i)
            p0, p1 = self.perm[i], self.perm[i + 1]
            rv = np.zeros((n0, K))
            rv[n0 - K:] = Bm                       # [0; B_i] in the old numbering of block i
            rw = np.zeros((n1, K))
            rw[:K] = Cm                            # [C_{i+1}; 0] in that of block i+1
            Vh = self.block_solve(i, _to_new(p0, rv))        # entire spikes, new numbering
            Wh = self.block_solve(i + 1, _to_new(p1, rw))
            Vb = Vh[_tip_rows_v(p0, n0, K)]                   # V^(b)_i
            Wt = Wh[_tip_rows_w(p1, K)]                       # W^(t)_{i+1}
            R = np.eye(K) - Wt @ Vb                           # Eq. (2.5a)
            st, lu, piv = dense_getrf(R)
            if st != 0:
                raise ValueError(f"interface {i}: singular reduced matrix")
            self.B.append(Bm)
            self.C.append(Cm)
            self.Vfull.append(Vh)
            self.Wfull.append(Wh)
            self.Vb.append(Vb)
            self.Wt.append(Wt)
            self.R.append((R, lu, piv))

    # ---- application z = M^{-1} r ----
    def apply(self, r):
        r = np.asarray(r, dtype=np.float64)
        off, K = self.off, self.K
        g = np.concatenate([self.block_apply(i, r[off[i]:off[i + 1]]) for i in range(self.P)])
        if self.variant == SAP_D or self.P == 1:
            return g                                             # Eq. (2.3)
        xb, xt = [], []
        for i in range(self.P - 1):                              # Eq. (2.5b,c)
            s = int(off[i + 1])
            gb, gt = g[s - K:s], g[s:s + K]
            _, lu, piv = self.R[i]
            x_t = dense_getrs(lu, piv, gt - self.Wt[i] @ gb)
            xb.append(gb - self.Vb[i] @ x_t)
            xt.append(x_t)
        z = np.empty(self.N)
        for i in range(self.P):
            s, e = int(off[i]), int(off[i + 1])
            ri = r[s:e].copy()
            if i > 0:
                ri[:K] -= self.C[i - 1] @ xb[i - 1]
            if i < self.P - 1:
                ri[e - s - K:] -= self.B[i] @ xt[i]
            z[s:e] = self.block_apply(i, ri)
        return z
