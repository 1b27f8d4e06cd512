"""Oracle of the sparse front end (Sec. 2.2: diagonal boosting, Cuthill-McKee
bandwidth reduction, band assembly), plain numpy / Python, for the small
matrices of the tests.

TEST INFRASTRUCTURE ONLY: the tests may use this module; the library never
imports it, and it shares no code with the library (whose matching is a sparse
Dijkstra search and whose ordering is C++; here the matching is the textbook
dense Hungarian method and the ordering a direct transcription of the rule).

Conventions: CSR with int64 row pointers, int32 column indices sorted within
each row, float64 values.  A permutation p given as "new index of old index"
(p[old] = new).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

INF = math.inf


def csr_to_dense(n, rowptr, col, val):
    A = np.zeros((n, n))
    for i in range(n):
        for p in range(rowptr[i], rowptr[i + 1]):
            A[i, col[p]] = val[p]
    return A


# ---- Diagonal boosting (Sec. 2.2, Eq. (DBrelated)) ----

def db_costs(n, rowptr, col, val):
    """a_i = max_j |a_ij| and the edge weights c_ij = log a_i - log |a_ij|
    (infinite for a zero entry), one per stored entry."""
    a = np.zeros(n)
    c = np.empty(len(val))
    for i in range(n):
        lo, hi = rowptr[i], rowptr[i + 1]
        a[i] = max((abs(val[p]) for p in range(lo, hi)), default=0.0)
        for p in range(lo, hi):
            c[p] = math.log(a[i]) - math.log(abs(val[p])) if val[p] != 0.0 else INF
    return a, c


def hungarian(cost):
    """Minimum-cost perfect assignment of a dense n x n cost matrix (INF =
    no edge) by the Hungarian method in its shortest-augmenting-path form:
    rows are added one at a time; a Dijkstra-like scan over the columns with
    reduced costs cost[i][j] - u[i] - v[j] finds the cheapest way to place
    the new row, the potentials are updated by the scan distances and the
    path is flipped.  Returns (assign[row] = column, u, v) with
    cost[i][j] - u[i] - v[j] >= 0 for every edge and = 0 on the assignment.
    Raises ValueError when no perfect assignment exists."""
    n = len(cost)
    u = [0.0] * (n + 1)            # potentials, 1-based with a dummy 0
    v = [0.0] * (n + 1)
    match = [0] * (n + 1)          # match[j] = row (1-based) on column j, 0 = free
    way = [0] * (n + 1)
    for i in range(1, n + 1):
        match[0] = i
        j0 = 0
        minv = [INF] * (n + 1)
        used = [False] * (n + 1)
        while True:
            used[j0] = True
            i0 = match[j0]
            delta, j1 = INF, -1
            for j in range(1, n + 1):
                if used[j]:
                    continue
                cij = cost[i0 - 1][j - 1]
                cur = cij - u[i0] - v[j] if cij != INF else INF
                if cur < minv[j]:
                    minv[j] = cur
                    way[j] = j0
                if minv[j] < delta:
                    delta, j1 = minv[j], j
            if j1 < 0 or delta == INF:
                raise ValueError("structurally singular: no perfect matching")
            for j in range(n + 1):
                if used[j]:
                    u[match[j]] += delta
                    v[j] -= delta
                else:
                    minv[j] -= delta
            j0 = j1
            if match[j0] == 0:
                break
        while True:                # flip the augmenting path
            j1 = way[j0]
            match[j0] = match[j1]
            j0 = j1
            if j0 == 0:
                break
    assign = [0] * n
    for j in range(1, n + 1):
        assign[match[j] - 1] = j - 1
    return np.array(assign, dtype=np.int64), np.array(u[1:]), np.array(v[1:])


@dataclass
class DBResult:
    sigma: np.ndarray     # sigma[i] = column matched to row i = the new index of row i
    a: np.ndarray         # row maxima
    u: np.ndarray         # row potentials
    v: np.ndarray         # column potentials
    cost: float           # sum_i c_{i sigma_i}
    logprod: float        # sum_i log |a_{i sigma_i}|


def db_match(n, rowptr, col, val):
    """The permutation sigma maximising prod_i |a_{i sigma(i)}|, i.e. the
    minimum perfect matching of the bipartite graph with weights c_ij
    (Sec. 2.2), and the dual potentials of the assignment."""
    a, c = db_costs(n, rowptr, col, val)
    cost = [[INF] * n for _ in range(n)]
    for i in range(n):
        for p in range(rowptr[i], rowptr[i + 1]):
            cost[i][col[p]] = c[p]
    sigma, u, v = hungarian(cost)
    tot = sum(cost[i][sigma[i]] for i in range(n))
    lp = 0.0
    for i in range(n):
        for p in range(rowptr[i], rowptr[i + 1]):
            if col[p] == sigma[i]:
                lp += math.log(abs(val[p]))
    return DBResult(sigma, a, u, v, tot, lp)


def db_scaling(a, u, v):
    """Row and column scale factors from the potentials: r_i = exp(u_i) / a_i,
    s_j = exp(v_j); then |r_i a_ij s_j| = exp(u_i + v_j - c_ij) <= 1 with
    equality on the matching (an I-matrix after the row permutation)."""
    return np.exp(u) / a, np.exp(v)


# ---- Cuthill-McKee (Sec. 2.2 bandwidth reduction, Sec. 3.3) ----

def sym_pattern(n, rowptr, col, rownew=None):
    """Neighbour lists (sorted, no self loops) of the pattern of B + B^T,
    B the matrix with row i moved to rownew[i] (identity if None)."""
    nb = [set() for _ in range(n)]
    for i in range(n):
        r = i if rownew is None else int(rownew[i])
        for p in range(rowptr[i], rowptr[i + 1]):
            j = int(col[p])
            if j != r:
                nb[r].add(j)
                nb[j].add(r)
    return [sorted(s) for s in nb]


CM_MAX_STARTS = 5


def _levels(nb, start, alive):
    """BFS levels from start over the nodes in `alive`."""
    lev = [[start]]
    seen = {start}
    while True:
        nxt = []
        for x in lev[-1]:
            for y in nb[x]:
                if y in alive and y not in seen:
                    seen.add(y)
                    nxt.append(y)
        if not nxt:
            return lev
        lev.append(nxt)


def cm_order(n, nb):
    """Cuthill-McKee ordering (Sec. 2.2): a BFS in which the unvisited
    neighbours of each node are taken in non-descending degree.  Per connected
    component: start from its node of lowest degree (lowest index on ties);
    up to CM_MAX_STARTS trials, each next start the not yet tried node of
    lowest degree in the last BFS level; a trial is kept while its tree is
    taller and narrower (fewer nodes in its widest level) than the best so
    far, else the search stops (Sec. 3.3).  Ties in degree go to the lower
    index.  Returns perm with perm[old] = new."""
    deg = [len(x) for x in nb]
    key = lambda x: (deg[x], x)
    remaining = set(range(n))
    order = []
    while remaining:
        s = min(remaining, key=key)
        comp = set()
        best = None
        tried = set()
        for _ in range(CM_MAX_STARTS):
            lev = _levels(nb, s, remaining)
            if not comp:
                comp = set(y for L in lev for y in L)
            h, w = len(lev), max(len(L) for L in lev)
            if best is None:
                best = (s, h, w)
            elif h > best[1] and w < best[2]:
                best = (s, h, w)
            else:
                break
            tried.add(s)
            cand = [y for y in lev[-1] if y not in tried]
            if not cand:
                break
            s = min(cand, key=key)
        start = best[0]
        seen = {start}
        q = [start]
        k = 0
        while k < len(q):
            x = q[k]
            k += 1
            for y in sorted((y for y in nb[x] if y in comp and y not in seen), key=key):
                seen.add(y)
                q.append(y)
        order.extend(q)
        remaining -= comp
    perm = np.empty(n, dtype=np.int64)
    perm[np.array(order, dtype=np.int64)] = np.arange(n)
    return perm


# ---- bandwidth and band assembly ----

def bandwidth(n, rowptr, col, rownew, colnew):
    """max |rownew[i] - colnew[j]| over the stored entries (i, j)."""
    K = 0
    for i in range(n):
        for p in range(rowptr[i], rowptr[i + 1]):
            K = max(K, abs(int(rownew[i]) - int(colnew[col[p]])))
    return K


def to_band(n, rowptr, col, val, rownew, colnew, K, r=None, s=None, drop=False):
    """Band storage ((2K+1) * n, band[(K + I - J) * n + J] = entry (I, J)) of
    the matrix with entry (i, j) moved to (rownew[i], colnew[j]) and scaled to
    (r_i a_ij) s_j when scale factors are given.  An entry outside the band is
    dropped (drop) or an error."""
    band = np.zeros((2 * K + 1) * n)
    for i in range(n):
        I = int(rownew[i])
        for p in range(rowptr[i], rowptr[i + 1]):
            j = int(col[p])
            J = int(colnew[j])
            if abs(I - J) > K:
                if drop:
                    continue
                raise ValueError("entry outside the band")
            x = val[p] if r is None else (r[i] * val[p]) * s[j]
            band[(K + I - J) * n + J] = x
    return band


# ---- element drop-off (Sec. 2.2) ----

def dist_weights(n, rowptr, col, val, rownew, colnew, K, r=None, s=None):
    """w[d] = sum of |(r_i a_ij) s_j| over the entries at distance |I - J| = d."""
    w = np.zeros(K + 1)
    for i in range(n):
        I = int(rownew[i])
        for p in range(rowptr[i], rowptr[i + 1]):
            j = int(col[p])
            d = abs(I - int(colnew[j]))
            w[d] += abs(val[p]) if r is None else abs((r[i] * val[p]) * s[j])
    return w


def drop_bandwidth(w, frac):
    """The smallest K' with sum_{d > K'} w[d] <= frac * sum_d w[d]."""
    total = float(np.sum(w))
    for Kp in range(len(w)):
        if float(np.sum(w[Kp + 1:])) <= frac * total:
            return Kp
    return len(w) - 1
