"""Python front end of the FP64 CPU oracle (``sap_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this module; the library itself never
imports it.  It shares no code with the CUDA path.

The C file is compiled with gcc into ``_liboracle.so`` next to it on first
use (or by :func:`build`).  Every routine works on float64 numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sap_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_LIB_OMP = os.path.join(_HERE, "_liboracle_omp.so")

OK, INVALID_ARG, OOM, NOT_CONVERGED, BREAKDOWN, SINGULAR = 0, 1, 2, 3, 4, 8
SAP_D, SAP_C = 0, 1
FP64_EPS = 2.0 ** -53
FP32_EPS = 2.0 ** -24


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no FMA
    contraction so that every operation rounds as written).  omp=True builds
    the OpenMP variant (the per-block loops in parallel, same arithmetic)."""
    out = _LIB_OMP if omp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"] +
                              (["-fopenmp"] if omp else []) + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


_lib = None
_lib_omp = None


def _load(omp: bool = False):
    global _lib, _lib_omp
    if omp:
        if _lib_omp is None:
            _lib_omp = _declare(C.CDLL(build(omp=True)))
        return _lib_omp
    if _lib is None:
        _lib = _declare(C.CDLL(build()))
    return _lib


def omp_threads() -> int:
    """Threads the OpenMP variant uses (its OMP_NUM_THREADS / the host's cores)."""
    lib = _load(omp=True)
    try:
        f = lib.omp_get_max_threads
    except AttributeError:
        return 1
    f.restype = C.c_int
    return int(f())


def _declare(lib):
    if True:
        i64, i32, dbl, vp = C.c_int64, C.c_int32, C.c_double, C.c_void_p
        P = C.POINTER
        lib.orc_partition.argtypes = [i64, i32, P(i64)]
        lib.orc_spmv.argtypes = [P(dbl), i64, C.c_int, P(dbl), P(dbl), C.c_int]
        lib.orc_factor.argtypes = [P(dbl), i64, C.c_int, C.c_int, C.c_int, dbl, P(vp)]
        lib.orc_factor.restype = C.c_int
        lib.orc_free.argtypes = [vp]
        lib.orc_apply.argtypes = [vp, P(dbl), P(dbl)]
        lib.orc_bicgstab2.argtypes = [vp, P(dbl), P(dbl), P(dbl), dbl, C.c_int, vp, P(dbl), C.c_int]
        lib.orc_bicgstab2.restype = C.c_int
        lib.orc_pcg.argtypes = [vp, P(dbl), P(dbl), P(dbl), dbl, C.c_int, vp, P(dbl), C.c_int]
        lib.orc_pcg.restype = C.c_int
        lib.orc_transpose_band.argtypes = [P(dbl), i64, C.c_int, P(dbl)]
        lib.orc_grad_band.argtypes = [i64, C.c_int, P(dbl), P(dbl), P(dbl)]
        lib.orc_n_boosted.argtypes = [vp]
        lib.orc_n_boosted.restype = i64
        lib.orc_offsets.argtypes = [vp, P(i64)]
        lib.orc_get_block.argtypes = [vp, C.c_int, C.c_int, P(dbl)]
        lib.orc_get_block.restype = C.c_int
        lib.orc_get_interface.argtypes = [vp, C.c_int, C.c_int, P(dbl)]
        lib.orc_get_interface.restype = C.c_int
        lib.orc_band_absmax.argtypes = [P(dbl), i64, C.c_int]
        lib.orc_band_absmax.restype = dbl
        lib.orc_block_lu.argtypes = [P(dbl), i64, C.c_int, dbl]
        lib.orc_block_lu.restype = i64
        lib.orc_block_ul.argtypes = [P(dbl), i64, C.c_int, dbl]
        lib.orc_block_ul.restype = i64
        lib.orc_dense_getrf.argtypes = [P(dbl), C.c_int, P(i32)]
        lib.orc_dense_getrf.restype = C.c_int
        lib.orc_dense_getrs.argtypes = [P(dbl), C.c_int, P(i32), P(dbl)]
        lib.orc_reduced_solve.argtypes = [vp, C.c_int, P(dbl), P(dbl), P(dbl), P(dbl)]
    return lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _Info(C.Structure):
    _fields_ = [("iters", C.c_double), ("relres", C.c_double),
                ("n_matvec", C.c_int64), ("n_restarts", C.c_int64)]


@dataclass
class SolveInfo:
    status: int
    iters: float
    relres: float
    n_matvec: int
    n_restarts: int
    trace: np.ndarray | None = None


def partition(N: int, P: int) -> np.ndarray:
    """Block offsets (P+1) of Section 3.1."""
    off = np.zeros(P + 1, dtype=np.int64)
    _load().orc_partition(N, P, off.ctypes.data_as(C.POINTER(C.c_int64)))
    return off


def spmv(band: np.ndarray, N: int, K: int, x: np.ndarray, transpose: bool = False) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(N)
    _load().orc_spmv(_d(band), N, K, _d(x), _d(y), int(transpose))
    return y


def band_absmax(band: np.ndarray, N: int, K: int) -> float:
    return _load().orc_band_absmax(_d(band), N, K)


def transpose_band(band: np.ndarray, N: int, K: int) -> np.ndarray:
    out = np.empty_like(band)
    _load().orc_transpose_band(_d(band), N, K, _d(out))
    return out


def grad_band(N: int, K: int, lam: np.ndarray, x: np.ndarray) -> np.ndarray:
    g = np.empty((2 * K + 1) * N)
    _load().orc_grad_band(N, K, _d(np.ascontiguousarray(lam)), _d(np.ascontiguousarray(x)), _d(g))
    return g


def block_lu(f: np.ndarray, n: int, K: int, tau: float) -> int:
    """In-place LU of a dense-band row-major block (n x (2K+1)); returns boosts."""
    return int(_load().orc_block_lu(_d(f), n, K, tau))


def block_ul(f: np.ndarray, n: int, K: int, tau: float) -> int:
    return int(_load().orc_block_ul(_d(f), n, K, tau))


def dense_getrf(a: np.ndarray):
    a = np.ascontiguousarray(a, dtype=np.float64).copy()
    n = a.shape[0]
    piv = np.zeros(n, dtype=np.int32)
    st = _load().orc_dense_getrf(_d(a), n, piv.ctypes.data_as(C.POINTER(C.c_int32)))
    return st, a, piv


def dense_getrs(lu: np.ndarray, piv: np.ndarray, b: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(b, dtype=np.float64).copy()
    _load().orc_dense_getrs(_d(np.ascontiguousarray(lu)), lu.shape[0],
                            piv.ctypes.data_as(C.POINTER(C.c_int32)), _d(x))
    return x


class Sap:
    """The oracle's SaP preconditioner for one banded matrix.

    ``boost_eps`` is relative: the boosting threshold is
    tau = boost_eps * max |a_ij| over the band (default: FP64 unit roundoff)."""

    def __init__(self, band: np.ndarray, N: int, K: int, P: int, variant: int = SAP_D,
                 boost_eps: float | None = None, tau: float | None = None, omp: bool = False):
        self._L = _load(omp)
        self.band = np.ascontiguousarray(band, dtype=np.float64)
        self.N, self.K, self.P, self.variant = int(N), int(K), int(P), int(variant)
        if tau is None:
            eps = FP64_EPS if boost_eps is None else boost_eps
            tau = eps * band_absmax(self.band, N, K)
        self.tau = float(tau)
        h = C.c_void_p()
        st = self._L.orc_factor(_d(self.band), N, K, P, variant, self.tau, C.byref(h))
        if st != OK:
            raise ValueError(f"oracle factor failed with status {st}")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) is not None and getattr(self, "_L", None) is not None:
            self._L.orc_free(self._h)
            self._h = None

    @property
    def n_boosted(self) -> int:
        return int(self._L.orc_n_boosted(self._h))

    @property
    def offsets(self) -> np.ndarray:
        off = np.zeros(self.P + 1, dtype=np.int64)
        self._L.orc_offsets(self._h, off.ctypes.data_as(C.POINTER(C.c_int64)))
        return off

    def block(self, i: int, which: int = 0) -> np.ndarray:
        """Factors of block i, dense-band row-major (n_i, 2K+1); which 0 = LU, 1 = UL."""
        off = self.offsets
        n = int(off[i + 1] - off[i])
        out = np.empty((n, 2 * self.K + 1))
        if self._L.orc_get_block(self._h, i, which, _d(out)) != OK:
            raise ValueError("no such block")
        return out

    def interface(self, i: int, which: str) -> np.ndarray:
        """K x K matrix of interface i: 'B', 'C', 'V', 'W' or 'R' (unfactored Rbar)."""
        code = {"B": 0, "C": 1, "V": 2, "W": 3, "R": 4}[which]
        out = np.empty((self.K, self.K))
        if self._L.orc_get_interface(self._h, i, code, _d(out)) != OK:
            raise ValueError("no such interface")
        return out

    def reduced_solve(self, i: int, gb: np.ndarray, gt: np.ndarray):
        """Truncated reduced solve of interface i (Eq. (2.5)); returns (xb, xt)."""
        gb = np.ascontiguousarray(gb, dtype=np.float64)
        gt = np.ascontiguousarray(gt, dtype=np.float64)
        xb, xt = np.empty(self.K), np.empty(self.K)
        self._L.orc_reduced_solve(self._h, i, _d(gb), _d(gt), _d(xb), _d(xt))
        return xb, xt

    def apply(self, r: np.ndarray) -> np.ndarray:
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.empty(self.N)
        self._L.orc_apply(self._h, _d(r), _d(z))
        return z

    def solve(self, b: np.ndarray, tol: float = 1e-10, max_iters: int = 500,
              trace: bool = False) -> tuple[np.ndarray, SolveInfo]:
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty(self.N)
        info = _Info()
        cap = 4 * max_iters + 8
        tr = np.zeros(4 * cap) if trace else None
        st = self._L.orc_bicgstab2(self._h, _d(self.band), _d(b), _d(x), tol, max_iters,
                                   C.byref(info), _d(tr) if trace else None, cap)
        t = None
        if trace:
            t = tr.reshape(-1, 4)
            t = t[t[:, 0] > 0]
        return x, SolveInfo(st, info.iters, info.relres, info.n_matvec, info.n_restarts, t)

    def solve_cg(self, b: np.ndarray, tol: float = 1e-10, max_iters: int = 500,
                 trace: bool = False) -> tuple[np.ndarray, SolveInfo]:
        """Preconditioned conjugate gradient for an SPD A (Section 3), M the
        SaP factorisation; iterations are whole CG steps.  trace rows:
        (iteration, ||r||, (r, z) before the step, true relres or -1)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty(self.N)
        info = _Info()
        cap = max_iters + 2
        tr = np.zeros(4 * cap) if trace else None
        st = self._L.orc_pcg(self._h, _d(self.band), _d(b), _d(x), tol, max_iters,
                             C.byref(info), _d(tr) if trace else None, cap)
        t = None
        if trace:
            t = tr.reshape(-1, 4)
            t = t[t[:, 0] > 0]
        return x, SolveInfo(st, info.iters, info.relres, info.n_matvec, info.n_restarts, t)


def solve_cg(band, N, K, b, P, variant=SAP_D, tol=1e-10, max_iters=500, **kw):
    """Factor and solve the SPD system A x = b by preconditioned CG; returns
    (x, info, sap)."""
    s = Sap(band, N, K, P, variant, **kw)
    x, info = s.solve_cg(b, tol=tol, max_iters=max_iters)
    return x, info, s


def solve(band, N, K, b, P, variant=SAP_D, tol=1e-10, max_iters=500, **kw):
    """Factor and solve A x = b with the oracle; returns (x, info, sap)."""
    s = Sap(band, N, K, P, variant, **kw)
    x, info = s.solve(b, tol=tol, max_iters=max_iters)
    return x, info, s


def solve_adjoint(band, N, K, gbar, P, variant=SAP_D, tol=1e-10, max_iters=500, **kw):
    """Solve A^T lambda = gbar with SaP built on A^T (same partition)."""
    bt = transpose_band(band, N, K)
    s = Sap(bt, N, K, P, variant, **kw)
    lam, info = s.solve(gbar, tol=tol, max_iters=max_iters)
    return lam, info, s
