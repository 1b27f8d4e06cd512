"""GB300-native dense-banded SaP solver: Python binding of libsap.

The binding is argument marshalling only: every step of the solver runs in
the CUDA kernels of ``libsap.so`` (built in-tree by ``_build.build()``).
Importing this package loads the library and raises if it is missing; there
is no CPU fallback.  Tensors are torch CUDA float64 tensors; the stream is
torch's current CUDA stream unless one is given.

The functions below carry the names of the C entry points in
``include/sap.h``.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsap.so")

SAP_OK, SAP_ERR_INVALID_ARG, SAP_ERR_OOM, SAP_ERR_NOT_CONVERGED, SAP_ERR_BREAKDOWN = 0, 1, 2, 3, 4
SAP_ERR_TIMEOUT, SAP_ERR_CUDA, SAP_ERR_NOT_IMPLEMENTED, SAP_ERR_SINGULAR = 5, 6, 7, 8
SAP_D, SAP_C = 0, 1
SAP_FP64, SAP_FP32, SAP_FP32_BF16TU = 0, 1, 2
SAP_KRYLOV_BICGSTAB2, SAP_KRYLOV_CG = 0, 1


class SapError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {sap_status_string(status)} (status {status})")


class sap_options_t(C.Structure):
    _fields_ = [("P", C.c_int32), ("variant", C.c_int32), ("precision", C.c_int32),
                ("max_iters", C.c_int32), ("tol", C.c_double), ("boost_eps", C.c_double),
                ("spin_limit", C.c_int64), ("segments", C.c_int32), ("krylov", C.c_int32)]


class sap_info_t(C.Structure):
    _fields_ = [("iters", C.c_double), ("relres", C.c_double), ("n_boosted", C.c_int64),
                ("n_matvec", C.c_int64), ("n_restarts", C.c_int64),
                ("t_factor_ms", C.c_float), ("t_solve_ms", C.c_float), ("t_lu_ms", C.c_float),
                ("t_ul_ms", C.c_float), ("t_spk_ms", C.c_float), ("segments", C.c_int32),
                ("graphed", C.c_int32), ("tc_update", C.c_int32), ("P", C.c_int32),
                ("t_bc_ms", C.c_float), ("t_rdcd_ms", C.c_float), ("t_kry_ms", C.c_float),
                ("t_prep_ms", C.c_float), ("reserved1", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsap.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    P = C.POINTER
    sig = {
        "sap_default_options": (None, [P(sap_options_t)]),
        "sap_factor": (C.c_int, [vp, i64, i32, P(sap_options_t), vp, P(vp)]),
        "sap_refactor": (C.c_int, [vp, vp]),
        "sap_solve": (C.c_int, [vp, vp, vp, P(sap_info_t), vp]),
        "sap_solve_adjoint": (C.c_int, [vp, vp, vp, P(sap_info_t), vp]),
        "sap_solve_pair": (C.c_int, [vp, vp, vp, vp, vp, P(sap_info_t), P(sap_info_t), vp]),
        "sap_grad_band": (C.c_int, [vp, vp, vp, vp, vp]),
        "sap_apply_preconditioner": (C.c_int, [vp, vp, vp, i32, vp]),
        "sap_spmv": (C.c_int, [vp, i64, i32, vp, vp, i32, vp]),
        "sap_solve_host": (C.c_int, [vp, vp, vp, P(sap_info_t), vp]),
        "sap_factor_host": (C.c_int, [vp, i64, i32, P(sap_options_t), vp, P(vp)]),
        "sap_refactor_host": (C.c_int, [vp, vp, vp]),
        "sap_solve_pair_host": (C.c_int, [vp, vp, vp, vp, vp, P(sap_info_t), P(sap_info_t), vp]),
        "sap_get_partition": (C.c_int, [vp, vp]),
        "sap_get_block_lu": (C.c_int, [vp, i32, vp, vp]),
        "sap_get_interface": (C.c_int, [vp, i32, i32, i32, vp, vp]),
        "sap_n_boosted": (i64, [vp]),
        "sap_num_partitions": (i32, [vp]),
        "sap_destroy": (C.c_int, [vp]),
        "sap_status_string": (C.c_char_p, [C.c_int]),
        "sap_max_K": (i32, [i32]),
        "sap_kernel_launches": (i64, []),
        "sap_selftest_wait_timeout": (C.c_int, [i32, vp]),
        "sap_band_solve_noalloc": (C.c_int, [vp, i64, i32, vp, vp, i32, vp, vp]),
        "sap_factor_batched": (C.c_int, [i32, vp, vp, vp, P(sap_options_t), vp, P(vp)]),
        "sap_autotune": (C.c_int, [vp, i64, i32, P(sap_options_t), vp, i32, vp, i32, vp, vp,
                                   P(C.c_int32), P(C.c_int32), vp, P(C.c_int32)]),
        "sap_refactor_batched": (C.c_int, [vp, vp]),
        "sap_solve_batched": (C.c_int, [vp, vp, vp, vp, vp, vp]),
        "sap_solve_adjoint_batched": (C.c_int, [vp, vp, vp, vp, vp, vp]),
        "sap_solve_pair_batched": (C.c_int, [vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "sap_grad_band_batched": (C.c_int, [vp, vp, vp, vp, vp]),
        "sap_batch_size": (i32, [vp]),
        "sap_batch_partitions": (i32, [vp, i32]),
        "sap_batch_destroy": (C.c_int, [vp]),
        "sap_db_reorder": (C.c_int, [i64, i64, vp, vp, vp, vp, vp, vp, P(C.c_double), vp]),
        "sap_cm_reorder": (C.c_int, [i64, i64, vp, vp, vp, vp, P(C.c_int32), vp]),
        "sap_perm_compose": (C.c_int, [i64, vp, vp, vp, vp]),
        "sap_sparse_bandwidth": (C.c_int, [i64, i64, vp, vp, vp, vp, P(C.c_int32), vp]),
        "sap_sparse_to_band": (C.c_int, [i64, i64, vp, vp, vp, vp, vp, vp, vp, i32, i32, vp, vp]),
        "sap_sparse_drop_bandwidth": (C.c_int, [i64, i64, vp, vp, vp, vp, vp, vp, vp, i32, dbl, P(C.c_int32), vp]),
        "sap_set_operator_csr": (C.c_int, [vp, i64, i64, vp, vp, vp, vp, vp, vp, vp]),
        "sap_sparse_permute_rhs": (C.c_int, [i64, vp, vp, vp, vp, vp]),
        "sap_sparse_unpermute_solution": (C.c_int, [i64, vp, vp, vp, vp, vp]),
        "sap_block_cm_reorder": (C.c_int, [vp, i64, i32, i32, vp, vp, vp]),
        "sap_factor_blocks": (C.c_int, [vp, i64, i32, vp, P(sap_options_t), vp, P(vp)]),
        "sap_get_block_bandwidths": (C.c_int, [vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor) -> int:
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA float64 tensor")
    return t.data_ptr()


def _check(st: int, where: str, ok=(SAP_OK,)):
    if st not in ok:
        raise SapError(st, where)
    return st


def sap_status_string(status: int) -> str:
    return _lib.sap_status_string(int(status)).decode()


def sap_max_K(precision: int = SAP_FP32) -> int:
    return int(_lib.sap_max_K(precision))


def sap_default_options(**kw) -> sap_options_t:
    o = sap_options_t()
    _lib.sap_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Handle:
    """Owns a sap_handle_t and keeps the borrowed band tensor alive."""

    def __init__(self, ptr: int, band: torch.Tensor, N: int, K: int, opts: sap_options_t):
        self.ptr = C.c_void_p(ptr)
        self.band, self.N, self.K, self.opts = band, N, K, opts

    def __del__(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value and _lib is not None:
            _lib.sap_destroy(self.ptr)
            self.ptr = None


def sap_factor(band: torch.Tensor, N: int, K: int, opts: sap_options_t | None = None, stream=None,
               **kw) -> Handle:
    opts = opts or sap_default_options(**kw)
    out = C.c_void_p()
    st = _lib.sap_factor(_ptr(band), N, K, C.byref(opts), _stream(stream), C.byref(out))
    _check(st, "sap_factor")
    return Handle(out.value, band, N, K, opts)


def sap_refactor(h: Handle, stream=None) -> None:
    """Refactor after the values of h.band changed (no allocation)."""
    _check(_lib.sap_refactor(h.ptr, _stream(stream)), "sap_refactor")


def sap_solve(h: Handle, b: torch.Tensor, x: torch.Tensor | None = None, stream=None,
              raise_on_error: bool = True):
    x = torch.empty_like(b) if x is None else x
    info = sap_info_t()
    st = _lib.sap_solve(h.ptr, _ptr(b), _ptr(x), C.byref(info), _stream(stream))
    if raise_on_error:
        _check(st, "sap_solve")
    return x, info, st


def sap_solve_adjoint(h: Handle, gbar: torch.Tensor, lam: torch.Tensor | None = None, stream=None,
                      raise_on_error: bool = True):
    lam = torch.empty_like(gbar) if lam is None else lam
    info = sap_info_t()
    st = _lib.sap_solve_adjoint(h.ptr, _ptr(gbar), _ptr(lam), C.byref(info), _stream(stream))
    if raise_on_error:
        _check(st, "sap_solve_adjoint")
    return lam, info, st


def sap_solve_pair(h: Handle, b: torch.Tensor, gbar: torch.Tensor, x: torch.Tensor | None = None,
                   lam: torch.Tensor | None = None, stream=None, raise_on_error: bool = True):
    """x = A^{-1} b and lambda = A^{-T} gbar, solved concurrently (gbar independent of x)."""
    x = torch.empty_like(b) if x is None else x
    lam = torch.empty_like(gbar) if lam is None else lam
    ix, il = sap_info_t(), sap_info_t()
    st = _lib.sap_solve_pair(h.ptr, _ptr(b), _ptr(x), _ptr(gbar), _ptr(lam), C.byref(ix), C.byref(il),
                             _stream(stream))
    if raise_on_error:
        _check(st, "sap_solve_pair")
    return x, lam, ix, il, st


def sap_solve_host(h: Handle, b_host, x_host, stream=None, raise_on_error: bool = True):
    """b_host / x_host: CPU float64 tensors (pinned for best transfer speed)."""
    info = sap_info_t()
    st = _lib.sap_solve_host(h.ptr, C.c_void_p(b_host.data_ptr()), C.c_void_p(x_host.data_ptr()),
                             C.byref(info), _stream(stream))
    if raise_on_error:
        _check(st, "sap_solve_host")
    return x_host, info, st


def _hptr(t) -> int:
    if not (t.device.type == "cpu" and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous CPU float64 tensor")
    return t.data_ptr()


def sap_factor_host(band_host: torch.Tensor, N: int, K: int, opts: sap_options_t | None = None, stream=None,
                    **kw) -> Handle:
    """Factor from a host band; the handle owns the device copy."""
    opts = opts or sap_default_options(**kw)
    out = C.c_void_p()
    _check(_lib.sap_factor_host(_hptr(band_host), N, K, C.byref(opts), _stream(stream), C.byref(out)),
           "sap_factor_host")
    return Handle(out.value, band_host, N, K, opts)


def sap_refactor_host(h: Handle, band_host: torch.Tensor, stream=None) -> None:
    _check(_lib.sap_refactor_host(h.ptr, _hptr(band_host), _stream(stream)), "sap_refactor_host")


def sap_solve_pair_host(h: Handle, b_host, g_host, x_host, lam_host, stream=None, raise_on_error: bool = True):
    """x = A^{-1} b and lambda = A^{-T} g with host buffers, copies inside the call."""
    ix, il = sap_info_t(), sap_info_t()
    st = _lib.sap_solve_pair_host(h.ptr, _hptr(b_host), _hptr(g_host), _hptr(x_host), _hptr(lam_host),
                                  C.byref(ix), C.byref(il), _stream(stream))
    if raise_on_error:
        _check(st, "sap_solve_pair_host")
    return x_host, lam_host, ix, il, st


def sap_grad_band(h: Handle, lam: torch.Tensor, x: torch.Tensor, out: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(h.band.numel(), dtype=torch.float64, device=lam.device)
    _check(_lib.sap_grad_band(h.ptr, _ptr(lam), _ptr(x), _ptr(out), _stream(stream)), "sap_grad_band")
    return out


def sap_apply_preconditioner(h: Handle, r: torch.Tensor, z: torch.Tensor | None = None,
                             transpose: bool = False, stream=None) -> torch.Tensor:
    z = torch.empty_like(r) if z is None else z
    _check(_lib.sap_apply_preconditioner(h.ptr, _ptr(r), _ptr(z), int(transpose), _stream(stream)),
           "sap_apply_preconditioner")
    return z


def sap_spmv(band: torch.Tensor, N: int, K: int, x: torch.Tensor, y: torch.Tensor | None = None,
             transpose: bool = False, stream=None) -> torch.Tensor:
    y = torch.empty_like(x) if y is None else y
    _check(_lib.sap_spmv(_ptr(band), N, K, _ptr(x), _ptr(y), int(transpose), _stream(stream)), "sap_spmv")
    return y


def sap_num_partitions(h: Handle) -> int:
    return int(_lib.sap_num_partitions(h.ptr))


def sap_get_partition(h: Handle):
    import numpy as np
    off = np.zeros(sap_num_partitions(h) + 1, dtype=np.int64)
    _check(_lib.sap_get_partition(h.ptr, C.c_void_p(off.ctypes.data)), "sap_get_partition")
    return off


def sap_get_block_lu(h: Handle, i: int, stream=None):
    import numpy as np
    off = sap_get_partition(h)
    n = int(off[i + 1] - off[i])
    f = np.zeros((n, 2 * h.K + 1))
    _check(_lib.sap_get_block_lu(h.ptr, i, C.c_void_p(f.ctypes.data), _stream(stream)), "sap_get_block_lu")
    return f


def sap_get_interface(h: Handle, i: int, which: str, adjoint: bool = False, stream=None):
    import numpy as np
    code = {"B": 0, "C": 1, "V": 2, "W": 3, "R": 4}[which]
    m = np.zeros((h.K, h.K))
    _check(_lib.sap_get_interface(h.ptr, i, code, int(adjoint), C.c_void_p(m.ctypes.data), _stream(stream)),
           "sap_get_interface")
    return m


def sap_band_solve_noalloc(band: torch.Tensor, N: int, K: int, b: torch.Tensor, x: torch.Tensor,
                           precision: int = SAP_FP64, timeout: torch.Tensor | None = None,
                           stream=None) -> torch.Tensor:
    """Allocation-free direct banded solve (see include/sap.h).  timeout: an
    optional CUDA int32 tensor of one element that receives 1 if a bounded
    device wait of the call gave up."""
    tp = None
    if timeout is not None:
        if not (timeout.is_cuda and timeout.dtype == torch.int32 and timeout.numel() >= 1):
            raise ValueError("timeout must be a CUDA int32 tensor")
        tp = timeout.data_ptr()
    _check(_lib.sap_band_solve_noalloc(_ptr(band), N, K, _ptr(b), _ptr(x), precision, tp, _stream(stream)),
           "sap_band_solve_noalloc")
    return x


def sap_autotune(band: torch.Tensor, N: int, K: int, P_cands=None, seg_cands=None, b: torch.Tensor | None = None,
                 stream=None, **kw):
    """Measured choice of (P, segments); returns (P, segments, {(P, S): ms})."""
    opts = sap_default_options(**kw)
    Pc = list(P_cands or [])
    Sc = list(seg_cands or [])
    PA = (C.c_int32 * max(1, len(Pc)))(*Pc) if Pc else None
    SA = (C.c_int32 * max(1, len(Sc)))(*Sc) if Sc else None
    ms = (C.c_float * (16 * max(1, len(Sc))))()
    bp, bs_, nused = C.c_int32(), C.c_int32(), C.c_int32()
    st = _lib.sap_autotune(_ptr(band), N, K, C.byref(opts), PA, len(Pc), SA, len(Sc),
                           _ptr(b) if b is not None else None, _stream(stream), C.byref(bp), C.byref(bs_),
                           ms, C.byref(nused))
    _check(st, "sap_autotune")
    table = {}
    Slist = Sc or [0]
    # candidate P values in the library's order are not returned; rebuild them as it does
    if Pc:
        Plist = [p for p in Pc if 1 <= p <= N][:16]
    else:
        pmax = max(1, N // (2 * K)) if opts.variant == SAP_C else max(1, N // 64)
        Plist = []
        for rows in (16000, 8000, 4000, 2000, 1000):
            p = max(1, min(pmax, (N + rows // 2) // rows))
            if p not in Plist:
                Plist.append(p)
        for p in (152, 304):
            if p <= pmax and p not in Plist:
                Plist.append(p)
    for i, p in enumerate(Plist[:nused.value]):
        for j, sg in enumerate(Slist):
            table[(p, sg)] = float(ms[i * len(Slist) + j])
    return bp.value, bs_.value, table


class BatchHandle:
    """Owns a sap_batch_t and keeps the borrowed band tensors alive."""

    def __init__(self, ptr: int, bands, Ns, Ks, opts: sap_options_t):
        self.ptr = C.c_void_p(ptr)
        self.bands, self.Ns, self.Ks, self.opts = list(bands), list(Ns), list(Ks), opts

    def __len__(self):
        return len(self.bands)

    def __del__(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value and _lib is not None:
            _lib.sap_batch_destroy(self.ptr)
            self.ptr = None


def _ptr_array(ts):
    return (C.c_void_p * len(ts))(*[_ptr(t) for t in ts])


def sap_factor_batched(bands, Ns, Ks, opts: sap_options_t | None = None, stream=None, **kw) -> BatchHandle:
    """Factor a batch of systems (P=0 picks the partition count per system)."""
    kw.setdefault("P", 0)
    opts = opts or sap_default_options(**kw)
    n = len(bands)
    if not (len(Ns) == len(Ks) == n):
        raise ValueError("bands, Ns and Ks must have the same length")
    NA = (C.c_int64 * n)(*[int(v) for v in Ns])
    KA = (C.c_int32 * n)(*[int(v) for v in Ks])
    out = C.c_void_p()
    st = _lib.sap_factor_batched(n, _ptr_array(bands), NA, KA, C.byref(opts), _stream(stream), C.byref(out))
    _check(st, "sap_factor_batched")
    return BatchHandle(out.value, bands, Ns, Ks, opts)


def sap_refactor_batched(bh: BatchHandle, stream=None) -> None:
    _check(_lib.sap_refactor_batched(bh.ptr, _stream(stream)), "sap_refactor_batched")


def _solve_batched(fn, name, bh, ins, outs, stream, raise_on_error):
    n = len(bh)
    outs = [torch.empty_like(t) for t in ins] if outs is None else list(outs)
    infos = (sap_info_t * n)()
    stats = (C.c_int32 * n)()
    st = fn(bh.ptr, _ptr_array(ins), _ptr_array(outs), infos, stats, _stream(stream))
    if raise_on_error:
        _check(st, name)
    return outs, list(infos), list(stats), st


def sap_solve_batched(bh: BatchHandle, bs, xs=None, stream=None, raise_on_error: bool = True):
    return _solve_batched(_lib.sap_solve_batched, "sap_solve_batched", bh, bs, xs, stream, raise_on_error)


def sap_solve_adjoint_batched(bh: BatchHandle, gs, lams=None, stream=None, raise_on_error: bool = True):
    return _solve_batched(_lib.sap_solve_adjoint_batched, "sap_solve_adjoint_batched", bh, gs, lams, stream,
                          raise_on_error)


def sap_solve_pair_batched(bh: BatchHandle, bs, gs, xs=None, lams=None, stream=None, raise_on_error: bool = True):
    """Every system's x_i = A_i^{-1} b_i and lambda_i = A_i^{-T} g_i, solved concurrently."""
    n = len(bh)
    xs = [torch.empty_like(t) for t in bs] if xs is None else list(xs)
    lams = [torch.empty_like(t) for t in gs] if lams is None else list(lams)
    ix, il = (sap_info_t * n)(), (sap_info_t * n)()
    stats = (C.c_int32 * (2 * n))()
    st = _lib.sap_solve_pair_batched(bh.ptr, _ptr_array(bs), _ptr_array(xs), _ptr_array(gs), _ptr_array(lams),
                                     ix, il, stats, _stream(stream))
    if raise_on_error:
        _check(st, "sap_solve_pair_batched")
    return xs, lams, list(ix), list(il), list(stats), st


def sap_grad_band_batched(bh: BatchHandle, lams, xs, outs=None, stream=None):
    outs = [torch.empty_like(bd) for bd in bh.bands] if outs is None else list(outs)
    _check(_lib.sap_grad_band_batched(bh.ptr, _ptr_array(lams), _ptr_array(xs), _ptr_array(outs),
                                      _stream(stream)), "sap_grad_band_batched")
    return outs


def sap_batch_partitions(bh: BatchHandle):
    return [int(_lib.sap_batch_partitions(bh.ptr, i)) for i in range(len(bh))]


def sap_kernel_launches() -> int:
    """Kernels launched by libsap in this process so far."""
    return int(_lib.sap_kernel_launches())


def sap_selftest_wait_timeout(spin_limit: int = 1000, stream=None) -> int:
    """Failure-detection self-test: one bounded device wait on a barrier that
    nothing completes; returns the status (SAP_ERR_TIMEOUT expected)."""
    return int(_lib.sap_selftest_wait_timeout(int(spin_limit), _stream(stream)))


def sap_n_boosted(h: Handle) -> int:
    return int(_lib.sap_n_boosted(h.ptr))


from .autograd import SapSolve, SapSolveBatched, sap_solve_autograd, sap_solve_batched_autograd  # noqa: E402

__all__ = [n for n in dir() if n.startswith("sap_") or n in ("Handle", "BatchHandle", "SapError", "SapSolve",
                                                                 "SapSolveBatched")]


# ---- sparse front end (include/sap_sparse.h) ----

class Csr:
    """A CSR matrix on the device: rowptr int64 (n + 1), col int32, val float64."""

    def __init__(self, n: int, rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor):
        self.n, self.rowptr, self.col, self.val = n, rowptr, col, val
        self.nnz = int(col.numel())


def _tptr(t: torch.Tensor | None, dtype=torch.float64):
    """Device pointer of a contiguous CUDA tensor of `dtype` (None: NULL)."""
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor")
    return t.data_ptr()


def _i32(t):
    return _tptr(t, torch.int32)


def _csr(A: "Csr"):
    return A.n, A.nnz, _tptr(A.rowptr, torch.int64), _i32(A.col)


def sap_db_reorder(A: Csr, scale: bool = True, stream=None):
    """Diagonal boosting: returns (rownew, rscale, cscale, logprod); the scale
    factors are None when scale is False."""
    dev = A.val.device
    rownew = torch.empty(A.n, dtype=torch.int32, device=dev)
    r = torch.empty(A.n, dtype=torch.float64, device=dev) if scale else None
    s = torch.empty(A.n, dtype=torch.float64, device=dev) if scale else None
    lp = C.c_double()
    _check(_lib.sap_db_reorder(*_csr(A), _ptr(A.val), _i32(rownew), _tptr(r), _tptr(s), C.byref(lp),
                               _stream(stream)), "sap_db_reorder")
    return rownew, r, s, lp.value


def sap_cm_reorder(A: Csr, rownew: torch.Tensor | None = None, stream=None):
    """Cuthill-McKee of the pattern of B + B^T (B: A with rows moved to
    rownew): returns (perm, K)."""
    perm = torch.empty(A.n, dtype=torch.int32, device=A.col.device)
    K = C.c_int32()
    _check(_lib.sap_cm_reorder(*_csr(A), _i32(rownew), _i32(perm), C.byref(K), _stream(stream)), "sap_cm_reorder")
    return perm, K.value


def sap_perm_compose(outer: torch.Tensor, inner: torch.Tensor, stream=None) -> torch.Tensor:
    out = torch.empty_like(inner)
    _check(_lib.sap_perm_compose(inner.numel(), _i32(outer), _i32(inner), _i32(out), _stream(stream)),
           "sap_perm_compose")
    return out


def sap_sparse_bandwidth(A: Csr, rownew=None, colnew=None, stream=None) -> int:
    K = C.c_int32()
    _check(_lib.sap_sparse_bandwidth(*_csr(A), _i32(rownew), _i32(colnew), C.byref(K), _stream(stream)), "sap_sparse_bandwidth")
    return K.value


def sap_sparse_to_band(A: Csr, rownew, colnew, K: int, rscale=None, cscale=None, drop: bool = False,
                       stream=None) -> torch.Tensor:
    band = torch.empty((2 * K + 1) * A.n, dtype=torch.float64, device=A.val.device)
    _check(_lib.sap_sparse_to_band(*_csr(A), _ptr(A.val), _i32(rownew), _i32(colnew), _tptr(rscale),
                                   _tptr(cscale), K, int(drop), _ptr(band), _stream(stream)), "sap_sparse_to_band")
    return band


def sap_sparse_drop_bandwidth(A: Csr, rownew, colnew, K: int, frac: float, rscale=None, cscale=None,
                              stream=None) -> int:
    Kd = C.c_int32()
    _check(_lib.sap_sparse_drop_bandwidth(*_csr(A), _ptr(A.val), _i32(rownew), _i32(colnew), _tptr(rscale),
                                          _tptr(cscale), K, float(frac), C.byref(Kd), _stream(stream)),
           "sap_sparse_drop_bandwidth")
    return Kd.value


def sap_set_operator_csr(h: Handle, A: Csr | None, rownew=None, colnew=None, rscale=None, cscale=None) -> None:
    """Make the reordered sparse matrix the handle's Krylov operator (A None:
    the band again); the tensors must outlive their use by the handle."""
    if A is None:
        _check(_lib.sap_set_operator_csr(h.ptr, 0, 0, None, None, None, None, None, None, None),
               "sap_set_operator_csr")
        h._csr_keep = None
        return
    _check(_lib.sap_set_operator_csr(h.ptr, *_csr(A), _ptr(A.val), _i32(rownew), _i32(colnew), _tptr(rscale),
                                     _tptr(cscale)), "sap_set_operator_csr")
    h._csr_keep = (A, rownew, colnew, rscale, cscale)


def sap_sparse_permute_rhs(b: torch.Tensor, rownew: torch.Tensor, rscale=None, stream=None) -> torch.Tensor:
    out = torch.empty_like(b)
    _check(_lib.sap_sparse_permute_rhs(b.numel(), _ptr(b), _i32(rownew), _tptr(rscale), _ptr(out),
                                       _stream(stream)), "sap_sparse_permute_rhs")
    return out


def sap_sparse_unpermute_solution(y: torch.Tensor, colnew: torch.Tensor, cscale=None, stream=None) -> torch.Tensor:
    x = torch.empty_like(y)
    _check(_lib.sap_sparse_unpermute_solution(y.numel(), _ptr(y), _i32(colnew), _tptr(cscale), _ptr(x),
                                              _stream(stream)), "sap_sparse_unpermute_solution")
    return x



# ---- per-block bandwidths: the third-stage reordering (include/sap_blocks.h) ----

def sap_block_cm_reorder(band: torch.Tensor, N: int, K: int, P: int, stream=None):
    """Cuthill-McKee of every block of the partition on its own: returns
    (perm, K_i), perm (int32, device) local to each block, K_i (list)."""
    perm = torch.empty(N, dtype=torch.int32, device=band.device)
    Ki = (C.c_int32 * P)()
    _check(_lib.sap_block_cm_reorder(_ptr(band), N, K, P, _i32(perm), Ki, _stream(stream)),
           "sap_block_cm_reorder")
    return perm, list(Ki)


def sap_factor_blocks(band: torch.Tensor, N: int, K: int, perm: torch.Tensor, opts: sap_options_t | None = None,
                      stream=None, **kw) -> Handle:
    """SaP with every block reordered by perm and factored at its own K_i."""
    opts = opts or sap_default_options(**kw)
    out = C.c_void_p()
    _check(_lib.sap_factor_blocks(_ptr(band), N, K, _i32(perm), C.byref(opts), _stream(stream), C.byref(out)),
           "sap_factor_blocks")
    return Handle(out.value, band, N, K, opts)


def sap_get_block_bandwidths(h: Handle) -> list:
    P = sap_num_partitions(h)
    Ki = (C.c_int32 * P)()
    _check(_lib.sap_get_block_bandwidths(h.ptr, Ki), "sap_get_block_bandwidths")
    return list(Ki)
