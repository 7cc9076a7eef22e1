"""ctypes binding of ``libpsvd.so`` (include/psvd.h), same names as the C-ABI.

Argument marshalling only: every step of the streaming SVD runs in the library's
CUDA kernels.  If the library cannot be loaded (not built, no nvcc, wrong
architecture) every entry point raises ``PsvdError``; there is no fallback.

Matrices are column-major ``(rows, cols)`` tensors/arrays (``stride(0) == 1``),
i.e. each snapshot (column) is contiguous, matching the paper's data matrix
(rows = grid points, columns = snapshots, Sec. 3.1).  torch tensors (CUDA or
CPU) and numpy arrays are accepted; host inputs are staged by the library.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

PSVD_OK = 0
PSVD_WARN_RANK_DEFICIENT = 1
PSVD_WARN_NOT_CONVERGED = 2
PSVD_WARN_DEGENERATE = 3
PSVD_ERR_INVALID_ARG = -1
PSVD_ERR_NOT_INITIALIZED = -2
PSVD_ERR_SHAPE = -3
PSVD_ERR_NONFINITE = -4
PSVD_ERR_CUDA = -5
PSVD_ERR_ALLOC = -6
PSVD_ERR_IO = -7
PSVD_ERR_UNSUPPORTED = -8
PSVD_ERR_TIMEOUT = -9

PSVD_F32, PSVD_BF16, PSVD_F64 = 0, 1, 2
PSVD_PREC_FP32, PSVD_PREC_BF16_TC, PSVD_PREC_FP64 = 0, 1, 2


class PsvdError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class psvd_config(C.Structure):
    _fields_ = [("M", C.c_int64), ("K", C.c_int32), ("max_batch", C.c_int32), ("ff", C.c_double),
                ("precision", C.c_int32), ("low_rank", C.c_int32), ("oversample", C.c_int32),
                ("power_iters", C.c_int32), ("seed", C.c_uint64), ("stream", C.c_void_p)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads (building first if needed) the in-tree libpsvd.so."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not _build.up_to_date():
            if not build_if_missing:
                raise PsvdError(PSVD_ERR_UNSUPPORTED, f"libpsvd.so missing at {path}")
            try:
                path = _build.build()
            except Exception as e:  # no fallback: surface the build failure
                raise RuntimeError(f"cannot build libpsvd.so: {e}") from e
        lib = C.CDLL(path)
        vp, i64, i32, u64 = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64
        dp, fp = C.POINTER(C.c_double), C.c_void_p
        lib.psvd_create.argtypes = [C.POINTER(vp), C.POINTER(psvd_config)]
        lib.psvd_destroy.argtypes = [vp]
        lib.psvd_destroy.restype = None
        lib.psvd_initialize.argtypes = [vp, vp, i64, i32, i32]
        lib.psvd_incorporate_data.argtypes = [vp, vp, i64, i32, i32]
        lib.psvd_incorporate_batches.argtypes = [vp, C.POINTER(vp), i32, i64, i32, i32, vp]
        lib.psvd_parallel_qr.argtypes = [vp, vp, i64, i32, i32, vp]
        lib.psvd_parallel_svd.argtypes = [vp, vp, i64, C.POINTER(C.c_int64), i32, i32, i32, i32,
                                          i32, fp, i64, vp]
        lib.psvd_get_modes.argtypes = [vp, fp, i64]
        lib.psvd_get_modes_f64.argtypes = [vp, vp, i64]
        lib.psvd_get_singular_values.argtypes = [vp, vp]
        lib.psvd_num_modes.argtypes = [vp]
        lib.psvd_save.argtypes = [vp, C.c_char_p]
        lib.psvd_load.argtypes = [C.POINTER(vp), C.c_char_p, vp]
        lib.psvd_gaussian_sketch.argtypes = [u64, u64, i64, i64, fp, vp]
        lib.psvd_status_string.argtypes = [C.c_int]
        lib.psvd_status_string.restype = C.c_char_p
        lib.psvd_last_info.argtypes = [vp, C.POINTER(C.c_int32)]
        lib.psvd_debug_set_wait_budget.argtypes = [i32, i64]
        lib.psvd_parallel_qr_static.argtypes = [vp, i64, i64, i32, i32, vp, vp]
        lib.psvd_update_adjoint.argtypes = [vp, i32, vp, i64, vp, vp, i64, i32, i32, i32, vp, i64,
                                            vp, vp, i64, vp, vp, i64, vp, vp, i64]
        lib.psvd_group_create.argtypes = [C.POINTER(vp), i32, C.POINTER(psvd_config)]
        lib.psvd_group_destroy.argtypes = [vp]
        lib.psvd_group_destroy.restype = None
        lib.psvd_group_initialize.argtypes = [vp, C.POINTER(vp), i64, i32, i32]
        lib.psvd_group_incorporate_data.argtypes = [vp, C.POINTER(vp), i64, i32, i32]
        lib.psvd_group_member.argtypes = [vp, i32]
        lib.psvd_group_member.restype = vp
        lib.psvd_group_status.argtypes = [vp]
        lib.psvd_group_stats.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        lib.psvd_autotune.argtypes = [vp, vp, i64, i32, i32, C.POINTER(C.c_int32)]
        lib.psvd_set_profiling.argtypes = [vp, i32]
        lib.psvd_get_profile.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                         C.POINTER(C.c_int64)]
        _lib = lib
        return lib


def status_string(status: int) -> str:
    try:
        return load().psvd_status_string(int(status)).decode()
    except Exception:
        return "library unavailable"


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise PsvdError(rc, where)
    return rc


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _mat(x, name: str, allow_f64: bool = False):
    """(pointer, ld, rows, cols, dtype code, keepalive) of a column-major matrix."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        if x.dim() == 1:
            x = x[:, None]
        if x.dim() != 2:
            raise ValueError(f"{name}: expected a 2-D matrix")
        rows, cols = x.shape
        if cols > 1 and x.stride(0) != 1:
            raise ValueError(f"{name}: must be column-major (stride(0) == 1)")
        ld = x.stride(1) if cols > 1 else rows
        code = {torch.float32: PSVD_F32, torch.bfloat16: PSVD_BF16, torch.float64: PSVD_F64}.get(x.dtype)
        if code is None or (code == PSVD_F64 and not allow_f64):
            raise ValueError(f"{name}: unsupported dtype {x.dtype}")
        return x.data_ptr(), ld, rows, cols, code, x
    a = np.asarray(x)
    if a.ndim == 1:
        a = a[:, None]
    if a.ndim != 2:
        raise ValueError(f"{name}: expected a 2-D matrix")
    rows, cols = a.shape
    if a.dtype == np.float32:
        code = PSVD_F32
    elif a.dtype == np.float64 and allow_f64:
        code = PSVD_F64
    else:
        raise ValueError(f"{name}: unsupported dtype {a.dtype}")
    if cols > 1 and a.strides[0] != a.itemsize:
        raise ValueError(f"{name}: must be column-major (Fortran order)")
    ld = a.strides[1] // a.itemsize if cols > 1 else rows
    return a.ctypes.data, ld, rows, cols, code, a


def psvd_create(M: int, K: int, max_batch: int, ff: float = 1.0, precision: int = PSVD_PREC_FP32,
                low_rank: int = 0, oversample: int = 10, power_iters: int = 0, seed: int = 0,
                stream=None) -> int:
    lib = load()
    cfg = psvd_config(int(M), int(K), int(max_batch), float(ff), int(precision), int(low_rank),
                      int(oversample), int(power_iters), int(seed), _stream_ptr(stream))
    h = C.c_void_p()
    _check(lib.psvd_create(C.byref(h), C.byref(cfg)), "psvd_create")
    return h.value


def psvd_destroy(h: int) -> None:
    load().psvd_destroy(h)


def psvd_initialize(h: int, A0) -> int:
    p, ld, _, B, code, _keep = _mat(A0, "A0", allow_f64=True)
    return _check(load().psvd_initialize(h, p, ld, B, code), "psvd_initialize")


def psvd_incorporate_data(h: int, A) -> int:
    p, ld, _, B, code, _keep = _mat(A, "A", allow_f64=True)
    return _check(load().psvd_incorporate_data(h, p, ld, B, code), "psvd_incorporate_data")


def psvd_incorporate_batches(h: int, batches, s_out=None, K=None) -> int:
    """psvd_incorporate_data on every batch in order: host batches are copied to the
    device while the previous batch is processed.  All batches share lda, B and dtype.
    s_out (optional): contiguous float64, count x K (the handle's K; its size is
    checked when K is given); row i receives batch i's singular values.  Returns
    after enqueuing."""
    ptrs, ld, B, code, _keep = _batch_list(batches, "batches")
    sp = None
    if s_out is not None:
        if hasattr(s_out, "data_ptr"):
            import torch
            if s_out.dtype != torch.float64 or not s_out.is_contiguous():
                raise ValueError("s_out: expected a contiguous float64 tensor")
            sp, n = s_out.data_ptr(), s_out.numel()
        else:
            a = np.asarray(s_out)
            if a.dtype != np.float64 or not a.flags.c_contiguous:
                raise ValueError("s_out: expected a contiguous float64 array")
            sp, n = a.ctypes.data, a.size
        if K is not None and n < len(ptrs) * K:
            raise ValueError(f"s_out: needs {len(ptrs)} x {K} elements")
    return _check(load().psvd_incorporate_batches(h, ptrs, len(ptrs), ld, B, code, sp),
                  "psvd_incorporate_batches")


def psvd_parallel_qr(h: int, P, R_out) -> int:
    p, ld, _, n, code, _keep = _mat(P, "P", allow_f64=True)
    r, _, rr, rc_, rcode, _keep2 = _mat(R_out, "R_out", allow_f64=True)
    if rcode != PSVD_F64 or rr != n or rc_ != n:
        raise ValueError("R_out: must be an n x n float64 matrix")
    return _check(load().psvd_parallel_qr(h, p, ld, n, code, r), "psvd_parallel_qr")


def psvd_parallel_qr_static(P, R_out, stream=None) -> int:
    """R of psvd_parallel_qr without any allocation (see include/psvd.h): for callers
    that cannot allocate device memory when they need the factor.  P must be a
    device matrix with at most 128 columns; calls that overlap on the GPU race."""
    p, ld, M, n, code, _keep = _mat(P, "P")
    r, _, rr, rc_, rcode, _keep2 = _mat(R_out, "R_out", allow_f64=True)
    if rcode != PSVD_F64 or rr != n or rc_ != n:
        raise ValueError("R_out: must be an n x n float64 matrix")
    return _check(load().psvd_parallel_qr_static(p, ld, M, n, code, r, _stream_ptr(stream)),
                  "psvd_parallel_qr_static")


def psvd_parallel_svd(h: int, A, part_offsets, r1: int, r2: int, U_out, L_out) -> int:
    p, ld, _, N, code, _keep = _mat(A, "A")
    off = np.ascontiguousarray(part_offsets, dtype=np.int64)
    u, ldu, _, _, ucode, _keep2 = _mat(U_out, "U_out")
    l, _, _, _, lcode, _keep3 = _mat(L_out, "L_out", allow_f64=True)
    if ucode != PSVD_F32 or lcode != PSVD_F64:
        raise ValueError("U_out must be float32 and L_out float64")
    return _check(load().psvd_parallel_svd(h, p, ld, off.ctypes.data_as(C.POINTER(C.c_int64)),
                                           off.size - 1, N, code, int(r1), int(r2), u, ldu, l),
                  "psvd_parallel_svd")


def psvd_get_modes(h: int, U_out) -> int:
    p, ld, _, _, code, _keep = _mat(U_out, "U_out")
    if code != PSVD_F32:
        raise ValueError("U_out must be float32")
    return _check(load().psvd_get_modes(h, p, ld), "psvd_get_modes")


def psvd_get_modes_f64(h: int, U_out) -> int:
    p, ld, _, _, code, _keep = _mat(U_out, "U_out", allow_f64=True)
    if code != PSVD_F64:
        raise ValueError("U_out must be float64")
    return _check(load().psvd_get_modes_f64(h, p, ld), "psvd_get_modes_f64")


def psvd_get_singular_values(h: int, s_out) -> int:
    p, _, _, _, code, _keep = _mat(s_out, "s_out", allow_f64=True)
    if code != PSVD_F64:
        raise ValueError("s_out must be float64")
    return _check(load().psvd_get_singular_values(h, p), "psvd_get_singular_values")


def psvd_num_modes(h: int) -> int:
    return _check(load().psvd_num_modes(h), "psvd_num_modes")


def psvd_save(h: int, path: str) -> int:
    return _check(load().psvd_save(h, os.fsencode(path)), "psvd_save")


def psvd_load(path: str, stream=None) -> int:
    h = C.c_void_p()
    _check(load().psvd_load(C.byref(h), os.fsencode(path), _stream_ptr(stream)), "psvd_load")
    return h.value


def psvd_gaussian_sketch(seed: int, stream_id: int, out, stream=None) -> int:
    p, ld, rows, cols, code, _keep = _mat(out, "out")
    if code != PSVD_F32 or ld != rows:
        raise ValueError("out must be a contiguous column-major float32 matrix")
    return _check(load().psvd_gaussian_sketch(int(seed), int(stream_id), rows, cols, p,
                                              _stream_ptr(stream)), "psvd_gaussian_sketch")


def psvd_update_adjoint(h: int, U, D, A, U_new, D_new, U_new_bar, D_new_bar, U_bar, D_bar,
                        A_bar) -> int:
    """Cotangents (U_bar, D_bar, A_bar) of one step's inputs from those of its outputs
    (include/psvd.h).  U, D, U_bar, D_bar are None for the initialisation step.
    Returns PSVD_OK or PSVD_WARN_DEGENERATE."""
    a, lda, M, B, acode, _k1 = _mat(A, "A")
    un, ldn, _, k1, ucode, _k2 = _mat(U_new, "U_new")
    ub, ldb, _, _, bcode, _k3 = _mat(U_new_bar, "U_new_bar")
    ab, ldab, _, _, abcode, _k4 = _mat(A_bar, "A_bar")
    dn, _, _, _, dcode, _k5 = _mat(D_new, "D_new", allow_f64=True)
    db, _, _, _, dbcode, _k6 = _mat(D_new_bar, "D_new_bar", allow_f64=True)
    if ucode != PSVD_F32 or bcode != PSVD_F32 or abcode != PSVD_F32:
        raise ValueError("U_new, U_new_bar and A_bar must be float32")
    if dcode != PSVD_F64 or dbcode != PSVD_F64:
        raise ValueError("D_new and D_new_bar must be float64")
    if U is None:
        kc, u, ldu, d, ubar, ldub, dbar = 0, None, M, None, None, M, None
        keep = ()
    else:
        u, ldu, _, kc, c1, k7 = _mat(U, "U")
        d, _, _, _, c2, k8 = _mat(D, "D", allow_f64=True)
        ubar, ldub, _, _, c3, k9 = _mat(U_bar, "U_bar")
        dbar, _, _, _, c4, k10 = _mat(D_bar, "D_bar", allow_f64=True)
        if c1 != PSVD_F32 or c3 != PSVD_F32 or c2 != PSVD_F64 or c4 != PSVD_F64:
            raise ValueError("U, U_bar must be float32 and D, D_bar float64")
        keep = (k7, k8, k9, k10)
    rc = load().psvd_update_adjoint(h, kc, u, ldu, d, a, lda, B, acode, k1, un, ldn, dn, ub, ldb,
                                    db, ubar, ldub, dbar, ab, ldab)
    del keep
    return _check(rc, "psvd_update_adjoint")


def psvd_autotune(h: int, A):
    """Times the handle's launch-shape choices on the representative device batch A and
    keeps the fastest.  Returns (Gram CTAs per SM, update tile rows) for an FP32 handle,
    (Gram clusters, update CTAs, update stages) for a tensor-core handle."""
    p, ld, _, B, code, _keep = _mat(A, "A", allow_f64=True)
    ch = (C.c_int32 * 3)()
    _check(load().psvd_autotune(h, p, ld, B, code, ch), "psvd_autotune")
    if ch[2] == 0:
        return int(ch[0]), int(ch[1])
    return int(ch[0]), int(ch[1]), int(ch[2])


def psvd_last_info(h: int):
    info = (C.c_int32 * 4)()
    rc = _check(load().psvd_last_info(h, info), "psvd_last_info")
    return rc, [int(x) for x in info]


PSVD_DEBUG_UPDATE_KERNEL = 1


def psvd_debug_set_wait_budget(kernel: int, cycles: int) -> int:
    """Testing hook: clock-cycle budget of the tensor-core update kernel's pipeline
    waits for later launches (0 restores the default); see include/psvd.h."""
    return _check(load().psvd_debug_set_wait_budget(int(kernel), int(cycles)),
                  "psvd_debug_set_wait_budget")


def psvd_set_profiling(h: int, enable: bool) -> int:
    return _check(load().psvd_set_profiling(h, 1 if enable else 0), "psvd_set_profiling")


def psvd_get_profile(h: int):
    """(ms[3], counts[3], launches): per-phase device time (Gram, small solve, update)."""
    ms = (C.c_double * 3)()
    cnt = (C.c_int64 * 3)()
    nl = C.c_int64()
    _check(load().psvd_get_profile(h, ms, cnt, C.byref(nl)), "psvd_get_profile")
    return [float(x) for x in ms], [int(x) for x in cnt], int(nl.value)


def _batch_list(batches, where: str):
    mats = [_mat(b, f"{where}[{i}]", allow_f64=True) for i, b in enumerate(batches)]
    if not mats:
        raise ValueError(f"{where}: no batches")
    ld, B, code = mats[0][1], mats[0][3], mats[0][4]
    for m in mats:
        if (m[1], m[3], m[4]) != (ld, B, code):
            raise ValueError(f"{where}: every batch needs the same lda, B and dtype")
    ptrs = (C.c_void_p * len(mats))(*[m[0] for m in mats])
    return ptrs, ld, B, code, mats


def psvd_group_create(count: int, M: int, K: int, max_batch: int, ff: float = 1.0,
                      precision: int = PSVD_PREC_FP32, low_rank: int = 0, oversample: int = 10,
                      power_iters: int = 0, seed: int = 0, stream=None) -> int:
    lib = load()
    cfg = psvd_config(int(M), int(K), int(max_batch), float(ff), int(precision), int(low_rank),
                      int(oversample), int(power_iters), int(seed), _stream_ptr(stream))
    g = C.c_void_p()
    _check(lib.psvd_group_create(C.byref(g), int(count), C.byref(cfg)), "psvd_group_create")
    return g.value


def psvd_group_destroy(g: int) -> None:
    load().psvd_group_destroy(g)


def psvd_group_initialize(g: int, batches) -> int:
    ptrs, ld, B, code, _keep = _batch_list(batches, "batches")
    return _check(load().psvd_group_initialize(g, ptrs, ld, B, code), "psvd_group_initialize")


def psvd_group_incorporate_data(g: int, batches) -> int:
    ptrs, ld, B, code, _keep = _batch_list(batches, "batches")
    return _check(load().psvd_group_incorporate_data(g, ptrs, ld, B, code),
                  "psvd_group_incorporate_data")


def psvd_group_member(g: int, i: int) -> int:
    h = load().psvd_group_member(g, int(i))
    if not h:
        raise PsvdError(PSVD_ERR_INVALID_ARG, "psvd_group_member")
    return h


def psvd_group_status(g: int) -> int:
    return _check(load().psvd_group_status(g), "psvd_group_status")


def psvd_group_stats(g: int):
    """(captures, replays): calls that captured a CUDA graph, calls that replayed one."""
    c, r = C.c_int64(), C.c_int64()
    _check(load().psvd_group_stats(g, C.byref(c), C.byref(r)), "psvd_group_stats")
    return int(c.value), int(r.value)


class StreamingSVD:
    """Convenience owner of one handle (Algorithm 1 state) with torch outputs."""

    def __init__(self, M, K, max_batch, ff=1.0, precision=PSVD_PREC_FP32, low_rank=0,
                 oversample=10, power_iters=0, seed=0, stream=None):
        self.M, self.K, self.precision = int(M), int(K), int(precision)
        self.h = psvd_create(M, K, max_batch, ff, precision, low_rank, oversample, power_iters,
                             seed, stream)

    def initialize(self, A0):
        return psvd_initialize(self.h, A0)

    def incorporate_data(self, A):
        return psvd_incorporate_data(self.h, A)

    def incorporate_batches(self, batches, s_out=None):
        return psvd_incorporate_batches(self.h, batches, s_out, self.K)

    @property
    def num_modes(self) -> int:
        return psvd_num_modes(self.h)

    def modes(self, device="cuda"):
        """Current modes, column-major: float64 for a PSVD_PREC_FP64 handle, else float32."""
        import torch
        k = self.num_modes
        if self.precision == PSVD_PREC_FP64:
            U = torch.empty((k, self.M), dtype=torch.float64, device=device).T
            psvd_get_modes_f64(self.h, U)
        else:
            U = torch.empty((k, self.M), dtype=torch.float32, device=device).T
            psvd_get_modes(self.h, U)
        return U

    def singular_values(self, device="cuda"):
        import torch
        s = torch.empty(self.num_modes, dtype=torch.float64, device=device)
        psvd_get_singular_values(self.h, s)
        return s

    def close(self):
        if self.h:
            psvd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
