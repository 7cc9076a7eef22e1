"""FP64 CPU oracle for the streaming, partitioned, randomized SVD of arXiv 2108.08845.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s ``cpu_baseline`` / ``--impl reference`` legs may import this
package.  It shares no code with the CUDA library in ``paper_2108_08845_gb300``.

Every routine runs the paper's steps in the paper's order, in plain FP64 C
(``oracle.c``): Householder QR, one-sided Jacobi SVD, Algorithm 1 (streaming
update, Sec. 3.1), Algorithm 2 (APMOS, Sec. 3.2), the randomized low-rank SVD of
Sec. 3.3, and the Philox4x32-10 Gaussian test matrix.  Inputs of any float dtype
are widened exactly to float64 here; outputs are float64.

Readings of the paper taken where it is silent:
  * Algorithm 1 always truncates to K modes after each batch (steps 3 and 5),
  * the forget factor scales U*D (the singular values), not their squares,
  * singular values are sorted descending with a stable order for ties,
  * the Gaussian test matrix has unit variance (Sec. 3.3) and is drawn from
    Philox4x32-10 with a Box-Muller transform on self-written log/sin/cos.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

MAX_SWEEPS = 60
JACOBI_TOL = 1e-15

ORC_OK = 0
ORC_ERR_SHAPE = -1
ORC_ERR_NOT_CONVERGED = -2


class OracleError(RuntimeError):
    pass


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = C.CDLL(path)
        dp, i64, i32, u64, dbl = (C.POINTER(C.c_double), C.c_int64, C.c_int, C.c_uint64,
                                  C.c_double)
        i64p = C.POINTER(C.c_int64)
        lib.orc_householder_qr.argtypes = [i64, i64, dp, i64, dp, i64, dp, i64]
        lib.orc_jacobi_svd.argtypes = [i64, i64, dp, i64, dp, i64, dp, i32, dbl]
        lib.orc_sort_desc.argtypes = [i64, dp, i64p]
        lib.orc_stream_initialize.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, i32, dbl]
        lib.orc_stream_update.argtypes = [i64, i64, i64, i64, dbl, dp, i64, dp, dp, i64, i32, dbl]
        lib.orc_tsqr_r.argtypes = [i64, i64, dp, i64, i64, i64p, dp, i64]
        lib.orc_apmos.argtypes = [i64, i64, dp, i64, i64, i64p, i64, i64, dp, i64, dp, i32, dbl]
        lib.orc_rsvd_panel.argtypes = [i64, i64, dp, i64, i64, i64, dp, i64, i64, dp, i64, dp,
                                       i32, dbl]
        u32p = C.POINTER(C.c_uint32)
        u64p = C.POINTER(C.c_uint64)
        lib.orc_philox4x32.argtypes = [u32p, u32p, i32, u32p]
        lib.orc_philox4x32.restype = None
        lib.orc_philox4x64.argtypes = [u64p, u64p, i32, u64p]
        lib.orc_philox4x64.restype = None
        lib.orc_ln.argtypes = [dbl]
        lib.orc_ln.restype = dbl
        lib.orc_sincos_2pi.argtypes = [dbl, dp, dp]
        lib.orc_sincos_2pi.restype = None
        lib.orc_gaussian.argtypes = [u64, u64, u64, i64, dp]
        lib.orc_gaussian.restype = None
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    """Exact widening to a Fortran-ordered float64 copy (any real float dtype)."""
    a = np.asarray(a)
    if a.dtype.kind != "f" and a.dtype.name != "bfloat16":
        a = a.astype(np.float64)
    return np.array(a, dtype=np.float64, order="F", copy=True)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(rc: int, what: str):
    if rc < 0:
        raise OracleError(f"{what} failed with status {rc}")
    return rc


def householder_qr(A):
    """Thin Householder QR with diag(R) >= 0.  Returns (Q m x n, R n x n)."""
    lib = _load()
    A = _f64(A)
    m, n = A.shape
    Q = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    _check(lib.orc_householder_qr(m, n, _ptr(A), m, _ptr(Q), m, _ptr(R), n), "householder_qr")
    return Q, R


def jacobi_svd(A, max_sweeps=MAX_SWEEPS, tol=JACOBI_TOL):
    """Thin SVD by one-sided Jacobi on the columns of A (m x n).

    Returns (U, s, V) sorted by descending s with A V = U diag(s); a zero
    singular value leaves its U column zero.  Also returns the sweep count.
    """
    lib = _load()
    W = _f64(A)
    m, n = W.shape
    V = np.zeros((n, n), order="F")
    s = np.zeros(n)
    sweeps = _check(lib.orc_jacobi_svd(m, n, _ptr(W), m, _ptr(V), n, _ptr(s), max_sweeps, tol),
                    "jacobi_svd")
    order = sort_desc(s)
    s = s[order]
    W = W[:, order]
    V = V[:, order]
    U = np.zeros_like(W)
    nz = s > 0
    U[:, nz] = W[:, nz] / s[nz]
    return U, s, V, sweeps


def sort_desc(s) -> np.ndarray:
    """Stable descending order (ties keep the lower index first)."""
    lib = _load()
    s = np.ascontiguousarray(s, dtype=np.float64)
    order = np.zeros(s.shape[0], dtype=np.int64)
    lib.orc_sort_desc(s.shape[0], _ptr(s), order.ctypes.data_as(C.POINTER(C.c_int64)))
    return order


def stream_initialize(A0, K, max_sweeps=MAX_SWEEPS, tol=JACOBI_TOL):
    """Algorithm 1 I1-I2: returns (U m x k0, D k0), k0 = min(K, B), from A0 (m x B)."""
    lib = _load()
    A0 = _f64(A0)
    m, B = A0.shape
    U = np.zeros((m, K), order="F")
    D = np.zeros(K)
    k0 = _check(lib.orc_stream_initialize(m, B, K, _ptr(A0), m, _ptr(U), m, _ptr(D),
                                          max_sweeps, tol), "stream_initialize")
    return np.asfortranarray(U[:, :k0]), D[:k0].copy()


def stream_update(U, D, A, ff, K=None, max_sweeps=MAX_SWEEPS, tol=JACOBI_TOL):
    """Algorithm 1 steps 1-5 for one batch; returns the new (U, D) with
    min(K, kc + B) modes (K defaults to the current mode count kc)."""
    lib = _load()
    U = _f64(U)
    D = np.array(D, dtype=np.float64)
    A = _f64(A)
    m, kc = U.shape
    K = kc if K is None else int(K)
    B = A.shape[1]
    Ub = np.zeros((m, max(K, 1)), order="F")
    Ub[:, :kc] = U
    Db = np.zeros(max(K, 1))
    Db[:kc] = D
    k1 = _check(lib.orc_stream_update(m, kc, K, B, float(ff), _ptr(Ub), m, _ptr(Db), _ptr(A), m,
                                      max_sweeps, tol), "stream_update")
    return np.asfortranarray(Ub[:, :k1]), Db[:k1].copy()


def stream_run(batches, K, ff):
    """Algorithm 1 over a list of batches: initialise on the first, update on the rest."""
    U, D = stream_initialize(batches[0], K)
    for A in batches[1:]:
        U, D = stream_update(U, D, A, ff, K)
    return U, D


def panel(U, D, A, ff):
    """The Algorithm 1 step-1 panel [ff U diag(D) | A] in float64."""
    return np.concatenate([_f64(U) * (ff * np.asarray(D, np.float64))[None, :], _f64(A)], axis=1)


def tsqr_r(A, offsets):
    """R factor (diag >= 0) of the row-partitioned QR (local QRs, then QR of stacked R)."""
    lib = _load()
    A = _f64(A)
    m, n = A.shape
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    R = np.zeros((n, n), order="F")
    _check(lib.orc_tsqr_r(m, n, _ptr(A), m, off.shape[0] - 1,
                          off.ctypes.data_as(C.POINTER(C.c_int64)), _ptr(R), n), "tsqr_r")
    return R


def apmos(A, offsets, r1, r2, max_sweeps=MAX_SWEEPS, tol=JACOBI_TOL):
    """Algorithm 2 (APMOS).  Returns (U m x r2, Lambda r2)."""
    lib = _load()
    A = _f64(A)
    m, N = A.shape
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    U = np.zeros((m, r2), order="F")
    L = np.zeros(r2)
    _check(lib.orc_apmos(m, N, _ptr(A), m, off.shape[0] - 1,
                         off.ctypes.data_as(C.POINTER(C.c_int64)), r1, r2, _ptr(U), m, _ptr(L),
                         max_sweeps, tol), "apmos")
    return U, L


def rsvd_panel(P, K, Omega, q, max_sweeps=MAX_SWEEPS, tol=JACOBI_TOL):
    """Randomized rank-K SVD of the panel P with Gaussian Omega (n x l) and q power steps."""
    lib = _load()
    P = _f64(P)
    Om = _f64(Omega)
    m, n = P.shape
    l = Om.shape[1]
    U = np.zeros((m, K), order="F")
    D = np.zeros(K)
    _check(lib.orc_rsvd_panel(m, n, _ptr(P), m, K, l, _ptr(Om), n, q, _ptr(U), m, _ptr(D),
                              max_sweeps, tol), "rsvd_panel")
    return U, D


def rsvd_update(U, D, A, ff, Omega, q):
    """Streaming update whose panel SVD is the randomized low-rank SVD (Sec. 3.3)."""
    K = np.asarray(D).shape[0]
    return rsvd_panel(panel(U, D, A, ff), K, Omega, q)


def rsvd_initialize(A0, K, Omega, q):
    """Initialisation whose SVD of the first batch is the randomized low-rank SVD."""
    return rsvd_panel(_f64(A0), K, Omega, q)


def rsvd_run(batches, K, ff, p, q, seed):
    """Algorithm 1 whose panel SVDs are the randomized low-rank SVD (Sec. 3.3).

    Batch t (t = 0 is the initialisation) draws its Gaussian test matrix as stream t
    of the Philox key `seed`: n x l with n = k + B the panel width (k = 0 at t = 0)
    and l = min(K + p, n), kept modes k1 = min(K, n) (l >= k1)."""
    U = D = None
    for t, A in enumerate(batches):
        A = _f64(A)
        P = A if U is None else panel(U, D, A, ff)
        n = P.shape[1]
        k1 = min(K, n)
        l = max(min(K + p, n), k1)
        U, D = rsvd_panel(P, k1, gaussian_matrix(seed, t, n, l), q)
    return U, D


# Philox stream of the sketch of the literal low_rank_svd(W) in Algorithm 2 (an
# identifier that no batch index of the streaming sketches reaches)
APMOS_SKETCH_STREAM = 0x41504D4F53


def apmos_local_factors(A, offsets, r1, max_sweeps=MAX_SWEEPS, tol=JACOBI_TOL):
    """Algorithm 2's local step: for every row block A_b, the thin SVD (Householder QR,
    then one-sided Jacobi on R) and its leading r1 right factors W_b = V_b diag(s_b),
    each column signed so that its entries sum to >= 0.  Returns W (N x r1*nparts)."""
    A = _f64(A)
    off = np.asarray(offsets, dtype=np.int64)
    cols = []
    for b in range(off.shape[0] - 1):
        _, R = householder_qr(A[off[b]:off[b + 1], :])
        _, s, V, _ = jacobi_svd(R)
        Wb = V[:, :r1] * s[None, :r1]
        sg = np.where(Wb.sum(axis=0) >= 0, 1.0, -1.0)
        cols.append(Wb * sg[None, :])
    return np.concatenate(cols, axis=1)


def rsvd_wide(W, k, Omega, q, max_sweeps=MAX_SWEEPS, tol=JACOBI_TOL):
    """Randomized rank-k SVD of any N x m matrix W (Halko, Martinsson & Tropp, Alg. 4.4):
    Y = W Omega, Q = orth(Y); q times: Q^ = orth(W^T Q), Q = orth(W Q^); B = Q^T W;
    the left singular vectors of B (Jacobi SVD of B^T) give X = Q U_B.  orth() is the
    oracle's Householder QR.  Returns (X N x k, s k)."""
    W = _f64(W)
    Q, _ = householder_qr(W @ _f64(Omega))
    for _ in range(int(q)):
        Qh, _ = householder_qr(W.T @ Q)
        Q, _ = householder_qr(W @ Qh)
    B = Q.T @ W
    _, s, Vb, _ = jacobi_svd(B.T)  # B^T Vb = Ub diag(s): B's left vectors are Vb
    return Q @ Vb[:, :k], s[:k].copy()


def apmos_low_rank(A, offsets, r1, r2, p, q, seed, max_sweeps=MAX_SWEEPS, tol=JACOBI_TOL):
    """Algorithm 2 with the paper's low_rank_svd on the gathered W (Listing 3 with
    low_rank set): W = [W_0 ... W_{nparts-1}] (N x m, m = r1 nparts), then the
    randomized SVD of W (Halko, Martinsson & Tropp, Alg. 4.4) with the Gaussian test
    matrix Omega (m x l, l = min(r2 + p, N), stream APMOS_SKETCH_STREAM of the seed)
    and q power steps gives X~ (N x r2) and L~; U = A X~ diag(1/L~) (zero where
    L~ = 0).  Returns (U m x r2, L~)."""
    A = _f64(A)
    W = apmos_local_factors(A, offsets, r1, max_sweeps, tol)
    N, m = W.shape
    l = min(r2 + p, N, m)
    Om = gaussian_matrix(seed, APMOS_SKETCH_STREAM, m, l)
    X, L = rsvd_wide(W, r2, Om, q, max_sweeps, tol)
    inv = np.zeros_like(L)
    inv[L > 0] = 1.0 / L[L > 0]
    return A @ (X * inv[None, :]), L


def philox4x32(ctr, key, rounds=10):
    lib = _load()
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib.orc_philox4x32(c, k, rounds, o)
    return [int(x) for x in o]


def philox4x64(ctr, key, rounds=10):
    lib = _load()
    M = (1 << 64) - 1
    c = (C.c_uint64 * 4)(*[int(x) & M for x in ctr])
    k = (C.c_uint64 * 2)(*[int(x) & M for x in key])
    o = (C.c_uint64 * 4)()
    lib.orc_philox4x64(c, k, rounds, o)
    return [int(x) for x in o]


def ln(x: float) -> float:
    return _load().orc_ln(float(x))


def sincos_2pi(u: float):
    s = C.c_double()
    c = C.c_double()
    _load().orc_sincos_2pi(float(u), C.byref(s), C.byref(c))
    return s.value, c.value


def gaussian(seed: int, stream: int, count: int, first: int = 0) -> np.ndarray:
    """Gaussian variates first..first+count-1 of Philox stream (seed, stream), float64."""
    out = np.zeros(int(count))
    _load().orc_gaussian(int(seed), int(stream), int(first), int(count), _ptr(out))
    return out


def gaussian_matrix(seed: int, stream: int, rows: int, cols: int) -> np.ndarray:
    """Column-major rows x cols sketch: element (i, j) is variate i + j*rows, rounded to
    float32 (the precision the sketch is applied in) and widened back to float64."""
    g = gaussian(seed, stream, rows * cols).astype(np.float32).astype(np.float64)
    return g.reshape((cols, rows)).T.copy(order="F")


def _omp(name):
    try:
        return getattr(_load(), name)
    except AttributeError:  # built without OpenMP: one thread
        return None


def threads() -> int:
    """Threads the oracle's parallel loops use (1 when built without OpenMP)."""
    f = _omp("omp_get_max_threads")
    if f is None:
        return 1
    f.restype = C.c_int
    return int(f())


def set_threads(n: int) -> None:
    """Thread count of the oracle's parallel loops (results do not depend on it)."""
    f = _omp("omp_set_num_threads")
    if f is not None:
        f.argtypes = [C.c_int]
        f(int(n))
