"""Pins the FP64 oracle to things other than itself (CPU only).

Each test checks an oracle routine against a closed form, an invariant, brute
force, or an independent library routine (LAPACK through numpy, numpy's own
Philox4x64), chosen so that a plausible slip -- a dropped term, a wrong sign or
index, a transposed operand, a wrong truncation or ordering -- fails at least one.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2108_08845_gb300 import synthetic
from tests.helpers import max_principal_angle, rel_err

RNG = np.random.default_rng(20210819)


# --------------------------------------------------------------------------- QR
@pytest.mark.parametrize("m,n", [(60, 9), (9, 9), (200, 35), (33, 1)])
def test_qr_factorisation_properties(m, n):
    A = RNG.standard_normal((m, n))
    Q, R = oracle.householder_qr(A)
    assert np.abs(Q @ R - A).max() <= 1e-13 * np.abs(A).max() * n
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 1e-14 * max(n, 4)
    assert np.all(np.tril(R, -1) == 0)
    assert np.all(np.diag(R) >= 0)


def test_qr_R_equals_cholesky_factor_of_gram():
    # for full-rank A the QR with diag(R) > 0 is unique: R = chol(A^T A)^T (LAPACK potrf)
    A = RNG.standard_normal((120, 17))
    _, R = oracle.householder_qr(A)
    L = np.linalg.cholesky(A.T @ A)
    assert np.abs(R - L.T).max() <= 1e-12 * np.abs(R).max()


def test_qr_rank_deficient_still_orthonormal():
    A = RNG.standard_normal((40, 6))
    A[:, 3] = 0.0
    A[:, 5] = A[:, 1]
    Q, R = oracle.householder_qr(A)
    assert np.abs(Q @ R - A).max() <= 1e-13
    assert np.abs(Q.T @ Q - np.eye(6)).max() <= 1e-14


# ------------------------------------------------------------------- Jacobi SVD
def test_jacobi_recovers_constructed_singular_values():
    m, n = 80, 12
    s = np.array([10.0 ** (-i / 4.0) for i in range(n)])
    U0 = np.linalg.qr(RNG.standard_normal((m, n)))[0]
    V0 = np.linalg.qr(RNG.standard_normal((n, n)))[0]
    A = (U0 * s) @ V0.T
    U, sv, V, _ = oracle.jacobi_svd(A)
    assert rel_err(sv, s).max() <= 1e-12
    # distinct singular values: vectors unique up to sign
    sg = np.sign(np.sum(U * U0, axis=0))
    assert np.abs(U * sg - U0).max() <= 1e-10
    assert np.abs(V * sg - V0).max() <= 1e-10
    assert np.abs(A @ V - U * sv).max() <= 1e-14


@pytest.mark.parametrize("m,n", [(50, 20), (20, 20), (7, 3), (5, 9)])
def test_jacobi_matches_lapack_svd(m, n):
    A = RNG.standard_normal((m, n))
    U, s, V, sweeps = oracle.jacobi_svd(A)
    ref = np.linalg.svd(A, compute_uv=False)
    k = min(m, n)
    assert rel_err(s[:k], ref).max() <= 1e-12
    assert np.all(s[k:] <= 1e-12 * s[0])
    assert np.all(np.diff(s) <= 0)
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-13
    assert sweeps <= 20


def test_jacobi_repeated_singular_values_subspace():
    m, n = 60, 8
    s = np.array([3.0, 3.0, 3.0, 2.0, 1.0, 1.0, 0.5, 0.1])
    U0 = np.linalg.qr(RNG.standard_normal((m, n)))[0]
    V0 = np.linalg.qr(RNG.standard_normal((n, n)))[0]
    U, sv, V, _ = oracle.jacobi_svd((U0 * s) @ V0.T)
    assert rel_err(sv, s).max() <= 1e-13
    assert max_principal_angle(U[:, :3], U0[:, :3]) <= 1e-12
    assert max_principal_angle(U[:, 4:6], U0[:, 4:6]) <= 1e-12


def test_jacobi_zero_and_scalar():
    U, s, V, _ = oracle.jacobi_svd(np.zeros((5, 3)))
    assert np.all(s == 0) and np.all(U == 0)
    U, s, V, _ = oracle.jacobi_svd(np.array([[-2.5]]))
    assert s[0] == 2.5 and U[0, 0] * V[0, 0] == -1.0


def test_sort_is_stable_descending():
    s = np.array([1.0, 3.0, 2.0, 3.0, 1.0])
    assert list(oracle.sort_desc(s)) == [1, 3, 2, 0, 4]


# ------------------------------------------------------- Algorithm 1 (streaming)
def _batches(A, B):
    return [A[:, i:i + B] for i in range(0, A.shape[1], B)]


def test_stream_ff1_rank_le_K_recovers_closed_form():
    # rank-10 data, K = 10, ff = 1: no information is ever truncated, so the
    # streaming result equals the one-shot SVD (Sec. 3.1: ff = 1 converges to the
    # regular SVD), i.e. exactly the constructed s and span(U0).
    A, U0, s, _ = synthetic.low_rank(300, 60, 10, 0.0, seed=11)
    A = A.numpy()
    U, D = oracle.stream_run(_batches(A, 20), K=10, ff=1.0)
    assert rel_err(D, s.numpy()).max() <= 1e-12
    assert max_principal_angle(U, U0.numpy()) <= 1e-11
    assert np.abs(U.T @ U - np.eye(10)).max() <= 1e-13


def test_stream_ff1_K_ge_rank_matches_full_svd():
    # low-rank structure at M = 500 with K = 40 = rank: equals LAPACK SVD of all data
    A, _, _, _ = synthetic.low_rank(500, 100, 40, 1e-8, seed=12)
    A = A.numpy()
    ref_U, ref_s, _ = np.linalg.svd(A, full_matrices=False)
    U, D = oracle.stream_run(_batches(A, 25), K=40, ff=1.0)
    # the first 35 directions are far above the 1e-8 noise floor
    assert rel_err(D[:35], ref_s[:35]).max() <= 1e-9
    assert max_principal_angle(U[:, :20], ref_U[:, :20]) <= 1e-10


def test_stream_forget_factor_closed_form():
    # no truncation (rank 8 = K): the result is the SVD of the weighted
    # concatenation [ff^(T-1) A_0, ..., ff A_(T-2), A_(T-1)] (ff scales U*D).
    A, _, _, _ = synthetic.low_rank(200, 48, 8, 0.0, seed=13)
    A = A.numpy()
    bs = _batches(A, 12)
    ff = 0.9
    T = len(bs)
    W = np.concatenate([ff ** (T - 1 - i) * b for i, b in enumerate(bs)], axis=1)
    ref_U, ref_s, _ = np.linalg.svd(W, full_matrices=False)
    U, D = oracle.stream_run(bs, K=8, ff=ff)
    assert rel_err(D, ref_s[:8]).max() <= 1e-12
    assert max_principal_angle(U, ref_U[:, :8]) <= 1e-10
    # energy invariant without truncation
    assert abs(np.sum(D ** 2) - np.sum(W ** 2)) <= 1e-12 * np.sum(W ** 2)


def _listing1_numpy(batches, K, ff):
    """Algorithm 1 restated with LAPACK (numpy qr / svd) as an independent check."""
    q, r = np.linalg.qr(batches[0])
    ui, d, _ = np.linalg.svd(r)
    U, D = (q @ ui)[:, :K], d[:K]
    for A in batches[1:]:
        P = np.concatenate([ff * U * D[None, :], A], axis=1)
        q, r = np.linalg.qr(P)
        ut, dt, _ = np.linalg.svd(r)
        keep = np.argsort(-dt, kind="stable")[:K]
        U, D = q @ ut[:, keep], dt[keep]
    return U, D


@pytest.mark.parametrize("ff", [1.0, 0.95])
def test_stream_truncating_matches_lapack_restatement(ff):
    # K = 6 < rank: truncation after every batch; both must agree step by step
    A, _, _, _ = synthetic.low_rank(400, 120, 30, 1e-6, seed=14)
    bs = _batches(A.numpy(), 20)
    U, D = oracle.stream_run(bs, K=6, ff=ff)
    Ur, Dr = _listing1_numpy(bs, 6, ff)
    assert rel_err(D, Dr).max() <= 1e-11
    assert max_principal_angle(U, Ur) <= 1e-9
    assert np.abs(U.T @ U - np.eye(6)).max() <= 1e-13


def test_stream_truncation_energy_bound():
    # with truncation, the kept energy never exceeds the weighted total
    A, _, _, _ = synthetic.low_rank(300, 90, 30, 1e-6, seed=15)
    bs = _batches(A.numpy(), 15)
    U, D = oracle.stream_run(bs, K=5, ff=1.0)
    assert np.sum(D ** 2) <= np.sum(A.numpy() ** 2) * (1 + 1e-12)
    # and sigma_1 can only be bounded by the true sigma_1 of all data
    assert D[0] <= np.linalg.svd(A.numpy(), compute_uv=False)[0] * (1 + 1e-12)


def test_stream_initialize_shape_errors():
    with pytest.raises(oracle.OracleError):
        oracle.stream_initialize(np.ones((3, 10)), K=4)  # B > M
    with pytest.raises(oracle.OracleError):
        oracle.stream_update(np.ones((10, 6)), np.ones(6), np.ones((10, 6)), 1.0)  # M < K+B


# ----------------------------------------------------------- partitioned QR (TSQR)
def test_tsqr_R_equals_direct_R():
    A = RNG.standard_normal((300, 12))
    R = oracle.tsqr_r(A, [0, 40, 150, 151 + 20, 300])
    _, R0 = oracle.householder_qr(A)
    assert np.abs(R - R0).max() <= 1e-12 * np.abs(R0).max()
    assert np.abs(R - np.linalg.cholesky(A.T @ A).T).max() <= 1e-11 * np.abs(R0).max()


# ---------------------------------------------------------- Algorithm 2 (APMOS)
def test_apmos_exact_when_r1_covers_local_rank():
    # r1 = N keeps all local information: W W^T = A^T A, so X = V and Lambda = sigma(A)
    A = RNG.standard_normal((240, 10)) * (2.0 ** -np.arange(10))[None, :]
    off = [0, 50, 130, 240]
    U, L = oracle.apmos(A, off, r1=10, r2=6)
    Ur, sr, _ = np.linalg.svd(A, full_matrices=False)
    assert rel_err(L, sr[:6]).max() <= 1e-12
    sg = np.sign(np.sum(U * Ur[:, :6], axis=0))
    assert np.abs(U * sg - Ur[:, :6]).max() <= 1e-10


def test_apmos_single_partition_equals_serial_svd():
    A = RNG.standard_normal((90, 8))
    U, L = oracle.apmos(A, [0, 90], r1=8, r2=8)
    Ur, sr, _ = np.linalg.svd(A, full_matrices=False)
    assert rel_err(L, sr).max() <= 1e-12
    assert max_principal_angle(U[:, :3], Ur[:, :3]) <= 1e-11


def test_apmos_truncated_modes_are_partition_consistent():
    # r1 < N: an approximation, but each global mode satisfies A^i X_j / L_j on every
    # block, so the assembled U equals A X~ L~^-1 computed in one piece
    A, _, _, _ = synthetic.low_rank(360, 24, 24, 0.0, seed=16,
                                    s=[2.0 ** (-i) for i in range(24)])
    A = A.numpy()
    U, L = oracle.apmos(A, [0, 100, 200, 360], r1=6, r2=4)
    assert np.all(np.diff(L) <= 0) and L[-1] > 0
    # leading global mode is close to the exact one (fast decay, r1 = 6)
    Ur, sr, _ = np.linalg.svd(A, full_matrices=False)
    assert abs(L[0] - sr[0]) / sr[0] < 1e-3
    assert max_principal_angle(U[:, :1], Ur[:, :1]) < 1e-2


# ------------------------------------------------------ randomized SVD (Sec. 3.3)
@pytest.mark.parametrize("q", [0, 1])
def test_rsvd_exact_when_sketch_covers_rank(q):
    A, _, _, _ = synthetic.low_rank(250, 60, 10, 0.0, seed=17)
    bs = _batches(A.numpy(), 20)
    U, D = oracle.stream_initialize(bs[0], K=8)
    P = oracle.panel(U, D, bs[1], 0.95)  # 28 columns, rank <= 10
    Om = oracle.gaussian_matrix(5, 1, P.shape[1], 14)
    Ur, Dr = oracle.rsvd_panel(P, 8, Om, q)
    Ud, Dd = oracle.stream_update(U, D, bs[1], 0.95)
    assert rel_err(Dr, Dd).max() <= 1e-10
    assert max_principal_angle(Ur, Ud) <= 1e-9
    # sign convention of the randomized modes: (P 1)^T u_j >= 0
    assert np.all(P.sum(axis=1) @ Ur >= 0.0)
    # ... and otherwise the same vectors as the exact update (distinct sigmas)
    sg = np.sign(np.sum(Ur * Ud, axis=0))
    assert np.abs(Ur - Ud * sg[None, :]).max() <= 1e-8


def test_rsvd_power_iteration_improves_accuracy():
    A, _, _, _ = synthetic.low_rank(400, 80, 80, 0.0, seed=18,
                                    s=[1.0 / (1 + i) for i in range(80)])
    P = A.numpy()
    ref = np.linalg.svd(P, compute_uv=False)[:10]
    Om = oracle.gaussian_matrix(9, 2, 80, 14)
    e0 = rel_err(oracle.rsvd_panel(P, 10, Om, 0)[1], ref).max()
    e2 = rel_err(oracle.rsvd_panel(P, 10, Om, 2)[1], ref).max()
    assert e2 < e0 and e2 < 0.05


def test_rsvd_run_with_full_sketch_equals_exact_stream():
    # p >= B gives l = n at every batch: Q spans the whole panel, so each
    # randomized update reduces to the exact one
    A, _, _, _ = synthetic.low_rank(300, 60, 30, 1e-6, seed=19, s=[0.8 ** i for i in range(30)])
    bs = _batches(A.numpy(), 15)
    Ur, Dr = oracle.rsvd_run(bs, 6, 0.9, p=15, q=0, seed=3)
    Ud, Dd = oracle.stream_run(bs, 6, 0.9)
    assert rel_err(Dr, Dd).max() <= 1e-10
    assert max_principal_angle(Ur, Ud) <= 1e-8


# --------------------------------------------------------------------- Philox
@pytest.mark.parametrize("ctr,key", [
    ([5, 7, 9, 2 ** 64 - 1], [0x0123456789ABCDEF, 0xFEDCBA9876543210]),
    ([0, 0, 0, 0], [0, 0]),
    ([2 ** 64 - 2, 2 ** 63, 1, 3], [2 ** 64 - 1, 12345]),
])
def test_philox4x64_matches_numpy_bit_generator(ctr, key):
    # numpy.random.Philox is an independent Philox4x64-10; it increments the
    # counter before each block.  This pins the round function, the key
    # schedule and the word order shared with the 4x32 instantiation.
    bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64),
                          key=np.array(key, dtype=np.uint64))
    raw = [int(x) for x in bg.random_raw(8)]
    c1 = list(ctr)
    out = []
    for _ in range(2):
        c1[0] = (c1[0] + 1) % 2 ** 64
        if c1[0] == 0:
            c1[1] = (c1[1] + 1) % 2 ** 64
        out += oracle.philox4x64(c1, key)
    assert out == raw


def _philox_kat():
    path = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.txt")
    rows = []
    for line in open(path):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        w = [int(x, 16) for x in f[2:]]
        rows.append((f[0], int(f[1]), w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("gen,rounds,ctr,key,expect", _philox_kat())
def test_philox_published_known_answers(gen, rounds, ctr, key, expect):
    # the published known-answer vectors of Philox4x32-10 (the generator of the
    # Gaussian test matrix) and Philox4x64-10: a mistyped multiplier, Weyl constant
    # or word order changes every output word
    f = oracle.philox4x32 if gen == "philox4x32" else oracle.philox4x64
    assert list(f(ctr, key, rounds)) == expect


def test_philox4x32_bit_statistics_and_avalanche():
    key = [0xDEADBEEF, 0x12345678]
    n = 20000
    words = np.array([oracle.philox4x32([i, 0, 3, 0], key) for i in range(n)],
                     dtype=np.uint64).reshape(-1)
    bits = ((words[:, None] >> np.arange(32, dtype=np.uint64)[None, :]) & 1).astype(np.float64)
    p = bits.mean(axis=0)
    assert np.all(np.abs(p - 0.5) < 6 * 0.5 / math.sqrt(words.size))
    # flipping one counter bit flips about half of the 128 output bits
    flips = []
    for i in range(200):
        a = oracle.philox4x32([i, 77, 3, 9], key)
        b = oracle.philox4x32([i ^ (1 << (i % 32)), 77, 3, 9], key)
        flips.append(sum(bin(x ^ y).count("1") for x, y in zip(a, b)))
    assert 60 < np.mean(flips) < 68
    # fewer rounds give different words (the round loop is really applied 10 times)
    assert oracle.philox4x32([1, 2, 3, 4], key, rounds=9) != oracle.philox4x32([1, 2, 3, 4], key)


# ---------------------------------------------------------- Gaussian transform
def test_own_log_matches_libm():
    xs = [2.0 ** -53, 1e-300 * 0 + 2.0 ** -40, 1e-9, 0.1, 0.3, 0.5, 0.7071067811865476,
          0.7071067811865475, 0.9, 0.999999, 1.0 - 2.0 ** -53, 1.0]
    xs += list(RNG.uniform(0, 1, 2000))
    for x in xs:
        if x <= 0:
            continue
        got, ref = oracle.ln(x), math.log(x)
        assert abs(got - ref) <= 2 * math.ulp(ref) + 1e-300, (x, got, ref)
    assert oracle.ln(1.0) == 0.0


def test_own_sincos_matches_libm():
    us = [0.0, 0.125, 0.25, 0.5, 0.75, 1.0 - 2.0 ** -53] + list(RNG.uniform(0, 1, 2000))
    for u in us:
        s, c = oracle.sincos_2pi(u)
        # the reference argument 2*pi*u itself carries up to ~9e-16 absolute rounding
        assert abs(s - math.sin(2 * math.pi * u)) <= 1e-15
        assert abs(c - math.cos(2 * math.pi * u)) <= 1e-15


def test_gaussian_moments_and_ks():
    from scipy import stats
    g = oracle.gaussian(seed=42, stream=7, count=400000)
    n = g.size
    assert abs(g.mean()) < 5 / math.sqrt(n)
    assert abs(g.var() - 1) < 5 * math.sqrt(2 / n)
    assert abs(stats.skew(g)) < 5 * math.sqrt(6 / n)
    assert abs(stats.kurtosis(g)) < 5 * math.sqrt(24 / n)
    assert stats.kstest(g, "norm").pvalue > 1e-4


def test_gaussian_is_counter_based():
    a = oracle.gaussian(3, 11, 50, first=0)
    b = oracle.gaussian(3, 11, 20, first=30)
    assert np.array_equal(a[30:50], b)
    c = oracle.gaussian(3, 12, 50)
    assert not np.array_equal(a, c)
    m = oracle.gaussian_matrix(3, 11, 5, 10)
    assert m[2, 3] == np.float32(a[2 + 3 * 5])
