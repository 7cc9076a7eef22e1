"""Pins of the literal randomization placement (the paper's low_rank_svd applied to
the small factors: rfinal in the streaming update, W in Algorithm 2), no GPU.

* rfinal: for P = Q R, P Omega = Q (R Omega), so the randomized SVD of R with a
  given Omega, mapped through Q, is the randomized SVD of the panel P with the same
  Omega (the sign convention (P 1)^T u >= 0 maps to (R 1)^T u_R >= 0 too).  The
  oracle's two runs must agree to rounding.
* W: with a sketch as wide as W's rank, the randomized APMOS equals the exact one
  (oracle.apmos); with a narrower sketch it equals the same subspace iteration
  restated with LAPACK (numpy QR and SVD) on the same W and Omega.
"""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("q", [0, 1, 2])
def test_rsvd_of_rfinal_equals_panel_front_end(q):
    rng = np.random.default_rng(61)
    M, n, K, l = 400, 30, 8, 14
    P = rng.standard_normal((M, n)) * (0.8 ** np.arange(n))[None, :]
    Om = rng.standard_normal((n, l))
    Up, Dp = oracle.rsvd_panel(P, K, Om, q)
    Q, R = oracle.householder_qr(P)
    Ur, Dr = oracle.rsvd_panel(R, K, Om, q)
    assert np.abs(Dp / Dr - 1).max() <= 1e-12
    assert np.abs(Up - Q @ Ur).max() <= 1e-10


def _blocks(N, sizes, rank, seed):
    rng = np.random.default_rng(seed)
    M = sum(sizes)
    U0 = np.linalg.qr(rng.standard_normal((M, rank)))[0]
    V0 = np.linalg.qr(rng.standard_normal((N, rank)))[0]
    A = (U0 * 1.15 ** -np.arange(rank)) @ V0.T
    return np.asfortranarray(A), np.concatenate([[0], np.cumsum(sizes)])


def _angle(U1, U2):
    Q1, Q2 = np.linalg.qr(U1)[0], np.linalg.qr(U2)[0]
    return float(np.arcsin(min(1.0, np.linalg.norm(Q2 - Q1 @ (Q1.T @ Q2), 2))))


@pytest.mark.parametrize("q", [0, 1])
def test_apmos_low_rank_exact_when_sketch_covers_rank(q):
    N, r1, r2 = 12, 4, 5
    A, off = _blocks(N, [60, 45, 80, 50, 70], N, seed=62)
    # l = min(r2 + p, N) = N: the sketch spans the range of W
    U, L = oracle.apmos_low_rank(A, off, r1, r2, p=20, q=q, seed=5)
    Ue, Le = oracle.apmos(A, off, r1, r2)
    assert np.abs(L / Le - 1).max() <= 1e-10
    assert _angle(U, Ue) <= 1e-9


def test_apmos_low_rank_matches_lapack_subspace_iteration():
    N, r1, r2, p, q, seed = 40, 10, 6, 4, 1, 7
    A, off = _blocks(N, [300, 200, 260, 240], 40, seed=63)
    U, L = oracle.apmos_low_rank(A, off, r1, r2, p, q, seed)
    W = oracle.apmos_local_factors(A, off, r1)
    l = min(r2 + p, N)
    Om = oracle.gaussian_matrix(seed, oracle.APMOS_SKETCH_STREAM, W.shape[1], l)
    Y = W @ Om
    for _ in range(q):
        Y = W @ (W.T @ np.linalg.qr(Y)[0])
    Qy = np.linalg.qr(Y)[0]
    Ub, s, _ = np.linalg.svd(Qy.T @ W, full_matrices=False)
    X = Qy @ Ub[:, :r2]
    assert np.abs(L / s[:r2] - 1).max() <= 1e-10
    assert _angle(U, A @ (X / s[None, :r2])) <= 1e-9
    # a sketch narrower than the rank is a genuine approximation of the exact APMOS
    Le = oracle.apmos(A, off, r1, r2)[1]
    assert np.abs(L / Le - 1).max() > 1e-8
