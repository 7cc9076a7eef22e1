"""Pins of the FP64 adjoint oracle (no GPU).

The oracle's reverse sweep (QR and SVD backward, oracle/adjoint.py) is held to
things other than itself:
  * central finite differences (h = 1e-6) of the C oracle's forward Algorithm 1
    (a separate code path: orc_stream_initialize / orc_stream_update) on every
    entry of every batch of a tiny problem;
  * the closed-form gradient of the Ky Fan k-norm sum_{k<K} sigma_k of one SVD,
    U_K V_K^T, with the factors from numpy's LAPACK SVD;
  * homogeneity of the streaming map: scaling every batch by c scales every
    singular value by c and leaves the modes unchanged, so
    sum_t <Abar_t, A_t> equals sum_k sigma_k for the singular-value loss and 0
    for any loss of the modes alone.
"""
import numpy as np
import pytest

import oracle
from oracle import adjoint as adj


def _batches(M, B, T, seed, rank=None):
    rng = np.random.default_rng(seed)
    if rank is None:
        return [rng.standard_normal((M, B)) for _ in range(T)]
    U0 = np.linalg.qr(rng.standard_normal((M, rank)))[0]
    V0 = np.linalg.qr(rng.standard_normal((B * T, rank)))[0]
    s = 1.15 ** -np.arange(rank)
    A = (U0 * s) @ V0.T
    return [np.asfortranarray(A[:, t * B:(t + 1) * B]) for t in range(T)]


def _loss_c_oracle(batches, K, ff, p, w):
    U, D = oracle.stream_run(batches, K, ff)
    return float(np.sum(w * (p @ U) ** 2) + np.sum(D))


@pytest.mark.parametrize("ff", [1.0, 0.9])
def test_adjoint_matches_central_differences(ff):
    M, B, K, T = 30, 4, 3, 3
    batches = _batches(M, B, T, seed=11)
    rng = np.random.default_rng(12)
    p = rng.standard_normal(M)
    w = rng.uniform(0.5, 1.5, K)
    U, D, tape = adj.forward(batches, K, ff)
    U_c, D_c = oracle.stream_run(batches, K, ff)
    assert np.allclose(D, D_c, rtol=1e-12, atol=0)
    _, Ubar, Dbar = adj.probe_loss(U, D, p, w)
    grads = adj.backward(tape, Ubar, Dbar)
    h = 1e-6
    gmax = max(np.abs(g).max() for g in grads)
    for t in range(T):
        fd = np.zeros((M, B))
        for i in range(M):
            for j in range(B):
                bp = [b.copy() for b in batches]
                bm = [b.copy() for b in batches]
                bp[t][i, j] += h
                bm[t][i, j] -= h
                fd[i, j] = (_loss_c_oracle(bp, K, ff, p, w) - _loss_c_oracle(bm, K, ff, p, w)) / (2 * h)
        err = np.abs(fd - grads[t]).max()
        assert err <= 1e-6 * gmax, (t, err, gmax)


def test_adjoint_ky_fan_closed_form():
    # one SVD (the initialisation step): d/dP sum_{k<K} sigma_k = U_K V_K^T
    rng = np.random.default_rng(21)
    M, n, K = 50, 6, 3
    P = rng.standard_normal((M, n))
    U, D, tape = adj.forward([P], K, 1.0)
    (g,) = adj.backward(tape, np.zeros((M, K)), np.ones(K))
    Un, sn, Vtn = np.linalg.svd(P, full_matrices=False)
    assert np.allclose(D, sn[:K], rtol=1e-12)
    ref = Un[:, :K] @ Vtn[:K, :]
    assert np.abs(g - ref).max() <= 1e-12


@pytest.mark.parametrize("ff", [1.0, 0.95])
def test_adjoint_homogeneity(ff):
    M, B, K, T = 2000, 8, 5, 4
    batches = _batches(M, B, T, seed=31, rank=24)
    U, D, tape = adj.forward(batches, K, ff)
    # singular-value loss: sum_t <Abar_t, A_t> = sum_k sigma_k
    g = adj.backward(tape, np.zeros_like(U), np.ones_like(D))
    lhs = sum(float(np.sum(gt * At)) for gt, At in zip(g, batches))
    assert abs(lhs - D.sum()) <= 1e-10 * D.sum()
    # mode loss: sum_t <Abar_t, A_t> = 0
    rng = np.random.default_rng(32)
    p = rng.standard_normal(M)
    w = rng.uniform(0.5, 1.5, K)
    _, Ubar, _ = adj.probe_loss(U, D, p, w)
    g = adj.backward(tape, Ubar, np.zeros_like(D))
    lhs = sum(float(np.sum(gt * At)) for gt, At in zip(g, batches))
    scale = sum(np.linalg.norm(gt) * np.linalg.norm(At) for gt, At in zip(g, batches))
    assert abs(lhs) <= 1e-10 * scale


def test_qr_backward_matches_central_differences():
    # the QR step alone, for a loss that uses Q and R directly (gauge fixed by diag(R) > 0)
    rng = np.random.default_rng(41)
    M, n = 12, 4
    P = rng.standard_normal((M, n))
    C1 = rng.standard_normal((M, n))
    C2 = np.triu(rng.standard_normal((n, n)))

    def loss(Pm):
        Q, R = oracle.householder_qr(Pm)
        return float(np.sum(C1 * Q) + np.sum(C2 * R))

    Q, R = oracle.householder_qr(P)
    g = adj.qr_backward(Q, R, C1, C2)
    h = 1e-6
    fd = np.zeros_like(P)
    for i in range(M):
        for j in range(n):
            Pp, Pm = P.copy(), P.copy()
            Pp[i, j] += h
            Pm[i, j] -= h
            fd[i, j] = (loss(Pp) - loss(Pm)) / (2 * h)
    assert np.abs(fd - g).max() <= 1e-7 * np.abs(g).max()


def test_svd_backward_matches_central_differences():
    # the square SVD step alone, for a sign-invariant loss of (Ur, s)
    rng = np.random.default_rng(42)
    n, k = 5, 3
    R = rng.standard_normal((n, n))
    a = rng.standard_normal(n)
    c = rng.uniform(0.5, 1.5, k)

    def factors(Rm):
        Ur, s, Vr, _ = oracle.jacobi_svd(Rm)
        return Ur, s, Vr

    def loss(Rm):
        Ur, s, _ = factors(Rm)
        return float(np.sum(c * (a @ Ur[:, :k]) ** 2) + np.sum(s[:k] ** 1.5))

    Ur, s, Vr = factors(R)
    Urbar = np.zeros((n, n))
    Urbar[:, :k] = np.outer(a, 2 * c * (a @ Ur[:, :k]))
    sbar = np.zeros(n)
    sbar[:k] = 1.5 * s[:k] ** 0.5
    live = np.zeros((n, n), dtype=bool)
    live[:k, :] = True
    live[:, :k] = True
    np.fill_diagonal(live, False)
    g = adj.svd_backward(Ur, s, Vr, Urbar, sbar, live)
    h = 1e-6
    fd = np.zeros_like(R)
    for i in range(n):
        for j in range(n):
            Rp, Rm = R.copy(), R.copy()
            Rp[i, j] += h
            Rm[i, j] -= h
            fd[i, j] = (loss(Rp) - loss(Rm)) / (2 * h)
    assert np.abs(fd - g).max() <= 1e-7 * np.abs(g).max()
