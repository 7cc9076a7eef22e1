"""The library's adjoint formulation, restated in numpy, equals the oracle's literal
QR + SVD backward (no GPU).

The CUDA adjoint never forms Q or the dropped singular vectors.  It recovers
V_k = P^T U' S_k^-1 from the output modes, takes the dropped directions through
the shifted solves (s_j^2 I - Pi H Pi)^-1 Pi P^T ybar_j, and returns
Pbar = P N + Ybar E.  This test writes that sequence out in FP64 (same steps,
no blocking) and checks it against oracle/adjoint.py, which differentiates the
Householder QR and the square SVD of R.  A mistake in the derivation would show up
here independently of the kernels.
"""
import numpy as np
import pytest

from oracle import adjoint as adj


def _formulation(U, D, A, ff, Unew, s, Ybar, sbar):
    kc = 0 if U is None else U.shape[1]
    L = A if U is None else np.concatenate([U, A], 1)
    n = L.shape[1]
    k1 = Unew.shape[1]
    Sd = np.concatenate([ff * D, np.ones(A.shape[1])]) if kc else np.ones(n)
    G = L.T @ np.concatenate([L, Unew, Ybar], 1)          # the one Gram pass
    H = Sd[:, None] * G[:, :n] * Sd[None, :]
    V = Sd[:, None] * G[:, n:n + k1] / s[None, :]        # V_k = P^T U' / s
    Cb = Sd[:, None] * G[:, n + k1:]                     # P^T Ybar
    Z = V.T @ Cb
    Bp = Cb - V @ Z                                      # Pi P^T Ybar
    HV = H @ V
    Hp = H - HV @ V.T - V @ HV.T + V @ (V.T @ HV) @ V.T  # Pi H Pi
    X = np.column_stack([np.linalg.solve(s[j] ** 2 * np.eye(n) - Hp, Bp[:, j])
                         for j in range(k1)])
    W = np.zeros((k1, k1))
    for i in range(k1):
        for j in range(k1):
            if i == j:
                W[i, i] = (sbar[i] - Z[i, i] / s[i] ** 2) / s[i]
            else:
                F = 1.0 / (s[j] ** 2 - s[i] ** 2)
                W[i, j] = (F * (Z[i, j] * s[j] / s[i] - Z[j, i]) - Z[i, j] / (s[i] * s[j])) / s[i]
    Xs = X / s[None, :]
    N = (V @ W + Xs) @ V.T + V @ Xs.T
    E = V.T / s[:, None]
    Pbar = L @ (Sd[:, None] * N) + Ybar @ E              # the apply pass
    if kc == 0:
        return None, None, Pbar
    SN = Sd[:, None] * N
    Dbar = ff * (np.einsum("kr,rk->k", G[:kc, :n], SN[:, :kc])
                 + np.einsum("kj,jk->k", G[:kc, n + k1:], E[:, :kc]))
    return Pbar[:, :kc] * (ff * D)[None, :], Dbar, Pbar[:, kc:]


@pytest.mark.parametrize("ff,K,B", [(1.0, 5, 8), (0.9, 5, 8), (0.95, 12, 8)])
def test_formulation_equals_qr_svd_backward(ff, K, B):
    # K = 12 > B at the first step: the initialisation keeps every column (no dropped
    # directions); the later steps truncate
    rng = np.random.default_rng(7)
    M, T, r = 1500, 4, 24
    U0 = np.linalg.qr(rng.standard_normal((M, r)))[0]
    V0 = np.linalg.qr(rng.standard_normal((B * T, r)))[0]
    A = (U0 * 1.15 ** -np.arange(r)) @ V0.T
    batches = [A[:, t * B:(t + 1) * B].copy() for t in range(T)]
    Uf, Df, tape = adj.forward(batches, K, ff)
    p = rng.standard_normal(M)
    w = rng.uniform(0.5, 1.5, Uf.shape[1])
    _, Ub, Db = adj.probe_loss(Uf, Df, p, w)
    ref = adj.backward(tape, Ub, Db)
    Us, Ds = [None], [None]
    U = D = None
    for Ab in batches:
        U, D, _ = adj.forward_step(U, D, Ab, ff, K)
        Us.append(U)
        Ds.append(D)
    g = [None] * T
    for t in range(T - 1, -1, -1):
        Ub, Db, g[t] = _formulation(Us[t], Ds[t], batches[t], ff, Us[t + 1], Ds[t + 1], Ub, Db)
    scale = max(np.abs(r_).max() for r_ in ref)
    assert max(np.abs(a - b).max() for a, b in zip(g, ref)) <= 1e-11 * scale
