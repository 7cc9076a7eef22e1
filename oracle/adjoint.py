"""FP64 CPU oracle of the adjoint (reverse-mode derivative) of Algorithm 1.

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU legs may import it.  It shares no code with the CUDA library.

The forward step is the paper's, restated in FP64 with the oracle's own Householder
QR and one-sided Jacobi SVD (Alg. 1 steps 1-5, Sec. 3.1):

    P = [ff U diag(D) | A]          (M x n, n = kc + B; kc = 0 at the
                                      initialisation I1-I2, where P = A_0)
    P = Q R                          (thin Householder QR, diag(R) >= 0)
    R = Ur diag(s) Vr^T              (square SVD, s descending)
    U' = Q Ur[:, :k1],  D' = s[:k1]  (truncation to k1 = min(K, n) modes)

and its adjoint is taken literally through those factors, in reverse order:

    1. Y = Q Ur_k          ->  Qbar = Ybar Ur_k^T,  Urbar = [Q^T Ybar | 0]
    2. SVD backward of the square R (V unused by the loss):
         Rbar = Ur [diag(sbar) + (F o (X - X^T)) diag(s)] Vr^T,
         X = Ur^T Urbar,  F_ij = 1 / (s_j^2 - s_i^2) (i != j, 0 on the diagonal)
    3. QR backward of the thin QR:
         Mq = R Rbar^T - Qbar^T Q,
         Pbar = (Qbar + Q copyltu(Mq)) R^-T,  copyltu(Mq) = tril(Mq) + tril(Mq, -1)^T
    4. P = [ff U diag(D) | A]  ->  Ubar = ff Pbar_U diag(D),
         Dbar_k = ff <U_k, Pbar_U,k>,  Abar = Pbar_A.

Steps 2 and 3 follow from differentiating R = Ur S Vr^T and P = Q R (the first-order
perturbation of each factor, solved for its antisymmetric / triangular parts).  Both
need distinct kept singular values and a full-rank panel; the pins in
``tests/test_adjoint_pins.py`` hold this oracle to central finite differences of the
C oracle's forward (the whole sweep, and the QR and SVD steps each on their own), to
the closed form of the Ky Fan k-norm's gradient, and to the homogeneity identities
of the streaming map.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import householder_qr, jacobi_svd, _f64


@dataclass
class Step:
    """What the reverse sweep needs from one forward step."""
    U: np.ndarray | None  # M x kc modes before the step (None at the initialisation)
    D: np.ndarray | None  # kc singular values before the step
    ff: float
    Q: np.ndarray         # M x n
    R: np.ndarray         # n x n
    Ur: np.ndarray        # n x n
    s: np.ndarray         # n
    Vr: np.ndarray        # n x n
    k1: int


def forward_step(U, D, A, ff, K):
    """One step of Algorithm 1 in FP64 by QR + SVD of R.  Returns (U', D', Step)."""
    A = _f64(A)
    if U is None:
        P = A
        kc = 0
    else:
        U = _f64(U)
        D = np.asarray(D, np.float64)
        P = np.concatenate([U * (ff * D)[None, :], A], axis=1)
        kc = U.shape[1]
    n = P.shape[1]
    Q, R = householder_qr(P)
    Ur, s, Vr, _ = jacobi_svd(R)
    if np.any(s <= 0):
        raise ValueError("the adjoint oracle needs a full-rank panel")
    k1 = min(int(K), n)
    Unew = Q @ Ur[:, :k1]
    return Unew, s[:k1].copy(), Step(U, D if kc else None, float(ff), Q, R, Ur, s, Vr, k1)


def forward(batches, K, ff):
    """Algorithm 1 over the batches (first one initialises); returns (U, D, tape)."""
    U = D = None
    tape = []
    for A in batches:
        U, D, st = forward_step(U, D, A, ff, K)
        tape.append(st)
    return U, D, tape


def _copyltu(M):
    return np.tril(M) + np.tril(M, -1).T


def qr_backward(Q, R, Qbar, Rbar):
    """Cotangent of P for the thin QR P = Q R (diag(R) > 0): (Qbar + Q copyltu(Mq)) R^-T."""
    Mq = R @ Rbar.T - Qbar.T @ Q
    G = Qbar + Q @ _copyltu(Mq)
    return np.linalg.solve(R, G.T).T


def svd_backward(Ur, s, Vr, Urbar, sbar, live):
    """Cotangent of the square R = Ur diag(s) Vr^T for a loss of (Ur, s) only:
    Ur [diag(sbar) + (F o (X - X^T)) diag(s)] Vr^T, X = Ur^T Urbar, F_ij = 1/(s_j^2 - s_i^2)
    on the pairs marked live (off-diagonal pairs that touch a column the loss uses)."""
    n = s.shape[0]
    X = Ur.T @ Urbar
    s2 = s ** 2
    diff = s2[None, :] - s2[:, None]  # (i, j) -> s_j^2 - s_i^2
    F = np.zeros((n, n))
    F[live] = 1.0 / diff[live]
    inner = np.diag(sbar) + (F * (X - X.T)) * s[None, :]
    return Ur @ inner @ Vr.T


def backward_step(st: Step, Ybar, sbar):
    """Reverse one forward step: (Ybar M x k1, sbar k1) -> (Ubar, Dbar, Abar)."""
    n = st.R.shape[0]
    k1 = st.k1
    Ybar = np.asarray(Ybar, np.float64)
    sbar_full = np.zeros(n)
    sbar_full[:k1] = sbar
    # 1. Y = Q Ur_k
    Qbar = Ybar @ st.Ur[:, :k1].T
    Urbar = np.zeros((n, n))
    Urbar[:, :k1] = st.Q.T @ Ybar
    # 2. square SVD backward
    live = np.zeros((n, n), dtype=bool)
    live[:k1, :] = True
    live[:, :k1] = True
    np.fill_diagonal(live, False)
    Rbar = svd_backward(st.Ur, st.s, st.Vr, Urbar, sbar_full, live)
    # 3. thin QR backward
    Pbar = qr_backward(st.Q, st.R, Qbar, Rbar)
    # 4. split the panel
    if st.U is None:
        return None, None, Pbar
    kc = st.U.shape[1]
    PU = Pbar[:, :kc]
    Ubar = st.ff * PU * st.D[None, :]
    Dbar = st.ff * np.sum(st.U * PU, axis=0)
    return Ubar, Dbar, Pbar[:, kc:]


def backward(tape, Ubar, Dbar):
    """Reverse sweep over the tape; returns the list of Abar, one per batch."""
    grads = [None] * len(tape)
    Ub, Db = np.asarray(Ubar, np.float64), np.asarray(Dbar, np.float64)
    for t in range(len(tape) - 1, -1, -1):
        Ub, Db, grads[t] = backward_step(tape[t], Ub, Db)
    return grads


def probe_loss(U, D, p, w):
    """The differentiation workload's loss  sum_k w_k (p^T u_k)^2 + sum_k sigma_k
    and its cotangents (Ubar, Dbar)."""
    U = np.asarray(U, np.float64)
    c = p @ U
    loss = float(np.sum(w * c * c) + np.sum(D))
    Ubar = np.outer(p, 2.0 * w * c)
    Dbar = np.ones_like(np.asarray(D, np.float64))
    return loss, Ubar, Dbar
