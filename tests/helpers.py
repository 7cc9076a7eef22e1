"""Comparison helpers shared by the tests (plain numpy, float64)."""
from __future__ import annotations

import numpy as np


def orth(X):
    Q, _ = np.linalg.qr(np.asarray(X, dtype=np.float64))
    return Q


def max_principal_angle(U1, U2) -> float:
    """Largest principal angle (radians) between span(U1) and span(U2), same dimension.

    Computed as arcsin of the spectral norm of (I - Q1 Q1^T) Q2, which is accurate for
    small angles (the cosine form loses everything below ~1e-8)."""
    Q1, Q2 = orth(U1), orth(U2)
    R = Q2 - Q1 @ (Q1.T @ Q2)
    s = np.linalg.norm(R, 2) if R.size else 0.0
    return float(np.arcsin(min(1.0, s)))


def column_angles(U1, U2) -> np.ndarray:
    """Per-column angle between matching columns after sign alignment."""
    U1 = np.asarray(U1, np.float64)
    U2 = np.asarray(U2, np.float64)
    out = []
    for j in range(U1.shape[1]):
        a, b = U1[:, j], U2[:, j]
        na, nb = np.linalg.norm(a), np.linalg.norm(b)
        c = abs(a @ b) / (na * nb)
        d = np.linalg.norm(a / na - np.sign(a @ b) * b / nb)
        out.append(2.0 * np.arcsin(min(1.0, d / 2.0)) if c > 0.5 else np.pi / 2)
    return np.array(out)


def rel_err(a, b) -> np.ndarray:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), np.finfo(np.float64).tiny)
