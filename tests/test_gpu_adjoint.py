"""GPU parity of the hand-written adjoint of Algorithm 1 (psvd_update_adjoint through
the torch.autograd.Function) against the FP64 adjoint oracle.

Loss (the differentiation workload): L = sum_k w_k (p^T u_k)^2 + sum_k sigma_k for a
seeded probe p and weights w.  Its gradient with respect to every entry of every
batch comes from the library; the oracle's comes from the literal QR + SVD backward
of oracle/adjoint.py (itself pinned by central differences in
test_adjoint_pins.py).  Both sides read the same FP32 (or BF16) batch values.

Tolerance: the FP32 forward's modes carry ~1e-7 relative rounding (a few u32 from
the compensated Gram and the update), which the gradient map amplifies by at most the
largest 1/(1 - s_j^2/s_i^2) between kept and dropped indices (~4 for the 13 % gap of
the workload) over a few steps, and the adjoint's FP32 panel passes add ~1e-7; an
error of 5e-6 of the largest gradient entry bounds that with a margin of ~10 (the
measured errors are 2e-8 to 3e-7), while a wrong term (sign, index, a dropped
block) moves the gradient by O(1) of its size.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint as adj
from paper_2108_08845_gb300 import psvd, synthetic
from paper_2108_08845_gb300.autograd import streaming_svd

pytestmark = pytest.mark.gpu

TOL = 5e-6


def _workload(M, B, T, rank, seed, dtype=torch.float32):
    A, *_ = synthetic.spectrum(M, B * T, [1.15 ** -i for i in range(rank)], seed)
    A = synthetic.to_storage(A, dtype)
    host = [np.asfortranarray(A[:, t * B:(t + 1) * B].to(torch.float64).numpy()) for t in range(T)]
    dev = [A[:, t * B:(t + 1) * B].cuda().T.contiguous().T.requires_grad_(True) for t in range(T)]
    return host, dev


def _gpu_grads(dev, K, ff, p, w):
    U, D = streaming_svd(dev, K, ff)
    pt = torch.as_tensor(p, dtype=torch.float32, device="cuda")
    wt = torch.as_tensor(w, dtype=torch.float32, device="cuda")
    loss = (wt * (pt @ U) ** 2).sum() + D.sum()
    grads = torch.autograd.grad(loss, dev)
    return U.detach(), D.detach(), [g.double().cpu().numpy() for g in grads]


def _oracle_grads(host, K, ff, p, w):
    U, D, tape = adj.forward(host, K, ff)
    _, Ub, Db = adj.probe_loss(U, D, p, w)
    return D, adj.backward(tape, Ub, Db), tape


def _rel_err(g, ref):
    scale = max(np.abs(r).max() for r in ref)
    return max(np.abs(a - b).max() for a, b in zip(g, ref)) / scale


def test_adjoint_matches_oracle_all_entries():
    M, B, K, T, ff = 4096, 16, 8, 4, 0.9
    host, dev = _workload(M, B, T, 40, seed=501)
    rng = np.random.default_rng(502)
    p = rng.standard_normal(M)
    w = rng.uniform(0.5, 1.5, K)
    _, D, g = _gpu_grads(dev, K, ff, p, w)
    Do, go, _ = _oracle_grads(host, K, ff, p, w)
    assert np.abs(D.cpu().numpy() / Do - 1).max() <= 1e-5
    err = _rel_err(g, go)
    print(f"gradient error {err:.3e} of the largest entry")
    assert err <= TOL
    # the reductions run in a fixed order: a second sweep is bit-identical
    _, _, g2 = _gpu_grads(dev, K, ff, p, w)
    assert all(np.array_equal(a, b) for a, b in zip(g, g2))


def test_adjoint_ragged_rows_bf16_and_untruncated_steps():
    # M not a multiple of the 64-row tiles; the initialisation keeps every column
    # (k1 = n: no dropped directions), the later steps truncate
    M, B, K, T, ff = 3001, 8, 12, 3, 0.95
    host, dev = _workload(M, B, T, 20, seed=511, dtype=torch.bfloat16)
    rng = np.random.default_rng(512)
    p = rng.standard_normal(M)
    w = rng.uniform(0.5, 1.5, K)
    _, D, g = _gpu_grads(dev, K, ff, p, w)
    Do, go, _ = _oracle_grads(host, K, ff, p, w)
    assert np.abs(D.cpu().numpy() / Do - 1).max() <= 1e-5
    # the gradient of a BF16 input is returned in BF16 (torch keeps a gradient in its
    # input's dtype): with 8 significant bits, each entry then carries a round-to-nearest
    # error <= 2^-8 of itself (the FP32 gradient itself is checked in the other tests)
    scale = max(np.abs(r).max() for r in go)
    err = max((np.abs(a - b) - 2.0 ** -8 * np.abs(b)).max() for a, b in zip(g, go)) / scale
    print(f"gradient error beyond BF16 rounding {err:.3e} of the largest entry")
    assert err <= TOL


def test_adjoint_differentiation_workload_full_size():
    # M = 262,144, K = 16, 8 batches of B = 32, ff = 1, spectrum 1.15^-i (rank 64)
    M, B, K, T, ff = 262144, 32, 16, 8, 1.0
    host, dev = _workload(M, B, T, 64, seed=1238)
    rng = np.random.default_rng(1239)
    p = rng.standard_normal(M)
    w = rng.uniform(0.5, 1.5, K)
    _, D, g = _gpu_grads(dev, K, ff, p, w)
    # homogeneity of the streaming map: sum_t <Abar_t, A_t> = sum_k sigma_k
    lhs = sum(float(np.sum(gt * At)) for gt, At in zip(g, host))
    assert abs(lhs / float(D.sum()) - 1) <= 1e-4
    # 64 random entries against the oracle's analytic gradient
    Do, go, tape = _oracle_grads(host, K, ff, p, w)
    scale = max(np.abs(r).max() for r in go)
    ts = rng.integers(0, T, 64)
    rs = rng.integers(0, M, 64)
    cs = rng.integers(0, B, 64)
    err = max(abs(g[t][r, c] - go[t][r, c]) for t, r, c in zip(ts, rs, cs)) / scale
    print(f"sampled gradient error {err:.3e}, homogeneity {lhs / float(D.sum()) - 1:.2e}")
    assert err <= TOL
    # central differences (h = 1e-6) of the FP64 oracle forward on entries of the
    # last two batches, restarted from the oracle's state before that batch
    h = 1e-6

    def loss_from(t, batch_t):
        U = D_ = None
        if t > 0:
            st = tape[t]
            U, D_ = st.U, st.D
        seq = [batch_t] + host[t + 1:]
        for A in seq:
            U, D_, _ = adj.forward_step(U, D_, A, ff, K)
        return float(np.sum(w * (p @ U) ** 2) + np.sum(D_))

    for t in (T - 1, T - 2):
        for _ in range(3):
            r, c = int(rng.integers(0, M)), int(rng.integers(0, B))
            bp, bm = host[t].copy(), host[t].copy()
            bp[r, c] += h
            bm[r, c] -= h
            fd = (loss_from(t, bp) - loss_from(t, bm)) / (2 * h)
            print(f"FD batch {t}: {abs(fd - g[t][r, c]) / scale:.3e}")
            assert abs(fd - g[t][r, c]) <= TOL * scale, (t, r, c, fd, g[t][r, c])


def test_adjoint_degenerate_pair_warns():
    # two orthogonal columns of equal norm, one mode kept: the kept and the dropped
    # singular value coincide and the derivative does not exist
    M = 1024
    A0 = torch.zeros(M, 2, dtype=torch.float32)
    A0[3, 0] = 3.0
    A0[700, 1] = 3.0
    A0 = A0.cuda().T.contiguous().T
    s = psvd.StreamingSVD(M, 1, 2, 1.0, psvd.PSVD_PREC_FP32)
    s.initialize(A0)
    U, D = s.modes(), s.singular_values()
    Ub = torch.ones_like(U)
    Db = torch.ones_like(D)
    Abar = torch.empty(2, M, dtype=torch.float32, device="cuda").T
    rc = psvd.psvd_update_adjoint(s.h, None, None, A0, U, D, Ub, Db, None, None, Abar)
    assert rc == psvd.PSVD_WARN_DEGENERATE
    s.close()
