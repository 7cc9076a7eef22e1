"""``torch.autograd`` interface to Algorithm 1 (Sec. 3.1) with the library's
hand-written adjoint as its backward.

``streaming_svd(batches, K, ff)`` runs the streaming update through the C-ABI
(``psvd_initialize`` on the first batch, ``psvd_incorporate_data`` on the rest, FP32
path) and returns the final modes U (M x k, column-major FP32) and singular values D
(k, FP64).  Its backward sweeps the steps in reverse with ``psvd_update_adjoint``:
each step's cotangents (Ubar, Dbar) become those of the previous step's outputs,
and every batch receives its own gradient.  The tape is the per-step modes and
singular values (M x k FP32 + k FP64 per step); no QR factor is kept.
Marshalling only: every step of the forward and the backward runs in the library.
"""
from __future__ import annotations

import warnings

import torch

from . import psvd as _p


def _colmajor(x: torch.Tensor, dtype) -> torch.Tensor:
    x = x.to(dtype)
    return x if x.dim() == 1 or x.stride(0) == 1 else x.T.contiguous().T


class StreamingSVDFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, K, ff, *batches):
        if not batches:
            raise ValueError("streaming_svd: no batches")
        dev = batches[0].device
        if dev.type != "cuda":
            raise ValueError("streaming_svd: batches must be CUDA tensors")
        M = batches[0].shape[0]
        maxB = max(int(b.shape[1]) for b in batches)
        owner = _p.StreamingSVD(M, K, maxB, ff, _p.PSVD_PREC_FP32)
        Us, Ds = [], []
        for t, A in enumerate(batches):
            if t == 0:
                owner.initialize(A)
            else:
                owner.incorporate_data(A)
            Us.append(owner.modes(dev))
            Ds.append(owner.singular_values(dev))
        ctx.owner = owner
        ctx.Us, ctx.Ds = Us, Ds
        ctx.save_for_backward(*batches)
        return Us[-1].clone(), Ds[-1].clone()

    @staticmethod
    def backward(ctx, gU, gD):
        batches = ctx.saved_tensors
        Us, Ds, h = ctx.Us, ctx.Ds, ctx.owner.h
        M = batches[0].shape[0]
        dev = batches[0].device
        k = Us[-1].shape[1]
        Ub = _colmajor(gU if gU is not None else torch.zeros(M, k, device=dev), torch.float32)
        Db = (gD if gD is not None else torch.zeros(k, device=dev)).to(torch.float64).contiguous()
        grads = [None] * len(batches)
        degenerate = False
        for t in range(len(batches) - 1, -1, -1):
            A = batches[t]
            Abar = torch.empty((A.shape[1], M), dtype=torch.float32, device=dev).T
            if t == 0:
                U = D = Ubp = Dbp = None
            else:
                U, D = Us[t - 1], Ds[t - 1]
                Ubp = torch.empty((U.shape[1], M), dtype=torch.float32, device=dev).T
                Dbp = torch.empty(U.shape[1], dtype=torch.float64, device=dev)
            rc = _p.psvd_update_adjoint(h, U, D, A, Us[t], Ds[t], Ub, Db, Ubp, Dbp, Abar)
            degenerate |= rc == _p.PSVD_WARN_DEGENERATE
            grads[t] = Abar if A.dtype == torch.float32 else Abar.to(A.dtype)
            Ub, Db = Ubp, Dbp
        if degenerate:
            warnings.warn("streaming_svd backward: coincident singular values at a kept index; "
                          "the gradient is undefined there", RuntimeWarning)
        return (None, None, *grads)


def streaming_svd(batches, K: int, ff: float = 1.0):
    """Final (U, D) of Algorithm 1 over `batches` (column-major CUDA tensors, FP32 or
    BF16), differentiable with respect to every batch."""
    return StreamingSVDFunction.apply(int(K), float(ff), *batches)
