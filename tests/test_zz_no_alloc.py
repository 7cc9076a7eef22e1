"""The allocation-free R factor (psvd_parallel_qr_static) against psvd_parallel_qr.

psvd_parallel_qr_static exists for callers that cannot allocate device memory
when they need the factor (device memory reserved by another allocator, or a
loop that must not pay cudaMalloc's implicit synchronisation); it keeps its
scratch in a fixed device array instead.  This file is collected last so that a
failure here leaves every other test already run; it also passes on its own.
"""
import numpy as np
import pytest
import torch

from paper_2108_08845_gb300 import psvd

pytestmark = pytest.mark.gpu

REL_TOL = 1e-9  # both paths reduce a compensated FP32 Gram in FP64; only the chunking differs


def _panel(seed, M, n, dtype):
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(M, n, generator=g, dtype=torch.float64) * torch.logspace(0, -2, n, dtype=torch.float64)
    return A.to(dtype).T.contiguous().T.cuda()


def _reference_R(P):
    M, n = P.shape
    h = psvd.psvd_create(M, 8, n)
    R = torch.zeros((n, n), dtype=torch.float64, device="cuda").T
    psvd.psvd_parallel_qr(h, P, R)
    psvd.psvd_destroy(h)
    return R.cpu().numpy()


def test_static_scratch_matches_allocating_entry_point_twice():
    # two calls in a row on different panels: the second must not see the first's scratch
    for seed, M, n, dtype in [(1, 6001, 40, torch.float32), (2, 20000, 128, torch.bfloat16)]:
        P = _panel(seed, M, n, dtype)
        R_ref = _reference_R(P)
        R = torch.zeros((n, n), dtype=torch.float64, device="cuda").T
        psvd.psvd_parallel_qr_static(P, R)
        err = np.abs(R.cpu().numpy() - R_ref).max() / np.abs(R_ref).max()
        assert err <= REL_TOL, f"n={n}: rel diff {err:.3e}"


def test_static_scratch_rejects_oversize():
    P = _panel(3, 500, 129, torch.float32)
    R = torch.zeros((129, 129), dtype=torch.float64, device="cuda").T
    with pytest.raises(psvd.PsvdError) as e:
        psvd.psvd_parallel_qr_static(P, R)
    assert e.value.status == psvd.PSVD_ERR_SHAPE
