"""The allocation-free R factor (psvd_parallel_qr_static), through the C-ABI.

psvd_parallel_qr_static exists for callers that cannot allocate device memory
when they need the factor (device memory reserved by another allocator, or a
loop that must not pay cudaMalloc's implicit synchronisation); it keeps its
scratch in a fixed device array instead.  Its R is checked against the
allocating entry point (same Gram kernels, different row chunking) and against
the oracle's Householder R, on two calls in a row (the second must not see the
first's scratch), on a side stream, and on a panel holding a NaN.  This file is
collected last so that a failure here leaves every other test already run; it
also passes on its own.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_08845_gb300 import psvd

pytestmark = pytest.mark.gpu

REL_TOL = 1e-9     # both paths reduce a compensated FP32 Gram in FP64; only the chunking differs
ORACLE_TOL = 1e-6  # Cholesky of the compensated Gram against Householder, relative to max |R|


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


def _static_R(P, stream=None):
    n = P.shape[1]
    R = torch.zeros((n, n), dtype=torch.float64, device="cuda").T
    psvd.psvd_parallel_qr_static(P, R, stream)
    if stream is not None:
        stream.synchronize()
    return R.cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_static_scratch_matches_allocating_entry_point_and_oracle_twice():
    # two calls in a row on different panels: the second must not see the first's scratch
    for seed, M, n, dtype in [(1, 6001, 40, torch.float32), (2, 20000, 128, torch.bfloat16)]:
        P = _panel(seed, M, n, dtype)
        R = _static_R(P)
        err = _rel(R, _reference_R(P))
        assert err <= REL_TOL, f"n={n}: rel diff to psvd_parallel_qr {err:.3e}"
        _, Ro = oracle.householder_qr(P.cpu().double().numpy())
        err_o = _rel(R, Ro)
        assert err_o <= ORACLE_TOL, f"n={n}: rel diff to the oracle's Householder R {err_o:.3e}"


def test_static_scratch_on_a_side_stream():
    P = _panel(4, 9000, 96, torch.float32)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        R = _static_R(P, stream=s)
    _, Ro = oracle.householder_qr(P.cpu().double().numpy())
    assert _rel(R, Ro) <= ORACLE_TOL


def test_static_scratch_nan_panel_then_clean_panel():
    P = _panel(5, 3000, 32, torch.float32)
    bad = P.clone()
    bad[17, 5] = float("nan")
    R = torch.zeros((32, 32), dtype=torch.float64, device="cuda").T
    with pytest.raises(psvd.PsvdError) as e:
        psvd.psvd_parallel_qr_static(bad, R)
    assert e.value.status == psvd.PSVD_ERR_NONFINITE
    # the status word is cleared by the next call
    Rc = _static_R(P)
    _, Ro = oracle.householder_qr(P.cpu().double().numpy())
    assert _rel(Rc, Ro) <= ORACLE_TOL


def test_static_scratch_rejects_oversize_and_host_panels():
    P = _panel(3, 500, 129, torch.float32)
    R = torch.zeros((129, 129), dtype=torch.float64, device="cuda").T
    with pytest.raises(psvd.PsvdError) as e:
        psvd.psvd_parallel_qr_static(P, R)
    assert e.value.status == psvd.PSVD_ERR_SHAPE
    Ph = _panel(3, 500, 16, torch.float32).cpu().T.contiguous().T
    R = torch.zeros((16, 16), dtype=torch.float64, device="cuda").T
    with pytest.raises(psvd.PsvdError) as e:
        psvd.psvd_parallel_qr_static(Ph, R)
    assert e.value.status == psvd.PSVD_ERR_INVALID_ARG
