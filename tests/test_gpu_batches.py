"""psvd_incorporate_batches: several batches in one call, host batches copied on a
copy stream while the previous batch is processed.  The result must be the one of
the single calls, bit for bit (the same kernels on the same values), for host
batches on both paths and device batches on the FP32 path, and each batch's
singular values must land in s_out.  Device batches on the tensor-core path take the
A^T A look-ahead (the next batch's A^T A block summed during the small solve, the
other blocks by the two-CTA Gram): a different summation order of the same Gram, so
those results are compared with the single calls and the oracle at the path's bars."""
import numpy as np
import pytest
import torch

from paper_2108_08845_gb300 import psvd, synthetic
from tests.test_gpu_fp32 import _compare, _oracle_run_gap

pytestmark = pytest.mark.gpu


def _run_single(bs, K, ff, prec):
    s = psvd.StreamingSVD(bs[0].shape[0], K, bs[0].shape[1], ff, prec)
    sig = []
    try:
        s.initialize(bs[0].cuda())
        for b in bs[1:]:
            s.incorporate_data(b.cuda())
            sig.append(s.singular_values().cpu().numpy())
        return s.modes().cpu().numpy(), s.singular_values().cpu().numpy(), sig
    finally:
        s.close()


def _run_batched(bs, K, ff, prec, host):
    M, B = bs[0].shape
    s = psvd.StreamingSVD(M, K, B, ff, prec)
    try:
        s.initialize(bs[0].cuda())
        rest = [b.pin_memory() if host else b.cuda() for b in bs[1:]]
        s_out = torch.zeros((len(rest), K), dtype=torch.float64).pin_memory()
        s.incorporate_batches(rest, s_out)
        U, D = s.modes().cpu().numpy(), s.singular_values().cpu().numpy()
        return U, D, s_out.numpy()
    finally:
        s.close()


@pytest.mark.parametrize("prec,dt", [(psvd.PSVD_PREC_FP32, torch.float32),
                                     (psvd.PSVD_PREC_BF16_TC, torch.bfloat16)])
@pytest.mark.parametrize("host", [True, False])
def test_batches_equal_single_calls(prec, dt, host):
    gen = synthetic.TravellingWaves(96, 128, 64, 1.5, 1e-3, seed=71)
    bs = [synthetic.to_storage(gen.batch(i, 48), dt) for i in range(6)]
    U1, D1, sig1 = _run_single(bs, 24, 0.95, prec)
    U2, D2, sig2 = _run_batched(bs, 24, 0.95, prec, host)
    tc = prec == psvd.PSVD_PREC_BF16_TC
    unit = 2.0 ** -17 if tc else 2.0 ** -24
    sig_tol, ang_tol = (1e-4, 1e-3) if tc else (1e-5, 1e-4)
    if tc and not host:
        _compare(U2.astype(np.float64), D2, U1.astype(np.float64), D1, sig_tol=sig_tol,
                 ang_tol=ang_tol, unit=unit, gram_res=2e-9)
        for i, s in enumerate(sig1):
            assert np.allclose(sig2[i, :len(s)], s, rtol=1e-4, atol=0)
    else:
        assert np.array_equal(U1, U2) and np.array_equal(D1, D2)
        for i, s in enumerate(sig1):
            assert np.array_equal(sig2[i, :len(s)], s)
    # and against the oracle
    Uo, Do, s_next = _oracle_run_gap(bs, 24, 0.95)
    _compare(U2.astype(np.float64), D2, Uo, Do, sig_tol=sig_tol, ang_tol=ang_tol, unit=unit,
             s_next=s_next)


def test_batches_reject_mismatched_shapes():
    s = psvd.StreamingSVD(4096, 8, 32, 1.0)
    try:
        a = torch.randn(4096, 32).T.contiguous().T.cuda()
        s.initialize(a)
        with pytest.raises(ValueError):
            psvd.psvd_incorporate_batches(s.h, [a, a[:, :16]])
        with pytest.raises(psvd.PsvdError) as e:
            psvd.psvd_incorporate_batches(s.h, [torch.randn(4096, 40).T.contiguous().T.cuda()])
        assert e.value.status == psvd.PSVD_ERR_SHAPE
    finally:
        s.close()


@pytest.mark.parametrize("ny,nx,B,nb,K", [
    (128, 256, 128, 5, 64),   # K = 64, B = 128: [Uh | Ul] and A one slab each
    (125, 256, 100, 5, 64),   # ragged last row tile, B not a multiple of 16
    (96, 128, 40, 6, 64),     # k grows 40 -> 64: the split starts at the third step
    (96, 128, 100, 4, 57),    # K = 57: mode planes padded to 64 columns
    (64, 128, 8, 12, 60),     # a one-box snapshot slab (B = 8)
])
def test_tensor_core_lookahead_matches_single_calls_and_oracle(ny, nx, B, nb, K):
    gen = synthetic.TravellingWaves(ny, nx, 256, 1.2, 1e-4, seed=ny + B)
    bs = [synthetic.to_storage(gen.batch(i, B), torch.bfloat16) for i in range(nb)]
    TC = psvd.PSVD_PREC_BF16_TC
    U1, D1, sig1 = _run_single(bs, K, 0.95, TC)
    U2, D2, sig2 = _run_batched(bs, K, 0.95, TC, host=False)
    unit = 2.0 ** -17
    _compare(U2.astype(np.float64), D2, U1.astype(np.float64), D1, sig_tol=1e-4, ang_tol=1e-3,
             unit=unit, gram_res=2e-9)
    Uo, Do, s_next = _oracle_run_gap(bs, K, 0.95)
    _compare(U2.astype(np.float64), D2, Uo, Do, sig_tol=1e-4, ang_tol=1e-3, unit=unit,
             s_next=s_next)
    # each batch's singular values: the same as the single calls' at the path's bar
    for i, s in enumerate(sig1):
        assert np.allclose(sig2[i, :len(s)], s, rtol=1e-4, atol=1e-4 * s[0])


def test_mixed_host_and_device_batches():
    # host (pinned and pageable) and device batches in one call: the look-ahead runs
    # only ahead of device batches; every batch still lands as with single calls
    gen = synthetic.TravellingWaves(128, 256, 256, 1.2, 1e-4, seed=77)
    bs = [synthetic.to_storage(gen.batch(i, 128), torch.bfloat16) for i in range(6)]
    TC = psvd.PSVD_PREC_BF16_TC
    U1, D1, _ = _run_single(bs, 64, 0.95, TC)
    M = bs[0].shape[0]
    s = psvd.StreamingSVD(M, 64, 128, 0.95, TC)
    try:
        s.initialize(bs[0].cuda())
        mixed = [bs[1].pin_memory(), bs[2].cuda(), bs[3].clone(), bs[4].cuda(), bs[5].cuda()]
        s_out = torch.zeros((5, 64), dtype=torch.float64).pin_memory()
        s.incorporate_batches(mixed, s_out)
        U2, D2 = s.modes().cpu().numpy(), s.singular_values().cpu().numpy()
    finally:
        s.close()
    unit = 2.0 ** -17
    _compare(U2.astype(np.float64), D2, U1.astype(np.float64), D1, sig_tol=1e-4, ang_tol=1e-3,
             unit=unit, gram_res=2e-9)
    assert np.array_equal(s_out.numpy()[4], D2)
    Uo, Do, s_next = _oracle_run_gap(bs, 64, 0.95)
    _compare(U2.astype(np.float64), D2, Uo, Do, sig_tol=1e-4, ang_tol=1e-3, unit=unit,
             s_next=s_next)


def test_single_batch_and_pageable_numpy_fp32():
    # count = 1, and pageable numpy batches on the FP32 path: bit for bit the single calls
    gen = synthetic.TravellingWaves(64, 128, 64, 1.5, 1e-3, seed=78)
    bs = [synthetic.to_storage(gen.batch(i, 32), torch.float32) for i in range(4)]
    U1, D1, _ = _run_single(bs, 16, 0.9, psvd.PSVD_PREC_FP32)
    s = psvd.StreamingSVD(bs[0].shape[0], 16, 32, 0.9, psvd.PSVD_PREC_FP32)
    try:
        s.initialize(bs[0].cuda())
        s.incorporate_batches([np.asfortranarray(bs[1].numpy())])
        s.incorporate_batches([np.asfortranarray(b.numpy()) for b in bs[2:]])
        U2, D2 = s.modes().cpu().numpy(), s.singular_values().cpu().numpy()
    finally:
        s.close()
    assert np.array_equal(U1, U2) and np.array_equal(D1, D2)
