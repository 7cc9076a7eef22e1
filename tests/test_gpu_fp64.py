"""Parity of the FP64 path (PSVD_PREC_FP64) with the FP64 oracle, through the C-ABI.

The FP64 path keeps the modes and the panel passes in FP64; the small solve is
the same scale-level FP32 solve with FP64 refinement as on the other paths.
Its bars are four decades tighter than the FP32 path's: singular values within
1e-9 relative and the kept subspace within 1e-8 rad, widened by the FP64
representation floor u64 * sigma_1 / sigma_i (and / gap for the subspace).
"""
import os
import tempfile

import numpy as np
import pytest
import torch

import oracle
from paper_2108_08845_gb300 import psvd, synthetic
from tests.test_gpu_fp32 import _batches, _compare, _gpu_run, _oracle_run

pytestmark = pytest.mark.gpu

F64 = psvd.PSVD_PREC_FP64
U64 = 2.0 ** -53


def _f64(bs):
    return [b.clone().T.contiguous().T for b in bs]  # float64, column-major


def test_fp64_low_rank():
    # rank-40 data, s_i = 10^(-i/8), noise 1e-8, K = 10, four batches of 25
    A, _, _, _ = synthetic.low_rank(4096, 100, 40, 1e-8, seed=1234)
    bs = _f64(_batches(A, 25))
    U, D, info = _gpu_run(bs, K=10, ff=1.0, precision=F64)
    Uo, Do = _oracle_run(bs, 10, 1.0)
    _compare(U, D, Uo, Do, sig_tol=1e-9, ang_tol=1e-8, unit=U64, floor=64.0)


def test_fp64_travelling_waves_ff():
    # travelling-wave recipe (64 modes, amplitudes j^-1.5, noise 1e-3) on a
    # 64 x 128 grid, K = 32, B = 64, ff = 0.95
    gen = synthetic.TravellingWaves(64, 128, 64, 1.5, 1e-3, seed=1235)
    bs = _f64([gen.batch(i, 64) for i in range(4)])
    U, D, _ = _gpu_run(bs, K=32, ff=0.95, precision=F64)
    Uo, Do = _oracle_run(bs, 32, 0.95)
    _compare(U, D, Uo, Do, sig_tol=1e-9, ang_tol=1e-8, unit=U64, floor=64.0)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_fp64_handle_widens_narrow_inputs(dtype):
    # FP32 / BF16 snapshots are widened exactly: the oracle sees the same values
    A, _, _, _ = synthetic.low_rank(3001, 75, 30, 1e-6, seed=77)
    bs = [synthetic.to_storage(b, dtype) for b in _batches(A, 25)]
    U, D, _ = _gpu_run(bs, K=12, ff=0.9, precision=F64)
    Uo, Do = _oracle_run(bs, 12, 0.9)
    _compare(U, D, Uo, Do, sig_tol=1e-9, ang_tol=1e-8, unit=U64, floor=64.0)


def test_fp64_modes_f32_view_and_host_inputs():
    A, _, _, _ = synthetic.low_rank(2048, 60, 20, 1e-7, seed=5)
    bs = _f64(_batches(A, 20))
    s = psvd.StreamingSVD(2048, 8, 20, 1.0, F64)
    try:
        for i, b in enumerate(bs):  # host (numpy, Fortran order) inputs are staged
            (s.initialize if i == 0 else s.incorporate_data)(np.asfortranarray(b.numpy()))
        U64_ = s.modes().cpu().numpy()
        U32_ = torch.empty((s.num_modes, 2048), dtype=torch.float32, device="cuda").T
        psvd.psvd_get_modes(s.h, U32_)
        assert U64_.dtype == np.float64
        assert np.array_equal(U32_.cpu().numpy(), U64_.astype(np.float32))
    finally:
        s.close()


def test_fp64_save_load_continues_bit_identically():
    A, _, _, _ = synthetic.low_rank(4000, 100, 30, 1e-7, seed=8)
    bs = [b.cuda() for b in _f64(_batches(A, 25))]
    ref = psvd.StreamingSVD(4000, 10, 25, 0.95, F64)
    s = psvd.StreamingSVD(4000, 10, 25, 0.95, F64)
    try:
        for h in (ref, s):
            h.initialize(bs[0])
            h.incorporate_data(bs[1])
        with tempfile.TemporaryDirectory() as d:
            path = os.path.join(d, "h.psvd")
            psvd.psvd_save(s.h, path)
            s.close()
            s = psvd.StreamingSVD.__new__(psvd.StreamingSVD)
            s.M, s.K, s.precision = 4000, 10, F64
            s.h = psvd.psvd_load(path)
        for h in (ref, s):
            for b in bs[2:]:
                h.incorporate_data(b)
        assert torch.equal(ref.modes(), s.modes())
        assert torch.equal(ref.singular_values(), s.singular_values())
    finally:
        ref.close()
        s.close()


def test_fp64_parallel_qr():
    A, _, _, _ = synthetic.low_rank(5000, 48, 48, 1e-6, seed=21)
    P = A.clone().T.contiguous().T.cuda()
    h = psvd.psvd_create(5000, 48, 48, 1.0, F64)
    try:
        R = torch.zeros((48, 48), dtype=torch.float64, device="cuda").T
        psvd.psvd_parallel_qr(h, P, R)
    finally:
        psvd.psvd_destroy(h)
    Rn = np.linalg.cholesky(A.numpy().T @ A.numpy()).T
    R = R.cpu().numpy()
    assert np.max(np.abs(R - Rn)) <= 1e-10 * np.max(np.abs(Rn))


def test_fp64_errors():
    with pytest.raises(psvd.PsvdError) as ei:
        psvd.psvd_create(4096, 8, 16, 1.0, F64, 1, 10, 0, 0)  # no randomized front end
    assert ei.value.status == psvd.PSVD_ERR_UNSUPPORTED
    A = torch.zeros((4096, 16), dtype=torch.float64).T.contiguous().T.cuda()
    h = psvd.psvd_create(4096, 8, 16, 1.0, psvd.PSVD_PREC_FP32)
    try:
        with pytest.raises(psvd.PsvdError) as ei:  # FP64 snapshots need an FP64 handle
            psvd.psvd_initialize(h, A)
        assert ei.value.status == psvd.PSVD_ERR_UNSUPPORTED
        U = torch.zeros((8, 4096), dtype=torch.float64, device="cuda").T
        with pytest.raises(psvd.PsvdError) as ei:
            psvd.psvd_get_modes_f64(h, U)
        assert ei.value.status == psvd.PSVD_ERR_UNSUPPORTED
    finally:
        psvd.psvd_destroy(h)
