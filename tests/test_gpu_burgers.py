"""The paper's Burgers validation (Sec. 4.3) on the GPU, through the C-ABI.

16,384 grid points, snapshots of the analytic viscous Burgers solution at
Re = 1000 on t in [0, 2].  The paper compares the first two singular vectors of
a 4-rank parallel SVD with a serial one.  The eigen-solver here takes panels of
at most 192 columns, so the comparison runs two ways: the streaming update
(Algorithm 1, ff = 1) over all 800 snapshots in batches, and APMOS (Algorithm 2)
with 4 row partitions of 4,096 rows on every fifth snapshot.  Both are checked
against the oracle (same algorithm, FP64) and against the serial SVD's modes 1-2.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_08845_gb300 import psvd, synthetic
from tests.test_gpu_fp32 import U32, _compare, _gpu_run, _oracle_run

pytestmark = pytest.mark.gpu

U17 = 2.0 ** -17


@pytest.fixture(scope="module")
def burgers():
    return synthetic.burgers(16384, 800)


def _mode_checks(U, D, Us, ss, sig_tol, ang_tol):
    # modes 1-2 against the serial SVD (sign-free), singular values relative
    for j in range(2):
        u = U[:, j] / np.linalg.norm(U[:, j])
        ang = float(np.arccos(min(1.0, abs(u @ Us[:, j]))))
        assert ang <= ang_tol, f"mode {j + 1}: {ang:.3e} rad"
    e = np.abs(D[:2] - ss[:2]) / ss[:2]
    assert np.all(e <= sig_tol), f"sigma 1-2 rel err {e.max():.3e}"


@pytest.mark.parametrize("precision,dtype,K,B,sig_tol,ang_tol,unit", [
    (psvd.PSVD_PREC_FP32, torch.float32, 40, 80, 1e-5, 1e-4, U32),
    (psvd.PSVD_PREC_BF16_TC, torch.bfloat16, 64, 128, 1e-4, 1e-3, U17),
    (psvd.PSVD_PREC_FP64, torch.float64, 40, 80, 1e-9, 1e-8, 2.0 ** -53),
])
def test_burgers_streaming_matches_serial(burgers, precision, dtype, K, B, sig_tol, ang_tol, unit):
    A = burgers.to(dtype).T.contiguous().T
    bs = [A[:, i:i + B] for i in range(0, 800, B)]  # the last batch is ragged for B = 128
    U, D, _ = _gpu_run(bs, K=K, ff=1.0, precision=precision)
    Uo, Do = _oracle_run(bs, K, 1.0)
    _compare(U, D, Uo, Do, sig_tol=sig_tol, ang_tol=ang_tol, unit=unit,
             floor=64.0 if precision == psvd.PSVD_PREC_FP64 else 8.0)
    Us, ss, _ = np.linalg.svd(A.double().numpy(), full_matrices=False)
    _mode_checks(U, D, Us, ss, sig_tol, ang_tol)


def test_burgers_apmos_four_partitions(burgers):
    S = synthetic.to_storage(burgers[:, ::5], torch.float32)  # 16,384 x 160
    off = np.array([0, 4096, 8192, 12288, 16384], dtype=np.int64)
    h = psvd.psvd_create(16384, 8, 8, 1.0)
    try:
        U = torch.zeros((10, 16384), dtype=torch.float32, device="cuda").T
        L = torch.zeros(10, dtype=torch.float64, device="cuda")
        rc = psvd.psvd_parallel_svd(h, S.cuda(), off, 20, 10, U, L)
    finally:
        psvd.psvd_destroy(h)
    # the last block (x >= 0.75, where u ~ 1e-10) has local modes at the rounding
    # level: Lambda_j ~ 0 is reported as a warning, the global result stands
    assert rc in (psvd.PSVD_OK, psvd.PSVD_WARN_RANK_DEFICIENT)
    U, L = U.cpu().double().numpy(), L.cpu().numpy()
    Sd = S.double().numpy()
    Uo, Lo = oracle.apmos(Sd, off, 20, 10)
    e = np.abs(L - Lo) / Lo
    assert np.all(e <= 1e-5 + 8 * U32 * Lo[0] / Lo), f"L vs oracle {e.max():.3e}"
    Us, ss, _ = np.linalg.svd(Sd, full_matrices=False)
    _mode_checks(U, L, Us, ss, 1e-5, 1e-4)
