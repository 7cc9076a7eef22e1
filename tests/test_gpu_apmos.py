"""Parity of psvd_parallel_svd (Algorithm 2, APMOS) with the FP64 oracle, via the C-ABI.

Row blocks of uneven sizes stand in for the paper's ranks.  Tolerances are the
FP32 ones of the streaming path (see test_gpu_fp32): 1e-5 relative on the
singular values and 1e-4 rad on the leading subspace, flat, widened by the FP32
representation floor u32 * sigma_1 / sigma_i only for sigma_i below 1e-2 sigma_1.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_08845_gb300 import psvd, synthetic
from tests.helpers import max_principal_angle

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _offsets(sizes):
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def _gpu_apmos(A, offsets, r1, r2, device="cuda"):
    Mtot, N = A.shape
    h = psvd.psvd_create(int(Mtot), 8, 8, 1.0)
    try:
        if device == "cuda":
            Ad = A.cuda()
            U = torch.zeros((r2, Mtot), dtype=torch.float32, device="cuda").T
            L = torch.zeros(r2, dtype=torch.float64, device="cuda")
        else:
            Ad = A
            U = np.zeros((Mtot, r2), dtype=np.float32, order="F")
            L = np.zeros(r2)
        rc = psvd.psvd_parallel_svd(h, Ad, offsets, r1, r2, U, L)
    finally:
        psvd.psvd_destroy(h)
    if device == "cuda":
        U, L = U.cpu().double().numpy(), L.cpu().numpy()
    return np.asarray(U, dtype=np.float64), np.asarray(L), rc


def _compare(U, L, Uo, Lo, k=None):
    # flat bars; the FP32 representation floor only where sigma_i (or the gap) is
    # below 1e-2 sigma_1
    tol = 1e-5 + np.where(Lo < 1e-2 * Lo[0], 8 * U32 * Lo[0] / Lo, 0.0)
    e = np.abs(L - Lo) / Lo
    assert np.all(e <= tol), f"L rel err {e.max():.3e}"
    k = k or len(Lo)
    # columns are A x_j / L_j: compare the spans of the leading k after normalising
    Un = U[:, :k] / np.linalg.norm(U[:, :k], axis=0)
    Uon = Uo[:, :k] / np.linalg.norm(Uo[:, :k], axis=0)
    gap = Lo[k - 1] - Lo[k] if k < len(Lo) else Lo[k - 1]
    ang = max_principal_angle(Un, Uon)
    atol = 1e-4 + (8 * U32 * Lo[0] / gap if gap < 1e-2 * Lo[0] else 0.0)
    assert ang <= atol, f"subspace angle {ang:.3e} > {atol:.3e}"
    return e.max(), ang


def test_apmos_uneven_partitions():
    # uneven row blocks (the paper's ranks), scaled down: 6 blocks of 2,000-9,000 rows, 64 snapshots,
    # r1 = r2 = 20.  The spectrum (s_i = 0.85^i, 60 modes, noise 1e-5) puts the
    # local truncation at sigma_20 / sigma_1 ~ 0.04, inside what a Gram-based
    # local SVD of FP32 data resolves (the travelling-wave recipe has only ~15
    # significant modes in 64 snapshots, so r1 = 20 would cut its noise floor)
    rng = np.random.default_rng(1237)
    sizes = rng.integers(2000, 9001, size=6)
    A64, _, _, _ = synthetic.low_rank(int(sizes.sum()), 64, 60, 1e-5, seed=1237,
                                      s=[0.85 ** i for i in range(60)])
    A = synthetic.to_storage(A64, torch.float32)
    off = _offsets(sizes)
    U, L, rc = _gpu_apmos(A, off, 20, 20)
    assert rc == psvd.PSVD_OK
    Uo, Lo = oracle.apmos(A.double().numpy(), off, 20, 20)
    _compare(U, L, Uo, Lo, k=16)


def test_apmos_exact_when_r1_covers_local_rank():
    # rank-10 data: r1 = 12 >= every block's rank, so W W^T = A^T A and the
    # result is the SVD of A (Alg. 2 is exact here)
    s = [0.8 ** i for i in range(10)]
    A64, _, _, _ = synthetic.low_rank(9000, 40, 10, 0.0, seed=5, s=s)
    A = synthetic.to_storage(A64, torch.float32)
    off = _offsets([2000, 3500, 3500])
    U, L, rc = _gpu_apmos(A, off, 12, 10)
    Ad = A.double().numpy()
    Us, ss, _ = np.linalg.svd(Ad, full_matrices=False)
    e = np.abs(L - ss[:10]) / ss[:10]
    assert e.max() <= 1e-5 + 8 * U32 * ss[0] / ss[9], f"L vs svd {e.max():.3e}"
    Un = U / np.linalg.norm(U, axis=0)
    assert max_principal_angle(Un, Us[:, :10]) <= 1e-4


def test_apmos_single_block_is_the_serial_svd():
    A64, _, _, _ = synthetic.low_rank(5000, 48, 48, 1e-6, seed=9,
                                      s=[10.0 ** (-i / 24.0) for i in range(48)])
    A = synthetic.to_storage(A64, torch.float32)
    U, L, _ = _gpu_apmos(A, _offsets([5000]), 48, 16)
    Ad = A.double().numpy()
    Us, ss, _ = np.linalg.svd(Ad, full_matrices=False)
    _compare(U, L, Us[:, :16] * ss[:16], ss[:16], k=12)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_apmos_host_buffers_and_bf16(dtype):
    rng = np.random.default_rng(3)
    sizes = rng.integers(300, 900, size=5)
    A64, _, _, _ = synthetic.low_rank(int(sizes.sum()), 32, 20, 1e-4, seed=3,
                                      s=[0.85 ** i for i in range(20)])
    A = synthetic.to_storage(A64, dtype)
    off = _offsets(sizes)
    Ug, Lg, _ = _gpu_apmos(A, off, 10, 8, device="cuda")
    # host input and host outputs: staged through device buffers, same result
    Uh, Lh, _ = _gpu_apmos(A, off, 10, 8, device="cpu")
    assert np.array_equal(Ug, Uh) and np.array_equal(Lg, Lh)
    Uo, Lo = oracle.apmos(A.double().numpy(), off, 10, 8)
    _compare(Ug, Lg, Uo, Lo, k=6)


@pytest.mark.parametrize("sizes,r1,r2,status", [
    ([100, 20], 8, 8, psvd.PSVD_ERR_SHAPE),     # a block shorter than N = 32
    ([200, 200], 4, 9, psvd.PSVD_ERR_SHAPE),    # r2 > r1 * nparts
    ([200, 200], 40, 8, psvd.PSVD_ERR_SHAPE),   # r1 > N
])
def test_apmos_argument_errors(sizes, r1, r2, status):
    A = torch.zeros((sum(sizes), 32), dtype=torch.float32).T.contiguous().T.cuda()
    with pytest.raises(psvd.PsvdError) as ei:
        _gpu_apmos(A, _offsets(sizes), r1, r2)
    assert ei.value.status == status


def test_apmos_many_partitions_concurrent_lanes():
    # 40 uneven row blocks: more blocks than concurrent lanes, so every lane takes
    # several; the result must not depend on the lanes' timing (fixed-order gather)
    rng = np.random.default_rng(4242)
    sizes = rng.integers(1000, 4001, size=40)
    A64, _, _, _ = synthetic.low_rank(int(sizes.sum()), 48, 40, 1e-5, seed=4242,
                                      s=[0.85 ** i for i in range(40)])
    A = synthetic.to_storage(A64, torch.float32)
    off = _offsets(sizes)
    U1, L1, rc = _gpu_apmos(A, off, 16, 12)
    U2, L2, _ = _gpu_apmos(A, off, 16, 12)
    assert rc in (psvd.PSVD_OK, psvd.PSVD_WARN_RANK_DEFICIENT)
    assert np.array_equal(U1, U2) and np.array_equal(L1, L2)
    Uo, Lo = oracle.apmos(A.double().numpy(), off, 16, 12)
    _compare(U1, L1, Uo, Lo, k=10)


@pytest.mark.parametrize("p,q", [(6, 0), (2, 1)])
def test_apmos_low_rank_svd_of_w_matches_oracle(p, q):
    # the paper's literal placement: low_rank_svd on the gathered W (Listing 3 with
    # low_rank set).  8 uneven blocks, N = 48 snapshots of a full-rank 1.15^-i
    # spectrum, r1 = 10 (W is 48 x 80 of rank 48), r2 = 10 with a 16- or 12-column
    # sketch (q = 0: a genuine approximation, 3.7e-4 from the exact APMOS; q = 1: the
    # power step), compared with the oracle run on the same Philox sketch and the
    # same sign convention for the local factors
    sizes = synthetic.partition_sizes(8, 2000, 6000, seed=1241)
    off = _offsets(sizes)
    N, r1, r2, seed = 48, 10, 10, 99
    A, *_ = synthetic.spectrum(int(off[-1]), N, [1.15 ** -i for i in range(N)], 1242)
    A = synthetic.to_storage(A, torch.float32)
    Mtot = int(off[-1])
    h = psvd.psvd_create(Mtot, 8, 8, 1.0, psvd.PSVD_PREC_FP32, low_rank=1, oversample=p,
                         power_iters=q, seed=seed)
    U = torch.zeros((r2, Mtot), dtype=torch.float32, device="cuda").T
    L = torch.zeros(r2, dtype=torch.float64, device="cuda")
    rc = psvd.psvd_parallel_svd(h, A.cuda(), off, r1, r2, U, L)
    psvd.psvd_destroy(h)
    assert rc == psvd.PSVD_OK
    Uo, Lo = oracle.apmos_low_rank(A.double().numpy(), off, r1, r2, p, q, seed)
    _compare(U.cpu().double().numpy(), L.cpu().numpy(), Uo, Lo, k=6)
    if q == 0:
        # an approximation: the exact APMOS differs beyond rounding
        Le = oracle.apmos(A.double().numpy(), off, r1, r2)[1]
        assert np.abs(Lo / Le - 1).max() > 1e-5


def test_apmos_batching_workload_64_partitions():
    # the batching workload at its full size: 64 row partitions of uniformly drawn
    # 16,384 - 262,144 rows (about 8.7 M rows in all), N = 64 snapshots, r1 = r2 = 20.
    # A graded spectrum s_i = 0.85^i over 60 modes plus 1e-5 noise puts every local
    # truncation at sigma_20 / sigma_1 ~ 0.04 (see test_apmos_uneven_partitions)
    sizes = synthetic.partition_sizes(64, 16384, 262144, seed=1239)
    off = _offsets(sizes)
    Mtot = int(off[-1])
    A64, _, _, _ = synthetic.low_rank(Mtot, 64, 60, 1e-5, seed=1239,
                                      s=[0.85 ** i for i in range(60)])
    A = synthetic.to_storage(A64, torch.float32)
    del A64
    U, L, rc = _gpu_apmos(A, off, 20, 20)
    assert rc == psvd.PSVD_OK
    Uo, Lo = oracle.apmos(A.double().numpy(), off, 20, 20)
    _compare(U, L, Uo, Lo, k=16)
