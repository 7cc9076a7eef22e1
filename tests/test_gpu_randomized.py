"""Parity of the randomized front end (Sec. 3.3) with the FP64 oracle, via the C-ABI.

Both sides draw the same Philox Gaussian test matrix for batch t (stream t of the
seed), so they compute the same randomized approximation; the tolerances are the
ones of the exact path (see test_gpu_fp32 and test_gpu_tc), with one difference
below 1e-2 sigma_1: a Gaussian sketch column mixes all n = K + B coordinates of the
panel, so the Gram's resolution (1e-9 lambda_1 per coordinate) enters the range
finder n-fold and the resolution floor is taken at n * 1e-9.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_08845_gb300 import psvd, synthetic
from tests.test_gpu_fp32 import U32, _batches, _compare, _gpu_run

pytestmark = pytest.mark.gpu

U17 = 2.0 ** -17


def _f32(bs):
    return [synthetic.to_storage(b, torch.float32) for b in bs]


def _gpu_rsvd(batches, K, ff, p, q, seed, precision=psvd.PSVD_PREC_FP32):
    M = batches[0].shape[0]
    maxB = max(b.shape[1] for b in batches)
    s = psvd.StreamingSVD(M, K, maxB, ff, precision, low_rank=1, oversample=p, power_iters=q,
                          seed=seed)
    try:
        codes = [s.initialize(batches[0].cuda())]
        for b in batches[1:]:
            codes.append(s.incorporate_data(b.cuda()))
        U = s.modes().cpu().double().numpy()
        D = s.singular_values().cpu().numpy()
    finally:
        s.close()
    return U, D, codes


def _oracle_rsvd(batches, K, ff, p, q, seed):
    return oracle.rsvd_run([b.double().numpy() for b in batches], K, ff, p, q, seed)


def test_randomized_travelling_waves_64_modes():
    # travelling-wave recipe (64 modes, amplitudes j^-1.5, noise 1e-3,
    # K = 32, B = 64, ff = 0.95, p = 10, q = 1) on a 128 x 128 grid
    gen = synthetic.TravellingWaves(128, 128, 64, 1.5, 1e-3, seed=1235)
    bs = _f32([gen.batch(i, 64) for i in range(4)])
    U, D, codes = _gpu_rsvd(bs, 32, 0.95, 10, 1, seed=42)
    assert all(c >= 0 for c in codes)
    Uo, Do = _oracle_rsvd(bs, 32, 0.95, 10, 1, seed=42)
    _compare(U, D, Uo, Do, gram_res=96e-9)


@pytest.mark.parametrize("M,K,B,nb,ff,p,q", [
    (5001, 10, 25, 4, 1.0, 5, 0),    # ragged rows, no power iteration
    (3001, 40, 25, 3, 0.95, 8, 2),   # l = n at the first batch, modes grow 25 -> 40
    (8192, 16, 48, 4, 0.9, 0, 1),    # no oversampling
])
def test_randomized_shapes(M, K, B, nb, ff, p, q):
    s = [10.0 ** (-i / 24.0) for i in range(48)]
    A, _, _, _ = synthetic.low_rank(M, B * nb, 48, 1e-7, seed=M + K, s=s)
    bs = _f32(_batches(A, B))
    U, D, _ = _gpu_rsvd(bs, K, ff, p, q, seed=7)
    Uo, Do = _oracle_rsvd(bs, K, ff, p, q, seed=7)
    _compare(U, D, Uo, Do, gram_res=(K + B) * 1e-9)


def test_randomized_sketch_wider_than_rank():
    # exact rank 12 < l = 26: the range finder keeps the 12 directions of the data.  The
    # oracle (FP64 Householder on the panel) puts sigma_13.. at the rounding level of the
    # FP32 data; the library's Gram-based range finder resolves singular values only
    # down to its resolution, lambda = 4 n 1e-9 lambda_1 (the Gram's 1e-9 per coordinate,
    # mixed over the n = K + B = 48 coordinates of each sketch column), i.e. sigma =
    # 2 sqrt(n 1e-9) sigma_1.  Below it the two must agree to that resolution; above it
    # to the FP32 bars.
    A, _, _, _ = synthetic.low_rank(4000, 96, 12, 0.0, seed=3,
                                    s=[0.7 ** i for i in range(12)])
    bs = _f32(_batches(A, 32))
    U, D, codes = _gpu_rsvd(bs, 16, 0.95, 10, 1, seed=1)
    assert all(c in (psvd.PSVD_OK, psvd.PSVD_WARN_RANK_DEFICIENT) for c in codes)
    Uo, Do = _oracle_rsvd(bs, 16, 0.95, 10, 1, seed=1)
    res = 2.0 * np.sqrt(48 * 1e-9) * Do[0]
    assert np.all(Do[12:] <= res)
    assert np.all(np.abs(D[12:] - Do[12:]) <= res), (D[12:] / Do[0], Do[12:] / Do[0])
    e = np.abs(D[:12] - Do[:12]) / Do[:12]
    assert e.max() <= 1e-5, f"sigma rel err {e.max():.3e}"
    from tests.helpers import max_principal_angle
    ang = max_principal_angle(U[:, :12], Uo[:, :12])
    assert ang <= 1e-4, f"subspace angle {ang:.3e}"


def test_randomized_full_sketch_equals_exact_path():
    # p >= B makes l = n at every batch: the randomized update is the exact one
    gen = synthetic.TravellingWaves(64, 96, 48, 1.5, 1e-3, seed=5)
    bs = _f32([gen.batch(i, 32) for i in range(4)])
    Ur, Dr, _ = _gpu_rsvd(bs, 16, 0.95, 32, 0, seed=9)
    Ue, De, _ = _gpu_run(bs, 16, 0.95)
    _compare(Ur, Dr, Ue, De, gram_res=49e-9)  # both sides carry the Gram's noise


def test_randomized_deterministic_and_seeded():
    gen = synthetic.TravellingWaves(64, 64, 48, 1.2, 1e-2, seed=6)
    bs = _f32([gen.batch(i, 32) for i in range(3)])
    U1, D1, _ = _gpu_rsvd(bs, 24, 0.95, 4, 0, seed=11)
    U2, D2, _ = _gpu_rsvd(bs, 24, 0.95, 4, 0, seed=11)
    U3, D3, _ = _gpu_rsvd(bs, 24, 0.95, 4, 0, seed=12)
    assert np.array_equal(U1, U2) and np.array_equal(D1, D2)
    assert not np.array_equal(D1, D3)  # another sketch, another approximation


def test_randomized_tensor_core_256_mode_waves():
    # travelling-wave recipe (256 modes, j^-1.2, noise 1e-4, K = 64, B = 128, BF16) with
    # the range finder (p = 10, q = 1) on a 125 x 256 grid
    gen = synthetic.TravellingWaves(125, 256, 256, 1.2, 1e-4, seed=1236)
    bs = [synthetic.to_storage(gen.batch(i, 128), torch.bfloat16) for i in range(3)]
    U, D, _ = _gpu_rsvd(bs, 64, 0.95, 10, 1, seed=5, precision=psvd.PSVD_PREC_BF16_TC)
    Uo, Do = _oracle_rsvd(bs, 64, 0.95, 10, 1, seed=5)
    _compare(U, D, Uo, Do, sig_tol=1e-4, ang_tol=1e-3, unit=U17, gram_res=192e-9)


@pytest.mark.parametrize("p,q", [(-1, 0), (10, -1), (10, 17)])
def test_randomized_bad_config(p, q):
    with pytest.raises(psvd.PsvdError) as ei:
        psvd.psvd_create(4096, 8, 16, 1.0, psvd.PSVD_PREC_FP32, 1, p, q, 0)
    assert ei.value.status == psvd.PSVD_ERR_INVALID_ARG


def test_randomized_tensor_core_batches_lookahead():
    # psvd_incorporate_batches on a randomized tensor-core handle with resident
    # batches (K = 64, so the A^T A look-ahead runs): the same sketches as the
    # oracle's, the H of each step assembled from the split Gram and the look-ahead
    gen = synthetic.TravellingWaves(128, 256, 256, 1.2, 1e-4, seed=1238)
    bs = [synthetic.to_storage(gen.batch(i, 96), torch.bfloat16) for i in range(4)]
    M = bs[0].shape[0]
    s = psvd.StreamingSVD(M, 64, 96, 0.95, psvd.PSVD_PREC_BF16_TC, low_rank=1, oversample=10,
                          power_iters=1, seed=7)
    try:
        s.initialize(bs[0].cuda())
        s.incorporate_batches([b.cuda() for b in bs[1:]])
        U = s.modes().cpu().double().numpy()
        D = s.singular_values().cpu().numpy()
        assert psvd.psvd_last_info(s.h)[0] >= 0
    finally:
        s.close()
    Uo, Do = _oracle_rsvd(bs, 64, 0.95, 10, 1, seed=7)
    _compare(U, D, Uo, Do, sig_tol=1e-4, ang_tol=1e-3, unit=U17, gram_res=160e-9)
