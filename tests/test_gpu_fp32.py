"""Parity of the FP32 CUDA path with the FP64 oracle, through the C-ABI.

Tolerances for the FP32 path: singular values within 1e-5 relative and the kept
mode subspace within 1e-4 rad (largest principal angle), on the same seeded
inputs (float32 bits widened exactly to float64 for the oracle).

The bars are flat for every mode with sigma_i >= 1e-2 sigma_1.  Below that two
floors of the method are added to the singular-value bar, each derived, not
fitted: FP32-stored modes perturb the panel by ~u32 sigma_1, which moves sigma_i
by a relative ~u32 sigma_1 / sigma_i (8 u32 sigma_1 / sigma_i); and a Gram-based
factorisation resolves eigenvalues of the Gram to ~1e-9 lambda_1 (the library's
stated resolution), which moves sigma_i by a relative 1e-9 sigma_1^2 / (2 sigma_i^2)
(taken 4x).  The subspace bar is flat, over the largest leading k <= K (k = K
when the oracle's last panel gives sigma_K+1) that the oracle separates from the
rest by a relative gap of 1 % and whose eigenvalue gap lambda_k - lambda_k+1
resolves that bar at the Gram's resolution (4e-9 lambda_1 / gap <= the bar).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_08845_gb300 import psvd, synthetic
from tests.helpers import max_principal_angle, rel_err

pytestmark = pytest.mark.gpu

SIG_TOL = 1e-5
ANG_TOL = 1e-4
U32 = 2.0 ** -24
U64 = 2.0 ** -53
REL_GAP = 1e-2      # a leading subspace is compared when sigma_k - sigma_k+1 >= REL_GAP sigma_k
FLOOR_BELOW = 1e-2  # the method's floors apply to sigma_i < FLOOR_BELOW sigma_1
GRAM_RES = 1e-9     # resolution of the FP32 and tensor-core Grams, relative to lambda_1


def _batches(A, B):
    return [A[:, i:i + B] for i in range(0, A.shape[1], B)]


def _gpu_run(batches, K, ff, precision=psvd.PSVD_PREC_FP32, device="cuda"):
    M = batches[0].shape[0]
    maxB = max(b.shape[1] for b in batches)
    s = psvd.StreamingSVD(M, K, maxB, ff, precision)
    try:
        s.initialize(batches[0].to(device))
        for b in batches[1:]:
            s.incorporate_data(b.to(device))
        U = s.modes().cpu().double().numpy()
        D = s.singular_values().cpu().numpy()
        _, info = psvd.psvd_last_info(s.h)
    finally:
        s.close()
    return U, D, info


def _oracle_run(batches, K, ff):
    return oracle.stream_run([b.double().numpy() for b in batches], K, ff)


def _oracle_run_gap(batches, K, ff):
    """The oracle's (U, D) and sigma_K+1, the largest singular value its last step
    dropped (of the panel [ff U D | A_last], or of A_0 with one batch; 0 if none)."""
    bs = [b.double().numpy() for b in batches]
    if len(bs) == 1:
        s_all = np.linalg.svd(bs[0], compute_uv=False)
        U, D = oracle.stream_initialize(bs[0], K)
    else:
        U, D = oracle.stream_run(bs[:-1], K, ff)
        s_all = np.linalg.svd(oracle.panel(U, D, bs[-1], ff), compute_uv=False)
        U, D = oracle.stream_update(U, D, bs[-1], ff, K)
    k = len(D)
    return U, D, (float(s_all[k]) if len(s_all) > k else 0.0)


def subspace_dim(Do, s_next=None, ang_tol=ANG_TOL, gram_res=GRAM_RES, rel_gap=REL_GAP):
    """Largest k <= K whose leading-k subspace is separated from the rest by a
    relative gap (sigma_k - sigma_k+1 >= rel_gap sigma_k) that the Gram's resolution
    resolves at the angle bar (4 gram_res sigma_1^2 / (sigma_k^2 - sigma_k+1^2) <=
    ang_tol); sigma_K+1 = s_next (None: unknown, so k = K is not taken)."""
    s = list(Do) + ([s_next] if s_next is not None else [])
    for k in range(len(Do), 0, -1):
        if k >= len(s):
            continue
        gap, lgap = s[k - 1] - s[k], s[k - 1] ** 2 - s[k] ** 2
        if gap >= rel_gap * s[k - 1] and 4.0 * gram_res * s[0] ** 2 <= ang_tol * lgap:
            return k
    return 1


def _compare(U, D, Uo, Do, sig_tol=SIG_TOL, ang_tol=ANG_TOL, unit=U32, floor=8.0, s_next=None,
             gram_res=None):
    """unit: rounding unit of the stored modes (u32 FP32, 2^-17 BF16 hi/lo pair, u64 FP64);
    the storage floor applies to FP32 and FP64 storage.  gram_res: the Gram's resolution
    relative to lambda_1 (1e-9 for the FP32 and tensor-core Grams, 1e-13 for FP64)."""
    assert U.shape == Uo.shape and D.shape == Do.shape
    if gram_res is None:
        gram_res = 1e-13 if unit == U64 else GRAM_RES
    tol = np.full(len(Do), sig_tol)
    low = Do < FLOOR_BELOW * Do[0]
    tol[low] += 4.0 * gram_res * Do[0] ** 2 / (2.0 * Do[low] ** 2)
    if unit in (U32, U64):
        tol[low] += floor * unit * Do[0] / Do[low]
    e = rel_err(D, Do)
    assert np.all(e <= tol), f"sigma rel err {e.max():.3e} (worst ratio {np.max(e / tol):.2f})"
    k = subspace_dim(Do, s_next, ang_tol, gram_res)
    e_ang = max_principal_angle(U[:, :k], Uo[:, :k])
    assert e_ang <= ang_tol, f"subspace angle {e_ang:.3e} > {ang_tol:.3e} (k={k} of {len(Do)})"
    # U_new = P V / sigma in finite precision: column i is orthonormal to ~u*sigma_1/sigma_i
    cond = Do[0] / np.minimum.outer(Do, Do)
    orth = np.abs(U.T @ U - np.eye(U.shape[1]))
    assert np.all(orth <= 1e-4 + floor * unit * cond), f"orthonormality {orth.max():.3e}"
    return e.max(), e_ang


def test_low_rank_fp32():
    # M=4096, K=10, 4 batches of B=25, ff=1, rank-40 data, s_i = 10^(-i/8), noise 1e-8
    A, _, _, _ = synthetic.low_rank(4096, 100, 40, 1e-8, seed=1234)
    bs = [synthetic.to_storage(b, torch.float32) for b in _batches(A, 25)]
    U, D, info = _gpu_run(bs, K=10, ff=1.0)
    Uo, Do, s_next = _oracle_run_gap(bs, 10, 1.0)
    _compare(U, D, Uo, Do, s_next=s_next)


@pytest.mark.parametrize("M,K,B,nb,ff", [
    (4099, 10, 25, 4, 1.0),    # ragged tail in every tile
    (3001, 40, 25, 3, 1.0),    # K > B at initialisation: the mode count grows
    (10000, 16, 48, 5, 0.95),  # forget factor
    (2048, 33, 31, 4, 0.9),    # odd n = K + B
])
def test_low_rank_shapes_fp32(M, K, B, nb, ff):
    # rank-48 data with s_i = 10^(-i/24): every kept mode has sigma/sigma_1 >= 0.02.
    # Storing the modes in FP32 perturbs the panel by ~u*sigma_1, a relative error
    # of ~u*sigma_1/sigma_i in sigma_i for any FP32 method, so 1e-5 needs
    # sigma_i/sigma_1 above ~1e-2.
    s = [10.0 ** (-i / 24.0) for i in range(48)]
    A, _, _, _ = synthetic.low_rank(M, B * nb, 48, 1e-7, seed=M + K, s=s)
    bs = [synthetic.to_storage(b, torch.float32) for b in _batches(A, B)]
    U, D, _ = _gpu_run(bs, K=K, ff=ff)
    Uo, Do, s_next = _oracle_run_gap(bs, K, ff)
    _compare(U, D, Uo, Do, s_next=s_next)


def test_rank_deficient_modes_are_zeroed_and_flagged():
    # rank-12 data, K = 20: modes 13..20 have sigma at the 1e-9 noise level, far
    # below what the panel Gram resolves; they come back as zero with a warning
    A, _, _, _ = synthetic.low_rank(3000, 60, 12, 1e-9, seed=21)
    bs = [synthetic.to_storage(b, torch.float32) for b in _batches(A, 30)]
    U, D, info = _gpu_run(bs, K=20, ff=1.0)
    Uo, Do = _oracle_run(bs, 20, 1.0)
    assert info[2] & 1  # PSVD_WARN_RANK_DEFICIENT
    assert np.all(D[12:] == 0) and np.all(U[:, 12:] == 0)
    _compare(U[:, :12], D[:12], Uo[:, :12], Do[:12])


def test_travelling_waves_fp32():
    # travelling-wave recipe on a 64 x 64 grid: 64 modes, amplitudes j^-1.5,
    # noise 1e-3, K = 32, B = 64, ff = 0.95
    gen = synthetic.TravellingWaves(64, 64, 64, 1.5, 1e-3, seed=1235)
    bs = [synthetic.to_storage(gen.batch(i, 64), torch.float32) for i in range(4)]
    U, D, _ = _gpu_run(bs, K=32, ff=0.95)
    Uo, Do, s_next = _oracle_run_gap(bs, 32, 0.95)
    _compare(U, D, Uo, Do, s_next=s_next)


def test_bf16_inputs_on_fp32_path():
    A, _, _, _ = synthetic.low_rank(5000, 60, 30, 1e-6, seed=77)
    bs = [synthetic.to_storage(b, torch.bfloat16) for b in _batches(A, 20)]
    U, D, _ = _gpu_run(bs, K=8, ff=1.0)
    Uo, Do, s_next = _oracle_run_gap(bs, 8, 1.0)
    _compare(U, D, Uo, Do, s_next=s_next)


@pytest.mark.parametrize("M", [5000, 3001])
def test_bf16_odd_and_even_leading_dimension(M):
    # BF16 snapshots on the FP32 path: an even leading dimension is read as 4-byte row
    # pairs, an odd one (M = 3001, unpadded) one row at a time; both match the oracle
    A, _, _, _ = synthetic.low_rank(M, 60, 30, 1e-6, seed=M)
    bs = [synthetic.to_storage(b, torch.bfloat16) for b in _batches(A, 20)]
    U, D, _ = _gpu_run(bs, K=8, ff=1.0)
    Uo, Do, s_next = _oracle_run_gap(bs, 8, 1.0)
    _compare(U, D, Uo, Do, s_next=s_next)


def test_host_and_device_inputs_identical():
    A, _, _, _ = synthetic.low_rank(3000, 60, 20, 1e-6, seed=5)
    bs = [synthetic.to_storage(b, torch.float32) for b in _batches(A, 20)]
    Ud, Dd, _ = _gpu_run(bs, K=8, ff=0.95, device="cuda")
    Uh, Dh, _ = _gpu_run(bs, K=8, ff=0.95, device="cpu")
    assert np.array_equal(Ud, Uh) and np.array_equal(Dd, Dh)


def test_save_load_resumes_bit_identically(tmp_path):
    A, _, _, _ = synthetic.low_rank(2500, 100, 30, 1e-6, seed=6)
    bs = [synthetic.to_storage(b, torch.float32).cuda() for b in _batches(A, 20)]
    s = psvd.StreamingSVD(2500, 8, 20, 0.95)
    s.initialize(bs[0])
    s.incorporate_data(bs[1])
    path = str(tmp_path / "state.psvd")
    psvd.psvd_save(s.h, path)
    h2 = psvd.psvd_load(path)
    for b in bs[2:]:
        s.incorporate_data(b)
        psvd.psvd_incorporate_data(h2, b)
    U1 = s.modes()
    U2 = torch.empty_like(U1.T).T
    psvd.psvd_get_modes(h2, U2)
    s1 = s.singular_values()
    s2 = torch.empty_like(s1)
    psvd.psvd_get_singular_values(h2, s2)
    psvd.psvd_destroy(h2)
    s.close()
    assert torch.equal(U1, U2) and torch.equal(s1, s2)


def test_parallel_qr_R_matches_householder():
    A = np.asfortranarray(np.random.default_rng(3).standard_normal((6000, 40)).astype(np.float32))
    h = psvd.psvd_create(6000, 8, 40)
    R = torch.zeros((40, 40), dtype=torch.float64, device="cuda").T
    psvd.psvd_parallel_qr(h, torch.from_numpy(A).cuda().T.contiguous().T, R)
    psvd.psvd_destroy(h)
    _, Ro = oracle.householder_qr(A.astype(np.float64))
    assert np.abs(R.cpu().numpy() - Ro).max() <= 1e-5 * np.abs(Ro).max()


def test_gaussian_sketch_bit_exact():
    for rows, cols, seed, sid in [(96, 42, 1234, 0), (1000, 7, 2 ** 40 + 3, 2 ** 33 + 1), (1, 1, 0, 0)]:
        out = torch.empty((cols, rows), dtype=torch.float32, device="cuda").T
        psvd.psvd_gaussian_sketch(seed, sid, out)
        ref = oracle.gaussian_matrix(seed, sid, rows, cols).astype(np.float32)
        got = out.cpu().numpy()
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_errors_are_reported():
    h = psvd.psvd_create(1000, 4, 16)
    x = torch.zeros((1000, 8), dtype=torch.float32, device="cuda").T.contiguous().T
    with pytest.raises(psvd.PsvdError) as e:
        psvd.psvd_incorporate_data(h, x)
    assert e.value.status == psvd.PSVD_ERR_NOT_INITIALIZED
    big = torch.zeros((1000, 17), dtype=torch.float32, device="cuda").T.contiguous().T
    with pytest.raises(psvd.PsvdError) as e:
        psvd.psvd_initialize(h, big)
    assert e.value.status == psvd.PSVD_ERR_SHAPE
    psvd.psvd_destroy(h)
    with pytest.raises(psvd.PsvdError):
        psvd.psvd_create(1000, 100, 100)  # K + max_batch > 192
    with pytest.raises(psvd.PsvdError):
        psvd.psvd_create(1000, 4, 16, ff=1.5)


def test_nan_input_reports_nonfinite():
    A = torch.randn(2000, 16, dtype=torch.float64)
    A[5, 3] = float("nan")
    h = psvd.psvd_create(2000, 4, 16)
    psvd.psvd_initialize(h, synthetic.to_storage(A, torch.float32).cuda())
    s = torch.empty(4, dtype=torch.float64, device="cuda")
    with pytest.raises(psvd.PsvdError) as e:
        psvd.psvd_get_singular_values(h, s)
    assert e.value.status == psvd.PSVD_ERR_NONFINITE
    psvd.psvd_destroy(h)
