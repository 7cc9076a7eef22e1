"""The autotuner (psvd_autotune) of the FP32 and tensor-core paths: the choice is
one of the candidates, is cached per shape, leaves the handle's state untouched,
and a tuned run still matches the oracle with the path's tolerances."""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_08845_gb300 import psvd, synthetic
from tests.test_gpu_fp32 import _compare, _oracle_run_gap

pytestmark = pytest.mark.gpu


def _batches(M, B, T, seed):
    A, *_ = synthetic.low_rank(M, B * T, 60, 1e-6, seed)
    A = synthetic.to_storage(A, torch.float32)
    return [A[:, t * B:(t + 1) * B] for t in range(T)]


def test_autotune_choice_cache_state_and_parity():
    M, K, B, T, ff = 262144, 32, 64, 4, 0.95
    bs = _batches(M, B, T, seed=901)
    dev = [b.cuda() for b in bs]
    s = psvd.StreamingSVD(M, K, B, ff, psvd.PSVD_PREC_FP32)
    s.initialize(dev[0])
    U0, D0 = s.modes().cpu().numpy(), s.singular_values().cpu().numpy()
    cps, rows = psvd.psvd_autotune(s.h, dev[1])
    assert cps in (1, 2, 4, 8) and rows in (64, 128, 256)
    # the trials leave the modes, singular values and status as they were
    assert np.array_equal(s.modes().cpu().numpy(), U0)
    assert np.array_equal(s.singular_values().cpu().numpy(), D0)
    assert psvd.psvd_last_info(s.h)[0] == psvd.PSVD_OK
    for A in dev[1:]:
        s.incorporate_data(A)
    U, D = s.modes().cpu().numpy().astype(np.float64), s.singular_values().cpu().numpy()
    s.close()
    Uo, Do = oracle.stream_run([b.double().numpy() for b in bs], K, ff)
    _compare(U, D, Uo, Do)
    # a second handle of the same shape takes the cached choice
    s2 = psvd.StreamingSVD(M, K, B, ff, psvd.PSVD_PREC_FP32)
    assert psvd.psvd_autotune(s2.h, dev[2]) == (cps, rows)
    s2.close()


def test_autotune_tensor_core_choice_cache_state_and_parity():
    # travelling-wave recipe (K = 64, B = 128, BF16 snapshots) on a 256 x 512 grid
    M, K, B, ff = 131072, 64, 128, 0.95
    gen = synthetic.TravellingWaves(256, 512, 256, 1.2, 1e-4, seed=1237)
    bs = [synthetic.to_storage(gen.batch(i, B), torch.bfloat16) for i in range(4)]
    dev = [b.cuda() for b in bs]
    s = psvd.StreamingSVD(M, K, B, ff, psvd.PSVD_PREC_BF16_TC)
    s.initialize(dev[0])
    s.incorporate_data(dev[1])
    U0, D0 = s.modes().cpu().numpy(), s.singular_values().cpu().numpy()
    clusters, ctas, stages = psvd.psvd_autotune(s.h, dev[2])
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert 1 <= clusters <= sms and ctas in (sms, sms // 2) and 2 <= stages <= 4
    assert np.array_equal(s.modes().cpu().numpy(), U0)
    assert np.array_equal(s.singular_values().cpu().numpy(), D0)
    assert psvd.psvd_last_info(s.h)[0] == psvd.PSVD_OK
    for A in dev[2:]:
        s.incorporate_data(A)
    U, D = s.modes().cpu().numpy().astype(np.float64), s.singular_values().cpu().numpy()
    s.close()
    Uo, Do, s_next = _oracle_run_gap(bs, K, ff)
    _compare(U, D, Uo, Do, sig_tol=1e-4, ang_tol=1e-3, unit=2.0 ** -17, s_next=s_next)
    s2 = psvd.StreamingSVD(M, K, B, ff, psvd.PSVD_PREC_BF16_TC)
    assert psvd.psvd_autotune(s2.h, dev[3]) == (clusters, ctas, stages)
    s2.close()


def test_autotune_tensor_core_small_panel_stages():
    # K = 16, B = 16: the panel is narrow, so up to four update stages fit
    M, K, B = 65536, 16, 16
    A, *_ = synthetic.low_rank(M, 4 * B, 24, 1e-6, seed=905)
    bs = [synthetic.to_storage(A[:, t * B:(t + 1) * B], torch.bfloat16) for t in range(4)]
    dev = [b.cuda() for b in bs]
    ref = psvd.StreamingSVD(M, K, B, 1.0, psvd.PSVD_PREC_BF16_TC)
    s = psvd.StreamingSVD(M, K, B, 1.0, psvd.PSVD_PREC_BF16_TC)
    ref.initialize(dev[0])
    s.initialize(dev[0])
    choice = psvd.psvd_autotune(s.h, dev[1])
    assert len(choice) == 3 and 2 <= choice[2] <= 4
    for A in dev[1:]:
        ref.incorporate_data(A)
        s.incorporate_data(A)
    U, D = s.modes().cpu().numpy().astype(np.float64), s.singular_values().cpu().numpy()
    Ur, Dr = ref.modes().cpu().numpy().astype(np.float64), ref.singular_values().cpu().numpy()
    s.close()
    ref.close()
    Uo, Do, s_next = _oracle_run_gap(bs, K, 1.0)
    _compare(U, D, Uo, Do, sig_tol=1e-4, ang_tol=1e-3, unit=2.0 ** -17, s_next=s_next)
    # only the Gram's row split can change the rounding; the tuned run stays at the
    # default run's level
    _compare(U, D, Ur, Dr, sig_tol=1e-4, ang_tol=1e-3, unit=2.0 ** -17, gram_res=2e-9)


def test_autotune_rejects_fp64_handles():
    s = psvd.StreamingSVD(4096, 8, 16, 1.0, psvd.PSVD_PREC_FP64)
    A = torch.zeros(16, 4096, dtype=torch.float64, device="cuda").T
    with pytest.raises(psvd.PsvdError) as e:
        psvd.psvd_autotune(s.h, A)
    assert e.value.status == psvd.PSVD_ERR_UNSUPPORTED
    s.close()
