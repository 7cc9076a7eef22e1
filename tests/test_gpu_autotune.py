"""The FP32 path's autotuner (psvd_autotune): the choice is one of the candidates,
is cached per shape, leaves the handle's state untouched, and a tuned run still
matches the oracle with the plain path's tolerances."""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_08845_gb300 import psvd, synthetic
from tests.test_gpu_fp32 import _compare

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
    assert cps in (1, 2, 4, 8) and rows in (64, 128)
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


def test_autotune_rejects_tensor_core_handles():
    s = psvd.StreamingSVD(4096, 8, 16, 1.0, psvd.PSVD_PREC_BF16_TC)
    A = torch.zeros(16, 4096, dtype=torch.bfloat16, device="cuda").T
    with pytest.raises(psvd.PsvdError) as e:
        psvd.psvd_autotune(s.h, A)
    assert e.value.status == psvd.PSVD_ERR_UNSUPPORTED
    s.close()
