"""Device-side failure detection without a GPU fault (Sec. 5 of the design: every
wait of the tensor-core kernels is bounded).

The update kernel's pipeline-wait budget is set, through the library's testing hook,
below the latency of any copy: its first wait runs out, the kernel stops issuing
work, drains the copies and tensor-core products it had already issued (those waits
keep the full budget), frees its tensor memory and returns, and the handle reports
PSVD_ERR_TIMEOUT.  The kernel makes no cross-CTA waits (no cluster), so every copy
that can land in a CTA's shared memory is one that CTA issued and drains.  The
context stays usable: a new handle then runs to the oracle's result."""
import numpy as np
import pytest
import torch

from paper_2108_08845_gb300 import psvd, synthetic
from tests.test_gpu_fp32 import _compare, _gpu_run, _oracle_run_gap

pytestmark = pytest.mark.gpu

TC = psvd.PSVD_PREC_BF16_TC


def _bf16_batches():
    A, _, _, _ = synthetic.low_rank(8192, 64, 40, 1e-7, seed=77,
                                    s=[10.0 ** (-i / 24.0) for i in range(40)])
    return [synthetic.to_storage(A[:, i:i + 32], torch.bfloat16) for i in range(0, 64, 32)]


def test_update_wait_budget_runs_out_and_reports_timeout():
    bs = _bf16_batches()
    s = psvd.StreamingSVD(8192, 16, 32, 1.0, TC)
    try:
        s.initialize(bs[0].cuda())
        psvd.psvd_debug_set_wait_budget(psvd.PSVD_DEBUG_UPDATE_KERNEL, 1)
        try:
            s.incorporate_data(bs[1].cuda())
            out = torch.empty(16, dtype=torch.float64, device="cuda")
            with pytest.raises(psvd.PsvdError) as e:
                psvd.psvd_get_singular_values(s.h, out)
            assert e.value.status == psvd.PSVD_ERR_TIMEOUT
        finally:
            psvd.psvd_debug_set_wait_budget(psvd.PSVD_DEBUG_UPDATE_KERNEL, 0)
    finally:
        s.close()
    torch.cuda.synchronize()  # the context is still usable
    # a fresh handle with the default budget computes the oracle's result
    U, D, _ = _gpu_run(bs, K=16, ff=1.0, precision=TC)
    Uo, Do, s_next = _oracle_run_gap(bs, 16, 1.0)
    _compare(U, D, Uo, Do, sig_tol=1e-4, ang_tol=1e-3, unit=2.0 ** -17, s_next=s_next)
