"""Many independent snapshot streams updated together (psvd_group_*), including the
CUDA-graph replay path, against independently run handles and the FP64 oracle.

Each member runs the same kernels on the same inputs as a lone handle would, so the
group's results must be bit-identical to one handle per stream; two members are
also checked against the oracle with the FP32 tolerances of the plain path (and
their representation floor, as in test_gpu_fp32).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_08845_gb300 import psvd, synthetic
from tests.test_gpu_fp32 import _compare

pytestmark = pytest.mark.gpu


def _streams(count, M, B, T, seed, dtype=torch.float32):
    """count independent streams, T batches each (column-major on the host)."""
    out = []
    for i in range(count):
        A, *_ = synthetic.low_rank(M, B * T, 24, 1e-6, seed + 17 * i)
        A = synthetic.to_storage(A, dtype)
        out.append([A[:, t * B:(t + 1) * B] for t in range(T)])
    return out


def _run_group(streams, M, K, B, ff, prec=psvd.PSVD_PREC_FP32):
    count, T = len(streams), len(streams[0])
    g = psvd.psvd_group_create(count, M, K, B, ff, prec)
    # a ring of two input buffers per member: later calls repeat the pointers
    dt = streams[0][0].dtype
    ring = [[torch.empty(B, M, dtype=dt, device="cuda").T for _ in range(count)]
            for _ in range(2)]
    for t in range(T):
        buf = ring[t % 2]
        for i in range(count):
            buf[i].copy_(streams[i][t])
        if t == 0:
            psvd.psvd_group_initialize(g, buf)
        else:
            psvd.psvd_group_incorporate_data(g, buf)
    rc = psvd.psvd_group_status(g)
    stats = psvd.psvd_group_stats(g)
    res = []
    for i in range(count):
        h = psvd.psvd_group_member(g, i)
        k = psvd.psvd_num_modes(h)
        U = torch.empty(k, M, dtype=torch.float32, device="cuda").T
        D = torch.empty(k, dtype=torch.float64, device="cuda")
        psvd.psvd_get_modes(h, U)
        psvd.psvd_get_singular_values(h, D)
        res.append((U.cpu().numpy(), D.cpu().numpy()))
    psvd.psvd_group_destroy(g)
    return rc, stats, res


def _run_single(batches, M, K, B, ff, prec=psvd.PSVD_PREC_FP32):
    s = psvd.StreamingSVD(M, K, B, ff, prec)
    s.initialize(batches[0].cuda())
    for A in batches[1:]:
        s.incorporate_data(A.cuda())
    U, D = s.modes().cpu().numpy(), s.singular_values().cpu().numpy()
    s.close()
    return U, D


@pytest.mark.parametrize("count,M,T", [(8, 16384, 6), (32, 65536, 5)])
def test_group_matches_single_handles_and_replays(count, M, T):
    K, B, ff = 16, 16, 0.95
    streams = _streams(count, M, B, T, seed=700 + count)
    rc, (captures, replays), res = _run_group(streams, M, K, B, ff)
    assert rc == psvd.PSVD_OK
    # updates 1 and 2 capture one graph per buffer parity, later updates replay them
    assert captures == 2 and replays == T - 3, (captures, replays)
    for i in (0, count // 2, count - 1):
        U1, D1 = _run_single(streams[i], M, K, B, ff)
        assert np.array_equal(res[i][1], D1)
        assert np.array_equal(res[i][0], U1)
    for i in (0, count - 1):
        Uo, Do = oracle.stream_run([b.double().numpy() for b in streams[i]], K, ff)
        _compare(res[i][0].astype(np.float64), res[i][1], Uo, Do)


def test_tensor_core_group_matches_single_handles():
    # tensor-core members run their launches directly on their own streams (no
    # graph): still the same kernels on the same inputs as lone handles
    count, M, T, K, B, ff = 6, 12288, 5, 16, 16, 0.95
    TC = psvd.PSVD_PREC_BF16_TC
    streams = _streams(count, M, B, T, seed=900, dtype=torch.bfloat16)
    rc, _, res = _run_group(streams, M, K, B, ff, TC)
    assert rc == psvd.PSVD_OK
    for i in (0, count - 1):
        U1, D1 = _run_single(streams[i], M, K, B, ff, TC)
        assert np.array_equal(res[i][1], D1) and np.array_equal(res[i][0], U1)
        Uo, Do = oracle.stream_run([b.double().numpy() for b in streams[i]], K, ff)
        _compare(res[i][0].astype(np.float64), res[i][1], Uo, Do, sig_tol=1e-4, ang_tol=1e-3,
                 unit=2.0 ** -17)
