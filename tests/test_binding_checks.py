"""Host-side argument checks of the Python binding and the autograd entry point:
they reject bad layouts and dtypes before any library call (no GPU needed)."""
import numpy as np
import pytest
import torch

from paper_2108_08845_gb300 import psvd
from paper_2108_08845_gb300.autograd import streaming_svd


def test_matrices_must_be_column_major():
    a = np.zeros((8, 4), dtype=np.float32)  # C order: rows contiguous
    with pytest.raises(ValueError, match="column-major"):
        psvd._mat(a, "A")
    t = torch.zeros(8, 4)
    with pytest.raises(ValueError, match="column-major"):
        psvd._mat(t, "A")
    p, ld, rows, cols, code, _ = psvd._mat(torch.zeros(4, 8).T, "A")
    assert (ld, rows, cols, code) == (8, 8, 4, psvd.PSVD_F32)


def test_dtypes_are_checked():
    with pytest.raises(ValueError, match="unsupported dtype"):
        psvd._mat(np.zeros((8, 2), dtype=np.float64, order="F"), "A")  # FP64 not allowed here
    assert psvd._mat(np.zeros((8, 2), dtype=np.float64, order="F"), "A", allow_f64=True)[4] == \
        psvd.PSVD_F64
    with pytest.raises(ValueError, match="unsupported dtype"):
        psvd._mat(torch.zeros(2, 8, dtype=torch.int32).T, "A")


def test_group_batches_must_share_shape_and_dtype():
    a = torch.zeros(4, 8).T
    b = torch.zeros(3, 8).T
    with pytest.raises(ValueError, match="same lda, B and dtype"):
        psvd._batch_list([a, b], "batches")
    with pytest.raises(ValueError, match="no batches"):
        psvd._batch_list([], "batches")


def test_adjoint_binding_checks_dtypes_before_calling():
    M = 8
    A = torch.zeros(2, M).T
    U = torch.zeros(1, M).T
    D = torch.zeros(1, dtype=torch.float64)
    with pytest.raises(ValueError, match="U_new"):
        psvd.psvd_update_adjoint(0, None, None, A, U.double(), D, U, D, None, None,
                                 torch.zeros(2, M).T)
    with pytest.raises(ValueError, match="float64"):
        psvd.psvd_update_adjoint(0, None, None, A, U, D.float(), U, D, None, None,
                                 torch.zeros(2, M).T)


def test_streaming_svd_needs_cuda_tensors():
    with pytest.raises(ValueError, match="CUDA"):
        streaming_svd([torch.zeros(2, 16).T.requires_grad_(True)], 1, 1.0)


def test_incorporate_batches_checks_before_calling():
    a = torch.zeros(4, 8).T
    with pytest.raises(ValueError, match="same lda, B and dtype"):
        psvd.psvd_incorporate_batches(0, [a, torch.zeros(3, 8).T])
    with pytest.raises(ValueError, match="no batches"):
        psvd.psvd_incorporate_batches(0, [])
    with pytest.raises(ValueError, match="float64"):
        psvd.psvd_incorporate_batches(0, [a], torch.zeros(2, 4, dtype=torch.float32))
    with pytest.raises(ValueError, match="2 x 4 elements"):
        psvd.psvd_incorporate_batches(0, [a, a], torch.zeros(1, 4, dtype=torch.float64), K=4)
