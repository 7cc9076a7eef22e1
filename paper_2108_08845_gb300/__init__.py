"""GB300-native streaming, partitioned, randomized SVD (arXiv 2108.08845).

The hot path (Algorithm 1's per-batch update, Sec. 3.1) runs in hand-written CUDA
kernels for sm_103a behind the C-ABI library ``libpsvd.so`` declared in
``include/psvd.h``.  ``paper_2108_08845_gb300.psvd`` is the thin ctypes binding
with the same names; ``synthetic`` holds the seeded input generators.
"""
