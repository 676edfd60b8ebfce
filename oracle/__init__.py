"""CPU oracle for the kernel-selection GEMM library -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct reference implementations of what the GPU path
computes, written from the paper (Lawson, "Performance portability through
machine learning guided kernel selection in SYCL libraries"):

* ``gemm``    -- FP64 triple-loop GEMM and its componentwise error scale (Section 3).
* ``select``  -- normalisations (Section 3.4), k-means pruning and cluster
                 representatives (Sections 4.1-4.2), Top-N, the held-out
                 geometric-mean score (Section 4.3), the CART decision-tree
                 classifier (Section 5.1) and PCA (Section 3.3).
* ``mlp``     -- FP64 forward/backward/Adam of the 7-64-64-8 performance model.
* ``bf16``    -- round-to-nearest-even BF16 and the hi/lo split of an FP32 value.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It imports nothing from the CUDA
library and the library imports nothing from it.
"""
