"""GB300-native kernel-selection GEMM library (Lawson, arXiv 2008.13145, re-designed for sm_103a).

``kselect`` is the ctypes binding of the C-ABI library ``libkselect.so``;
``workloads`` holds the seeded synthetic shapes and inputs.  Importing the
package does not load the CUDA library; ``from paper_2008_13145_gb300 import
kselect`` does, and raises if it has not been built.
"""
