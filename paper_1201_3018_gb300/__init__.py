"""GB300-native approximate overlap-save convolution and cross-correlation
(companding + tight packing + block convolution core + unpacking), after
Anam & Andreopoulos, arXiv 1201.3018.

``paper_1201_3018_gb300.apx`` binds the C-ABI library ``libapx.so`` (hand-written
sm_103a CUDA kernels); ``paper_1201_3018_gb300.workloads`` holds the seeded
synthetic input generators.  Importing this package loads nothing: the CUDA
library is opened on first use of ``apx`` and fails loudly if it is missing.
"""
__all__ = ["apx", "workloads"]
