"""GB300-native single-GPU short-range MD hot path (arXiv:1412.3387).

The compute path is a C-ABI CUDA library (``csrc/``, header ``include/md.h``)
loaded through ``paper_1412_3387_gb300.md``.  Importing this package does not
load the library; ``inputs`` holds the seeded workload generators.
"""
