"""B300-native RNS-CKKS linear path of BLB (arXiv 2508.19525).

The compute path is the CUDA library libblb.so (C ABI in include/blb.h);
`paper_2508_19525_b300.blb` is its ctypes binding.  Importing this package does
not load CUDA; `workloads` holds the seeded synthetic inputs.
"""
__all__ = ["blb", "workloads"]
