"""DISK (arXiv 2512.04556) spatially-variant sparse-kernel-complex filtering,
GB300-native.  The compute path is the CUDA library ``libdisk.so`` (sm_103a)
behind a C ABI; ``paper_2512_04556_gb300.disk`` is its thin Python binding."""
