"""GB300-native ES adaptive moving-mesh RHD solver (Duan & Tang, arXiv 2107.12027).

The compute path lives in the CUDA library ``libesmm.so`` (C ABI, see
``include/esmm.h``); ``paper_2107_12027_gb300.esmm`` is its thin ctypes
binding.  Nothing is imported eagerly, so ``paper_2107_12027_gb300.workloads``
(the seeded input generators) works without a GPU.
"""
