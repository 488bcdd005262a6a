"""GB300 (sm_103a) library for the fine-level transient heat solve of the
spatiotemporal two-level method for laser powder bed fusion
(arXiv:2110.12932).

  tl         ctypes binding of the C ABI (include/tl.h) over libtl.so
  build      in-tree nvcc build of libtl.so
  workloads  seeded synthetic inputs (plates, patches, scan paths)

Importing the package loads nothing; ``tl.load()`` loads the CUDA library
and raises if it has not been built.
"""
