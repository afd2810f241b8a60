"""GB300-native spacetime-multigrid smoke control (Pan & Manocha, arXiv 1608.01102).

``stc``       -- Python binding of the C ABI in ``include/stc.h`` (libstc.so).
``build``     -- in-tree nvcc build of libstc.so for sm_103a.
``workloads`` -- seeded synthetic inputs shaped like the paper's benchmarks.
"""
