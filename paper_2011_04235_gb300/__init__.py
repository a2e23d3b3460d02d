"""FastPI on GB300: hub-and-spoke reordering, incremental low-rank SVD and the
pseudoinverse solve Z = V Sigma^+ U^T Y, as hand-written sm_103a CUDA kernels
behind a C ABI (include/fastpi.h).

``paper_2011_04235_gb300.fastpi`` holds the ctypes binding; ``build`` compiles
the library in-tree.  Importing this package does not load the library.
"""

__all__ = ["build", "fastpi"]
