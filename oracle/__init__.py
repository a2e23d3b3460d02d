"""FastPI CPU oracle (FP64, NumPy/SciPy).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library in
``paper_2011_04235_gb300`` never imports it, links it or calls it, and this
package imports nothing from the library: the two share no code.

Contents (each function cites the passage of the paper it follows):
  * :mod:`oracle.reorder`  -- Algorithm 2, hub-and-spoke reordering (integer).
  * :mod:`oracle.fastpi`   -- Algorithm 1: block SVD of A11 (Eq. 1), row
    incremental update (Eq. 2), column incremental update (Eq. 3), both in the
    paper's single-shot form and in the chunked (Brand) form the library uses,
    and the pseudoinverse apply of Problem 1 / Application 1.
  * :mod:`oracle.pinv`     -- dense Moore-Penrose pseudoinverse from a full
    SVD (Problem 1), the reference for untruncated special cases.
"""
