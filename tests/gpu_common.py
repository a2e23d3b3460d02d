"""Helpers shared by the GPU parity tests: build / load the library once and
compare its results with the oracle."""
import functools

import numpy as np
import scipy.sparse as sp


@functools.lru_cache(maxsize=1)
def binding():
    from paper_2011_04235_gb300 import build as _b
    _b.build()
    from paper_2011_04235_gb300 import fastpi
    fastpi.lib()
    return fastpi


def dense(m, n, rowptr, col, val):
    return sp.csr_matrix((val, col, rowptr), shape=(m, n)).toarray()


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
