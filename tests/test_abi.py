"""CPU checks of the C ABI: the library builds for sm_103a, loads without a
GPU, and exports every function that include/fastpi.h declares (no compute
call is made)."""
import ctypes
import numpy as np
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fastpi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fastpi_[A-Za-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2011_04235_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "fastpi_create" in names and "fastpi_apply" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_lists_every_declared_symbol():
    from paper_2011_04235_gb300 import fastpi
    assert sorted(fastpi.SYMBOLS) == _declared()
    lib = fastpi.lib()
    for n in fastpi.SYMBOLS:
        assert hasattr(lib, n)


def test_last_error_without_handle():
    from paper_2011_04235_gb300 import fastpi
    # a NULL handle is accepted and returns a (possibly empty) message
    assert isinstance(fastpi.lib().fastpi_last_error(None), bytes)


def test_binding_rejects_bad_dense_arguments():
    """The binding checks tensors before any pointer reaches the library: a
    host tensor, a non-tensor or a tensor on a non-CUDA device is refused with
    ValueError (no GPU needed: nothing is called)."""
    import pytest
    import torch
    from paper_2011_04235_gb300 import fastpi
    with pytest.raises(ValueError):
        fastpi._dense_dev(torch.zeros(4, 3, dtype=torch.float64), 4, "Y")         # host tensor
    with pytest.raises(ValueError):
        fastpi._dense_dev(np.zeros((4, 3)), 4, "Y")                              # not a tensor
    meta = torch.empty(4, 3, dtype=torch.float64, device="meta")
    with pytest.raises(ValueError):
        fastpi._dense_dev(meta, 4, "Y")                                          # not CUDA either


def test_missing_library_fails_loudly():
    """No CPU fallback: without libfastpi.so the binding raises instead of
    computing anything."""
    import pytest
    from paper_2011_04235_gb300 import fastpi
    missing = os.path.join(ROOT, "tests", "no_such_dir", "libfastpi.so")
    assert not os.path.exists(missing)
    with pytest.raises(ImportError):
        fastpi.load_library(missing)


def test_binding_residual_noalloc_checks_arguments():
    """residual_noalloc refuses, before any pointer reaches the library, the
    arguments whose sizes or types the C entry point would read past or
    misread: host tensors, an int32 rowptr, a rowptr of the wrong length,
    col / val of different lengths, a Y or Z with the wrong row count."""
    import pytest
    import torch
    from paper_2011_04235_gb300 import fastpi
    m, n = 4, 3
    rp = torch.tensor([0, 1, 2, 3, 4], dtype=torch.int64)
    cl = torch.tensor([0, 1, 2, 0], dtype=torch.int32)
    vl = torch.ones(4, dtype=torch.float64)
    Y = torch.zeros(m, 2, dtype=torch.float64)
    Z = torch.zeros(n, 2, dtype=torch.float64)
    cases = [
        (rp, cl, vl, Y, Z),                              # host tensors
        (rp.to(torch.int32), cl, vl, Y, Z),              # rowptr int32
        (rp[:-1], cl, vl, Y, Z),                         # rowptr of m entries
        (rp, cl, vl[:-1], Y, Z),                         # col and val lengths differ
        (rp, cl, vl, Y[:-1], Z),                         # Y with m - 1 rows
        (rp, cl, vl, Y, Z[:-1]),                         # Z with n - 1 rows
        (rp, cl.to(torch.int64), vl, Y, Z),              # col int64
    ]
    for args in cases:
        with pytest.raises(ValueError):
            fastpi.residual_noalloc(m, n, *args)
