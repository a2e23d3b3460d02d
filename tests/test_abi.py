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
