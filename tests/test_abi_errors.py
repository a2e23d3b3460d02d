"""The C ABI's argument checks, which run before any CUDA call: every entry
point returns FASTPI_ERR_ARG (1) for a NULL handle, impossible sizes or NULL
arrays, leaves a message where the header says so, and never aborts.  These
calls behave the same with or without a GPU, so they run on the CPU."""
import ctypes as C

import numpy as np
import pytest

ERR_ARG = 1


@pytest.fixture(scope="module")
def lib():
    from paper_2011_04235_gb300 import fastpi
    return fastpi.lib()


def test_null_handle_everywhere(lib):
    i64 = C.c_int64()
    d = C.c_double()
    calls = [
        lambda: lib.fastpi_factor(None, 10, 0.1, 0, 0, 0),
        lambda: lib.fastpi_reorder(None, 0.1),
        lambda: lib.fastpi_truncate(None, 3),
        lambda: lib.fastpi_apply(None, None, 0, 0, None, 0),
        lambda: lib.fastpi_apply_host(None, None, 0, 0, None, 0),
        lambda: lib.fastpi_apply_csr(None, 0, 0, None, None, None, None, 0),
        lambda: lib.fastpi_residual(None, None, 0, 0, None, 0, C.byref(d)),
        lambda: lib.fastpi_get_rank(None, C.byref(i64)),
        lambda: lib.fastpi_get_S(None, None),
        lambda: lib.fastpi_get_U(None, None, 0),
        lambda: lib.fastpi_get_V(None, None, 0),
        lambda: lib.fastpi_get_perm(None, None, None, None, None),
        lambda: lib.fastpi_get_blocks(None, None, None, None),
        lambda: lib.fastpi_get_info(None, None),
        lambda: lib.fastpi_get_counters(None),
    ]
    for call in calls:
        assert call() == ERR_ARG
    lib.fastpi_destroy(None)                       # a no-op
    assert isinstance(lib.fastpi_last_error(None), bytes)


def test_create_rejects_bad_sizes(lib):
    h = C.c_void_p(1234)                           # must come back NULL on error
    rp = np.array([0, 1, 2], dtype=np.int64)
    col = np.array([0, 1], dtype=np.int32)
    val = np.ones(2)
    ptrs = (rp.ctypes.data, col.ctypes.data, val.ctypes.data)
    assert lib.fastpi_create(None, 2, 2, 2, *ptrs, 0, None) == ERR_ARG
    for m, n, nnz in ((0, 2, 0), (2, 0, 0), (2, 2, -1), (2, 2, 5), (1 << 30, 1 << 30, 0)):
        assert lib.fastpi_create(C.byref(h), m, n, nnz, *ptrs, 0, None) == ERR_ARG
        assert h.value is None
        assert lib.fastpi_last_error(None)         # a message for the failed create
    assert lib.fastpi_create(C.byref(h), 2, 2, 2, None, ptrs[1], ptrs[2], 0, None) == ERR_ARG


def test_create_from_factors_checks_the_factors_first(lib):
    h = C.c_void_p()
    U = np.zeros((4, 2))
    V = np.zeros((3, 2))
    bad_order = np.array([1.0, 2.0])               # not descending
    negative = np.array([1.0, -0.5])
    for S in (bad_order, negative):
        assert lib.fastpi_create_from_factors(C.byref(h), 4, 3, 2, S.ctypes.data, U.ctypes.data, 2, V.ctypes.data,
                                              2, 0, 0, None) == ERR_ARG
    S = np.array([2.0, 1.0])
    assert lib.fastpi_create_from_factors(C.byref(h), 4, 3, 4, S.ctypes.data, U.ctypes.data, 2, V.ctypes.data,
                                          2, 0, 0, None) == ERR_ARG    # r > min(m, n)
    assert lib.fastpi_create_from_factors(C.byref(h), 4, 3, 2, S.ctypes.data, U.ctypes.data, 1, V.ctypes.data,
                                          2, 0, 0, None) == ERR_ARG    # ldu < r
    assert lib.fastpi_create_from_factors(C.byref(h), 4, 3, 2, S.ctypes.data, U.ctypes.data, 2, V.ctypes.data,
                                          2, 7, 0, None) == ERR_ARG    # unknown precision
    assert h.value is None


def test_batched_and_gemm_and_noalloc_argument_checks(lib):
    r = np.array([5], dtype=np.int64)
    assert lib.fastpi_factor_batched(None, 1, r.ctypes.data, 0.1, 0, 0, 0, 0, None) == ERR_ARG
    hs = (C.c_void_p * 1)(None)
    assert lib.fastpi_factor_batched(C.cast(hs, C.c_void_p), 1, r.ctypes.data, 0.1, 0, 0, 0, 0, None) == ERR_ARG
    assert lib.fastpi_factor_batched(C.cast(hs, C.c_void_p), 0, r.ctypes.data, 0.1, 0, 0, 0, 0, None) == ERR_ARG
    # gemm: unknown engine, negative size, leading dimension too small
    assert lib.fastpi_gemm_f32(0, 0, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, 2, None) == ERR_ARG
    assert lib.fastpi_gemm_f32(0, 0, -1, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, 0, None) == ERR_ARG
    assert lib.fastpi_gemm_f32(0, 0, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 3, 0, None) == ERR_ARG
    # the no-allocation residual: NULL out, and more rows than its static scratch
    d = C.c_double()
    rp = np.zeros(2, dtype=np.int64)
    assert lib.fastpi_residual_noalloc(1, 1, rp.ctypes.data, None, None, None, 0, 0, None, 0, None, None) == ERR_ARG
    assert lib.fastpi_residual_noalloc((1 << 20) + 1, 1, rp.ctypes.data, None, None, None, 0, 0, None, 0,
                                       C.byref(d), None) == ERR_ARG


def test_tuning_table_parsing(lib, tmp_path):
    """fastpi_load_tuning reads the autotuner's table (no GPU call): a
    well-formed file loads, a malformed line or a missing file is refused with
    FASTPI_ERR_ARG and a message, and NULL restores the built-in defaults."""
    good = tmp_path / "t.txt"
    good.write_text("# comment\ncore 600 16 4 0 1\ncore 1048576 32 8 1 1\nchunk 1 0 491 320\n"
                    "chunk 0 1 1099511627776 256\nbucket 1 256 1\ngemm 536870912\n")
    assert lib.fastpi_load_tuning(str(good).encode()) == 0
    for bad in ("core 600 24 4 0 1\n", "chunk 2 0 10 256\n", "bucket 1 256 9\n", "core 600 16\n", "foo 1\n", "gemm 0\n", "gemm\n"):
        p = tmp_path / "bad.txt"
        p.write_text(bad)
        assert lib.fastpi_load_tuning(str(p).encode()) == ERR_ARG
        assert lib.fastpi_last_error(None)
    assert lib.fastpi_load_tuning(str(tmp_path / "missing.txt").encode()) == ERR_ARG
    assert lib.fastpi_load_tuning(None) == 0
