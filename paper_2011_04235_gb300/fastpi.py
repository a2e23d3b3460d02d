"""Thin ctypes binding of libfastpi (include/fastpi.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Tensors are PyTorch tensors (device memory and streams come from
PyTorch); the library receives raw pointers and the current CUDA stream.
Importing this module loads ``libfastpi.so`` from this package directory and
raises if it is missing (build it with ``python -m paper_2011_04235_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfastpi.so")

FASTPI_FP64 = 0
FASTPI_MIXED_TF32 = 1
PRECISIONS = {"fp64": FASTPI_FP64, "mixed": FASTPI_MIXED_TF32, "tf32": FASTPI_MIXED_TF32}

STATUS = {0: "FASTPI_OK", 1: "FASTPI_ERR_ARG", 2: "FASTPI_ERR_CSR", 3: "FASTPI_ERR_OOM", 4: "FASTPI_ERR_CUDA",
          5: "FASTPI_ERR_NO_CONVERGENCE", 6: "FASTPI_ERR_STATE"}

# every symbol the header declares
SYMBOLS = ["fastpi_create", "fastpi_create_from_factors", "fastpi_truncate", "fastpi_factor",
           "fastpi_factor_batched", "fastpi_reorder", "fastpi_block_svd", "fastpi_apply", "fastpi_apply_host", "fastpi_apply_csr",
           "fastpi_residual", "fastpi_residual_noalloc", "fastpi_spmm", "fastpi_recon_error", "fastpi_get_rank", "fastpi_get_S", "fastpi_get_U",
           "fastpi_get_V",
           "fastpi_get_perm", "fastpi_get_blocks", "fastpi_get_info", "fastpi_get_counters",
           "fastpi_reset_counters", "fastpi_gemm_f32", "fastpi_core_svd_f32", "fastpi_load_tuning", "fastpi_last_error", "fastpi_destroy"]


class FastPIError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Info(C.Structure):
    _fields_ = [(name, C.c_int64) for name in
                ("m", "n", "nnz", "m1", "n1", "m2", "n2", "num_blocks", "iterations", "S", "s_row", "rank",
                 "chunk_row", "chunk_col", "row_chunks", "col_chunks", "dropped_directions",
                 "jacobi_sweeps_max")] + \
              [("min_trunc_gap", C.c_double), ("ms_reorder", C.c_double), ("ms_block_svd", C.c_double),
               ("ms_row_update", C.c_double), ("ms_col_update", C.c_double), ("ms_finalize", C.c_double),
               ("precision", C.c_int)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class Counters(C.Structure):
    _fields_ = [("kernel_launches", C.c_uint64), ("svd_launches", C.c_uint64 * 3), ("svd_ms", C.c_double * 3),
                ("svd_flops", C.c_double * 3), ("svd_flops_rot", C.c_double * 3),
                ("core_resident_launches", C.c_uint64)]


SVD_KINDS = ("blocks", "core32", "core64")


def counters() -> dict:
    """Process counters: kernel launches, and per SVD kind ("blocks": Eq. 1;
    "core32" / "core64": update cores) launches, event-timed ms, model flops
    and rotation flops."""
    c = Counters()
    _check(lib().fastpi_get_counters(C.byref(c)))
    out = {"kernel_launches": c.kernel_launches, "core_resident_launches": c.core_resident_launches}
    for i, kind in enumerate(SVD_KINDS):
        out[kind] = {"launches": c.svd_launches[i], "ms": c.svd_ms[i], "flops": c.svd_flops[i],
                     "flops_rot": c.svd_flops_rot[i]}
    return out


def reset_counters() -> None:
    lib().fastpi_reset_counters()


def residual_noalloc(m: int, n: int, rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor,
                     Y: torch.Tensor, Z: torch.Tensor) -> float:
    """|A Z - Y|_F through fastpi_residual_noalloc (device tensors, no allocation
    inside the library; A in CSR: rowptr int64 of m + 1 entries, col int32 and
    val float64 of equal length; Y m x L and Z n x L float64, row-major).  All
    tensors must be CUDA tensors on one device; anything else raises
    ValueError before the library is called (the library reads these buffers
    by the given sizes without checking them)."""
    m, n = int(m), int(n)
    for name, t, dt in (("rowptr", rowptr, torch.int64), ("col", col, torch.int32), ("val", val, torch.float64)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.dim() == 1):
            raise ValueError(f"{name} must be a 1-D CUDA {dt} tensor")
    if rowptr.numel() != m + 1:
        raise ValueError(f"rowptr must have m + 1 = {m + 1} entries")
    if col.numel() != val.numel():
        raise ValueError("col and val must have the same length")
    Y = _dense_dev(Y, m, "Y")
    Z = _dense_dev(Z, n, "Z")
    if Y.shape[1] != Z.shape[1]:
        raise ValueError("Y and Z must have the same number of columns")
    if len({t.device for t in (rowptr, col, val, Y, Z)}) != 1:
        raise ValueError("rowptr, col, val, Y and Z must be on one device")
    rowptr, col, val = rowptr.contiguous(), col.contiguous(), val.contiguous()
    out = C.c_double()
    st = torch.cuda.current_stream(Y.device).cuda_stream
    with torch.cuda.device(Y.device):
        _check(lib().fastpi_residual_noalloc(m, n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(Y),
                                             Y.shape[1], Y.stride(0), _ptr(Z), Z.stride(0), C.byref(out), st))
    return out.value


ENGINES = {"simt": 0, "tf32": 1, "tf32x3": 3}


def factor_batched(handles, ranks, k: float, precision="mixed", chunk_row: int = 0, chunk_col: int = 0,
                   concurrency: int = 0):
    """fastpi_factor_batched over FastPI objects (each created on its own stream
    for concurrency).  Returns the per-handle status list; raises on the first
    failure."""
    count = len(handles)
    hs = (C.c_void_p * count)(*[h._h for h in handles])
    rs = (C.c_int64 * count)(*[int(r) for r in ranks])
    st = (C.c_int * count)()
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    with torch.cuda.device(handles[0].device):
        _check(lib().fastpi_factor_batched(C.cast(hs, C.c_void_p), count, C.cast(rs, C.c_void_p), float(k), prec,
                                           int(chunk_row), int(chunk_col), int(concurrency),
                                           C.cast(st, C.c_void_p)))
    return list(st)


def gemm_f32(A: torch.Tensor, B: torch.Tensor, ta: bool = False, tb: bool = False, engine: str = "tf32x3",
             alpha: float = 1.0, beta: float = 0.0, Cout: torch.Tensor | None = None) -> torch.Tensor:
    """C = alpha op(A) op(B) + beta C through fastpi_gemm_f32 (device float32
    row-major tensors with unit column stride; op = transpose when ta / tb)."""
    M = A.shape[1] if ta else A.shape[0]
    K = A.shape[0] if ta else A.shape[1]
    N = B.shape[0] if tb else B.shape[1]
    if (B.shape[1] if tb else B.shape[0]) != K:
        raise ValueError("inner dimensions differ")
    if Cout is None:
        Cout = torch.zeros(M, N, dtype=torch.float32, device=A.device)
    st = torch.cuda.current_stream(A.device).cuda_stream
    with torch.cuda.device(A.device):
        _check(lib().fastpi_gemm_f32(int(ta), int(tb), M, N, K, float(alpha), _ptr(A), A.stride(0), _ptr(B),
                                     B.stride(0), float(beta), _ptr(Cout), Cout.stride(0), ENGINES[engine], st))
    return Cout


def core_svd_f32(K: torch.Tensor, panel: int = 16, parts: int = 0, resident: bool = False, fast: bool = True,
                 single_cta: bool = False):
    """SVD of a square FP32 matrix by the library's core-SVD kernel (block
    one-sided Jacobi) with the given tiling.  K: n x n CUDA tensor (any float
    dtype; copied).  Returns (S numpy float64 descending, U, V float32 CUDA
    tensors with singular vectors as columns, sweeps, kernel ms)."""
    n = int(K.shape[0])
    if K.dim() != 2 or K.shape[1] != n or not K.is_cuda:
        raise ValueError("K must be a square CUDA matrix")
    Kc = K.to(torch.float32).t().contiguous()           # column-major storage of K
    U = torch.empty((n, n), dtype=torch.float32, device=K.device)
    V = torch.empty((n, n), dtype=torch.float32, device=K.device)
    S = np.empty(n, dtype=np.float64)
    sw, ms = C.c_int(), C.c_float()
    flags = (1 if resident else 0) | (0 if fast else 2) | (4 if single_cta else 0)
    st = torch.cuda.current_stream(K.device).cuda_stream
    with torch.cuda.device(K.device):
        _check(lib().fastpi_core_svd_f32(n, _ptr(Kc), _ptr(U), S.ctypes.data, _ptr(V), int(panel), int(parts), flags,
                                         C.byref(sw), C.byref(ms), st))
    # column-major results: the singular vectors are the rows of the row-major views
    return S, U.t(), V.t(), sw.value, ms.value


TUNING_PATH = os.path.join(_HERE, "tuning.txt")


def load_tuning(path: str | None) -> None:
    """Replace the library's tuning table with the file at path (None: the
    built-in defaults)."""
    _check(lib().fastpi_load_tuning(None if path is None else os.fsencode(path)))


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libfastpi.so not built at {path}; run python -m paper_2011_04235_gb300.build")
    lib = C.CDLL(path)
    p, i64, i32, dbl, vp = C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_void_p
    sig = {
        "fastpi_create": ([C.POINTER(p), i64, i64, i64, vp, vp, vp, i32, vp], i32),
        "fastpi_factor": ([p, i64, dbl, i32, i64, i64], i32),
        "fastpi_reorder": ([p, dbl], i32),
        "fastpi_block_svd": ([p, i64, dbl, i32, vp, i64, C.POINTER(i64)], i32),
        "fastpi_create_from_factors": ([C.POINTER(p), i64, i64, i64, vp, vp, i64, vp, i64, i32, i32, vp], i32),
        "fastpi_truncate": ([p, i64], i32),
        "fastpi_factor_batched": ([vp, i32, vp, dbl, i32, i64, i64, i32, vp], i32),
        "fastpi_apply": ([p, vp, i64, i64, vp, i64], i32),
        "fastpi_apply_host": ([p, vp, i64, i64, vp, i64], i32),
        "fastpi_apply_csr": ([p, i64, i64, vp, vp, vp, vp, i64], i32),
        "fastpi_residual": ([p, vp, i64, i64, vp, i64, C.POINTER(dbl)], i32),
        "fastpi_spmm": ([p, vp, i64, i64, vp, i64], i32),
        "fastpi_recon_error": ([p, C.POINTER(dbl)], i32),
        "fastpi_residual_noalloc": ([i64, i64, vp, vp, vp, vp, i64, i64, vp, i64, C.POINTER(dbl), vp], i32),
        "fastpi_gemm_f32": ([i32, i32, i64, i64, i64, C.c_float, vp, i64, vp, i64, C.c_float, vp, i64, i32, vp],
                            i32),
        "fastpi_core_svd_f32": ([i32, vp, vp, vp, vp, i32, i32, i32, C.POINTER(i32), C.POINTER(C.c_float), vp],
                                i32),
        "fastpi_load_tuning": ([C.c_char_p], i32),
        "fastpi_get_rank": ([p, C.POINTER(i64)], i32),
        "fastpi_get_S": ([p, vp], i32),
        "fastpi_get_U": ([p, vp, i64], i32),
        "fastpi_get_V": ([p, vp, i64], i32),
        "fastpi_get_perm": ([p, vp, vp, C.POINTER(i64), C.POINTER(i64)], i32),
        "fastpi_get_blocks": ([p, C.POINTER(i64), vp, vp], i32),
        "fastpi_get_info": ([p, C.POINTER(Info)], i32),
        "fastpi_get_counters": ([C.POINTER(Counters)], i32),
        "fastpi_reset_counters": ([], None),
        "fastpi_last_error": ([p], C.c_char_p),
        "fastpi_destroy": ([p], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _check(st: int, h=None):
    if st != 0:
        msg = lib().fastpi_last_error(h)
        raise FastPIError(st, msg.decode() if msg else "")


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _dense_dev(t, rows: int, name: str, writable: bool = False) -> torch.Tensor:
    """A CUDA float64 matrix with `rows` rows and unit column stride (copied
    to that layout if needed; an output must already have it)."""
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.dim() == 2
            and t.shape[0] == rows):
        raise ValueError(f"{name} must be a 2-D CUDA float64 tensor with {rows} rows")
    if t.stride(1) != 1 or (t.shape[0] > 1 and t.stride(0) < t.shape[1]):
        if writable:
            raise ValueError(f"{name} must be row-major (unit column stride)")
        t = t.contiguous()
    return t


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


class FastPI:
    """A factorization handle.  ``A`` is given in CSR (rowptr int64, col int32,
    val float64), as numpy arrays (host) or CUDA tensors (device)."""

    def __init__(self, m: int, n: int, rowptr, col, val, device="cuda:0", stream=None):
        self.device = torch.device(device)
        self.m, self.n = int(m), int(n)
        on_dev = isinstance(rowptr, torch.Tensor) and rowptr.is_cuda
        if on_dev:
            rp = rowptr.to(torch.int64).contiguous()
            cl = col.to(torch.int32).contiguous()
            vl = val.to(torch.float64).contiguous()
            keep = (rp, cl, vl)
            ptrs = [_ptr(t) for t in keep]
        else:
            rp = np.ascontiguousarray(rowptr, dtype=np.int64)
            cl = np.ascontiguousarray(col, dtype=np.int32)
            vl = np.ascontiguousarray(val, dtype=np.float64)
            keep = (rp, cl, vl)
            ptrs = [a.ctypes.data for a in keep]
        self.nnz = int(cl.numel() if on_dev else cl.size)
        self._h = C.c_void_p()
        with torch.cuda.device(self.device):
            st = stream if stream is not None else _stream_ptr(self.device)
            self._stream = st
            _check(lib().fastpi_create(C.byref(self._h), self.m, self.n, self.nnz, ptrs[0], ptrs[1], ptrs[2],
                                       1 if on_dev else 0, st))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().fastpi_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def factor(self, r: int, k: float, precision="fp64", chunk_row: int = 0, chunk_col: int = 0):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        with torch.cuda.device(self.device):
            _check(lib().fastpi_factor(self._h, int(r), float(k), prec, int(chunk_row), int(chunk_col)), self._h)
        return self

    @classmethod
    def from_factors(cls, S, U: torch.Tensor, V: torch.Tensor, precision="fp64", device="cuda:0", stream=None):
        """A handle that serves applies from given factors (S host array, U and V
        FP64 device tensors, m x r and n x r, original row / column order)."""
        self = cls.__new__(cls)
        self.device = torch.device(device)
        self.m, self.n = int(U.shape[0]), int(V.shape[0])
        self.nnz = 0
        r = int(U.shape[1])
        S = np.ascontiguousarray(S, dtype=np.float64)
        U = U.to(self.device, torch.float64)
        V = V.to(self.device, torch.float64)
        U = U if U.stride(1) == 1 else U.contiguous()
        V = V if V.stride(1) == 1 else V.contiguous()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self._h = C.c_void_p()
        with torch.cuda.device(self.device):
            st = stream if stream is not None else _stream_ptr(self.device)
            self._stream = st
            _check(lib().fastpi_create_from_factors(C.byref(self._h), self.m, self.n, r, S.ctypes.data, _ptr(U),
                                                    max(U.stride(0), 1), _ptr(V), max(V.stride(0), 1), prec, 1,
                                                    st))
        return self

    def save(self, path: str):
        """Store (S, U, V) and the precision as a .npz file (factor reuse)."""
        inf = self.info()
        np.savez(path, S=self.S(), U=self.U().cpu().numpy(), V=self.V().cpu().numpy(),
                 precision=np.int64(inf["precision"]))

    @classmethod
    def load(cls, path: str, device="cuda:0", stream=None):
        d = np.load(path)
        return cls.from_factors(d["S"], torch.from_numpy(d["U"]), torch.from_numpy(d["V"]),
                                precision=int(d["precision"]), device=device, stream=stream)

    def truncate(self, r: int):
        _check(lib().fastpi_truncate(self._h, int(r)), self._h)
        return self

    def reorder(self, k: float):
        """Algorithm 2 alone (perm / blocks / info getters valid afterwards)."""
        with torch.cuda.device(self.device):
            _check(lib().fastpi_reorder(self._h, float(k)), self._h)
        return self

    def block_svd(self, r: int, k: float, precision="fp64") -> np.ndarray:
        """Eq. 1 alone (Algorithm 2, then the SVD of every A11 block): the kept
        block singular values, block by block, descending within a block."""
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        S = C.c_int64()
        cap = max(self.n, 1)
        sig = np.empty(cap, dtype=np.float64)
        with torch.cuda.device(self.device):
            _check(lib().fastpi_block_svd(self._h, int(r), float(k), prec, sig.ctypes.data, cap, C.byref(S)),
                   self._h)
        return sig[:S.value].copy()

    def apply(self, Y: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        Y = _dense_dev(Y, self.m, "Y")
        L = Y.shape[1]
        if out is None:
            Z = torch.empty((self.n, L), dtype=torch.float64, device=Y.device)
        else:
            Z = _dense_dev(out, self.n, "out", writable=True)
            if Z.shape[1] != L:
                raise ValueError(f"out must have {L} columns")
        with torch.cuda.device(self.device):
            _check(lib().fastpi_apply(self._h, _ptr(Y), L, Y.stride(0), _ptr(Z), Z.stride(0)), self._h)
        return Z

    def apply_host(self, Y: np.ndarray) -> np.ndarray:
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        Z = np.empty((self.n, Y.shape[1]), dtype=np.float64)
        with torch.cuda.device(self.device):
            _check(lib().fastpi_apply_host(self._h, Y.ctypes.data, Y.shape[1], Y.shape[1], Z.ctypes.data,
                                           Z.shape[1]), self._h)
        return Z

    def apply_csr(self, L: int, rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor) -> torch.Tensor:
        """Z = A^+ Y for a sparse label matrix Y (m x L, CSR on the device:
        rowptr int64[m+1], col int32 labels strictly increasing per row,
        val float64); the library checks Y and raises FastPIError on a
        malformed one."""
        if not all(isinstance(t, torch.Tensor) and t.is_cuda for t in (rowptr, col, val)):
            raise ValueError("rowptr, col and val must be CUDA tensors")
        if rowptr.numel() != self.m + 1 or col.numel() != val.numel():
            raise ValueError(f"need rowptr of {self.m + 1} entries and col, val of equal length")
        rowptr = rowptr.to(torch.int64).contiguous()
        col = col.to(torch.int32).contiguous()
        val = val.to(torch.float64).contiguous()
        Z = torch.empty((self.n, L), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            _check(lib().fastpi_apply_csr(self._h, int(L), int(col.numel()), _ptr(rowptr), _ptr(col), _ptr(val),
                                          _ptr(Z), L), self._h)
        return Z

    def residual(self, Y: torch.Tensor, Z: torch.Tensor) -> float:
        """||A Z - Y||_F in FP64 (Y: m x L, Z: n x L, CUDA float64)."""
        Y = _dense_dev(Y, self.m, "Y")
        Z = _dense_dev(Z, self.n, "Z")
        if Y.shape[1] != Z.shape[1]:
            raise ValueError("Y and Z must have the same number of columns")
        out = C.c_double()
        with torch.cuda.device(self.device):
            _check(lib().fastpi_residual(self._h, _ptr(Y), Y.shape[1], Y.stride(0), _ptr(Z), Z.stride(0),
                                         C.byref(out)), self._h)
        return out.value

    def spmm(self, X: torch.Tensor) -> torch.Tensor:
        """A X (m x L) for X n x L (CUDA float64)."""
        X = _dense_dev(X, self.n, "X")
        out = torch.empty((self.m, X.shape[1]), dtype=torch.float64, device=X.device)
        with torch.cuda.device(self.device):
            _check(lib().fastpi_spmm(self._h, _ptr(X), X.shape[1], X.stride(0), _ptr(out), out.stride(0)), self._h)
        return out

    def recon_error(self) -> float:
        """|A - U diag(S) V^T|_F / |A|_F from the stored factors (FP64, on the device)."""
        out = C.c_double()
        with torch.cuda.device(self.device):
            _check(lib().fastpi_recon_error(self._h, C.byref(out)), self._h)
        return out.value

    @property
    def rank(self) -> int:
        r = C.c_int64()
        _check(lib().fastpi_get_rank(self._h, C.byref(r)), self._h)
        return r.value

    def S(self) -> np.ndarray:
        s = np.empty(self.rank, dtype=np.float64)
        _check(lib().fastpi_get_S(self._h, s.ctypes.data), self._h)
        return s

    def U(self) -> torch.Tensor:
        r = self.rank
        U = torch.empty((self.m, max(r, 1)), dtype=torch.float64, device=self.device)[:, :r]
        with torch.cuda.device(self.device):
            _check(lib().fastpi_get_U(self._h, _ptr(U), U.stride(0)), self._h)
        return U

    def V(self) -> torch.Tensor:
        r = self.rank
        V = torch.empty((self.n, max(r, 1)), dtype=torch.float64, device=self.device)[:, :r]
        with torch.cuda.device(self.device):
            _check(lib().fastpi_get_V(self._h, _ptr(V), V.stride(0)), self._h)
        return V

    def perm(self):
        ro = np.empty(self.m, dtype=np.int32)
        co = np.empty(self.n, dtype=np.int32)
        m2, n2 = C.c_int64(), C.c_int64()
        with torch.cuda.device(self.device):
            _check(lib().fastpi_get_perm(self._h, ro.ctypes.data, co.ctypes.data, C.byref(m2), C.byref(n2)),
                   self._h)
        return ro, co, m2.value, n2.value

    def blocks(self):
        B = C.c_int64()
        _check(lib().fastpi_get_blocks(self._h, C.byref(B), None, None), self._h)
        ro = np.empty(B.value + 1, dtype=np.int64)
        co = np.empty(B.value + 1, dtype=np.int64)
        _check(lib().fastpi_get_blocks(self._h, C.byref(B), ro.ctypes.data, co.ctypes.data), self._h)
        return ro, co

    def info(self) -> dict:
        inf = Info()
        _check(lib().fastpi_get_info(self._h, C.byref(inf)), self._h)
        return inf.as_dict()
