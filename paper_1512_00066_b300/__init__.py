"""Python binding of ``libstc.so``: generalized sparse contraction on one B300.

Argument marshalling only.  Every step of every call runs in the CUDA library
(``csrc/``); this module passes device pointers of torch tensors, the current
CUDA stream and sizes through the C ABI declared in ``include/stc.h``, and maps
status codes to exceptions.  There is no CPU fallback: if the library cannot be
loaded, or no CUDA device is present, the calls raise.

Memory the library asks for (scratch and results) comes from torch's caching
allocator through the allocator callbacks of ``stc_create``, so results are
ordinary torch tensors.

Algebras (Solomonik & Hoefler, Section 3.1 Table 1 and Section 3.3.2):
``PLUS_TIMES_F32``, ``PLUS_TIMES_F64``, ``MIN_PLUS_I32``, ``MIN_PLUS_F32``,
``OR_AND_BOOL``, ``MULTPATH_I32_F64``.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

PLUS_TIMES_F32, PLUS_TIMES_F64, MIN_PLUS_I32, MIN_PLUS_F32, OR_AND_BOOL, MULTPATH_I32_F64 = range(6)
MIN_PLUS_I32_IDENTITY = 1073741823
ALGEBRA_NAMES = {0: "plus_times_f32", 1: "plus_times_f64", 2: "min_plus_i32", 3: "min_plus_f32",
                 4: "or_and_bool", 5: "multpath_i32_f64"}

STATUS = {0: "STC_OK", 1: "STC_ERR_INVALID_ARG", 2: "STC_ERR_SHAPE", 3: "STC_ERR_UNSORTED",
          4: "STC_ERR_ALGEBRA", 5: "STC_ERR_OOM", 6: "STC_ERR_CUDA", 7: "STC_ERR_NEG_CYCLE",
          8: "STC_ERR_TIMEOUT", 9: "STC_ERR_CAPACITY"}
NOALLOC_BF_MAX_VERTICES = 1 << 20
MLP_INPUTS, MLP_FEAT_STRIDE, MLP_HIDDEN, MLP_NUM_WEIGHTS = 67, 68, 64, 8577

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libstc.so")

# element types: (A, B/X, C/Y) as torch dtypes; multiplicity pairs are 16 raw bytes
_DT = {
    PLUS_TIMES_F32: (torch.float32, torch.float32, torch.float32),
    PLUS_TIMES_F64: (torch.float64, torch.float64, torch.float64),
    MIN_PLUS_I32: (torch.int32, torch.int32, torch.int32),
    MIN_PLUS_F32: (torch.float32, torch.float32, torch.float32),
    OR_AND_BOOL: (torch.uint8, torch.uint8, torch.uint8),
    MULTPATH_I32_F64: (torch.int32, "dsig", "dsig"),
}
DSIG_BYTES = 16


class StcError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({_status_text(status)})")


class _Csr(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("skip_validation", ctypes.c_int32), ("window_cols", ctypes.c_int32),
                ("light_rows", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class _LearnedStats(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("overflow_rows", ctypes.c_int64), ("scratch_entries", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("mean_abs_log2_error", ctypes.c_double),
                ("recomputed_rows", ctypes.c_int64)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_lib_lock = threading.Lock()


def lib():
    """Load libstc.so (building it with nvcc first if it is absent)."""
    global _lib
    with _lib_lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                from . import build as _b
                _b.build()
            L = ctypes.CDLL(LIB_PATH)
            p, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            L.stc_create.argtypes = [ctypes.POINTER(p), _ALLOC_FN, _FREE_FN, p]
            L.stc_create.restype = ctypes.c_int
            L.stc_destroy.argtypes = [p]
            L.stc_free.argtypes = [p, p, p]
            L.stc_status_str.argtypes = [ctypes.c_int]
            L.stc_status_str.restype = ctypes.c_char_p
            L.stc_version.restype = i32
            L.stc_contract_spgemm.argtypes = [p, ctypes.c_int, ctypes.POINTER(_Csr), ctypes.POINTER(_Csr),
                                              ctypes.POINTER(_Csr), ctypes.POINTER(_Opts), p]
            L.stc_contract_spgemm.restype = ctypes.c_int
            L.stc_contract_spgemm_batched.argtypes = [p, ctypes.c_int, i32, ctypes.POINTER(_Csr),
                                                      ctypes.POINTER(_Csr), ctypes.POINTER(_Csr),
                                                      ctypes.POINTER(_Opts), p]
            L.stc_contract_spgemm_batched.restype = ctypes.c_int
            L.stc_contract_spmm.argtypes = [p, ctypes.c_int, ctypes.POINTER(_Csr), p, i64, i32, p, i64, i32, p]
            L.stc_contract_spmm.restype = ctypes.c_int
            L.stc_contract_spmv.argtypes = [p, ctypes.c_int, ctypes.POINTER(_Csr), p, p, i32, p]
            L.stc_contract_spmv.restype = ctypes.c_int
            L.stc_check_device_status.argtypes = [p, p]
            L.stc_check_device_status.restype = ctypes.c_int
            L.stc_bellman_ford.argtypes = [p, ctypes.c_int, ctypes.POINTER(_Csr), i32, p,
                                           ctypes.POINTER(i32), ctypes.POINTER(i64), i32, p]
            L.stc_bellman_ford.restype = ctypes.c_int
            L.stc_set_timing.argtypes = [p, i32]
            L.stc_set_round_driver.argtypes = [p, i32]
            L.stc_autotune_spgemm.argtypes = [p, ctypes.c_int, ctypes.POINTER(_Csr), ctypes.POINTER(_Csr), p, p, p, p,
                                              p]
            L.stc_autotune_spgemm.restype = ctypes.c_int
            L.stc_contract_spgemm_masked.argtypes = [p, ctypes.c_int, ctypes.POINTER(_Csr), ctypes.POINTER(_Csr),
                                                     ctypes.POINTER(_Csr), p, p, p]
            L.stc_contract_spgemm_masked.restype = ctypes.c_int
            L.stc_apsp_path_doubling.argtypes = [p, ctypes.POINTER(_Csr), ctypes.POINTER(_Csr), p, p]
            L.stc_apsp_path_doubling.restype = ctypes.c_int
            L.stc_apsp_tiskin.argtypes = [p, ctypes.POINTER(_Csr), ctypes.POINTER(_Csr), p, p, p]
            L.stc_apsp_tiskin.restype = ctypes.c_int
            L.stc_selftest_barrier.argtypes = [p, i32, i32, p]
            L.stc_selftest_barrier.restype = ctypes.c_int
            L.stc_tune_save.argtypes = [p, ctypes.c_char_p]
            L.stc_tune_save.restype = ctypes.c_int
            L.stc_tune_load.argtypes = [p, ctypes.c_char_p]
            L.stc_tune_load.restype = ctypes.c_int
            L.stc_set_round_driver.restype = ctypes.c_int
            L.stc_set_timing.restype = ctypes.c_int
            L.stc_phase_times.argtypes = [p, ctypes.POINTER(ctypes.c_float), i32]
            L.stc_phase_times.restype = i32
            L.stc_kernel_launches.argtypes = [p]
            L.stc_kernel_launches.restype = i64
            L.stc_mfbc_sssp.argtypes = [p, ctypes.POINTER(_Csr), p, i32, p, p, ctypes.POINTER(i32), p]
            L.stc_mfbc_sssp.restype = ctypes.c_int
            L.stc_mfbc.argtypes = [p, ctypes.POINTER(_Csr), p, i32, i32, p, p]
            L.stc_mfbc.restype = ctypes.c_int
            L.stc_row_features.argtypes = [p, ctypes.POINTER(_Csr), ctypes.POINTER(_Csr), p, p]
            L.stc_row_features.restype = ctypes.c_int
            L.stc_mlp_forward.argtypes = [p, p, p, i64, p, p]
            L.stc_mlp_forward.restype = ctypes.c_int
            L.stc_mlp_forward_tc.argtypes = [p, p, p, i64, p, p]
            L.stc_mlp_forward_tc.restype = ctypes.c_int
            L.stc_mlp_grad.argtypes = [p, p, p, p, p, i64, ctypes.c_float, p, p, p]
            L.stc_mlp_grad.restype = ctypes.c_int
            L.stc_mlp_adam.argtypes = [p, p, p, p, p, i64, ctypes.c_float, p]
            L.stc_mlp_adam.restype = ctypes.c_int
            L.stc_mlp_init.argtypes = [p, ctypes.c_uint64, p]
            L.stc_mlp_init.restype = ctypes.c_int
            L.stc_mlp_train.argtypes = [p, p, p, p, i64, i32, i32, ctypes.c_float, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_float), p]
            L.stc_mlp_train.restype = ctypes.c_int
            L.stc_contract_spgemm_learned.argtypes = [p, ctypes.c_int, ctypes.POINTER(_Csr), ctypes.POINTER(_Csr),
                                                      ctypes.POINTER(_Csr), p, ctypes.c_float,
                                                      ctypes.POINTER(_LearnedStats), ctypes.POINTER(_Opts), p]
            L.stc_contract_spgemm_learned.restype = ctypes.c_int
            L.stc_row_counts.argtypes = [p, ctypes.POINTER(_Csr), ctypes.POINTER(_Csr), p, ctypes.POINTER(_Opts), p]
            L.stc_row_counts.restype = ctypes.c_int
            L.stc_training_rows.argtypes = [p, ctypes.POINTER(_Csr), ctypes.POINTER(_Csr), p, p, p]
            L.stc_training_rows.restype = ctypes.c_int
            L.stc_model_save.argtypes = [ctypes.c_char_p, p, p]
            L.stc_model_save.restype = ctypes.c_int
            L.stc_model_load.argtypes = [ctypes.c_char_p, p, p]
            L.stc_model_load.restype = ctypes.c_int
            L.stc_calibrate_accumulate.argtypes = [p, ctypes.c_int, ctypes.POINTER(ctypes.c_double), p]
            L.stc_calibrate_accumulate.restype = ctypes.c_int
            L.stc_bellman_ford_noalloc.argtypes = [ctypes.c_int, ctypes.POINTER(_Csr), i32, p,
                                                   ctypes.POINTER(i32), p]
            L.stc_bellman_ford_noalloc.restype = ctypes.c_int
            _lib = L
    return _lib


def _status_text(s: int) -> str:
    try:
        return lib().stc_status_str(int(s)).decode()
    except Exception:  # pragma: no cover - library not loadable
        return "?"


def _check(st: int, where: str):
    if st != 0:
        raise StcError(st, where)


def _check_dist(alg: int, G: "DeviceCsr", dist: torch.Tensor, where: str) -> None:
    """Reject a distance buffer the library would write out of bounds or misread.

    The Bellman-Ford kernels write G.nrows elements of the algebra's type (int32
    for MIN_PLUS_I32, fp32 for MIN_PLUS_F32) at dist's first element, so the
    buffer must be a contiguous tensor of that dtype with at least G.nrows
    elements on the device that holds G.  Raised before any device work."""
    want = {MIN_PLUS_I32: torch.int32, MIN_PLUS_F32: torch.float32}.get(alg)
    if want is None:
        raise ValueError(f"{where}: algebra {alg} has no Bellman-Ford (MIN_PLUS_I32 or MIN_PLUS_F32)")
    if not isinstance(dist, torch.Tensor):
        raise ValueError(f"{where}: dist must be a torch tensor")
    if dist.dtype != want:
        raise ValueError(f"{where}: dist has dtype {dist.dtype}, the algebra needs {want}")
    if not dist.is_contiguous():
        raise ValueError(f"{where}: dist must be contiguous")
    if dist.numel() < G.nrows:
        raise ValueError(f"{where}: dist holds {dist.numel()} elements, the graph has {G.nrows} vertices")
    if not dist.is_cuda or dist.device != G.col.device:
        raise ValueError(f"{where}: dist is on {dist.device}, the graph on {G.col.device}")


def _stream_ptr(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


# ----------------------------------------------------------------- device CSR

@dataclass
class DeviceCsr:
    """CSR matrix held in torch tensors on one CUDA device."""
    nrows: int
    ncols: int
    rowptr: torch.Tensor  # int64[nrows+1]
    col: torch.Tensor     # int32[nnz]
    val: Optional[torch.Tensor]  # typed [nnz], or uint8 [nnz, 16] for multiplicity pairs

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    # The C descriptor and its bytes are kept in the instance (_cd, _cb) and dropped
    # whenever a field is assigned, so that batched calls, which marshal thousands
    # of descriptors, read one attribute per matrix.
    def __setattr__(self, name, value):
        object.__setattr__(self, name, value)
        if name in ("nrows", "ncols", "rowptr", "col", "val"):
            self.__dict__.pop("_cd", None)
            self.__dict__.pop("_cb", None)

    def _c(self) -> _Csr:
        """The C descriptor."""
        c = self.__dict__.get("_cd")
        return c if c is not None else self._build_c()[0]

    def _c_bytes(self) -> bytes:
        """The C descriptor's bytes (for building descriptor arrays of batched calls)."""
        b = self.__dict__.get("_cb")
        return b if b is not None else self._build_c()[1]

    def _build_c(self):
        c = _Csr(self.nrows, self.ncols, self.nnz, self.rowptr.data_ptr(), self.col.data_ptr(),
                 self.val.data_ptr() if self.val is not None and self.val.numel() else None)
        b = bytes(c)
        self.__dict__["_cd"] = c
        self.__dict__["_cb"] = b
        return c, b

    @staticmethod
    def from_host(nrows, ncols, rowptr, col, val=None, device="cuda") -> "DeviceCsr":
        rp = torch.from_numpy(np.ascontiguousarray(rowptr, dtype=np.int64)).to(device)
        cl = torch.from_numpy(np.ascontiguousarray(col, dtype=np.int32)).to(device)
        v = None if val is None else values_to_device(val, device)
        return DeviceCsr(int(nrows), int(ncols), rp, cl, v)

    def to_host(self):
        """(rowptr, col, val) as numpy arrays; multiplicity pairs as raw uint8 [nnz, 16]."""
        return (self.rowptr.cpu().numpy(), self.col.cpu().numpy(),
                None if self.val is None else self.val.cpu().numpy())


def values_to_device(val: np.ndarray, device="cuda") -> torch.Tensor:
    a = np.ascontiguousarray(val)
    if a.dtype.names is not None or a.dtype.itemsize == DSIG_BYTES and a.dtype.kind == "V":
        raw = a.view(np.uint8).reshape(-1, DSIG_BYTES)
        return torch.from_numpy(raw.copy()).to(device)
    return torch.from_numpy(a).to(device)


class BatchedResult:
    """The results of one batched call: C_b as DeviceCsr views into the three
    shared allocations, made on first access (the offsets come from the
    descriptors the library filled in)."""

    def __init__(self, alg, C, rp, col, raw):
        nb = len(C)
        desc = np.frombuffer(memoryview(C).cast("B"), dtype=np.int64).reshape(nb, 6)
        self._alg = alg
        self._nrows = desc[:, 0].copy()
        self._ncols = desc[:, 1].copy()
        self._nnz = desc[:, 2].copy()
        self._r0 = (desc[:, 3] - desc[0, 3]) // 8
        self._c0 = (desc[:, 4] - desc[0, 4]) // 4
        self._rp, self._col, self._raw = rp, col, raw
        ct = _DT[alg][2]
        self._vb = DSIG_BYTES if ct == "dsig" else torch.empty(0, dtype=ct).element_size()
        self._cache = {}

    def __len__(self):
        return self._nrows.size

    @property
    def nnz_total(self) -> int:
        return int(self._nnz.sum())

    def __getitem__(self, b):
        if isinstance(b, slice):
            return [self[i] for i in range(*b.indices(len(self)))]
        b = int(b) + (len(self) if b < 0 else 0)
        if not 0 <= b < len(self):
            raise IndexError(b)
        v = self._cache.get(b)
        if v is None:
            nnz, r0, c0, n = int(self._nnz[b]), int(self._r0[b]), int(self._c0[b]), int(self._nrows[b])
            ct = _DT[self._alg][2]
            raw = self._raw[c0 * self._vb: (c0 + nnz) * self._vb]
            val = raw.view(nnz, DSIG_BYTES) if ct == "dsig" else raw.view(ct)
            v = self._cache[b] = DeviceCsr(n, int(self._ncols[b]), self._rp[r0: r0 + n + 1],
                                           self._col[c0: c0 + nnz], val)
        return v

    def __iter__(self):
        for b in range(len(self)):
            yield self[b]


# ----------------------------------------------------------------- handle

class Handle:
    """An stc_handle whose allocations come from torch's caching allocator."""

    def __init__(self, device: Optional[int] = None):
        if not torch.cuda.is_available():
            raise RuntimeError("stc: no CUDA device available (the library has no CPU path)")
        self.device = torch.cuda.current_device() if device is None else device
        self._live = {}
        self._alloc_cb = _ALLOC_FN(self._alloc)
        self._free_cb = _FREE_FN(self._free)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().stc_create(ctypes.byref(h), self._alloc_cb, self._free_cb, None), "stc_create")
        self._h = h

    def _alloc(self, nbytes, ctx, stream):
        try:
            t = torch.empty(int(nbytes), dtype=torch.uint8, device=f"cuda:{self.device}")
        except Exception:
            return None
        ptr = t.data_ptr()
        self._live[ptr] = t
        return ptr

    def _free(self, ptr, ctx, stream):
        self._live.pop(ptr, None)

    def _take(self, ptr: int) -> torch.Tensor:
        return self._live.pop(ptr)

    def close(self):
        if getattr(self, "_h", None):
            lib().stc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- calls

    def spgemm(self, alg: int, A: DeviceCsr, B: DeviceCsr, skip_validation: bool = False,
               window_cols: int = 0, light_rows: int = 0, stream=None) -> DeviceCsr:
        """C = A (x) B (plain two-pass SpGEMM); synchronises the stream once.
        light_rows: 0 tuned/default, -1 none, L > 0 light-row launch for rows with
        fewer than 2^L products (stc_opts.light_rows)."""
        C = _Csr()
        opts = _Opts(1 if skip_validation else 0, int(window_cols), int(light_rows))
        a, b = A._c(), B._c()
        st = lib().stc_contract_spgemm(self._h, alg, ctypes.byref(a), ctypes.byref(b), ctypes.byref(C),
                                       ctypes.byref(opts), _stream_ptr(stream))
        _check(st, "stc_contract_spgemm")
        nnz = int(C.nnz)
        rowptr = self._take(C.rowptr).view(torch.int64)[: C.nrows + 1]
        col = self._take(C.col).view(torch.int32)[:nnz]
        raw = self._take(C.val)
        ct = _DT[alg][2]
        if ct == "dsig":
            val = raw[: nnz * DSIG_BYTES].view(nnz, DSIG_BYTES)
        else:
            val = raw.view(ct)[:nnz]
        return DeviceCsr(int(C.nrows), int(C.ncols), rowptr, col, val)

    def apsp(self, G: DeviceCsr, stream=None):
        """All-pairs shortest distances by path doubling: (P as DeviceCsr, squarings)."""
        P = _Csr()
        sq = ctypes.c_int32(0)
        g = G._c()
        st = lib().stc_apsp_path_doubling(self._h, ctypes.byref(g), ctypes.byref(P), ctypes.byref(sq),
                                          _stream_ptr(stream))
        _check(st, "stc_apsp_path_doubling")
        nnz = int(P.nnz)
        rowptr = self._take(P.rowptr).view(torch.int64)[: P.nrows + 1]
        col = self._take(P.col).view(torch.int32)[:nnz]
        val = self._take(P.val).view(torch.int32)[:nnz]
        return DeviceCsr(int(P.nrows), int(P.ncols), rowptr, col, val), int(sq.value)

    def apsp_tiskin(self, G: DeviceCsr, stream=None):
        """All-pairs shortest distances by Tiskin's path doubling:
        (P as DeviceCsr, rounds, path products evaluated)."""
        P = _Csr()
        rounds = ctypes.c_int32(0)
        prods = ctypes.c_int64(0)
        g = G._c()
        st = lib().stc_apsp_tiskin(self._h, ctypes.byref(g), ctypes.byref(P), ctypes.byref(rounds),
                                   ctypes.byref(prods), _stream_ptr(stream))
        _check(st, "stc_apsp_tiskin")
        nnz = int(P.nnz)
        rowptr = self._take(P.rowptr).view(torch.int64)[: P.nrows + 1]
        col = self._take(P.col).view(torch.int32)[:nnz]
        val = self._take(P.val).view(torch.int32)[:nnz]
        return DeviceCsr(int(P.nrows), int(P.ncols), rowptr, col, val), int(rounds.value), int(prods.value)

    def spgemm_masked(self, alg: int, A: DeviceCsr, B: DeviceCsr, M: DeviceCsr, skip_validation: bool = False,
                      stream=None) -> DeviceCsr:
        """C<M> = A (x) B with the structure of M (identity where no product lands)."""
        ct = _DT[alg][2]
        dev = M.col.device
        if ct == "dsig":
            val = torch.empty((M.nnz, DSIG_BYTES), dtype=torch.uint8, device=dev)
        else:
            val = torch.empty(M.nnz, dtype=ct, device=dev)
        m = _Csr(M.nrows, M.ncols, M.nnz, M.rowptr.data_ptr(), M.col.data_ptr() if M.nnz else None, None)
        opts = _Opts(1 if skip_validation else 0, 0, 0)
        a, b = A._c(), B._c()
        st = lib().stc_contract_spgemm_masked(self._h, alg, ctypes.byref(a), ctypes.byref(b), ctypes.byref(m),
                                              val.data_ptr() if M.nnz else None, ctypes.byref(opts),
                                              _stream_ptr(stream))
        _check(st, "stc_contract_spgemm_masked")
        return DeviceCsr(M.nrows, M.ncols, M.rowptr, M.col, val)

    def spgemm_batched(self, alg: int, As, Bs, skip_validation: bool = False, light_rows: int = 0, stream=None):
        """C_b = A_b (x) B_b for every pair, in one batched call (one synchronisation).

        Returns a sequence of DeviceCsr (BatchedResult) whose tensors are views into
        three shared allocations (row pointers, columns, values); the views are
        made when an element is first read.
        """
        nb = len(As)
        assert nb == len(Bs) and nb > 0
        A = (_Csr * nb).from_buffer_copy(b"".join([a.__dict__.get("_cb") or a._c_bytes() for a in As]))
        B = (_Csr * nb).from_buffer_copy(b"".join([b.__dict__.get("_cb") or b._c_bytes() for b in Bs]))
        C = (_Csr * nb)()
        opts = _Opts(1 if skip_validation else 0, 0, int(light_rows))
        st = lib().stc_contract_spgemm_batched(self._h, alg, nb, A, B, C, ctypes.byref(opts), _stream_ptr(stream))
        _check(st, "stc_contract_spgemm_batched")
        rp = self._take(C[0].rowptr).view(torch.int64)
        col = self._take(C[0].col).view(torch.int32)
        raw = self._take(C[0].val)
        return BatchedResult(alg, C, rp, col, raw)

    def spmm(self, alg: int, A: DeviceCsr, X: torch.Tensor, Y: Optional[torch.Tensor] = None,
             accumulate: bool = False, stream=None) -> torch.Tensor:
        """Y = A (x) X, or Y (+)= A (x) X; X is [A.ncols, ncol] (or a vector)."""
        vec = X.dim() == 1 or (_DT[alg][1] == "dsig" and X.dim() == 2 and X.shape[-1] == DSIG_BYTES
                               and X.dtype == torch.uint8)
        if _DT[alg][1] == "dsig":
            ncol = 1 if vec else X.shape[1]
            ldx = ncol
        else:
            ncol = 1 if X.dim() == 1 else X.shape[1]
            ldx = ncol if X.dim() == 1 else X.stride(0)
        if Y is None:
            if accumulate:
                raise ValueError("accumulate needs Y")
            if _DT[alg][2] == "dsig":
                Y = torch.empty((A.nrows, DSIG_BYTES) if vec else (A.nrows, ncol, DSIG_BYTES),
                                dtype=torch.uint8, device=X.device)
            else:
                Y = torch.empty((A.nrows,) if vec else (A.nrows, ncol), dtype=_DT[alg][2], device=X.device)
        ldy = ncol if (vec or _DT[alg][2] == "dsig") else Y.stride(0)
        a = A._c()
        st = lib().stc_contract_spmm(self._h, alg, ctypes.byref(a), X.data_ptr(), ldx, ncol, Y.data_ptr(),
                                     ldy, 1 if accumulate else 0, _stream_ptr(stream))
        _check(st, "stc_contract_spmm")
        return Y

    def spmv(self, alg: int, A: DeviceCsr, x: torch.Tensor, y: Optional[torch.Tensor] = None,
             accumulate: bool = False, stream=None) -> torch.Tensor:
        return self.spmm(alg, A, x, y, accumulate, stream)

    def check_device_status(self, stream=None):
        _check(lib().stc_check_device_status(self._h, _stream_ptr(stream)), "stc_check_device_status")

    def bellman_ford(self, alg: int, G: DeviceCsr, source: int, persistent=True,
                     dist: Optional[torch.Tensor] = None, stream=None):
        """Shortest distances from `source` over out-edge CSR G; returns (dist, rounds).

        persistent: False / 0 host loop, True / 1 cooperative persistent launch,
        2 or "graph" CUDA graph with a conditional WHILE node."""
        persistent = 2 if persistent == "graph" else int(persistent)
        if dist is None:
            dist = torch.empty(G.nrows, dtype=torch.int32 if alg == MIN_PLUS_I32 else torch.float32,
                               device=G.col.device)
        else:
            _check_dist(alg, G, dist, "bellman_ford")
        rounds = ctypes.c_int32(0)
        relax = ctypes.c_int64(0)
        g = G._c()
        st = lib().stc_bellman_ford(self._h, alg, ctypes.byref(g), int(source), dist.data_ptr(),
                                    ctypes.byref(rounds), ctypes.byref(relax), persistent,
                                    _stream_ptr(stream))
        _check(st, "stc_bellman_ford")
        self.last_relaxations = int(relax.value)
        return dist, int(rounds.value)

    # -------------------------------------------------------------- learned sizing

    def row_features(self, A: DeviceCsr, B: DeviceCsr, stream=None) -> torch.Tensor:
        """Features of every output row of A B: float [A.nrows, 68]."""
        f = torch.empty((A.nrows, MLP_FEAT_STRIDE), dtype=torch.float32, device=A.col.device)
        a, b = A._c(), B._c()
        _check(lib().stc_row_features(self._h, ctypes.byref(a), ctypes.byref(b), f.data_ptr(), _stream_ptr(stream)),
               "stc_row_features")
        return f

    def row_counts(self, A: DeviceCsr, B: DeviceCsr, skip_validation: bool = False, stream=None) -> torch.Tensor:
        """Exact nnz of every row of A B (the symbolic phase alone): int64 [A.nrows]."""
        c = torch.empty(A.nrows, dtype=torch.int64, device=A.col.device)
        opts = _Opts(1 if skip_validation else 0, 0, 0)
        a, b = A._c(), B._c()
        _check(lib().stc_row_counts(self._h, ctypes.byref(a), ctypes.byref(b), c.data_ptr(), ctypes.byref(opts),
                                    _stream_ptr(stream)), "stc_row_counts")
        return c

    def training_rows_of(self, A: DeviceCsr, B: DeviceCsr, stream=None):
        """(feat [A.nrows, 68], target [A.nrows]) of the product A B, from stc_training_rows."""
        f = torch.empty((A.nrows, MLP_FEAT_STRIDE), dtype=torch.float32, device=A.col.device)
        t = torch.empty(A.nrows, dtype=torch.float32, device=A.col.device)
        a, b = A._c(), B._c()
        _check(lib().stc_training_rows(self._h, ctypes.byref(a), ctypes.byref(b), f.data_ptr(), t.data_ptr(),
                                       _stream_ptr(stream)), "stc_training_rows")
        return f, t

    def mlp_forward(self, weights: torch.Tensor, feat: torch.Tensor, stream=None) -> torch.Tensor:
        y = torch.empty(feat.shape[0], dtype=torch.float32, device=feat.device)
        _check(lib().stc_mlp_forward(self._h, weights.data_ptr(), feat.data_ptr(), feat.shape[0], y.data_ptr(),
                                     _stream_ptr(stream)), "stc_mlp_forward")
        return y

    def mlp_forward_tc(self, weights: torch.Tensor, feat: torch.Tensor, stream=None) -> torch.Tensor:
        """The model on the tensor cores (tcgen05); raises StcError on a device
        timeout (synchronises the stream)."""
        y = torch.empty(feat.shape[0], dtype=torch.float32, device=feat.device)
        _check(lib().stc_mlp_forward_tc(self._h, weights.data_ptr(), feat.data_ptr(), feat.shape[0], y.data_ptr(),
                                        _stream_ptr(stream)), "stc_mlp_forward_tc")
        self.check_device_status(stream)
        return y

    def mlp_grad(self, weights, feat, target, idx=None, scale=None, stream=None):
        """(gradient, sum of squared errors) of mean-squared error over the rows."""
        n = feat.shape[0] if idx is None else idx.numel()
        g = torch.zeros(MLP_NUM_WEIGHTS, dtype=torch.float32, device=feat.device)
        loss = torch.zeros(1, dtype=torch.float32, device=feat.device)
        _check(lib().stc_mlp_grad(self._h, weights.data_ptr(), feat.data_ptr(), target.data_ptr(),
                                  None if idx is None else idx.data_ptr(), n, float(scale or n), g.data_ptr(),
                                  loss.data_ptr(), _stream_ptr(stream)), "stc_mlp_grad")
        return g, loss

    def mlp_train(self, weights, feat, target, batch=4096, epochs=10, lr=1e-3, seed=0, stream=None):
        """Train `weights` in place; returns the mean loss of every epoch."""
        losses = (ctypes.c_float * max(epochs, 1))()
        _check(lib().stc_mlp_train(self._h, weights.data_ptr(), feat.data_ptr(), target.data_ptr(), feat.shape[0],
                                   int(batch), int(epochs), float(lr), int(seed), losses, _stream_ptr(stream)),
               "stc_mlp_train")
        return [float(losses[i]) for i in range(epochs)]

    def spgemm_learned(self, alg: int, A: DeviceCsr, B: DeviceCsr, weights: Optional[torch.Tensor] = None,
                       margin: float = 0.25, skip_validation: bool = False, stream=None):
        """Single-pass SpGEMM sized by the model (or by the upper bound): (C, stats)."""
        C = _Csr()
        st_ = _LearnedStats()
        opts = _Opts(1 if skip_validation else 0, 0)
        a, b = A._c(), B._c()
        st = lib().stc_contract_spgemm_learned(self._h, alg, ctypes.byref(a), ctypes.byref(b), ctypes.byref(C),
                                               None if weights is None else weights.data_ptr(), float(margin),
                                               ctypes.byref(st_), ctypes.byref(opts), _stream_ptr(stream))
        _check(st, "stc_contract_spgemm_learned")
        nnz = int(C.nnz)
        rowptr = self._take(C.rowptr).view(torch.int64)[: C.nrows + 1]
        col = self._take(C.col).view(torch.int32)[:nnz]
        raw = self._take(C.val)
        ct = _DT[alg][2]
        val = raw[: nnz * DSIG_BYTES].view(nnz, DSIG_BYTES) if ct == "dsig" else raw.view(ct)[:nnz]
        stats = {f: getattr(st_, f) for f, _ in _LearnedStats._fields_}
        return DeviceCsr(int(C.nrows), int(C.ncols), rowptr, col, val), stats

    def mfbc_sssp(self, G: DeviceCsr, sources, stream=None):
        """(d [n, S] int32, sigma [n, S] fp64, rounds) from up to 256 sources."""
        src = np.ascontiguousarray(sources, dtype=np.int32)
        S = int(src.size)
        d = torch.empty((G.nrows, S), dtype=torch.int32, device=G.col.device)
        sig = torch.empty((G.nrows, S), dtype=torch.float64, device=G.col.device)
        rounds = ctypes.c_int32(0)
        g = G._c()
        st = lib().stc_mfbc_sssp(self._h, ctypes.byref(g), src.ctypes.data_as(ctypes.c_void_p), S,
                                 d.data_ptr(), sig.data_ptr(), ctypes.byref(rounds), _stream_ptr(stream))
        _check(st, "stc_mfbc_sssp")
        return d, sig, int(rounds.value)

    def mfbc(self, G: DeviceCsr, sources, batch: int = 256, bc: Optional[torch.Tensor] = None,
             stream=None) -> torch.Tensor:
        """Betweenness centrality summed over `sources` (host ids), batches of `batch`."""
        src = np.ascontiguousarray(sources, dtype=np.int32)
        if bc is None:
            bc = torch.empty(G.nrows, dtype=torch.float64, device=G.col.device)
        g = G._c()
        st = lib().stc_mfbc(self._h, ctypes.byref(g), src.ctypes.data_as(ctypes.c_void_p), int(src.size),
                            int(batch), bc.data_ptr(), _stream_ptr(stream))
        _check(st, "stc_mfbc")
        return bc

    def autotune_spgemm(self, alg: int, A: DeviceCsr, B: DeviceCsr, stream=None) -> dict:
        """Time the candidate light-row thresholds on C = A (x) B and cache the best
        for this algebra and output width: {"best": L, "candidates": {L: ms}}."""
        best = ctypes.c_int32(0)
        n = ctypes.c_int32(0)
        cand = (ctypes.c_int32 * 8)()
        ms = (ctypes.c_float * 8)()
        a, b = A._c(), B._c()
        st = lib().stc_autotune_spgemm(self._h, alg, ctypes.byref(a), ctypes.byref(b), ctypes.byref(best), cand,
                                       ms, ctypes.byref(n), _stream_ptr(stream))
        _check(st, "stc_autotune_spgemm")
        return {"best": int(best.value), "candidates": {int(cand[i]): float(ms[i]) for i in range(n.value)}}

    def selftest_barrier(self, missing: int, spin_limit: int = 4096, stream=None) -> int:
        """Status of the bounded grid barrier with `missing` blocks that never arrive
        (0: passes; 1: gives up after spin_limit polls with STC_ERR_TIMEOUT)."""
        return int(lib().stc_selftest_barrier(self._h, int(missing), int(spin_limit), _stream_ptr(stream)))

    def tune_save(self, path: str):
        _check(lib().stc_tune_save(self._h, str(path).encode()), "stc_tune_save")

    def tune_load(self, path: str):
        _check(lib().stc_tune_load(self._h, str(path).encode()), "stc_tune_load")

    def set_round_driver(self, driver: str = "graph"):
        """Round loops of mfbc / mfbc_sssp: "graph" (one CUDA graph launch per
        batch, conditional WHILE nodes) or "host" (host-driven rounds)."""
        code = {"host": 0, "graph": 1}[driver]
        _check(lib().stc_set_round_driver(self._h, code), "stc_set_round_driver")

    # -------------------------------------------------------------- instrumentation

    def calibrate_accumulate(self, alg: int, stream=None) -> float:
        """Products per second the numeric pass's shared-memory accumulator absorbs
        on this device (stc_calibrate_accumulate)."""
        r = ctypes.c_double(0.0)
        _check(lib().stc_calibrate_accumulate(self._h, alg, ctypes.byref(r), _stream_ptr(stream)),
               "stc_calibrate_accumulate")
        return float(r.value)

    def set_timing(self, enable: bool = True):
        _check(lib().stc_set_timing(self._h, 1 if enable else 0), "stc_set_timing")

    def phase_times(self):
        """Durations (ms) of the phases of the last timed call (synchronises)."""
        buf = (ctypes.c_float * 8)()
        n = lib().stc_phase_times(self._h, buf, 8)
        return [float(buf[i]) for i in range(n)]

    def kernel_launches(self) -> int:
        return int(lib().stc_kernel_launches(self._h))


def bellman_ford_noalloc(alg: int, G: DeviceCsr, source: int, dist: torch.Tensor, stream=None) -> int:
    """Allocation-free Bellman-Ford (stc_bellman_ford_noalloc) into the caller's `dist`.

    For callers that must not allocate device memory during the call: the
    library's working memory is a fixed array compiled into it.  Returns the
    number of rounds; raises StcError (STC_ERR_CAPACITY) above
    NOALLOC_BF_MAX_VERTICES vertices.  `dist` must be a contiguous tensor of the
    algebra's type with at least G.nrows elements on G's device (ValueError
    otherwise, before any device work).
    """
    _check_dist(alg, G, dist, "bellman_ford_noalloc")
    rounds = ctypes.c_int32(0)
    g = G._c()
    st = lib().stc_bellman_ford_noalloc(alg, ctypes.byref(g), int(source), dist.data_ptr(),
                                        ctypes.byref(rounds), _stream_ptr(stream))
    _check(st, "stc_bellman_ford_noalloc")
    return int(rounds.value)


def mlp_init(seed: int = 0, device="cuda", stream=None) -> torch.Tensor:
    """New fp32 weight vector (He-normal layers, zero biases) on the device."""
    w = torch.empty(MLP_NUM_WEIGHTS, dtype=torch.float32, device=device)
    _check(lib().stc_mlp_init(w.data_ptr(), int(seed), _stream_ptr(stream)), "stc_mlp_init")
    return w


def training_rows(H: "Handle", pairs):
    """Features and exact targets log2(1 + nnz(C_i)) for every row of every (A, B)
    pair (DeviceCsr), both computed by the library (stc_training_rows):
    (feat [N, 68], target [N])."""
    feats, targets = [], []
    for A, B in pairs:
        f, t = H.training_rows_of(A, B)
        feats.append(f)
        targets.append(t)
    return torch.cat(feats), torch.cat(targets)


def model_save(path: str, weights: torch.Tensor, stream=None) -> None:
    """Write the model's weights (device fp32 [MLP_NUM_WEIGHTS]) to a file (stc_model_save)."""
    if weights.dtype != torch.float32 or weights.numel() != MLP_NUM_WEIGHTS or not weights.is_contiguous():
        raise ValueError(f"weights must be a contiguous float32 tensor of {MLP_NUM_WEIGHTS} values")
    _check(lib().stc_model_save(str(path).encode(), weights.data_ptr(), _stream_ptr(stream)), "stc_model_save")


def model_load(path: str, device="cuda", stream=None) -> torch.Tensor:
    """Read a model file written by model_save into a new device tensor (stc_model_load)."""
    w = torch.empty(MLP_NUM_WEIGHTS, dtype=torch.float32, device=device)
    _check(lib().stc_model_load(str(path).encode(), w.data_ptr(), _stream_ptr(stream)), "stc_model_load")
    return w


_default = {}


def handle() -> Handle:
    """Process-wide handle for the current device."""
    dev = torch.cuda.current_device()
    h = _default.get(dev)
    if h is None:
        h = _default[dev] = Handle(dev)
    return h


def version() -> int:
    return int(lib().stc_version())
