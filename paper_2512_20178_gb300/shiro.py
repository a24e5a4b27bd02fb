"""Python binding of libshiro (argument marshalling only; every step runs in the CUDA library).

The C entry points keep their names (``shiro_plan_create``, ``shiro_pack``, ``shiro_spmm`` ...).
PyTorch supplies device memory (workspace, packed buffers, outputs) and the current stream.
There is no fallback: if the compiled library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libshiro.so")

SHIRO_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "BAD_CSR", 3: "INSUFFICIENT_WORKSPACE",
                4: "UNSUPPORTED", 5: "CUDA", 6: "DEVICE_TIMEOUT"}
SHIRO_F32, SHIRO_BF16, SHIRO_F64 = 0, 1, 2
SHIRO_PLAN_LOCAL_DIAG = 0x1
SHIRO_PLAN_DIAG_ONLY = 0x2
SHIRO_PLAN_TRANSPOSE = 0x4
SHIRO_SPMM_ACCUMULATE = 0x1
SHIRO_NOALLOC_SCRATCH_BYTES = 16 << 20

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32
_sz = ctypes.c_size_t


class shiro_csr(ctypes.Structure):
    _fields_ = [("M", _i64), ("K", _i64), ("nnz", _i64), ("rowptr", _vp), ("col", _vp),
                ("val", _vp), ("vdt", ctypes.c_int)]


class shiro_partition(ctypes.Structure):
    _fields_ = [("P_r", _i32), ("P_c", _i32), ("row_bounds", _vp), ("col_bounds", _vp),
                ("flags", _u32)]


class shiro_opts(ctypes.Structure):
    _fields_ = [("long_row_nnz", _i32), ("chunk_nnz", _i32), ("group_nnz", _i32),
                ("group_rows", _i32), ("warps_per_cta", _i32), ("persistent", _i32),
                ("pipeline", _i32), ("stage_rows", _i32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class shiro_plan_info(ctypes.Structure):
    _fields_ = [("M", _i64), ("K", _i64), ("nnz", _i64), ("P_r", _i32), ("P_c", _i32),
                ("n_tiles", _i32), ("flags", _u32), ("vdt", ctypes.c_int),
                ("total_cols", _i64), ("packed_rows", _i64), ("n_items", _i64),
                ("n_long_rows", _i64), ("n_chunks", _i64), ("workspace_used", _sz),
                ("opts", shiro_opts)]


_P = ctypes.POINTER
# (name, restype, argtypes) of every entry point in include/shiro.h.
SIGNATURES = [
    ("shiro_plan_workspace", ctypes.c_int, [_P(shiro_csr), _P(shiro_partition), _P(shiro_opts), _P(_sz)]),
    ("shiro_plan_create", ctypes.c_int, [_P(shiro_csr), _P(shiro_partition), _P(shiro_opts), _vp, _sz, _vp, _P(_vp)]),
    ("shiro_plan_destroy", None, [_vp]),
    ("shiro_plan_query", ctypes.c_int, [_vp, _P(shiro_plan_info)]),
    ("shiro_plan_tile_stats", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    ("shiro_plan_volumes", ctypes.c_int, [_vp, _i32, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]),
    ("shiro_plan_joint", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    ("shiro_plan_joint_weighted", ctypes.c_int, [_vp, _vp, _vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp]),
    ("shiro_plan_row_based", ctypes.c_int, [_vp, _vp, _vp, _vp]),
    ("shiro_joint_split_sizes", ctypes.c_int, [_vp, _vp, _P(_i64), _P(_i64), _P(_i64)]),
    ("shiro_joint_split", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("shiro_plan_export", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    ("shiro_plan_export_transpose", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    ("shiro_plan_update_values", ctypes.c_int, [_vp, _vp, _vp]),
    ("shiro_plan_check", ctypes.c_int, [_vp, _vp]),
    ("shiro_plan_reschedule", ctypes.c_int, [_vp, _P(shiro_opts), _vp]),
    ("shiro_pack", ctypes.c_int, [_vp, _vp, _i64, _i32, ctypes.c_int, _vp, _i64, _vp]),
    ("shiro_spmm_scratch", ctypes.c_int, [_vp, _i32, ctypes.c_int, _P(_sz)]),
    ("shiro_spmm", ctypes.c_int, [_vp, _vp, _i64, _vp, _i64, _i32, ctypes.c_int, _vp, _i64, _u32, _vp, _sz, _vp]),
    ("shiro_pack_spmm", ctypes.c_int, [_vp, _vp, _i64, _i32, ctypes.c_int, _vp, _i64, _vp, _i64, _u32, _vp, _sz, _vp]),
    ("shiro_spmm_noalloc", ctypes.c_int, [_vp, _vp, _i64, _vp, _i64, _i32, ctypes.c_int, _vp, _i64, _u32, _vp]),
    ("shiro_sddmm", ctypes.c_int, [_vp, _vp, _i64, _vp, _i64, _vp, _i64, _i32, ctypes.c_int, _vp, _vp]),
    ("shiro_spmm_backward", ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, _i64, _vp, _i64, _i32, ctypes.c_int, _vp, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    ("shiro_batch_workspace", ctypes.c_int, [_i32, _P(shiro_csr), _P(shiro_opts), _P(_sz)]),
    ("shiro_batch_plan_create", ctypes.c_int, [_i32, _P(shiro_csr), _P(shiro_opts), _vp, _sz, _vp, _P(_vp)]),
    ("shiro_autotune", ctypes.c_int, [_vp, _vp, _i64, _vp, _i64, _i32, ctypes.c_int, _vp, _i64, _vp, _sz, _i32, _vp, _P(shiro_opts)]),
    ("shiro_set_device", ctypes.c_int, [_i32]),
    ("shiro_default_opts", None, [_P(shiro_opts)]),
    ("shiro_last_error", ctypes.c_char_p, []),
    ("shiro_version", _i32, []),
]

_lib = None


def lib():
    """The loaded libshiro (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libshiro.so not built at {LIB_PATH}; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class ShiroError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = lib().shiro_last_error().decode(errors="replace")
        super().__init__(f"{where}: SHIRO_ERR_{STATUS_NAMES.get(status, status)}: {msg}")


def check(status, where):
    if status != SHIRO_OK:
        raise ShiroError(status, where)


# Thin wrappers with the C names (status-checked).
def _wrap(name):
    def f(*args):
        fn = getattr(lib(), name)
        r = fn(*args)
        if fn.restype is ctypes.c_int:
            check(r, name)
        return r
    f.__name__ = name
    return f


for _name, _res, _args in SIGNATURES:
    globals()[_name] = _wrap(_name)


# ---------------------------------------------------------------------------------------------
# torch-facing convenience layer (still only marshalling)

_DT = {torch.float32: SHIRO_F32, torch.bfloat16: SHIRO_BF16, torch.float64: SHIRO_F64}
_ACC = {torch.float32: torch.float32, torch.bfloat16: torch.float32, torch.float64: torch.float64}


def dtype_code(t: torch.dtype) -> int:
    if t not in _DT:
        raise TypeError(f"unsupported dtype {t}")
    return _DT[t]


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _ensure_device(dev: torch.device):
    idx = dev.index if dev.index is not None else torch.cuda.current_device()
    shiro_set_device(_i32(idx))


def make_opts(**kw) -> shiro_opts:
    o = shiro_opts()
    lib().shiro_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


def _csr_struct(rowptr, col, val, M, K):
    if rowptr.dtype != torch.int64 or col.dtype != torch.int32:
        raise TypeError("rowptr must be int64 and col int32")
    if val.dtype not in (torch.float32, torch.float64):
        raise TypeError("values must be float32 or float64")
    for t in (rowptr, col, val):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("CSR arrays must be contiguous CUDA tensors")
    return shiro_csr(int(M), int(K), int(col.numel()), rowptr.data_ptr(), col.data_ptr(),
                     val.data_ptr(), dtype_code(val.dtype))


class Plan:
    """A plan (tile split, Cols sets, remap, schedule) living in a torch-allocated workspace."""

    def __init__(self, handle, workspace, keep, device, vdt):
        self.handle = ctypes.c_void_p(handle)
        self.workspace = workspace
        self._keep = keep
        self.device = device
        self.vdt = vdt
        self.refresh_info()

    @classmethod
    def create(cls, rowptr, col, val, M, K, P_r=1, P_c=1, row_bounds=None, col_bounds=None,
               flags=0, opts=None, stream=None):
        dev = rowptr.device
        _ensure_device(dev)
        A = _csr_struct(rowptr, col, val, M, K)
        rb = None if row_bounds is None else (ctypes.c_int64 * (P_r + 1))(*[int(x) for x in row_bounds])
        cb = None if col_bounds is None else (ctypes.c_int64 * (P_c + 1))(*[int(x) for x in col_bounds])
        part = shiro_partition(P_r, P_c, ctypes.cast(rb, _vp) if rb is not None else None,
                               ctypes.cast(cb, _vp) if cb is not None else None, flags)
        o = opts if opts is not None else make_opts()
        nbytes = _sz(0)
        shiro_plan_workspace(ctypes.byref(A), ctypes.byref(part), ctypes.byref(o), ctypes.byref(nbytes))
        ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=dev)
        h = _vp()
        shiro_plan_create(ctypes.byref(A), ctypes.byref(part), ctypes.byref(o), _ptr(ws),
                          ws.numel(), _stream(stream), ctypes.byref(h))
        return cls(h.value, ws, (rowptr, col, val), dev, val.dtype)

    @classmethod
    def create_batch(cls, graphs, opts=None, stream=None):
        """graphs: list of (rowptr, col, val, M, K) CUDA tensors; one DIAG_ONLY tile per graph."""
        dev = graphs[0][0].device
        _ensure_device(dev)
        arr = (shiro_csr * len(graphs))(*[_csr_struct(*g) for g in graphs])
        o = opts if opts is not None else make_opts()
        nbytes = _sz(0)
        shiro_batch_workspace(len(graphs), arr, ctypes.byref(o), ctypes.byref(nbytes))
        ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=dev)
        h = _vp()
        shiro_batch_plan_create(len(graphs), arr, ctypes.byref(o), _ptr(ws), ws.numel(),
                                _stream(stream), ctypes.byref(h))
        return cls(h.value, ws, None, dev, graphs[0][2].dtype)

    def refresh_info(self):
        info = shiro_plan_info()
        shiro_plan_query(self.handle, ctypes.byref(info))
        self.info = info
        return info

    def close(self):
        if self.handle is not None and self.handle.value:
            lib().shiro_plan_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- queries ----
    def tile_stats(self):
        T = self.info.n_tiles
        out = {k: torch.zeros(T + (1 if k.endswith("ptr") else 0), dtype=torch.int64)
               for k in ("tile_nnz", "tile_nrows", "tile_ncols", "tile_cols_ptr", "pack_ptr")}
        shiro_plan_tile_stats(self.handle, *[_ptr(out[k]) for k in
                                             ("tile_nnz", "tile_nrows", "tile_ncols", "tile_cols_ptr", "pack_ptr")])
        return out

    def volumes(self, N, dtype=torch.float32, c_dtype=None):
        """(V_block, V_col, V_row) per tile in bytes (Eq. 1-3) for B stored as ``dtype`` and
        partial C rows as ``c_dtype`` (default: the accumulator type, FP64 for FP64 B, else
        FP32)."""
        if c_dtype is None:
            c_dtype = torch.float64 if dtype == torch.float64 else torch.float32
        T = self.info.n_tiles
        vb, vc, vr = (torch.zeros(T, dtype=torch.int64) for _ in range(3))
        shiro_plan_volumes(self.handle, int(N), dtype_code(dtype), dtype_code(c_dtype), _ptr(vb),
                           _ptr(vc), _ptr(vr))
        return vb, vc, vr

    def joint(self, stream=None):
        """Per-tile minimum vertex cover (joint row-column strategy) and the side of every nonzero."""
        T, n = self.info.n_tiles, self.info.nnz
        mu, cr, cc = (torch.zeros(T, dtype=torch.int64) for _ in range(3))
        side = torch.zeros(max(n, 1), dtype=torch.uint8)
        shiro_plan_joint(self.handle, _ptr(mu), _ptr(cr), _ptr(cc), _ptr(side), _stream(stream))
        return {"mu": mu, "cover_rows": cr, "cover_cols": cc, "row_based": side[:n]}

    def joint_weighted(self, w_row=1, w_col=1, stream=None):
        """Per-tile minimum weighted vertex cover (Sec. 5.3.3 min cut, Dinic).  w_row / w_col are
        one cost for every row / column, or per-vertex int64 arrays of M / K entries."""
        T, n = self.info.n_tiles, self.info.nnz
        cost, cr, cc = (torch.zeros(T, dtype=torch.int64) for _ in range(3))
        side = torch.zeros(max(n, 1), dtype=torch.uint8)

        def arr(w, size):
            if isinstance(w, int):
                return None, w
            t = torch.as_tensor(w, dtype=torch.int64).contiguous().cpu()
            if t.numel() != size:
                raise ValueError(f"expected {size} costs, got {t.numel()}")
            return t, 0

        wr, wr_all = arr(w_row, self.info.M)
        wc, wc_all = arr(w_col, self.info.K)
        shiro_plan_joint_weighted(self.handle, _ptr(wr) if wr is not None else None,
                                  _ptr(wc) if wc is not None else None, wr_all, wc_all,
                                  _ptr(cost), _ptr(cr), _ptr(cc), _ptr(side), _stream(stream))
        return {"cost": cost, "cover_rows": cr, "cover_cols": cc, "row_based": side[:n]}

    def row_based(self, stream=None):
        """Row-based strategy (Eq. 3): |Rows| per communicated tile and the side of every nonzero."""
        T, n = self.info.n_tiles, self.info.nnz
        rows = torch.zeros(T, dtype=torch.int64)
        side = torch.zeros(max(n, 1), dtype=torch.uint8)
        shiro_plan_row_based(self.handle, _ptr(rows), _ptr(side), _stream(stream))
        return {"rows": rows, "row_based": side[:n]}

    def export(self, stream=None):
        i = self.info
        d = self.device
        cols = torch.empty(max(i.total_cols, 1), dtype=torch.int32, device=d)
        src = torch.empty(max(i.packed_rows, 1), dtype=torch.int32, device=d)
        cl = torch.empty(max(i.nnz, 1), dtype=torch.int32, device=d)
        rm = torch.empty(max(i.nnz, 1), dtype=torch.int32, device=d)
        shiro_plan_export(self.handle, _ptr(cols), _ptr(src), _ptr(cl), _ptr(rm), _stream(stream))
        return {"cols_sorted": cols[: i.total_cols], "pack_src": src[: i.packed_rows],
                "colidx_local": cl[: i.nnz], "remap": rm[: i.nnz]}

    def export_transpose(self, stream=None):
        i = self.info
        d = self.device
        rp = torch.empty(i.M + 1, dtype=torch.int64, device=d)
        col = torch.empty(max(i.nnz, 1), dtype=torch.int32, device=d)
        perm = torch.empty(max(i.nnz, 1), dtype=torch.int64, device=d)
        shiro_plan_export_transpose(self.handle, _ptr(rp), _ptr(col), _ptr(perm), _stream(stream))
        return rp, col[: i.nnz], perm[: i.nnz]

    def update_values(self, val, stream=None):
        shiro_plan_update_values(self.handle, _ptr(val), _stream(stream))

    def check(self, stream=None):
        shiro_plan_check(self.handle, _stream(stream))

    def reschedule(self, **kw):
        o = self.info.opts
        o2 = make_opts(**{**o.as_dict(), **kw})
        shiro_plan_reschedule(self.handle, ctypes.byref(o2), _stream(None))
        self.refresh_info()

    # ---- compute ----
    def scratch_bytes(self, N, dtype):
        n = _sz(0)
        shiro_spmm_scratch(self.handle, int(N), dtype_code(dtype), ctypes.byref(n))
        return n.value

    def new_scratch(self, N, dtype):
        n = self.scratch_bytes(N, dtype)
        return torch.empty(max(n, 1), dtype=torch.uint8, device=self.device) if n else None

    def pack(self, B, out=None, stream=None):
        N = B.shape[1]
        if out is None:
            out = torch.empty((self.info.packed_rows, N), dtype=B.dtype, device=B.device)
        shiro_pack(self.handle, _ptr(B), B.stride(0), N, dtype_code(B.dtype), _ptr(out),
                   out.stride(0) if out.dim() == 2 else N, _stream(stream))
        return out

    def spmm(self, Bpack, B=None, out=None, accumulate=False, scratch=None, N=None, stream=None):
        dt = Bpack.dtype
        N = Bpack.shape[1] if N is None else N
        if out is None:
            out = torch.empty((self.info.M, N), dtype=_ACC[dt], device=Bpack.device)
        if scratch is None:
            scratch = self.new_scratch(N, dt)
        sb = scratch.numel() if scratch is not None else 0
        ldb = B.stride(0) if B is not None else N
        shiro_spmm(self.handle, _ptr(Bpack), Bpack.stride(0) if Bpack.dim() == 2 else N,
                   _ptr(B), ldb, N, dtype_code(dt), _ptr(out), out.stride(0),
                   SHIRO_SPMM_ACCUMULATE if accumulate else 0, _ptr(scratch), sb, _stream(stream))
        return out

    def pack_spmm(self, B, Bpack=None, out=None, accumulate=False, scratch=None, stream=None):
        """Pack and SpMM in one call (shiro_pack_spmm): fills Bpack with B's packed rows and
        returns C = A B, bit-identical to pack() then spmm()."""
        dt = B.dtype
        N = B.shape[1]
        if Bpack is None:
            Bpack = torch.empty((self.info.packed_rows, N), dtype=dt, device=B.device)
        if out is None:
            out = torch.empty((self.info.M, N), dtype=_ACC[dt], device=B.device)
        if scratch is None:
            scratch = self.new_scratch(N, dt)
        sb = scratch.numel() if scratch is not None else 0
        shiro_pack_spmm(self.handle, _ptr(B), B.stride(0), N, dtype_code(dt), _ptr(Bpack),
                        Bpack.stride(0) if Bpack.dim() == 2 else N, _ptr(out), out.stride(0),
                        SHIRO_SPMM_ACCUMULATE if accumulate else 0, _ptr(scratch), sb,
                        _stream(stream))
        return out

    def sddmm(self, dC, Bpack, B=None, out=None, stream=None):
        N = dC.shape[1]
        if out is None:
            out = torch.empty(self.info.nnz, dtype=_ACC[dC.dtype], device=dC.device)
        ldb = B.stride(0) if B is not None else N
        shiro_sddmm(self.handle, _ptr(dC), dC.stride(0), _ptr(Bpack),
                    Bpack.stride(0) if Bpack.dim() == 2 else N, _ptr(B), ldb, N,
                    dtype_code(dC.dtype), _ptr(out), _stream(stream))
        return out

    def autotune(self, Bpack, B=None, C=None, scratch=None, reps=3, stream=None):
        dt = Bpack.dtype
        N = Bpack.shape[1]
        if C is None:
            C = torch.empty((self.info.M, N), dtype=_ACC[dt], device=Bpack.device)
        if scratch is None:
            # Room for the smallest candidate chunk (256 nonzeros) with every row split.
            n = max(self.scratch_bytes(N, dt), 1)
            scratch = torch.empty(max(4 * n, 1 << 20), dtype=torch.uint8, device=Bpack.device)
        best = shiro_opts()
        ldb = B.stride(0) if B is not None else N
        shiro_autotune(self.handle, _ptr(Bpack), Bpack.stride(0), _ptr(B), ldb, N,
                       dtype_code(dt), _ptr(C), C.stride(0), _ptr(scratch), scratch.numel(),
                       int(reps), _stream(stream), ctypes.byref(best))
        self.refresh_info()
        return best.as_dict()


def spmm_backward(plan: Plan, planT: Plan, dC, Bpack, B=None, want_dB=True, want_dA=True,
                  scratch=None, stream=None, dCpack=None, dB=None, dA=None):
    """dB = A^T dC (through planT) and dA on A's pattern, in one C call (one launch for rows of
    256 or 512 bytes when B is given).  dCpack, dB and dA may be passed preallocated."""
    N = dC.shape[1]
    dev = dC.device
    acc = _ACC[dC.dtype]
    if want_dB and dCpack is None:
        dCpack = torch.empty((planT.info.packed_rows, N), dtype=dC.dtype, device=dev)
    if want_dB and dB is None:
        dB = torch.empty((planT.info.M, N), dtype=acc, device=dev)
    if want_dA and dA is None:
        dA = torch.empty(plan.info.nnz, dtype=acc, device=dev)
    if not want_dB:
        dCpack = dB = None
    if not want_dA:
        dA = None
    if scratch is None and want_dB:
        scratch = planT.new_scratch(N, dC.dtype)
    sb = scratch.numel() if scratch is not None else 0
    ldb = B.stride(0) if B is not None else N
    lddp = dCpack.stride(0) if dCpack is not None and dCpack.dim() == 2 else N
    lddb = dB.stride(0) if dB is not None else N
    shiro_spmm_backward(plan.handle, planT.handle if planT is not None else None, _ptr(dC),
                        dC.stride(0), _ptr(Bpack), Bpack.stride(0) if Bpack.dim() == 2 else N,
                        _ptr(B), ldb, N, dtype_code(dC.dtype), _ptr(dCpack), lddp, _ptr(dB),
                        lddb, _ptr(dA), _ptr(scratch), sb, _stream(stream))
    return dB, dA


class JointSpMM:
    """C = A B by the joint row-column strategy (Sec. 5.2-5.3): A's tiles are split by a minimum
    vertex cover into column-based nonzeros (packed B rows, plan_col) and row-based ones (partial
    C rows computed where B lives, plan_rs, then added to C in tile order by plan_agg).  All the
    arithmetic runs in the library; this class only allocates and sequences the calls.

    strategy: "joint" (uniform costs, Hopcroft-Karp + Koenig), "weighted" (costs w_row / w_col,
    min cut by Dinic) or "row" (the row-based strategy of Eq. 3: every communicated nonzero is
    row-based)."""

    def __init__(self, plan: Plan, P_r, P_c, flags=0, row_bounds=None, col_bounds=None,
                 opts=None, strategy="joint", w_row=1, w_col=1):
        self.base = plan
        if strategy == "joint":
            self.cover = plan.joint()
        elif strategy == "weighted":
            self.cover = plan.joint_weighted(w_row, w_col)
        elif strategy == "row":
            self.cover = plan.row_based()
        else:
            raise ValueError(f"unknown strategy {strategy!r}")
        side = self.cover["row_based"].contiguous()
        info = plan.info
        dev = plan.device
        cn, R, rn = _i64(0), _i64(0), _i64(0)
        shiro_joint_split_sizes(plan.handle, _ptr(side), ctypes.byref(cn), ctypes.byref(R),
                                ctypes.byref(rn))
        self.split_rows = R.value
        vdt = plan.vdt
        M, K = info.M, info.K
        z = lambda n, dt: torch.empty(max(int(n), 1), dtype=dt, device=dev)
        self.col = (z(M + 1, torch.int64), z(cn.value, torch.int32), z(cn.value, vdt))
        self.rs = (z(R.value + 1, torch.int64), z(rn.value, torch.int32), z(rn.value, vdt))
        self.agg = (z(M + 1, torch.int64), z(R.value, torch.int32), z(R.value, vdt))
        shiro_joint_split(plan.handle, _ptr(side), *[_ptr(t) for t in self.col],
                          *[_ptr(t) for t in self.rs], *[_ptr(t) for t in self.agg],
                          _stream(None))
        col = (self.col[0], self.col[1][: cn.value], self.col[2][: cn.value])
        self.plan_col = Plan.create(*col, M, K, P_r, P_c, row_bounds=row_bounds,
                                    col_bounds=col_bounds, flags=flags, opts=opts)
        self.plan_rs = self.plan_agg = None
        if R.value > 0:
            rs = (self.rs[0][: R.value + 1], self.rs[1][: rn.value], self.rs[2][: rn.value])
            agg = (self.agg[0], self.agg[1][: R.value], self.agg[2][: R.value])
            self.plan_rs = Plan.create(*rs, R.value, K, 1, 1, flags=SHIRO_PLAN_LOCAL_DIAG, opts=opts)
            self.plan_agg = Plan.create(*agg, M, R.value, 1, 1, flags=SHIRO_PLAN_LOCAL_DIAG,
                                        opts=opts)

    def volumes(self):
        """(rows of B sent, partial C rows sent): the two parts of mu (Eq. 9)."""
        return self.plan_col.info.packed_rows, self.split_rows

    def spmm(self, B, out=None, stream=None):
        N = B.shape[1]
        Bp = self.plan_col.pack(B, stream=stream)
        C = self.plan_col.spmm(Bp, B=B, out=out, stream=stream)
        if self.plan_rs is not None:
            none = torch.empty((0, N), dtype=B.dtype, device=B.device)
            part = self.plan_rs.spmm(none, B=B, stream=stream)
            self.plan_agg.spmm(torch.empty((0, N), dtype=part.dtype, device=B.device), B=part,
                               out=C, accumulate=True, stream=stream)
        return C
