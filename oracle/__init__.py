"""FP64 CPU oracle for the sparsity-aware SpMM path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  It wraps ``oracle.c`` (plain C, FP64, compiled with ``-ffp-contract=off``) through
ctypes and shares no code with the CUDA library.

Functions mirror the definitions in ``oracle.c``; see that file for the passage of the paper each
one follows.  All arrays are numpy; floating-point inputs are converted to FP64 exactly.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", _SRC, "-o", _LIB]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-lm"], check=True)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
    return _lib


def use_library(path):
    """Swap the loaded oracle library (used by the planted-mistake tests); returns the old one."""
    global _lib
    old = _lib
    _lib = ctypes.CDLL(path) if isinstance(path, str) else path
    return old


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


def threads() -> int:
    return int(lib().oracle_threads())


def set_threads(n: int) -> None:
    lib().oracle_set_threads(_i32(n))


def uniform_bounds(n: int, P: int) -> np.ndarray:
    b = np.zeros(P + 1, dtype=np.int64)
    lib().oracle_uniform_bounds(_i64(n), _i32(P), _p(b))
    return b


@dataclass
class Plan:
    """Per-tile outputs of the plan (Tab. 1 notation; tile t = p * Pc + q, or t = p when diag_only)."""
    Pr: int
    Pc: int
    rb: np.ndarray
    cb: np.ndarray
    diag_only: bool
    tile_nnz: np.ndarray
    tile_nrows: np.ndarray
    tile_ncols: np.ndarray
    tile_cols_ptr: np.ndarray
    cols_sorted: np.ndarray
    colidx_local: np.ndarray

    @property
    def T(self) -> int:
        return len(self.tile_nnz)

    def tile_pq(self, t: int):
        return (t, t) if self.diag_only else (t // self.Pc, t % self.Pc)

    def cols_of(self, t: int) -> np.ndarray:
        return self.cols_sorted[self.tile_cols_ptr[t]:self.tile_cols_ptr[t + 1]]

    def packed_tiles(self, local_diag: bool) -> np.ndarray:
        """Tiles whose B rows are packed: all, or all but the diagonal ones in local_diag mode."""
        ts = np.arange(self.T)
        if local_diag and not self.diag_only:
            ts = ts[(ts // self.Pc) != (ts % self.Pc)]
        return ts

    def pack_layout(self, local_diag: bool = False):
        """(pack_ptr[T+1], pack_src): packed tiles' Cols concatenated in tile order."""
        keep = np.zeros(self.T, dtype=bool)
        keep[self.packed_tiles(local_diag)] = True
        cnt = np.where(keep, self.tile_ncols, 0)
        pack_ptr = np.zeros(self.T + 1, dtype=np.int64)
        np.cumsum(cnt, out=pack_ptr[1:])
        src = [self.cols_of(t) for t in range(self.T) if keep[t]]
        pack_src = np.concatenate(src).astype(np.int32) if src else np.zeros(0, np.int32)
        return pack_ptr, pack_src

    def volumes(self, N: int, sz: int, szc: int = 4, local_diag: bool = False):
        """(V_block, V_col, V_row) per tile in bytes (Eq. 1-3): B elements of sz bytes, partial C
        elements of szc bytes; local diagonal tiles report 0."""
        vb = np.zeros(self.T, dtype=np.int64)
        vc = np.zeros(self.T, dtype=np.int64)
        vr = np.zeros(self.T, dtype=np.int64)
        lib().oracle_volumes(_i32(self.Pr), _i32(self.Pc), ctypes.c_int(int(self.diag_only)),
                             ctypes.c_int(int(local_diag)), _p(self.cb), _p(self.tile_ncols),
                             _p(self.tile_nrows), _i32(N), _i32(sz), _i32(szc), _p(vb), _p(vc),
                             _p(vr))
        return vb, vc, vr


def plan(A, Pr: int, Pc: int, rb=None, cb=None, diag_only: bool = False) -> Plan:
    """Tile split, unique columns, remap (see oracle_plan in oracle.c)."""
    rb = uniform_bounds(A.M, Pr) if rb is None else np.ascontiguousarray(rb, dtype=np.int64)
    cb = uniform_bounds(A.K, Pc) if cb is None else np.ascontiguousarray(cb, dtype=np.int64)
    T = Pr if diag_only else Pr * Pc
    cap = max(1, A.nnz)
    tile_nnz = np.zeros(T, np.int64)
    tile_nrows = np.zeros(T, np.int64)
    tile_ncols = np.zeros(T, np.int64)
    tcp = np.zeros(T + 1, np.int64)
    cols = np.zeros(cap, np.int32)
    cl = np.full(max(1, A.nnz), -1, np.int32)
    rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int64)
    col = np.ascontiguousarray(A.col, dtype=np.int32)
    rc = lib().oracle_plan(_i64(A.M), _i64(A.K), _p(rowptr), _p(col), _i32(Pr), _i32(Pc), _p(rb),
                           _p(cb), ctypes.c_int(int(diag_only)), _p(tile_nnz), _p(tile_nrows),
                           _p(tile_ncols), _p(tcp), _p(cols), _i64(cap), _p(cl))
    if rc != 0:
        raise ValueError("oracle_plan rejected the matrix")
    return Plan(Pr, Pc, rb, cb, diag_only, tile_nnz, tile_nrows, tile_ncols, tcp,
                cols[: tcp[-1]].copy(), cl[: A.nnz].copy())


def pack(B: np.ndarray, src: np.ndarray) -> np.ndarray:
    """Bpack[r] = B[src[r]] (row copy of any dtype; bit-exact)."""
    B = np.ascontiguousarray(B)
    out = np.empty((len(src), B.shape[1]), dtype=B.dtype)
    src = np.ascontiguousarray(src, dtype=np.int32)
    lib().oracle_pack(_p(B), _i64(B.shape[1]), _i32(B.shape[1]), _i32(B.itemsize), _p(src),
                      _i64(len(src)), _p(out), _i64(B.shape[1]))
    return out


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def spmm(A, B, rows=None, val=None) -> np.ndarray:
    """C = A B in FP64; ``rows`` restricts to a list of rows (C then has len(rows) rows)."""
    B64 = _f64(B)
    v = _f64(A.val if val is None else val)
    N = B64.shape[1]
    rr = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    n = A.M if rr is None else len(rr)
    C = np.zeros((n, N), dtype=np.float64)
    lib().oracle_spmm(_i64(A.M), _p(np.ascontiguousarray(A.rowptr, np.int64)),
                      _p(np.ascontiguousarray(A.col, np.int32)), _p(v), _p(B64), _i64(N), _i32(N),
                      _p(rr), _i64(n), _p(C), _i64(N))
    return C


def spmm_packed(A, P: Plan, Bpack, B, local_diag: bool = False) -> np.ndarray:
    """C = A B read through the packed rows (Sec. 5.1 stages 3 and 5)."""
    pack_ptr, _ = P.pack_layout(local_diag)
    Bp = _f64(Bpack).reshape(-1, B.shape[1]) if len(Bpack) else np.zeros((1, B.shape[1]))
    B64 = _f64(B)
    N = B64.shape[1]
    C = np.zeros((A.M, N), dtype=np.float64)
    lib().oracle_spmm_packed(_i64(A.M), _p(np.ascontiguousarray(A.rowptr, np.int64)),
                             _p(np.ascontiguousarray(A.col, np.int32)), _p(_f64(A.val)),
                             _i32(P.Pr), _i32(P.Pc), _p(P.rb), _p(P.cb),
                             ctypes.c_int(int(P.diag_only)), ctypes.c_int(int(local_diag)),
                             _p(pack_ptr), _p(P.colidx_local), _p(Bp), _i64(N), _p(B64), _i64(N),
                             _i32(N), _p(C), _i64(N))
    return C


def abs_scale(A, B, rows=None) -> np.ndarray:
    """S[i,k] = sum_j |a_ij| |b_jk| (FP64), the per-element scale of the tolerance."""
    B64 = _f64(B)
    N = B64.shape[1]
    rr = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    n = A.M if rr is None else len(rr)
    S = np.zeros((n, N), dtype=np.float64)
    lib().oracle_abs_scale(_i64(A.M), _p(np.ascontiguousarray(A.rowptr, np.int64)),
                           _p(np.ascontiguousarray(A.col, np.int32)), _p(_f64(A.val)), _p(B64),
                           _i64(N), _i32(N), _p(rr), _i64(n), _p(S), _i64(N))
    return S


def spmm_t(A, dC, val=None) -> np.ndarray:
    """dB = A^T dC in FP64."""
    G = _f64(dC)
    N = G.shape[1]
    dB = np.zeros((A.K, N), dtype=np.float64)
    lib().oracle_spmm_t(_i64(A.M), _i64(A.K), _p(np.ascontiguousarray(A.rowptr, np.int64)),
                        _p(np.ascontiguousarray(A.col, np.int32)),
                        _p(_f64(A.val if val is None else val)), _p(G), _i64(N), _i32(N), _p(dB),
                        _i64(N))
    return dB


def sddmm(A, dC, B) -> np.ndarray:
    """out[e] = <dC[row e], B[col e]> in FP64 on A's pattern."""
    G = _f64(dC)
    B64 = _f64(B)
    N = G.shape[1]
    out = np.zeros(A.nnz, dtype=np.float64)
    lib().oracle_sddmm(_i64(A.M), _p(np.ascontiguousarray(A.rowptr, np.int64)),
                       _p(np.ascontiguousarray(A.col, np.int32)), _p(G), _i64(N), _p(B64),
                       _i64(N), _i32(N), _p(out))
    return out


def transpose(A):
    """(rowptrT, colT, perm) of A^T; rows of A^T list A's rows in ascending order."""
    rowptrT = np.zeros(A.K + 1, np.int64)
    colT = np.zeros(max(1, A.nnz), np.int32)
    perm = np.zeros(max(1, A.nnz), np.int64)
    lib().oracle_transpose(_i64(A.M), _i64(A.K), _p(np.ascontiguousarray(A.rowptr, np.int64)),
                           _p(np.ascontiguousarray(A.col, np.int32)), _p(rowptrT), _p(colT),
                           _p(perm))
    return rowptrT, colT[: A.nnz].copy(), perm[: A.nnz].copy()


def max_matching(nL: int, nR: int, ptr, adj) -> int:
    """Maximum matching of a bipartite graph (= minimum vertex cover size, Koenig)."""
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    adj = np.ascontiguousarray(adj if len(adj) else np.zeros(1, np.int32), dtype=np.int32)
    f = lib().oracle_max_matching
    f.restype = ctypes.c_int64
    return int(f(_i32(nL), _i32(nR), _p(ptr), _p(adj)))


def min_weight_cover(nL: int, nR: int, ptr, adj, w_row, w_col):
    """Minimum weighted vertex cover of a bipartite graph by the minimum cut of Sec. 5.3.3.
    Returns (max flow, cover_row bool[nL], cover_col bool[nR])."""
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    adj = np.ascontiguousarray(adj if len(adj) else np.zeros(1, np.int32), dtype=np.int32)
    wr = np.ascontiguousarray(w_row if nL else np.zeros(1), dtype=np.int64)
    wc = np.ascontiguousarray(w_col if nR else np.zeros(1), dtype=np.int64)
    cr = np.zeros(max(nL, 1), np.uint8)
    cc = np.zeros(max(nR, 1), np.uint8)
    f = lib().oracle_min_weight_cover
    f.restype = ctypes.c_int64
    flow = int(f(_i32(nL), _i32(nR), _p(ptr), _p(adj), _p(wr), _p(wc), _p(cr), _p(cc)))
    return flow, cr[:nL].astype(bool), cc[:nR].astype(bool)


def tile_graph(A, P: Plan, t: int):
    """Bipartite graph of tile t: left = the row block's rows (local ids), right = the tile's Cols
    positions, one edge per nonzero of the tile (input marshalling for max_matching)."""
    p, q = P.tile_pq(t)
    r0, r1 = int(P.rb[p]), int(P.rb[p + 1])
    c0, c1 = int(P.cb[q]), int(P.cb[q + 1])
    ptr = [0]
    adj = []
    for i in range(r0, r1):
        s, e = int(A.rowptr[i]), int(A.rowptr[i + 1])
        cols = A.col[s:e]
        loc = P.colidx_local[s:e]
        sel = (cols >= c0) & (cols < c1)
        adj.extend(loc[sel].tolist())
        ptr.append(len(adj))
    return r1 - r0, int(P.tile_ncols[t]), np.array(ptr, np.int64), np.array(adj, np.int32)


def scaled_error(C, C64, S, per_row: bool = False):
    """Maximum over elements of |C - C64| / S, where S = 0 requires C == 0 exactly (the element
    then counts 0, else +inf) and a NaN counts +inf (see oracle_scaled_error).  C may be any
    float dtype (converted to FP64 exactly).  With per_row, returns the per-row maxima instead."""
    C = _f64(C)
    C64 = _f64(C64)
    S = _f64(S)
    if C.ndim == 1:
        C, C64, S = C[:, None], C64[:, None], S[:, None]
    if not (C.shape == C64.shape == S.shape):
        raise ValueError(f"shape mismatch {C.shape} {C64.shape} {S.shape}")
    n, N = C.shape
    rm = np.zeros(max(n, 1), dtype=np.float64)
    f = lib().oracle_scaled_error
    f.restype = ctypes.c_double
    worst = float(f(_i64(n), _i32(N), _p(C), _i64(N), _p(C64), _i64(N), _p(S), _i64(N), _p(rm)))
    return rm[:n].copy() if per_row else worst
