"""Seeded synthetic inputs shaped like the paper's graphs (Tab. 2 and the GNN study of Sec. 7.6).

This module only *generates inputs*: CSR patterns, values and dense operands.  It holds none of
the method's arithmetic (no unique-column sets, no packing, no SpMM) and is the single source of
inputs for both the CUDA path and the CPU oracle, so the two always see the same bytes.

Random numbers come from a counter-based generator: the i-th output of SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) started
from a per-(seed, stream) state.  Output i of a stream is ``mix(state + (i + 1) * GAMMA)`` with
``state = mix(seed * GAMMA + stream)``, so any element can be drawn independently of the others
and the result does not depend on chunking or on the machine.

Workload recipes (the paper's SuiteSparse/OGB/IGB matrices are not available here; these seeded
stand-ins reproduce their shape: square, power-law degree, ~half the ids empty at scale 20+):

* ``er``    -- Erdos-Renyi G(n, p): every (i, j) is kept with probability p.
* ``rmat``  -- R-MAT (a, b, c, d) with ``scale`` levels, ``deg * n`` edge samples, duplicates merged
              (pattern first, values drawn afterwards in CSR order).  Endpoints >= n are rejected
              when n is not a power of two.
* ``gcn_normalized`` -- binary R-MAT pattern, symmetrised, self loops added,
              value 1/sqrt(d_i d_j) with d the row degree including the loop.
* ``batch_graphs`` -- G independent R-MAT graphs, n ~ U{lo..hi}, degree log-uniform.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_GEN_SRC = os.path.join(_HERE, "synth_gen.c")
_GEN_LIB = os.path.join(_HERE, "libsynthgen.so")
_gen = None


def build_gen(force: bool = False) -> str:
    """Compile synth_gen.c (the multi-threaded generators) next to this file."""
    if not force and os.path.exists(_GEN_LIB) and os.path.getmtime(_GEN_LIB) >= os.path.getmtime(_GEN_SRC):
        return _GEN_LIB
    tmp = _GEN_LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _GEN_SRC, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-lm"], check=True)
    os.replace(tmp, _GEN_LIB)
    return _GEN_LIB


def _lib():
    global _gen
    if _gen is None:
        build_gen()
        L = ctypes.CDLL(_GEN_LIB)
        u64, i64, i32, vp = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        L.synth_normal_f32.argtypes = [u64, u64, i64, ctypes.c_double, vp]
        L.synth_uniform_f32.argtypes = [u64, u64, i64, i64, vp]
        L.synth_rmat_keys.argtypes = [u64, u64, i32, i64, i64, i64, u64, u64, u64, vp]
        L.synth_keys_to_csr.argtypes = [vp, i64, i64, vp, vp]
        L.synth_keys_to_csr.restype = i64
        L.synth_f32_to_bf16.argtypes = [vp, i64, vp]
        _gen = L
    return _gen


def _vp(a):
    return a.ctypes.data_as(ctypes.c_void_p)

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK32 = np.uint64(0xFFFFFFFF)

# Stream ids (fixed so that every recipe draws from its own sequence).
STREAM_ER = 1
STREAM_RMAT = 16          # + level pair
STREAM_VAL = 2
STREAM_DENSE = 3
STREAM_BATCH = 4
STREAM_PERM = 5

_CHUNK = 1 << 22


def sorted_unique(x: np.ndarray) -> np.ndarray:
    """Ascending distinct values (sort + neighbour compare; faster than np.unique here)."""
    y = np.sort(x)
    if len(y) == 0:
        return y
    keep = np.empty(len(y), dtype=bool)
    keep[0] = True
    np.not_equal(y[1:], y[:-1], out=keep[1:])
    return y[keep]


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser (uint64 array in, uint64 array out, wrapping arithmetic)."""
    z = z ^ (z >> np.uint64(30))
    z = z * _M1
    z = z ^ (z >> np.uint64(27))
    z = z * _M2
    return z ^ (z >> np.uint64(31))


def stream_state(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([seed], dtype=np.uint64) * GAMMA + np.uint64(stream)
        return _mix(s)[0]


def draw_bits(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Outputs start..start+count-1 of the (seed, stream) SplitMix64 sequence as uint64."""
    st = stream_state(seed, stream)
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(st + i * GAMMA)


def uniform_f64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """U[0,1) doubles from the top 53 bits."""
    return (draw_bits(seed, stream, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_f32(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """U[0,1) floats from the top 24 bits (exactly representable in FP32)."""
    out = np.empty(count, dtype=np.float32)
    if count:
        _lib().synth_uniform_f32(seed, stream, start, count, _vp(out))
    return out


def normal_f32(seed: int, stream: int, count: int, std: float = 1.0) -> np.ndarray:
    """N(0, std^2) FP32 values by the Box-Muller transform, two outputs per 64-bit draw:
    draw k gives outputs 2k and 2k + 1 from u1 = (hi32 + 1/2) 2^-32 and u2 = (lo32 + 1/2) 2^-32."""
    out = np.empty(count, dtype=np.float32)
    if count:
        _lib().synth_normal_f32(seed, stream, count, float(std), _vp(out))
    return out


def dense_normal(rows: int, cols: int, seed: int, stream: int = STREAM_DENSE,
                 std: float = 1.0) -> np.ndarray:
    """Row-major rows x cols FP32 matrix with N(0, std^2) entries."""
    return normal_f32(seed, stream, rows * cols, std).reshape(rows, cols)


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round FP32 to BF16 (round to nearest, ties to even); returns the uint16 bit patterns.

    Inputs are finite; NaN handling is not needed for these generators."""
    src = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(src.shape, dtype=np.uint16)
    if src.size:
        _lib().synth_f32_to_bf16(_vp(src), src.size, _vp(out))
    return out


def bf16_bits_to_f32(h: np.ndarray) -> np.ndarray:
    return (h.astype(np.uint32) << np.uint32(16)).view(np.float32)


@dataclass
class CSR:
    """Square or rectangular CSR matrix on the host (int64 rowptr, int32 col, FP32 values)."""
    M: int
    K: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def row_ids(self) -> np.ndarray:
        return np.repeat(np.arange(self.M, dtype=np.int64), np.diff(self.rowptr))


def csr_from_sorted_keys(keys: np.ndarray, M: int, K: int, val: np.ndarray) -> CSR:
    rows = keys // K
    cols = (keys - rows * K).astype(np.int32)
    counts = np.bincount(rows, minlength=M).astype(np.int64)
    rowptr = np.zeros(M + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(M, K, rowptr, cols, val)


def er(n: int, avg_deg: float, seed: int, lo: float = -1.0, hi: float = 1.0) -> CSR:
    """G(n, p) with p = avg_deg / n: each (i, j) kept independently; values U(lo, hi)."""
    p = avg_deg / n
    keys = []
    total = n * n
    for s in range(0, total, _CHUNK):
        cnt = min(_CHUNK, total - s)
        u = uniform_f64(seed, STREAM_ER, s, cnt)
        keys.append(np.nonzero(u < p)[0].astype(np.int64) + s)
    k = np.concatenate(keys)
    u = uniform_f32(seed, STREAM_VAL, 0, len(k))
    val = (np.float32(lo) + np.float32(hi - lo) * u).astype(np.float32)
    return csr_from_sorted_keys(k, n, n, val)


def keys_to_pattern(keys: np.ndarray, n: int):
    """(rowptr, col) of the distinct keys row * n + col (negative keys skipped), columns ascending."""
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.empty(max(1, len(keys)), dtype=np.int32)
    nnz = _lib().synth_keys_to_csr(_vp(keys), len(keys), n, _vp(rowptr), _vp(col))
    return rowptr, col[:nnz].copy()


def rmat_samples(n: int, scale: int, samples: int, seed: int,
                 a: float = 0.57, b: float = 0.19, c: float = 0.19) -> np.ndarray:
    """Keys row * n + col of R-MAT edge samples (not deduplicated; -1 for rejected samples).

    Each sample descends ``scale`` levels, most significant bit first; at every level one
    32-bit uniform picks the quadrant (a: top-left, b: top-right, c: bottom-left, d: bottom-right).
    Samples with an endpoint >= n are rejected (only when n is not a power of two)."""
    ta, tab, tabc = int(a * 2 ** 32), int((a + b) * 2 ** 32), int((a + b + c) * 2 ** 32)
    keys = np.empty(max(1, samples), dtype=np.int64)
    if samples:
        _lib().synth_rmat_keys(seed, STREAM_RMAT, scale, n, 0, samples, ta, tab, tabc, _vp(keys))
    return keys[:samples]


def rmat_pattern(n: int, scale: int, samples: int, seed: int, a: float = 0.57, b: float = 0.19,
                 c: float = 0.19):
    """(rowptr, col) of an R-MAT pattern with duplicates merged."""
    return keys_to_pattern(rmat_samples(n, scale, samples, seed, a, b, c), n)


def rmat_keys(n: int, scale: int, samples: int, seed: int,
              a: float = 0.57, b: float = 0.19, c: float = 0.19) -> np.ndarray:
    """Sorted unique (row * n + col) keys of an R-MAT pattern with duplicates merged."""
    rowptr, col = rmat_pattern(n, scale, samples, seed, a, b, c)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    return rows * n + col.astype(np.int64)


def rmat(scale: int, avg_deg: int, seed: int, n: int | None = None,
         a: float = 0.57, b: float = 0.19, c: float = 0.19,
         lo: float = 0.0, hi: float = 1.0) -> CSR:
    """R-MAT CSR with avg_deg * n samples, duplicates merged, values U(lo, hi) in CSR order."""
    n = (1 << scale) if n is None else n
    rowptr, col = rmat_pattern(n, scale, avg_deg * n, seed, a, b, c)
    u = uniform_f32(seed, STREAM_VAL, 0, len(col))
    val = (np.float32(lo) + np.float32(hi - lo) * u).astype(np.float32)
    return CSR(n, n, rowptr, col, val)


def gcn_normalized(scale: int, avg_deg: int, seed: int) -> CSR:
    """Symmetric-normalised adjacency with self loops, D^-1/2 (A + A^T + I) D^-1/2 on the pattern.

    Built from a binary R-MAT pattern; the value of (i, j) is 1/sqrt(d_i d_j) computed in FP64
    and stored in FP32, d being the row count of the symmetrised pattern including the loop."""
    n = 1 << scale
    k = rmat_samples(n, scale, avg_deg * n, seed)
    k = k[k >= 0]
    r, c = k // n, k % n
    diag = np.arange(n, dtype=np.int64)
    rowptr, col = keys_to_pattern(np.concatenate([k, c * n + r, diag * n + diag]), n)
    d = np.diff(rowptr).astype(np.float64)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    val = (1.0 / np.sqrt(d[rows] * d[col])).astype(np.float32)
    return CSR(n, n, rowptr, col, val)


def induced_subgraph(A: CSR, n_sub: int) -> CSR:
    """Rows/cols < n_sub of A (values kept as they are)."""
    rows = A.row_ids()
    keep = (rows < n_sub) & (A.col < n_sub)
    keys = rows[keep] * n_sub + A.col[keep].astype(np.int64)
    return csr_from_sorted_keys(keys, n_sub, n_sub, A.val[keep].copy())


def renormalize_sym(A: CSR) -> CSR:
    """Recompute 1/sqrt(d_i d_j) on A's (symmetric) pattern, FP64 then FP32."""
    rows = A.row_ids()
    d = np.diff(A.rowptr).astype(np.float64)
    val = (1.0 / np.sqrt(d[rows] * d[A.col])).astype(np.float32)
    return CSR(A.M, A.K, A.rowptr.copy(), A.col.copy(), val)


@dataclass
class GraphBatch:
    graphs: list
    node_counts: np.ndarray
    degrees: np.ndarray


def batch_graphs(G: int, seed: int, n_lo: int = 100, n_hi: int = 20000,
                 d_lo: float = 4.0, d_hi: float = 40.0) -> GraphBatch:
    """G independent R-MAT graphs: n ~ U{n_lo..n_hi}, degree log-uniform on [d_lo, d_hi]."""
    u = uniform_f64(seed, STREAM_BATCH, 0, 2 * G)
    ns = (n_lo + np.floor(u[:G] * (n_hi - n_lo + 1))).astype(np.int64)
    ds = np.exp(math.log(d_lo) + u[G:] * (math.log(d_hi) - math.log(d_lo)))
    graphs = []
    for g in range(G):
        n = int(ns[g])
        scale = max(1, int(math.ceil(math.log2(n))))
        samples = int(round(ds[g] * n))
        sub_seed = seed * 1000003 + g
        rowptr, col = rmat_pattern(n, scale, samples, sub_seed)
        val = uniform_f32(sub_seed, STREAM_VAL, 0, len(col))
        graphs.append(CSR(n, n, rowptr, col, val))
    return GraphBatch(graphs, ns, ds)


def from_dense(D: np.ndarray) -> CSR:
    """CSR of the nonzeros of a small dense matrix (row-major, ascending columns)."""
    M, K = D.shape
    r, c = np.nonzero(D)
    keys = r.astype(np.int64) * K + c
    return csr_from_sorted_keys(keys, M, K, D[r, c].astype(np.float32))


def random_small(M: int, K: int, density: float, seed: int, lo: float = -1.0,
                 hi: float = 1.0, empty_rows: int = 0) -> CSR:
    """Small uniform random CSR for unit tests; ``empty_rows`` leading rows are forced empty."""
    u = uniform_f64(seed, STREAM_ER, 0, M * K).reshape(M, K)
    mask = u < density
    mask[:empty_rows] = False
    r, c = np.nonzero(mask)
    keys = r.astype(np.int64) * K + c
    v = uniform_f32(seed, STREAM_VAL, 0, len(keys))
    val = (np.float32(lo) + np.float32(hi - lo) * v).astype(np.float32)
    return csr_from_sorted_keys(keys, M, K, val)


def hub_matrix(M: int, K: int, hub_row: int, hub_nnz: int, base_deg: int, seed: int) -> CSR:
    """Uniform sparse rows plus one dense "hub" row with hub_nnz distinct columns (power-law stand-in)."""
    base = random_small(M, K, base_deg / K, seed, 0.0, 1.0) if M * K <= (1 << 26) else None
    rows = [] if base is None else [base.row_ids()]
    cols = [] if base is None else [base.col.astype(np.int64)]
    if base is not None:
        keep = rows[0] != hub_row
        rows[0], cols[0] = rows[0][keep], cols[0][keep]
    step = max(1, K // hub_nnz)
    hc = (np.arange(hub_nnz, dtype=np.int64) * step) % K
    hc = sorted_unique(hc)
    rows.append(np.full(len(hc), hub_row, dtype=np.int64))
    cols.append(hc)
    keys = sorted_unique(np.concatenate([r * K + c for r, c in zip(rows, cols)]))
    val = uniform_f32(seed, STREAM_VAL + 100, 0, len(keys))
    return csr_from_sorted_keys(keys, M, K, val)
