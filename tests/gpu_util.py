"""Helpers of the GPU parity tests: inputs to the device, oracle comparisons, tolerances.

Tolerance: FP32 SpMM within max scaled error 1e-5 of the FP64 oracle, the error of
element (i, k) being |C_ik - C64_ik| / sum_j |a_ij| |b_jk| (and exact zeros where the scale is 0).
The same bound is applied to dB (scale sum |a_ij| |dC_ik|) and dA (scale sum_k |dC_ik| |B_jk|).
BF16-stored operands are compared with the oracle run on the BF16-rounded values, which FP64
represents exactly, so the same 1e-5 bound applies to the FP32 accumulation.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2512_20178_gb300 import synth

TOL = 1e-5


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2512_20178_gb300 import shiro
    return shiro


def dev():
    return torch.device("cuda:0")


def to_dev(A: synth.CSR, vdt=torch.float32):
    d = dev()
    return (torch.from_numpy(np.ascontiguousarray(A.rowptr)).to(d),
            torch.from_numpy(np.ascontiguousarray(A.col)).to(d),
            torch.from_numpy(np.ascontiguousarray(A.val)).to(d).to(vdt))


def plan_of(A, Pr=1, Pc=1, flags=0, opts=None, vdt=torch.float32, row_bounds=None,
            col_bounds=None):
    shiro = lib()
    rp, col, val = to_dev(A, vdt)
    return shiro.Plan.create(rp, col, val, A.M, A.K, Pr, Pc, row_bounds=row_bounds,
                             col_bounds=col_bounds, flags=flags, opts=opts)


def assert_plan_matches(P, A, Pr, Pc, flags=0, rb=None, cb=None):
    """Integer outputs of the plan equal the oracle's bit for bit."""
    shiro = lib()
    diag_only = bool(flags & shiro.SHIRO_PLAN_DIAG_ONLY)
    local = bool(flags & shiro.SHIRO_PLAN_LOCAL_DIAG)
    O = oracle.plan(A, Pr, Pc, rb=rb, cb=cb, diag_only=diag_only)
    st = P.tile_stats()
    assert np.array_equal(st["tile_nnz"].numpy(), O.tile_nnz), "tile nnz"
    assert np.array_equal(st["tile_nrows"].numpy(), O.tile_nrows), "|Rows|"
    assert np.array_equal(st["tile_ncols"].numpy(), O.tile_ncols), "|Cols|"
    assert np.array_equal(st["tile_cols_ptr"].numpy(), O.tile_cols_ptr), "tile_cols_ptr"
    pack_ptr, pack_src = O.pack_layout(local)
    assert np.array_equal(st["pack_ptr"].numpy(), pack_ptr), "pack_ptr"
    ex = P.export()
    torch.cuda.synchronize()
    assert np.array_equal(ex["cols_sorted"].cpu().numpy(), O.cols_sorted), "Cols (sorted)"
    assert np.array_equal(ex["pack_src"].cpu().numpy(), pack_src), "pack list"
    assert np.array_equal(ex["colidx_local"].cpu().numpy(), O.colidx_local), "colidx_local"
    # remap: packed row, or -1 - col for local diagonal tiles.
    rows = A.row_ids()
    p = np.searchsorted(O.rb, rows, side="right") - 1
    q = np.searchsorted(O.cb, A.col, side="right") - 1
    t = p if diag_only else p * Pc + q
    expect = pack_ptr[t] + O.colidx_local
    if local:
        expect = np.where(p == q, -1 - A.col.astype(np.int64), expect)
    assert np.array_equal(ex["remap"].cpu().numpy(), expect.astype(np.int32)), "remap"
    for dt, sz in ((torch.float32, 4), (torch.bfloat16, 2)):
        vb, vc, vr = P.volumes(32, dt)
        ob, oc, orow = O.volumes(32, sz, 4, local)
        assert np.array_equal(vb.numpy(), ob) and np.array_equal(vc.numpy(), oc), "volumes"
        assert np.array_equal(vr.numpy(), orow), "V_row"
    return O


def scaled_err(C, C64, S):
    return oracle.scaled_error(C, C64, S)


def check_spmm(A, B_host, C_dev, rows=None, tol=TOL):
    """Scaled error of the GPU C against the FP64 oracle (optionally on sampled rows)."""
    C = C_dev.detach().cpu().numpy()
    if rows is not None:
        C = C[rows]
    C64 = oracle.spmm(A, B_host, rows=rows)
    S = oracle.abs_scale(A, B_host, rows=rows)
    err = scaled_err(C, C64, S)
    assert err <= tol, f"scaled error {err:.3e} > {tol}"
    return err


def sampled_rows_error(A, B_host, C_rows, rows):
    """Per-row maximum scaled error of C_rows (GPU rows `rows` of C) against the FP64 oracle, on a
    sub-problem holding only those rows and the B rows they touch (so a large B is never
    converted to FP64 whole)."""
    rows = np.asarray(rows, dtype=np.int64)
    lens = np.diff(A.rowptr)[rows]
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    idx = np.concatenate([np.arange(A.rowptr[r], A.rowptr[r + 1]) for r in rows]) \
        if rp[-1] else np.zeros(0, np.int64)
    cols = A.col[idx]
    ucols, local = np.unique(cols, return_inverse=True)
    S = synth.CSR(len(rows), max(1, len(ucols)), rp, local.astype(np.int32), A.val[idx])
    Bs = np.asarray(B_host[ucols]) if len(ucols) else np.zeros((1, B_host.shape[1]), np.float32)
    C64 = oracle.spmm(S, Bs)
    Sc = oracle.abs_scale(S, Bs)
    return oracle.scaled_error(np.asarray(C_rows), C64, Sc, per_row=True)


def sampled_sddmm_error(A, dC_host, B_host, dA_vals, es):
    """Maximum scaled error of the SDDMM values dA_vals (host array of all nnz) at the sampled
    nonzeros es against the FP64 oracle, on a sub-problem with one row per sampled nonzero: row r
    holds nonzero es[r] of A (its column remapped into the distinct sampled columns), so the
    oracle's dA of that row is <dC[row(es[r])], B[col(es[r])]>.  The scale is the same SDDMM on
    |dC| and |B|."""
    es = np.asarray(es, dtype=np.int64)
    rows_e = A.row_ids()[es]
    ucols, local = np.unique(A.col[es], return_inverse=True)
    S = synth.CSR(len(es), max(1, len(ucols)), np.arange(len(es) + 1, dtype=np.int64),
                  local.astype(np.int32), A.val[es])
    G = np.asarray(dC_host[rows_e])
    Bs = np.asarray(B_host[ucols])
    ref = oracle.sddmm(S, G, Bs)
    sc = oracle.sddmm(S, np.abs(G), np.abs(Bs))
    return oracle.scaled_error(np.asarray(dA_vals)[es], ref, sc)
