"""Plan parity on the GPU: tile split, Cols sets, remap, pack list, volumes -- bit-exact vs oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_20178_gb300 import synth
import gpu_util as gu

pytestmark = pytest.mark.gpu


def setup_module(_):
    gu.need_gpu()


CASES = {
    "er4096_2d_4x4": (lambda: synth.er(4096, 8, 1), 4, 4, 0),
    "er4096_1d_p4_localdiag": (lambda: synth.er(4096, 8, 1), 4, 4, 1),
    "rmat14_4x4": (lambda: synth.rmat(14, 16, 3), 4, 4, 0),
    "ragged_3x5": (lambda: synth.random_small(1000, 777, 0.01, 11), 3, 5, 0),
    "ragged_7x2": (lambda: synth.random_small(333, 1501, 0.02, 12, empty_rows=40), 7, 2, 0),
    "more_blocks_than_rows": (lambda: synth.random_small(5, 9, 0.5, 13), 8, 8, 0),
    "single_tile": (lambda: synth.rmat(10, 8, 4), 1, 1, 0),
    "wide_grid_16x16": (lambda: synth.rmat(12, 8, 5), 16, 16, 0),
    "hub_row_2e17": (lambda: synth.hub_matrix(64, 1 << 17, 5, 1 << 17, 2, 14), 2, 4, 0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_plan_parity(name):
    make, Pr, Pc, local = CASES[name]
    A = make()
    shiro = gu.lib()
    flags = shiro.SHIRO_PLAN_LOCAL_DIAG if local else 0
    P = gu.plan_of(A, Pr, Pc, flags)
    gu.assert_plan_matches(P, A, Pr, Pc, flags)


def test_custom_bounds():
    A = synth.rmat(12, 8, 6)
    rb = [0, 100, 100, 3000, A.M]
    cb = [0, 7, 2049, A.K]
    P = gu.plan_of(A, 4, 3, row_bounds=rb, col_bounds=cb)
    gu.assert_plan_matches(P, A, 4, 3, 0, rb=np.array(rb), cb=np.array(cb))


def test_diag_only_block_diagonal():
    gs = [synth.rmat(s, 6, 20 + s) for s in (5, 9, 7, 3)]
    n = sum(g.M for g in gs)
    rows, cols, vals, off = [], [], [], 0
    b = [0]
    for g in gs:
        rows.append(g.row_ids() + off)
        cols.append(g.col.astype(np.int64) + off)
        vals.append(g.val)
        off += g.M
        b.append(off)
    keys = np.concatenate([r * n + c for r, c in zip(rows, cols)])
    A = synth.csr_from_sorted_keys(keys, n, n, np.concatenate(vals))
    shiro = gu.lib()
    P = gu.plan_of(A, len(gs), len(gs), shiro.SHIRO_PLAN_DIAG_ONLY, row_bounds=b, col_bounds=b)
    gu.assert_plan_matches(P, A, len(gs), len(gs), shiro.SHIRO_PLAN_DIAG_ONLY,
                           rb=np.array(b), cb=np.array(b))


def test_empty_and_all_empty_rows():
    A = synth.CSR(100, 50, np.zeros(101, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    P = gu.plan_of(A, 3, 2)
    assert P.info.total_cols == 0 and P.info.packed_rows == 0
    gu.assert_plan_matches(P, A, 3, 2)


@pytest.mark.parametrize("bad", ["col_out_of_range", "negative_col", "rowptr_decreasing",
                                 "rowptr_end", "off_diagonal"])
def test_bad_csr_rejected(bad):
    shiro = gu.lib()
    A = synth.random_small(50, 40, 0.2, 3)
    rp, col, val = A.rowptr.copy(), A.col.copy(), A.val.copy()
    flags, bounds = 0, None
    if bad == "col_out_of_range":
        col[7] = 40
    elif bad == "negative_col":
        col[3] = -2
    elif bad == "rowptr_decreasing":
        rp[10] = rp[11] + 1
    elif bad == "rowptr_end":
        rp[-1] = rp[-1] - 1
    else:
        flags, bounds = shiro.SHIRO_PLAN_DIAG_ONLY, [0, 25, 50]
        A = synth.random_small(50, 50, 0.2, 3)
        rp, col, val = A.rowptr.copy(), A.col.copy(), A.val.copy()
    d = gu.dev()
    t = [torch.from_numpy(x).to(d) for x in (rp, col, val)]
    K = 50 if bad == "off_diagonal" else 40
    with pytest.raises(shiro.ShiroError) as ei:
        shiro.Plan.create(t[0], t[1], t[2], 50, K, 2, 2, row_bounds=bounds, col_bounds=bounds,
                          flags=flags)
    assert ei.value.status == 2
    # The device is still usable afterwards.
    P = gu.plan_of(synth.random_small(50, 40, 0.2, 4), 2, 2)
    assert P.info.nnz > 0


def test_full_size_rmat20_plan():
    """R-MAT 2^20, avg degree 16, 4x4 tiles (the benchmark workload): every integer output."""
    A = synth.rmat(20, 16, 2)
    P = gu.plan_of(A, 4, 4)
    gu.assert_plan_matches(P, A, 4, 4)
