"""Joint row-column strategy (Sec. 5.2-5.3) on the library's plans against the oracle.

For every tile: the library's cover size mu equals the oracle's maximum matching (Koenig), the
cover has mu vertices, the split of the nonzeros it implies sends exactly mu rows (distinct columns
of the column-based nonzeros + distinct rows of the row-based ones), and mu <= min(|Cols|, |Rows|)
(the joint strategy is never worse than either single strategy, Sec. 5.4)."""
import numpy as np
import pytest
import torch

import oracle
import oracle_pins as pins
from paper_2512_20178_gb300 import synth
import gpu_util as gu

pytestmark = pytest.mark.gpu


def setup_module(_):
    gu.need_gpu()


def check_joint(A, Pr, Pc, flags=0, rb=None, cb=None):
    shiro = gu.lib()
    diag_only = bool(flags & shiro.SHIRO_PLAN_DIAG_ONLY)
    local = bool(flags & shiro.SHIRO_PLAN_LOCAL_DIAG)
    P = gu.plan_of(A, Pr, Pc, flags, row_bounds=rb, col_bounds=cb)
    J = P.joint()
    O = oracle.plan(A, Pr, Pc, rb=None if rb is None else np.array(rb), cb=None if cb is None else np.array(cb),
                    diag_only=diag_only)
    rows = A.row_ids()
    p_of = np.searchsorted(O.rb, rows, side="right") - 1
    q_of = np.searchsorted(O.cb, A.col, side="right") - 1
    t_of = p_of if diag_only else p_of * Pc + q_of
    side = J["row_based"].numpy()
    total_mu, total_cols = 0, 0
    for t in range(O.T):
        p, q = O.tile_pq(t)
        mu = int(J["mu"][t])
        if local and p == q:
            assert mu == 0 and not side[t_of == t].any()
            continue
        assert mu == oracle.max_matching(*oracle.tile_graph(A, O, t)), f"tile {t}: mu differs"
        assert int(J["cover_rows"][t]) + int(J["cover_cols"][t]) == mu
        sel = t_of == t
        sent = len(np.unique(A.col[sel & (side == 0)])) + len(np.unique(rows[sel & (side == 1)]))
        assert sent == mu, f"tile {t}: the split sends {sent} rows, cover has {mu}"
        assert mu <= min(O.tile_ncols[t], O.tile_nrows[t])
        total_mu += mu
        total_cols += int(O.tile_ncols[t])
    return total_mu, total_cols


@pytest.mark.parametrize("name", ["rmat13_4x4", "er4096_1d_local", "ragged_3x5", "hub", "single"])
def test_joint_cover(name):
    shiro = gu.lib()
    if name == "rmat13_4x4":
        mu, cols = check_joint(synth.rmat(13, 8, 151), 4, 4)
        assert mu < cols, "power-law tiles should gain from the joint strategy"
    elif name == "er4096_1d_local":
        check_joint(synth.er(4096, 8, 1), 4, 4, shiro.SHIRO_PLAN_LOCAL_DIAG)
    elif name == "ragged_3x5":
        check_joint(synth.random_small(700, 900, 0.01, 152, empty_rows=50), 3, 5)
    elif name == "hub":
        check_joint(synth.hub_matrix(256, 4096, 3, 4000, 2, 153), 2, 2)
    else:
        check_joint(synth.rmat(10, 8, 154), 1, 1)


def test_joint_fig1_and_cross_pattern():
    nz, expect, meta = pins.read_golden("fig1_offdiag_tile.txt")
    D = np.zeros(meta["shape"], dtype=np.float32)
    for _, i, j in nz:
        D[i, j] = 1.0
    A = synth.from_dense(D)
    P = gu.plan_of(A, *meta["partition"])
    J = P.joint()
    assert int(J["mu"][1]) == expect["min_cover"][0]
    # A full row plus a full column (hubs on both sides): cover of 2 instead of 64.
    n = 64
    D = np.zeros((2 * n, 2 * n), dtype=np.float32)
    D[0, n:] = 1.0
    D[:n, n] = 1.0
    A = synth.from_dense(D)
    J = gu.plan_of(A, 2, 2).joint()
    assert int(J["mu"][1]) == 2


def test_joint_batch_diag_only():
    shiro = gu.lib()
    gb = synth.batch_graphs(6, 17, 100, 400)
    n = sum(g.M for g in gb.graphs)
    rows, cols, vals, b, off = [], [], [], [0], 0
    for g in gb.graphs:
        rows.append(g.row_ids() + off)
        cols.append(g.col.astype(np.int64) + off)
        vals.append(g.val)
        off += g.M
        b.append(off)
    keys = np.concatenate([r * n + c for r, c in zip(rows, cols)])
    A = synth.csr_from_sorted_keys(keys, n, n, np.concatenate(vals))
    check_joint(A, len(b) - 1, len(b) - 1, shiro.SHIRO_PLAN_DIAG_ONLY, rb=b, cb=b)


@pytest.mark.parametrize("name,N,dt", [("rmat13", 128, torch.float32), ("rmat13", 64, torch.bfloat16),
                                       ("er4096_local", 32, torch.float32), ("ragged", 100, torch.float32),
                                       ("hub", 128, torch.float32)])
def test_joint_spmm_matches_oracle(name, N, dt):
    """C by the joint strategy (packed cover-column B rows + partial C rows of the cover rows,
    added in tile order) within the SpMM tolerance of the FP64 oracle; its sends total mu."""
    shiro = gu.lib()
    flags, Pr, Pc = 0, 4, 4
    if name == "rmat13":
        A = synth.rmat(13, 8, 161)
    elif name == "er4096_local":
        A, flags = synth.er(4096, 8, 1), shiro.SHIRO_PLAN_LOCAL_DIAG
    elif name == "ragged":
        A, Pr, Pc = synth.random_small(700, 900, 0.01, 162, empty_rows=50), 3, 5
    else:
        A, Pr, Pc = synth.hub_matrix(256, 4096, 3, 4000, 2, 163), 2, 2
    P = gu.plan_of(A, Pr, Pc, flags)
    JS = shiro.JointSpMM(P, Pr, Pc, flags=flags)
    B = synth.dense_normal(A.K, N, 164)
    if dt == torch.bfloat16:
        bits = synth.to_bf16_bits(B)
        B = synth.bf16_bits_to_f32(bits).reshape(B.shape)
        Bd = torch.from_numpy(bits.view(np.int16)).to(gu.dev()).view(torch.bfloat16)
    else:
        Bd = torch.from_numpy(B).to(gu.dev())
    C = JS.spmm(Bd)
    torch.cuda.synchronize()
    gu.check_spmm(A, B, C)
    sent_b, sent_c = JS.volumes()
    mu = int(JS.cover["mu"].sum())
    assert sent_b + sent_c == mu, (sent_b, sent_c, mu)
    assert sent_b == int(JS.cover["cover_cols"].sum()) and sent_c == int(JS.cover["cover_rows"].sum())


def _weights(A, kind, seed):
    if kind == "unit":
        return 1, 1
    if kind == "bf16_b_fp32_c":
        # B rows in BF16 (2 bytes) against FP32 partial C rows (4 bytes), N = 64.
        return 4 * 64, 2 * 64
    u = synth.uniform_f64(seed, synth.STREAM_VAL, 0, A.M + A.K)
    return (1 + (u[:A.M] * 20).astype(np.int64)), (1 + (u[A.M:] * 20).astype(np.int64))


@pytest.mark.parametrize("name", ["rmat12_4x4", "er4096_1d_local", "ragged_3x5", "hub"])
@pytest.mark.parametrize("kind", ["unit", "bf16_b_fp32_c", "per_vertex"])
def test_weighted_cover_matches_oracle(name, kind):
    """Dinic's min cut in the library against the oracle's (Edmonds-Karp): per tile the same
    cost, and -- the source-side reachable set being unique -- the same side for every nonzero."""
    shiro = gu.lib()
    flags, Pr, Pc = 0, 4, 4
    if name == "rmat12_4x4":
        A = synth.rmat(12, 8, 171)
    elif name == "er4096_1d_local":
        A, flags = synth.er(4096, 8, 1), shiro.SHIRO_PLAN_LOCAL_DIAG
    elif name == "ragged_3x5":
        A, Pr, Pc = synth.random_small(700, 900, 0.01, 172, empty_rows=50), 3, 5
    else:
        A, Pr, Pc = synth.hub_matrix(256, 4096, 3, 4000, 2, 173), 2, 2
    w_row, w_col = _weights(A, kind, 174)
    P = gu.plan_of(A, Pr, Pc, flags)
    W = P.joint_weighted(w_row, w_col)
    O = oracle.plan(A, Pr, Pc)
    wr = np.full(A.M, w_row, np.int64) if isinstance(w_row, int) else w_row
    wc = np.full(A.K, w_col, np.int64) if isinstance(w_col, int) else w_col
    rows = A.row_ids()
    t_of = (np.searchsorted(O.rb, rows, side="right") - 1) * Pc + \
        (np.searchsorted(O.cb, A.col, side="right") - 1)
    side = W["row_based"].numpy()
    expect_side = np.zeros(A.nnz, np.uint8)
    for t in range(O.T):
        p, q = O.tile_pq(t)
        if flags & shiro.SHIRO_PLAN_LOCAL_DIAG and p == q:
            assert int(W["cost"][t]) == 0
            continue
        nL, nR, ptr, adj = oracle.tile_graph(A, O, t)
        gcols = O.cols_sorted[O.tile_cols_ptr[t]:O.tile_cols_ptr[t + 1]]
        flow, cr, cc = oracle.min_weight_cover(nL, nR, ptr, adj, wr[O.rb[p]:O.rb[p + 1]], wc[gcols])
        assert int(W["cost"][t]) == flow, f"tile {t}: cost {int(W['cost'][t])} != {flow}"
        assert int(W["cover_rows"][t]) == int(cr.sum()) and int(W["cover_cols"][t]) == int(cc.sum())
        sel = t_of == t
        expect_side[sel] = np.where(cc[O.colidx_local[sel]], 0, 1)
    assert np.array_equal(side, expect_side), "side of some nonzero differs from the oracle's cut"
    if kind == "unit":
        J = P.joint()
        assert np.array_equal(J["mu"].numpy(), W["cost"].numpy())
        assert np.array_equal(J["row_based"].numpy(), side), "unit costs must give Koenig's cover"


def test_row_based_strategy():
    """Row-based strategy (Eq. 3): every communicated tile sends |Rows| partial C rows and no B
    row; C through the split equals the oracle's."""
    shiro = gu.lib()
    A = synth.rmat(12, 8, 181)
    for flags in (0, shiro.SHIRO_PLAN_LOCAL_DIAG):
        P = gu.plan_of(A, 4, 4, flags)
        R = P.row_based()
        O = oracle.plan(A, 4, 4)
        for t in range(O.T):
            p, q = O.tile_pq(t)
            expect = 0 if (flags and p == q) else int(O.tile_nrows[t])
            assert int(R["rows"][t]) == expect
        JS = shiro.JointSpMM(P, 4, 4, flags=flags, strategy="row")
        B = synth.dense_normal(A.K, 64, 182)
        C = JS.spmm(torch.from_numpy(B).to(gu.dev()))
        torch.cuda.synchronize()
        gu.check_spmm(A, B, C)
        sent_b, sent_c = JS.volumes()
        if not flags:
            assert sent_b == 0
        assert sent_c == int(R["rows"].sum())


def test_weighted_spmm_bf16_b():
    """With BF16 B rows (cost 2N) and FP32 partial C rows (cost 4N) the weighted cover is at most
    as dear as the uniform cover, the column-based and the row-based plans priced the same way,
    and C through its split matches the oracle."""
    shiro = gu.lib()
    A = synth.rmat(13, 8, 191)
    N = 64
    P = gu.plan_of(A, 4, 4)
    W = P.joint_weighted(4 * N, 2 * N)
    J = P.joint()
    O = oracle.plan(A, 4, 4)
    uniform_priced = int((4 * N * J["cover_rows"] + 2 * N * J["cover_cols"]).sum())
    assert int(W["cost"].sum()) <= uniform_priced
    assert int(W["cost"].sum()) <= 2 * N * int(O.tile_ncols.sum())
    assert int(W["cost"].sum()) <= 4 * N * int(O.tile_nrows.sum())
    JS = shiro.JointSpMM(P, 4, 4, strategy="weighted", w_row=4 * N, w_col=2 * N)
    B = synth.dense_normal(A.K, N, 192)
    bits = synth.to_bf16_bits(B)
    Bh = synth.bf16_bits_to_f32(bits).reshape(B.shape)
    Bd = torch.from_numpy(bits.view(np.int16)).to(gu.dev()).view(torch.bfloat16)
    C = JS.spmm(Bd)
    torch.cuda.synchronize()
    gu.check_spmm(A, Bh, C)
    sent_b, sent_c = JS.volumes()
    assert 2 * N * sent_b + 4 * N * sent_c == int(W["cost"].sum())


def test_weighted_cover_rejects_bad_costs():
    shiro = gu.lib()
    A = synth.rmat(10, 8, 195)
    P = gu.plan_of(A, 2, 2)
    with pytest.raises(shiro.ShiroError):
        P.joint_weighted(-1, 1)
    bad = np.ones(A.K, np.int64)
    bad[3] = -5
    with pytest.raises(shiro.ShiroError):
        P.joint_weighted(1, bad)
    with pytest.raises(ValueError):
        P.joint_weighted(1, np.ones(A.K + 1, np.int64))
