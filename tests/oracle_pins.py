"""Checks that pin the FP64 oracle to facts outside itself.

Each ``check_*`` raises AssertionError on a mismatch.  The facts come from mathematics and from the
paper, never from the oracle's own code paths:

* dense FP64 matrix products (numpy) on tiny inputs -- the textbook definition of C = A B (Sec. 2.1),
  A^T dC and the sampled product dC B^T on A's pattern;
* identity, permutation and diagonal A, whose products are exact;
* Python ``set`` brute force for Cols/Rows of every tile (Tab. 1, Eq. 2, Eq. 3) and the invariants
  Cols_t[colidx_local[e]] == col[e], sum_q |Cols(A^(p,q))| == |Cols(A^(p,:))|, V_block >= V_col;
* |Cols(A^T tile (q,p))| == |Rows(A tile (p,q))|;
* the worked example of Fig. 1 / Sec. 5.2, rebuilt from its captions (tests/golden);
* brute-force minimum vertex covers (the 0-1 program of Eq. 4-6 by enumeration) for the matching
  size (Koenig's theorem), and a full row + full column pattern whose cover is 2.

The same checks run against deliberately broken builds of the oracle (test_oracle_mutants.py), so a
plausible mistake in it -- a dropped term, a wrong index or sign, a transposed operand, an
off-by-one tile boundary -- is shown to fail at least one of them.
"""
from __future__ import annotations

import itertools
import os

import numpy as np

import oracle
from paper_2512_20178_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def dense_of(A) -> np.ndarray:
    D = np.zeros((A.M, A.K), dtype=np.float64)
    rows = A.row_ids()
    np.add.at(D, (rows, A.col.astype(np.int64)), A.val.astype(np.float64))
    return D


def small_cases():
    """(A, N, seed) tiny cases: ragged shapes, empty rows, a dense row, a single column."""
    cases = []
    for k, (M, K, dens, N, er) in enumerate([(17, 23, 0.2, 3, 2), (64, 64, 0.1, 8, 5),
                                              (5, 40, 0.5, 1, 0), (40, 5, 0.4, 7, 3),
                                              (33, 1, 0.5, 4, 1), (1, 1, 1.0, 2, 0)]):
        cases.append((synth.random_small(M, K, dens, 100 + k, empty_rows=er), N, 200 + k))
    cases.append((synth.hub_matrix(48, 64, 7, 60, 2, 300), 5, 301))
    return cases


def check_spmm_dense():
    for A, N, seed in small_cases():
        B = synth.dense_normal(A.K, N, seed)
        C = oracle.spmm(A, B)
        ref = dense_of(A) @ B.astype(np.float64)
        S = np.abs(dense_of(A)) @ np.abs(B.astype(np.float64))
        assert np.all(np.abs(C - ref) <= 1e-12 * S + 1e-300), "spmm != dense A @ B"
        rows = np.array([0, A.M - 1, A.M // 2], dtype=np.int64)
        Cr = oracle.spmm(A, B, rows=rows)
        assert np.array_equal(Cr, C[rows]), "row-sampled spmm differs from the full one"


def check_spmm_exact_structures():
    n, N = 37, 6
    B = synth.dense_normal(n, N, 7)
    eye = synth.from_dense(np.eye(n, dtype=np.float32))
    assert np.array_equal(oracle.spmm(eye, B), B.astype(np.float64)), "I B != B"
    perm = np.argsort(synth.uniform_f64(3, synth.STREAM_PERM, 0, n))
    P = np.zeros((n, n), dtype=np.float32)
    P[np.arange(n), perm] = 1.0
    assert np.array_equal(oracle.spmm(synth.from_dense(P), B), B[perm].astype(np.float64)), \
        "permutation A gives wrong rows"
    d = (synth.uniform_f32(5, synth.STREAM_VAL, 0, n) - np.float32(0.5)).astype(np.float32)
    d[3] = 0.0
    D = synth.from_dense(np.diag(d))
    ref = d.astype(np.float64)[:, None] * B.astype(np.float64)
    assert np.array_equal(oracle.spmm(D, B), ref), "diagonal A does not scale rows"


def brute_tiles(A, rb, cb, diag_only=False):
    """{t: (cols_set, rows_set, nnz)} by Python sets."""
    Pr, Pc = len(rb) - 1, len(cb) - 1
    out = {}
    rows = A.row_ids()
    for p in range(Pr):
        qs = [p] if diag_only else range(Pc)
        for q in qs:
            t = p if diag_only else p * Pc + q
            cs, rs, n = set(), set(), 0
            for e in range(A.nnz):
                i, j = int(rows[e]), int(A.col[e])
                if rb[p] <= i < rb[p + 1] and cb[q] <= j < cb[q + 1]:
                    cs.add(j)
                    rs.add(i)
                    n += 1
            out[t] = (cs, rs, n)
    return out


def check_plan_bruteforce():
    grids = [(1, 1), (2, 3), (4, 4), (3, 1), (1, 5), (7, 6)]
    for (A, N, _), (Pr, Pc) in itertools.product(small_cases(), grids):
        P = oracle.plan(A, Pr, Pc)
        ref = brute_tiles(A, P.rb, P.cb)
        rows = A.row_ids()
        for t in range(P.T):
            cs, rs, n = ref[t]
            assert list(P.cols_of(t)) == sorted(cs), "Cols of a tile wrong or not ascending"
            assert P.tile_ncols[t] == len(cs) and P.tile_nrows[t] == len(rs), "|Cols|/|Rows| wrong"
            assert P.tile_nnz[t] == n, "tile nnz wrong"
        for e in range(A.nnz):
            p = int(np.searchsorted(P.rb, rows[e], side="right") - 1)
            q = int(np.searchsorted(P.cb, A.col[e], side="right") - 1)
            t = p * Pc + q
            assert P.cols_of(t)[P.colidx_local[e]] == A.col[e], "remap does not point back"
        for p in range(Pr):
            row_cols = {int(A.col[e]) for e in range(A.nnz) if P.rb[p] <= rows[e] < P.rb[p + 1]}
            assert sum(P.tile_ncols[p * Pc:(p + 1) * Pc]) == len(row_cols), \
                "sum_q |Cols(A^(p,q))| != |Cols(A^(p,:))|"
        assert P.tile_cols_ptr[-1] <= min(A.nnz, Pr * A.K)
        vb, vc, vr = P.volumes(N, 4)
        assert np.all(vb >= vc), "V_block < V_col"
        for t in range(P.T):
            cs, rs, _ = ref[t]
            # Eq. 2 and Eq. 3: bytes of the B rows the tile names, of its partial C rows.
            assert vc[t] == np.zeros((len(cs), N), np.float32).nbytes, "V_col"
            assert vr[t] == np.zeros((len(rs), N), np.float32).nbytes, "V_row"


def check_uniform_bounds():
    for n, P in [(10, 3), (10, 4), (5, 4), (4096, 4), (1, 3), (0, 2), (7, 7)]:
        b = oracle.uniform_bounds(n, P)
        step = -(-n // P) if n else 0
        assert b[0] == 0 and b[-1] == n, "bounds do not cover [0, n)"
        assert all(b[p] == min(p * step, n) for p in range(P + 1)), "bounds are not p*ceil(n/P)"


def check_plan_diag_only():
    gs = [synth.random_small(m, m, 0.3, 50 + m) for m in (3, 9, 1, 14)]
    n = sum(g.M for g in gs)
    D = np.zeros((n, n), dtype=np.float32)
    off = 0
    bounds = [0]
    for g in gs:
        D[off:off + g.M, off:off + g.M] = dense_of(g)
        off += g.M
        bounds.append(off)
    A = synth.from_dense(D)
    b = np.array(bounds, dtype=np.int64)
    P = oracle.plan(A, len(gs), len(gs), rb=b, cb=b, diag_only=True)
    for t, g in enumerate(gs):
        expect = sorted({int(c) + int(b[t]) for c in g.col})
        assert list(P.cols_of(t)) == expect, "diag-only Cols != the graph's nonempty columns"
    D2 = D.copy()
    D2[0, n - 1] = 1.0
    try:
        oracle.plan(synth.from_dense(D2), len(gs), len(gs), rb=b, cb=b, diag_only=True)
    except ValueError:
        pass
    else:
        raise AssertionError("diag-only plan accepted an off-diagonal nonzero")


def check_pack_and_packed_spmm():
    for (A, N, seed), (Pr, Pc) in itertools.product(small_cases(), [(2, 2), (3, 4), (4, 4)]):
        B = synth.dense_normal(A.K, N, seed)
        P = oracle.plan(A, Pr, Pc)
        for local_diag in (False, True):
            pack_ptr, src = P.pack_layout(local_diag)
            Bp = oracle.pack(B, src)
            assert np.array_equal(Bp, B[src]), "pack is not a row copy"
            bits = synth.to_bf16_bits(B)
            assert np.array_equal(oracle.pack(bits, src), bits[src]), "bf16 pack not bit-exact"
            C1 = oracle.spmm_packed(A, P, Bp, B, local_diag)
            assert np.array_equal(C1, oracle.spmm(A, B)), "packed path != direct path (FP64)"


def check_transpose_and_rows():
    for (A, N, seed), (Pr, Pc) in itertools.product(small_cases(), [(2, 3), (4, 4)]):
        rowptrT, colT, perm = oracle.transpose(A)
        rows = A.row_ids()
        pairs = sorted((int(A.col[e]), int(rows[e]), e) for e in range(A.nnz))
        assert [p[1] for p in pairs] == list(colT), "A^T rows not in ascending row order"
        assert [p[2] for p in pairs] == list(perm), "perm of A^T wrong"
        cnt = np.bincount(A.col, minlength=A.K)
        assert np.array_equal(np.diff(rowptrT), cnt), "rowptr of A^T wrong"
        AT = synth.CSR(A.K, A.M, rowptrT, colT, A.val[perm])
        P = oracle.plan(A, Pr, Pc)
        PT = oracle.plan(AT, Pc, Pr)
        for p in range(Pr):
            for q in range(Pc):
                assert PT.tile_ncols[q * Pr + p] == P.tile_nrows[p * Pc + q], \
                    "|Cols(A^T tile (q,p))| != |Rows(A tile (p,q))|"


def check_backward_dense():
    for A, N, seed in small_cases():
        G = synth.dense_normal(A.M, N, seed + 1)
        B = synth.dense_normal(A.K, N, seed)
        D = dense_of(A)
        dB = oracle.spmm_t(A, G)
        S = np.abs(D.T) @ np.abs(G.astype(np.float64))
        assert np.all(np.abs(dB - D.T @ G.astype(np.float64)) <= 1e-12 * S + 1e-300), \
            "A^T dC wrong"
        full = G.astype(np.float64) @ B.astype(np.float64).T
        rows = A.row_ids()
        ref = full[rows, A.col]
        got = oracle.sddmm(A, G, B)
        sc = np.abs(G.astype(np.float64)) @ np.abs(B.astype(np.float64)).T
        assert np.all(np.abs(got - ref) <= 1e-12 * sc[rows, A.col] + 1e-300), "SDDMM wrong"


def check_abs_scale():
    for A, N, seed in small_cases():
        B = synth.dense_normal(A.K, N, seed)
        S = oracle.abs_scale(A, B)
        ref = np.abs(dense_of(A)) @ np.abs(B.astype(np.float64))
        assert np.allclose(S, ref, rtol=1e-13, atol=0), "abs scale wrong"


def read_golden(name):
    nz, expect, meta = [], {}, {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = line.split()
            if w[0] == "nz":
                nz.append((w[1], int(w[2]), int(w[3])))
            elif w[0] == "expect":
                expect[w[1]] = [int(x) for x in w[2:]]
            else:
                meta[w[0]] = [int(x) for x in w[1:]]
    return nz, expect, meta


def check_fig1_golden():
    nz, expect, meta = read_golden("fig1_offdiag_tile.txt")
    M, K = meta["shape"]
    Pr, Pc = meta["partition"]
    D = np.zeros((M, K), dtype=np.float32)
    for _, i, j in nz:
        D[i, j] = 1.0
    A = synth.from_dense(D)
    P = oracle.plan(A, Pr, Pc)
    t = 0 * Pc + 1
    assert list(P.cols_of(t)) == expect["cols_tile_0_1"]
    assert P.tile_ncols[t] == expect["ncols_tile_0_1"][0]
    assert P.tile_nrows[t] == expect["nrows_tile_0_1"][0]
    assert P.tile_nnz[t] == expect["nnz_tile_0_1"][0]
    # Rows of the tile == Cols of the transposed tile (1, 0).
    rowptrT, colT, perm = oracle.transpose(A)
    PT = oracle.plan(synth.CSR(K, M, rowptrT, colT, A.val[perm]), Pc, Pr)
    assert list(PT.cols_of(1 * Pr + 0)) == expect["rows_tile_0_1"]
    # Smallest set of rows and columns covering every nonzero (Eq. 4-6), by brute force.
    verts = [("r", i) for i in expect["rows_tile_0_1"]] + [("c", j) for j in expect["cols_tile_0_1"]]
    best = min(len(s) for k in range(len(verts) + 1) for s in itertools.combinations(verts, k)
               if all(("r", i) in s or ("c", j) in s for _, i, j in nz))
    assert best == expect["min_cover"][0]


def check_er_band():
    """ER G(4096, 8/4096), 4x4 tiles: E|Cols_t| = 1024 (1 - (1 - p)^1024) ~ 885.4 (sanity band)."""
    A = synth.er(4096, 8, 1)
    P = oracle.plan(A, 4, 4)
    p = 8 / 4096
    mean = 1024 * (1 - (1 - p) ** 1024)
    assert abs(P.tile_ncols.mean() - mean) < 30, P.tile_ncols
    assert np.all(np.abs(P.tile_ncols - mean) < 80)


def brute_min_cover(nL, nR, edges):
    """Smallest set of rows and columns covering every edge (Eq. 4-6), by enumeration."""
    verts = [("r", i) for i in range(nL)] + [("c", j) for j in range(nR)]
    for k in range(len(verts) + 1):
        for sel in itertools.combinations(verts, k):
            ss = set(sel)
            if all(("r", i) in ss or ("c", j) in ss for i, j in edges):
                return k
    return len(verts)


def check_matching_is_min_cover():
    for seed in range(40):
        u = synth.uniform_f64(seed, synth.STREAM_PERM, 0, 3)
        nL, nR = 1 + int(u[0] * 6), 1 + int(u[1] * 6)
        dens = 0.15 + 0.6 * u[2]
        m = synth.uniform_f64(seed, synth.STREAM_ER, 0, nL * nR).reshape(nL, nR) < dens
        edges = [(i, j) for i in range(nL) for j in range(nR) if m[i, j]]
        ptr = np.zeros(nL + 1, np.int64)
        adj = []
        for i in range(nL):
            adj += [j for j in range(nR) if m[i, j]]
            ptr[i + 1] = len(adj)
        mu = oracle.max_matching(nL, nR, ptr, np.array(adj, np.int32))
        assert mu == brute_min_cover(nL, nR, edges), "matching size != minimum vertex cover"
    # Cross pattern (a full row and a full column, Sec. 5.4 pattern with hubs on both sides).
    n = 9
    adj = list(range(n)) + [0] * (n - 1)
    ptr = np.array([0, n] + [n + i for i in range(1, n)], np.int64)
    assert oracle.max_matching(n, n, ptr, np.array(adj, np.int32)) == 2


def check_fig1_joint_cover():
    nz, expect, meta = read_golden("fig1_offdiag_tile.txt")
    M, K = meta["shape"]
    Pr, Pc = meta["partition"]
    D = np.zeros((M, K), dtype=np.float32)
    for _, i, j in nz:
        D[i, j] = 1.0
    A = synth.from_dense(D)
    P = oracle.plan(A, Pr, Pc)
    assert oracle.max_matching(*oracle.tile_graph(A, P, 1)) == expect["min_cover"][0]


def _tiny_graph(seed, max_side=7):
    u = synth.uniform_f64(seed, synth.STREAM_PERM, 0, 3)
    nL, nR = 1 + int(u[0] * max_side), 1 + int(u[1] * max_side)
    dens = 0.15 + 0.6 * u[2]
    m = synth.uniform_f64(seed, synth.STREAM_ER, 0, nL * nR).reshape(nL, nR) < dens
    ptr = np.zeros(nL + 1, np.int64)
    adj = []
    for i in range(nL):
        adj += [j for j in range(nR) if m[i, j]]
        ptr[i + 1] = len(adj)
    return nL, nR, ptr, np.array(adj, np.int32), m


def brute_weighted_covers(nL, nR, m, w_row, w_col):
    """All covers of minimum cost (Eq. 4-6 with per-vertex costs), by enumerating the selected
    rows; the columns are then forced: every neighbour of an unselected row.  Returns the minimum
    cost and the list of (row set, column set) reaching it (costs > 0, so no extra vertex is ever
    free)."""
    best, covers = None, []
    for mask in range(1 << nL):
        rows = {i for i in range(nL) if mask >> i & 1}
        cols = {j for i in range(nL) if i not in rows for j in range(nR) if m[i, j]}
        c = sum(int(w_row[i]) for i in rows) + sum(int(w_col[j]) for j in cols)
        if best is None or c < best:
            best, covers = c, [(rows, cols)]
        elif c == best:
            covers.append((rows, cols))
    return best, covers


def check_weighted_cover_bruteforce():
    """Min cut of Sec. 5.3.3 = minimum weighted vertex cover (Eq. 4-6), and the selection read off
    the residual reachability is the minimum cover whose column set lies inside every other's."""
    for seed in range(60):
        nL, nR, ptr, adj, m = _tiny_graph(seed)
        w = synth.uniform_f64(seed, synth.STREAM_VAL, 0, nL + nR)
        w_row = 1 + (w[:nL] * 9).astype(np.int64)
        w_col = 1 + (w[nL:] * 9).astype(np.int64)
        flow, cr, cc = oracle.min_weight_cover(nL, nR, ptr, adj, w_row, w_col)
        best, covers = brute_weighted_covers(nL, nR, m, w_row, w_col)
        assert flow == best, f"max flow {flow} != minimum cover cost {best}"
        assert int(w_row[cr].sum() + w_col[cc].sum()) == flow, "cut cost != max flow"
        assert all(cr[i] or cc[j] for i in range(nL) for j in range(nR) if m[i, j]), "edge uncovered"
        inter = set(range(nR))
        for _, cols in covers:
            inter &= cols
        assert set(np.flatnonzero(cc).tolist()) == inter, "cover is not the source-minimal cut"
        assert not np.any(cr & (np.diff(ptr) == 0)), "isolated row selected"


def check_weighted_cover_special_cases():
    """Uniform costs reduce to Koenig (cost = c * maximum matching); one side far dearer than
    the other selects every non-isolated vertex of the cheap side; zero costs are free."""
    for seed in range(30):
        nL, nR, ptr, adj, m = _tiny_graph(100 + seed)
        mu = oracle.max_matching(nL, nR, ptr, adj)
        for c in (1, 7):
            flow, _, _ = oracle.min_weight_cover(nL, nR, ptr, adj, np.full(nL, c), np.full(nR, c))
            assert flow == c * mu, "uniform costs must give c * mu"
        used_cols = m.any(axis=0)
        used_rows = m.any(axis=1)
        big = 100 * (nL + nR)
        flow, cr, cc = oracle.min_weight_cover(nL, nR, ptr, adj, np.full(nL, big), np.ones(nR))
        assert flow == int(used_cols.sum()) and not cr.any() and np.array_equal(cc, used_cols)
        flow, cr, cc = oracle.min_weight_cover(nL, nR, ptr, adj, np.ones(nL), np.full(nR, big))
        assert flow == int(used_rows.sum()) and not cc.any() and np.array_equal(cr, used_rows)
        flow, cr, cc = oracle.min_weight_cover(nL, nR, ptr, adj, np.ones(nL), np.zeros(nR))
        assert flow == 0 and np.array_equal(cc, used_cols) and not cr.any()
    # A star: one row on five columns costs its row when rows are cheaper than five columns.
    ptr = np.array([0, 5], np.int64)
    adj = np.arange(5, dtype=np.int32)
    assert oracle.min_weight_cover(1, 5, ptr, adj, [4], np.ones(5))[0] == 4
    assert oracle.min_weight_cover(1, 5, ptr, adj, [6], np.ones(5))[0] == 5


def check_fig1_weighted_cover():
    """The off-diagonal tile of the Fig. 1 example: unit costs give the joint optimum of the
    golden file; its cover is a valid one of that size."""
    nz, expect, meta = read_golden("fig1_offdiag_tile.txt")
    M, K = meta["shape"]
    Pr, Pc = meta["partition"]
    D = np.zeros((M, K), dtype=np.float32)
    for _, i, j in nz:
        D[i, j] = 1.0
    A = synth.from_dense(D)
    P = oracle.plan(A, Pr, Pc)
    nL, nR, ptr, adj = oracle.tile_graph(A, P, 1)
    flow, cr, cc = oracle.min_weight_cover(nL, nR, ptr, adj, np.ones(nL), np.ones(nR))
    assert flow == expect["min_cover"][0] == int(cr.sum() + cc.sum())


def check_scaled_error_hand_cases():
    """The error metric every parity verdict goes through (the tolerance stated on C = A B,
    Sec. 2.1: |C_ik - C64_ik| / sum_j |a_ij||b_jk|, exact zeros where that scale is 0), on triples
    whose answer is worked out by hand.  The maximum sits where C < C64 and where S differs from
    |C64|, so a signed difference or a division by |C64| lands elsewhere."""
    inf = float("inf")
    C, C64, S = [[1.0, 2.0, 3.0]], [[1.0, 2.5, 2.0]], [[2.0, 4.0, 16.0]]
    # element errors 0, 0.5 / 4, 1 / 16: the maximum is 0.125, exactly representable.
    assert oracle.scaled_error(C, C64, S) == 0.125, "known maximum element"
    assert oracle.scaled_error([[0.0, -0.0]], [[0.0, 0.0]], [[0.0, 0.0]]) == 0.0, \
        "S = 0 and C = 0 must count 0"
    assert oracle.scaled_error([[1e-30, 0.0]], [[0.0, 0.0]], [[0.0, 1.0]]) == inf, \
        "S = 0 and C != 0 must fail"
    # Mixed rows: element errors (1/16, 0) and (0, 1/4); the maximum is 0.25 (a mean would be
    # 5/64, a per-row mean 1/8), the per-row maxima 1/16 and 1/4.
    C, C64, S = [[1.0, 1.0], [10.0, 10.0]], [[1.5, 1.0], [10.0, 10.25]], [[8.0, 1.0], [1.0, 1.0]]
    assert oracle.scaled_error(C, C64, S) == 0.25, "maximum over mixed rows"
    rm = oracle.scaled_error(C, C64, S, per_row=True)
    assert list(rm) == [0.0625, 0.25], "per-row maxima"
    assert oracle.scaled_error([[float("nan")]], [[1.0]], [[1.0]]) == inf, "NaN must fail"
    assert oracle.scaled_error(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 3))) == 0.0
    # 1-D results (SDDMM values): the same metric per nonzero.
    assert oracle.scaled_error([3.0, -1.0], [2.0, -1.0], [8.0, 2.0]) == 0.125


def check_scaled_error_fp32_bounds():
    """Facts of floating-point arithmetic the metric must reproduce on real products: the FP64
    result rounded once to FP32 has scaled error at most 2^-24 (|fl(x) - x| <= u |x| <= u S), and
    a plain FP32 sum of a row's FP32 products in CSR order has scaled error at most
    gamma_n = n u / (1 - n u) for n nonzeros in the row (the dot-product bound of Higham, Accuracy
    and Stability of Numerical Algorithms, Sec. 3.1), and above 0 somewhere."""
    u = 2.0 ** -24
    A = synth.random_small(64, 96, 0.3, 17, empty_rows=4)
    B = synth.dense_normal(A.K, 16, 18)
    C64 = oracle.spmm(A, B)
    S = oracle.abs_scale(A, B)
    assert oracle.scaled_error(C64.astype(np.float32), C64, S) <= u
    C32 = np.zeros((A.M, 16), dtype=np.float32)
    for i in range(A.M):
        acc = np.zeros(16, dtype=np.float32)
        for e in range(int(A.rowptr[i]), int(A.rowptr[i + 1])):
            acc = (acc + np.float32(A.val[e]) * B[A.col[e]]).astype(np.float32)
        C32[i] = acc
    rm = oracle.scaled_error(C32, C64, S, per_row=True)
    n = np.diff(A.rowptr)
    gamma = n * u / (1 - n * u)
    assert np.all(rm <= gamma), "FP32 sum beyond the dot-product error bound"
    assert rm.max() > 0, "an FP32 sum of these rows is inexact somewhere"
    assert np.all(rm[n == 0] == 0), "empty rows are exact"


def check_volumes_exact():
    """Eq. 1: a tile's block volume is the size in bytes of the block of B owned by the tile's
    column process, B^(q) = rows [k_q, k_(q+1)) of B; summed over the tiles of one row block it
    is the whole of B.  Ragged custom bounds with P_r != P_c, and every element size."""
    A = synth.random_small(13, 17, 0.4, 9)
    rb = np.array([0, 5, 6, 13], np.int64)
    cb = np.array([0, 3, 4, 11, 17], np.int64)
    P = oracle.plan(A, 3, 4, rb=rb, cb=cb)
    for N, dt in [(5, np.float32), (3, np.int16), (2, np.float64)]:
        B = np.zeros((A.K, N), dtype=dt)
        vb, vc, vr = P.volumes(N, B.itemsize, 8)
        assert np.array_equal(vr, P.tile_nrows * np.zeros((1, N), np.float64).nbytes)
        for p in range(3):
            for q in range(4):
                assert vb[p * 4 + q] == B[cb[q]:cb[q + 1]].nbytes, "V_block != bytes of B^(q)"
            assert vb[p * 4:(p + 1) * 4].sum() == B.nbytes, "V_block over a row block != |B|"
        assert np.all(vc <= vb)
    g = [synth.random_small(m, m, 0.5, 60 + m) for m in (2, 7, 4)]
    D = np.zeros((13, 13), dtype=np.float32)
    b = np.array([0, 2, 9, 13], np.int64)
    for t, gr in enumerate(g):
        D[b[t]:b[t + 1], b[t]:b[t + 1]] = dense_of(gr)
    Pd = oracle.plan(synth.from_dense(D), 3, 3, rb=b, cb=b, diag_only=True)
    B = np.zeros((13, 4), dtype=np.float32)
    vb, _, _ = Pd.volumes(4, 4)
    assert [int(x) for x in vb] == [B[b[t]:b[t + 1]].nbytes for t in range(3)], "diag-only V_block"
    # 1D plan with local diagonal tiles (Sec. 2.2): those tiles send nothing, the others are
    # unchanged.
    Pq = oracle.plan(A, 3, 3)
    full = Pq.volumes(4, 2)
    loc = Pq.volumes(4, 2, local_diag=True)
    for t in range(9):
        for f, l in zip(full, loc):
            assert l[t] == (0 if t // 3 == t % 3 else f[t]), "local diagonal tile volumes"


ALL_CHECKS = [check_weighted_cover_bruteforce, check_weighted_cover_special_cases,
              check_fig1_weighted_cover, check_matching_is_min_cover, check_fig1_joint_cover, check_spmm_dense, check_spmm_exact_structures, check_plan_bruteforce,
              check_uniform_bounds, check_plan_diag_only, check_pack_and_packed_spmm,
              check_transpose_and_rows, check_backward_dense, check_abs_scale, check_fig1_golden,
              check_er_band, check_scaled_error_hand_cases, check_scaled_error_fp32_bounds,
              check_volumes_exact]
