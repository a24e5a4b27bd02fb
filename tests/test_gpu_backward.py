"""Backward on the GPU: transposed plan (bit-exact), dB = A^T dC, dA by SDDMM, autograd, FD."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_20178_gb300 import synth
import gpu_util as gu

pytestmark = pytest.mark.gpu


def setup_module(_):
    gu.need_gpu()


def absA(A):
    return synth.CSR(A.M, A.K, A.rowptr, A.col, np.abs(A.val))


@pytest.mark.parametrize("name,Pr,Pc", [("rmat13", 4, 4), ("ragged", 3, 5), ("hub", 2, 2),
                                        ("empty_cols", 2, 3)])
def test_transpose_plan_parity(name, Pr, Pc):
    shiro = gu.lib()
    if name == "rmat13":
        A = synth.rmat(13, 8, 61)
    elif name == "ragged":
        A = synth.random_small(700, 1234, 0.01, 62)
    elif name == "hub":
        A = synth.hub_matrix(4096, 4096, 3, 4000, 3, 63)
    else:
        A = synth.random_small(300, 500, 0.005, 64, empty_rows=100)
    PT = gu.plan_of(A, Pr, Pc, shiro.SHIRO_PLAN_TRANSPOSE)
    rpT, colT, perm = PT.export_transpose()
    torch.cuda.synchronize()
    orp, ocol, operm = oracle.transpose(A)
    assert np.array_equal(rpT.cpu().numpy(), orp)
    assert np.array_equal(colT.cpu().numpy(), ocol)
    assert np.array_equal(perm.cpu().numpy(), operm)
    AT = synth.CSR(A.K, A.M, orp, ocol, A.val[operm])
    O = oracle.plan(A, Pr, Pc)
    OT = gu.assert_plan_matches(PT, AT, Pc, Pr)
    for p in range(Pr):
        for q in range(Pc):
            assert OT.tile_ncols[q * Pr + p] == O.tile_nrows[p * Pc + q]


def backward_case(A, N, Pr, Pc, dt=torch.float32, seed=70):
    shiro = gu.lib()
    B = synth.dense_normal(A.K, N, seed)
    G = synth.dense_normal(A.M, N, seed + 1)
    if dt == torch.bfloat16:
        Bq = synth.bf16_bits_to_f32(synth.to_bf16_bits(B)).reshape(B.shape)
        Gq = synth.bf16_bits_to_f32(synth.to_bf16_bits(G)).reshape(G.shape)
    else:
        Bq, Gq = B, G
    P = gu.plan_of(A, Pr, Pc)
    PT = gu.plan_of(A, Pr, Pc, shiro.SHIRO_PLAN_TRANSPOSE)
    d = gu.dev()
    Bd = torch.from_numpy(Bq).to(d).to(dt)
    Gd = torch.from_numpy(Gq).to(d).to(dt)
    Bp = P.pack(Bd)
    dB, dA = shiro.spmm_backward(P, PT, Gd, Bp, B=Bd)
    torch.cuda.synchronize()
    eB = gu.scaled_err(dB.cpu().numpy(), oracle.spmm_t(A, Gq), oracle.spmm_t(absA(A), np.abs(Gq)))
    eA = gu.scaled_err(dA.cpu().numpy(), oracle.sddmm(A, Gq, Bq),
                       oracle.sddmm(A, np.abs(Gq), np.abs(Bq)))
    assert eB <= gu.TOL, f"dB scaled error {eB}"
    assert eA <= gu.TOL, f"dA scaled error {eA}"
    return eB, eA


@pytest.mark.parametrize("N", [32, 64, 100, 128, 256])
def test_backward_rmat(N):
    backward_case(synth.rmat(13, 12, 71), N, 4, 4)


def test_backward_bf16():
    eB, eA = backward_case(synth.rmat(13, 12, 72), 128, 4, 4, torch.bfloat16)
    print("bf16 backward scaled errors", eB, eA)


def test_backward_hub_row():
    backward_case(synth.hub_matrix(64, 1 << 16, 5, 1 << 16, 2, 73), 128, 2, 2)


def test_autograd_matches_oracle():
    from paper_2512_20178_gb300 import autograd
    A = synth.rmat(12, 8, 74)
    N = 64
    B = synth.dense_normal(A.K, N, 75)
    G = synth.dense_normal(A.M, N, 76)
    rp, col, val = gu.to_dev(A)
    S = autograd.SparseMatrix(rp, col, val, A.M, A.K, 2, 2)
    v = S.val.requires_grad_(True)
    Bt = torch.from_numpy(B).to(gu.dev()).requires_grad_(True)
    C = autograd.spmm(S, Bt)
    C.backward(torch.from_numpy(G).to(gu.dev()))
    torch.cuda.synchronize()
    assert gu.scaled_err(C.detach().cpu().numpy(), oracle.spmm(A, B), oracle.abs_scale(A, B)) <= gu.TOL
    assert gu.scaled_err(Bt.grad.cpu().numpy(), oracle.spmm_t(A, G),
                         oracle.spmm_t(absA(A), np.abs(G))) <= gu.TOL
    assert gu.scaled_err(v.grad.cpu().numpy(), oracle.sddmm(A, G, B),
                         oracle.sddmm(A, np.abs(G), np.abs(B))) <= gu.TOL


def test_gcn_fd_fp64_subgraph():
    """GCN layer Y = A_hat (X W) on a 4096-node subgraph, FP64 on the GPU: central differences
    (h = 1e-6) on 64 entries each of X, W and A_hat's values against the analytic gradient."""
    from paper_2512_20178_gb300 import autograd
    full = synth.gcn_normalized(16, 16, 4)
    A = synth.renormalize_sym(synth.induced_subgraph(full, 4096))
    d = gu.dev()
    F, H = 64, 32
    X = torch.from_numpy(synth.dense_normal(A.M, F, 80, std=0.02)).to(d).double().requires_grad_(True)
    W = torch.from_numpy(synth.dense_normal(F, H, 81, std=0.02)).to(d).double().requires_grad_(True)
    Gl = torch.from_numpy(synth.dense_normal(A.M, H, 82)).to(d).double()
    rp, col, val = gu.to_dev(A, torch.float64)
    S = autograd.SparseMatrix(rp, col, val, A.M, A.K, 4, 4)
    v = S.val.requires_grad_(True)

    def loss():
        return (autograd.spmm(S, X @ W) * Gl).sum()

    L = loss()
    L.backward()
    gX, gW, gV = X.grad.clone(), W.grad.clone(), v.grad.clone()
    h = 1e-6
    pick = lambda n, s: (synth.uniform_f64(s, synth.STREAM_PERM, 0, 64) * n).astype(np.int64)
    with torch.no_grad():
        for T, g, s in ((X, gX, 90), (W, gW, 91), (v, gV, 92)):
            flat, gflat = T.view(-1), g.view(-1)
            for idx in pick(flat.numel(), s):
                old = flat[idx].item()
                flat[idx] = old + h
                lp = loss().item()
                flat[idx] = old - h
                lm = loss().item()
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                an = gflat[idx].item()
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (T.shape, int(idx), fd, an)


def test_gcn_full_fp32_vs_oracle():
    """GCN A_hat (R-MAT 2^20, avg degree 16, symmetrised + self loops), N = 128: forward, dH and dA
    in FP32 against the FP64 oracle (dH on every row, the others sampled)."""
    shiro = gu.lib()
    A = synth.gcn_normalized(20, 16, 4)
    N = 128
    Hh = synth.dense_normal(A.K, N, 93)
    G = synth.dense_normal(A.M, N, 94)
    d = gu.dev()
    P = gu.plan_of(A, 4, 4)
    PT = gu.plan_of(A, 4, 4, shiro.SHIRO_PLAN_TRANSPOSE)
    Hd = torch.from_numpy(Hh).to(d)
    Gd = torch.from_numpy(G).to(d)
    Hp = P.pack(Hd)
    Y = P.spmm(Hp)
    dH, dA = shiro.spmm_backward(P, PT, Gd, Hp, B=Hd)
    torch.cuda.synchronize()
    rows = np.unique((synth.uniform_f64(95, synth.STREAM_PERM, 0, 3000) * A.M).astype(np.int64))
    gu.check_spmm(A, Hh, Y, rows=rows)
    eB = gu.scaled_err(dH.cpu().numpy(), oracle.spmm_t(A, G), oracle.spmm_t(absA(A), np.abs(G)))
    assert eB <= gu.TOL, eB
    es = (synth.uniform_f64(96, synth.STREAM_PERM, 0, 200000) * A.nnz).astype(np.int64)
    eA = gu.sampled_sddmm_error(A, G, Hh, dA.cpu().numpy(), es)
    assert eA <= gu.TOL, f"dA (sampled) scaled error {eA}"


@pytest.mark.parametrize("case", ["f32_n128", "f32_n64", "bf16_n128", "bf16_n256", "hub",
                                  "local_diag", "empty_rows", "ragged"])
def test_sddmm_kernels(case):
    """dA by every SDDMM kernel -- lane groups of eight lanes per nonzero (the default for 16-byte
    aligned rows of 128 to 512 bytes), 48 registers with the shared-memory tile reduction
    (pipeline 6; pipeline 3 for BF16 and FP32 N = 64), 48 registers with the 4-wide shuffle
    butterfly (pipeline 3, FP32 N = 128) and 64 registers with the 8-wide butterfly (pipeline 5,
    persistent mode) -- within the oracle bound on the same inputs, including hub rows cut into
    chunks, 1D local diagonal tiles read from B in place, empty rows and a ragged last batch."""
    shiro = gu.lib()
    flags, dt, N = 0, torch.float32, 128
    A = synth.rmat(13, 12, 140)
    if case == "f32_n64":
        N = 64
    elif case.startswith("bf16"):
        dt = torch.bfloat16
        N = 256 if case.endswith("256") else 128
    elif case == "hub":
        A = synth.hub_matrix(300, 1 << 15, 7, 20000, 3, 141)
    elif case == "local_diag":
        flags = shiro.SHIRO_PLAN_LOCAL_DIAG
    elif case == "empty_rows":
        A = synth.random_small(900, 700, 0.02, 142, empty_rows=300)
    elif case == "ragged":
        A = synth.random_small(333, 517, 0.037, 143)
    B = synth.dense_normal(A.K, N, 144)
    G = synth.dense_normal(A.M, N, 145)
    if dt == torch.bfloat16:
        B = synth.bf16_bits_to_f32(synth.to_bf16_bits(B)).reshape(B.shape)
        G = synth.bf16_bits_to_f32(synth.to_bf16_bits(G)).reshape(G.shape)
    d = gu.dev()
    Bd = torch.from_numpy(B).to(d).to(dt)
    Gd = torch.from_numpy(G).to(d).to(dt)
    ref = oracle.sddmm(A, G, B)
    scale = oracle.sddmm(A, np.abs(G), np.abs(B))
    for pipe, pers in [(0, 0), (3, 0), (5, 0), (6, 0), (0, 1)]:
        opts = shiro.make_opts(pipeline=pipe, persistent=pers, long_row_nnz=128, chunk_nnz=64)
        P = gu.plan_of(A, 4, 4, flags, opts=opts)
        Bp = P.pack(Bd)
        dA = P.sddmm(Gd, Bp, B=Bd)
        torch.cuda.synchronize()
        err = gu.scaled_err(dA.cpu().numpy(), ref, scale)
        assert err <= gu.TOL, f"pipeline {pipe} persistent {pers}: dA scaled error {err}"
