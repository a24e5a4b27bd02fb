"""Pack and SpMM parity on the GPU against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_20178_gb300 import synth
import gpu_util as gu

pytestmark = pytest.mark.gpu


def setup_module(_):
    gu.need_gpu()


def run(A, B, Pr=1, Pc=1, flags=0, opts=None):
    P = gu.plan_of(A, Pr, Pc, flags, opts=opts)
    Bd = torch.from_numpy(B).to(gu.dev())
    Bp = P.pack(Bd)
    C = P.spmm(Bp, B=Bd)
    torch.cuda.synchronize()
    return P, Bd, Bp, C


SMALL_SPLIT = dict(long_row_nnz=64, chunk_nnz=32, group_nnz=40, group_rows=7)


@pytest.mark.parametrize("N", [1, 7, 32, 33, 64, 100, 128, 256, 512])
def test_spmm_n_sweep(N):
    A = synth.rmat(12, 8, 21)
    B = synth.dense_normal(A.K, N, 22)
    shiro = gu.lib()
    P, Bd, Bp, C = run(A, B, 4, 4, opts=shiro.make_opts(**SMALL_SPLIT))
    assert P.info.n_long_rows > 0
    src = P.export()["pack_src"].cpu().numpy()
    assert np.array_equal(Bp.cpu().numpy(), B[src]), "pack is not bit-exact"
    gu.check_spmm(A, B, C)


@pytest.mark.parametrize("case", ["er4096_1d_local", "rmat14", "rmat14_bf16_n256"])
def test_auto_groups_bit_identical(case):
    """group_nnz 0 (automatic) cuts small matrices into more, shorter items than 256-nonzero
    groups; rows are never split, so C and dA are bit-identical to the explicit 256 schedule."""
    shiro = gu.lib()
    flags = 0
    dt = torch.float32
    if case.startswith("er4096"):
        A, Pr, N = synth.er(4096, 8, 1), 4, 32
        flags = shiro.SHIRO_PLAN_LOCAL_DIAG
    else:
        A, Pr, N = synth.rmat(14, 16, 3), 4, 128
        if case.endswith("bf16_n256"):
            dt, N = torch.bfloat16, 256
    P = gu.plan_of(A, Pr, Pr, flags)
    assert P.info.opts.group_nnz == 0
    d = gu.dev()
    Bd = torch.from_numpy(synth.dense_normal(A.K, N, 5)).to(d).to(dt)
    dC = torch.from_numpy(synth.dense_normal(A.M, N, 6)).to(d).to(dt)
    out = {}
    for gn in (0, 256):
        P.reschedule(group_nnz=gn)
        Bp = P.pack(Bd)
        C = P.spmm(Bp, B=Bd)
        dA = P.sddmm(dC, Bp, B=Bd)
        torch.cuda.synchronize()
        P.check()
        out[gn] = (P.info.n_items, C, dA)
    assert out[0][0] > out[256][0], "automatic groups should give more items on a small matrix"
    assert torch.equal(out[0][1], out[256][1]) and torch.equal(out[0][2], out[256][2])
    if dt == torch.float32:
        gu.check_spmm(A, Bd.cpu().numpy(), out[0][1])


@pytest.mark.parametrize("name", ["er4096_2d", "er4096_1d_local", "ragged", "more_blocks",
                                  "empty_rows", "rmat14_default"])
def test_spmm_cases(name):
    shiro = gu.lib()
    flags = 0
    if name.startswith("er4096"):
        A, Pr, Pc, N = synth.er(4096, 8, 1), 4, 4, 32
        if name.endswith("local"):
            flags = shiro.SHIRO_PLAN_LOCAL_DIAG
    elif name == "ragged":
        A, Pr, Pc, N = synth.random_small(1000, 777, 0.01, 11), 3, 5, 64
    elif name == "more_blocks":
        A, Pr, Pc, N = synth.random_small(5, 9, 0.5, 13), 8, 8, 128
    elif name == "empty_rows":
        A, Pr, Pc, N = synth.random_small(300, 300, 0.02, 14, empty_rows=150), 2, 2, 128
    else:
        A, Pr, Pc, N = synth.rmat(14, 16, 3), 4, 4, 128
    B = synth.dense_normal(A.K, N, 5)
    P, Bd, Bp, C = run(A, B, Pr, Pc, flags)
    gu.check_spmm(A, B, C)
    # Packed path == direct path in FP64 (the oracle's own consistency at these inputs).
    O = oracle.plan(A, Pr, Pc)
    _, src = O.pack_layout(bool(flags))
    C1 = oracle.spmm_packed(A, O, B[src], B, bool(flags))
    assert np.array_equal(C1, oracle.spmm(A, B))


def test_empty_matrix_gives_zero_rows():
    A = synth.CSR(64, 32, np.zeros(65, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    B = synth.dense_normal(32, 128, 1)
    _, _, _, C = run(A, B, 2, 2)
    assert torch.count_nonzero(C).item() == 0


def test_hub_row_2e17_fp32_summation():
    """One row with 2^17 nonzeros: split into chunks, partial sums added in order."""
    A = synth.hub_matrix(64, 1 << 17, 5, 1 << 17, 2, 14)
    B = synth.dense_normal(A.K, 128, 15)
    P, Bd, Bp, C = run(A, B, 2, 4)
    assert P.info.n_long_rows >= 1
    err = gu.check_spmm(A, B, C)
    print("hub-row scaled error", err)


def test_accumulate_doubles_exactly():
    shiro = gu.lib()
    A = synth.rmat(12, 8, 31)
    B = synth.dense_normal(A.K, 128, 32)
    P, Bd, Bp, C = run(A, B, 2, 2, opts=shiro.make_opts(**SMALL_SPLIT))
    C2 = C.clone()
    P.spmm(Bp, B=Bd, out=C2, accumulate=True)
    torch.cuda.synchronize()
    assert torch.equal(C2, 2 * C)


def test_deterministic_and_persistent_identical():
    shiro = gu.lib()
    A = synth.rmat(14, 16, 41)
    B = synth.dense_normal(A.K, 128, 42)
    P, Bd, Bp, C = run(A, B, 4, 4, opts=shiro.make_opts(long_row_nnz=256, chunk_nnz=128))
    C_again = P.spmm(Bp, B=Bd)
    P.reschedule(persistent=1)
    C_pers = P.spmm(Bp, B=Bd)
    torch.cuda.synchronize()
    assert torch.equal(C, C_again), "SpMM not deterministic"
    assert torch.equal(C, C_pers), "persistent schedule changed the result"


def test_scratch_too_small_rejected():
    shiro = gu.lib()
    A = synth.rmat(12, 8, 21)
    P = gu.plan_of(A, 2, 2, opts=shiro.make_opts(**SMALL_SPLIT))
    Bd = torch.from_numpy(synth.dense_normal(A.K, 64, 1)).to(gu.dev())
    Bp = P.pack(Bd)
    small = torch.empty(16, dtype=torch.uint8, device=gu.dev())
    with pytest.raises(shiro.ShiroError) as ei:
        P.spmm(Bp, scratch=small)
    assert ei.value.status == 3


def test_huge_leading_dimension_rejected():
    """A B / Bpack stride of 2^32 elements or more is refused on the host (the gathers form row
    addresses from a 32-bit index times a 32-bit stride); nothing is launched."""
    shiro = gu.lib()
    A = synth.rmat(10, 4, 22)
    P = gu.plan_of(A, 2, 2)
    Bd = torch.from_numpy(synth.dense_normal(A.K, 32, 2)).to(gu.dev())
    Bp = P.pack(Bd)
    C = torch.empty((A.M, 32), dtype=torch.float32, device=gu.dev())
    f32 = shiro.dtype_code(torch.float32)
    with pytest.raises(shiro.ShiroError) as ei:
        shiro.shiro_spmm(P.handle, Bp.data_ptr(), 1 << 32, None, 0, 32, f32, C.data_ptr(), 32, 0,
                         None, 0, None)
    assert ei.value.status == 4
    with pytest.raises(shiro.ShiroError) as ei:
        shiro.shiro_sddmm(P.handle, C.data_ptr(), 32, Bp.data_ptr(), 1 << 32, None, 0, 32, f32,
                          C.data_ptr(), None)
    assert ei.value.status == 4


def test_autotune_keeps_result():
    A = synth.rmat(14, 16, 51)
    B = synth.dense_normal(A.K, 128, 52)
    P, Bd, Bp, C = run(A, B, 4, 4)
    best = P.autotune(Bp, B=Bd, reps=1)
    C2 = P.spmm(Bp, B=Bd)
    torch.cuda.synchronize()
    assert best["chunk_nnz"] >= 32
    gu.check_spmm(A, B, C2)


@pytest.fixture(scope="module")
def rmat20():
    A = synth.rmat(20, 16, 2)
    B = synth.dense_normal(A.K, 128, 2)
    return A, B


def test_full_size_rmat20_sampled_rows(rmat20):
    """The benchmark workload (R-MAT 2^20, N=128, 4x4 tiles, default schedule): sampled rows."""
    A, B = rmat20
    P, Bd, Bp, C = run(A, B, 4, 4)
    deg = np.diff(A.rowptr)
    rng_rows = (synth.uniform_f64(9, synth.STREAM_PERM, 0, 2000) * A.M).astype(np.int64)
    hubs = np.argsort(deg)[-64:]
    empties = np.nonzero(deg == 0)[0][:64]
    rows = np.unique(np.concatenate([rng_rows, hubs, empties, [0, A.M - 1]]))
    gu.check_spmm(A, B, C, rows=rows)
    # Packed rows are bit-exact copies (sampled).
    src = P.export()["pack_src"].cpu().numpy()
    pick = np.unique((synth.uniform_f64(10, synth.STREAM_PERM, 0, 4000) * len(src)).astype(np.int64))
    assert np.array_equal(Bp[torch.from_numpy(pick).to(gu.dev())].cpu().numpy(), B[src[pick]])


@pytest.mark.parametrize("case", ["f32_n128", "f32_n256", "f32_n64", "f32_n32", "bf16_n128",
                                  "bf16_n256", "bf16_n64", "f64_n128", "local_diag", "accumulate",
                                  "hub", "narrow_local_diag", "narrow_accumulate", "narrow_hub"])
def test_pipelines_bit_identical(case):
    """Register gathers (64- and 48-register forms), per-lane async copies and TMA bulk copies in
    two stages, the per-lane copy ring and the TMA gather4 ring (rows of 512 bytes) sum every row
    in the same order, so all pipelines give bit-identical C (and each passes the oracle bound)."""
    shiro = gu.lib()
    flags, vdt, dt, acc = 0, torch.float32, torch.float32, False
    A, N = synth.rmat(13, 12, 131), 128
    if case == "f32_n256":
        N = 256
    elif case == "f32_n64":
        N = 64
    elif case == "f32_n32":
        N = 32
    elif case.startswith("bf16"):
        dt = torch.bfloat16
        N = int(case.split("_n")[1])
    elif case == "f64_n128":
        vdt, dt = torch.float64, torch.float64
    if case.startswith("narrow"):
        N = 32  # rows of 128 bytes
    if case.endswith("local_diag"):
        flags = shiro.SHIRO_PLAN_LOCAL_DIAG
    elif case.endswith("accumulate"):
        acc = True
    elif case.endswith("hub"):
        A = synth.hub_matrix(64, 1 << 16, 5, 1 << 16, 2, 132)
    B = synth.dense_normal(A.K, N, 133)
    if dt == torch.bfloat16:
        bits = synth.to_bf16_bits(B)
        B = synth.bf16_bits_to_f32(bits).reshape(B.shape)
        Bd = torch.from_numpy(bits.view(np.int16)).to(gu.dev()).view(torch.bfloat16)
    else:
        Bd = torch.from_numpy(B).to(gu.dev()).to(dt)
    outs = []
    # (pipeline, stage_rows, persistent): forced register gathers, the two-stage copies, automatic,
    # the per-lane copy ring at each compiled depth (and persistent), the 48-register gathers
    # (and their persistent fallback).
    runs = [(5, 0, 0), (1, 0, 0), (2, 0, 0), (0, 0, 0), (4, 0, 0), (4, 4, 0), (4, 8, 0),
            (4, 12, 0), (4, 16, 1), (4, 32, 0), (6, 0, 0), (6, 0, 1), (7, 0, 0)]
    for pipe, rows, pers in runs:
        opts = shiro.make_opts(pipeline=pipe, long_row_nnz=128, chunk_nnz=64, group_nnz=256,
                               warps_per_cta=2, stage_rows=rows, persistent=pers)
        P = gu.plan_of(A, 4, 4, flags, opts=opts, vdt=vdt)
        Bp = P.pack(Bd)
        C = P.spmm(Bp, B=Bd)
        if acc:
            P.spmm(Bp, B=Bd, out=C, accumulate=True)
        P.check()
        torch.cuda.synchronize()
        outs.append(C.cpu())
    assert torch.equal(outs[0], outs[1]), "async pipeline differs from register gathers"
    assert torch.equal(outs[0], outs[2]), "bulk pipeline differs from register gathers"
    for (pipe, rows, pers), out in zip(runs[3:], outs[3:]):
        assert torch.equal(outs[0], out), \
            f"pipeline {pipe} (rows {rows}, persistent {pers}) differs from register gathers"
    C = outs[0].numpy() / (2.0 if acc else 1.0)
    err = gu.scaled_err(C, oracle.spmm(A, B), oracle.abs_scale(A, B))
    assert err <= gu.TOL, err


@pytest.mark.parametrize("case", ["f32_n32", "f32_n64", "bf16_n64", "bf16_n128", "local_diag",
                                  "accumulate", "hub", "empty_rows", "persistent"])
def test_grouped_pipeline(case):
    """Narrow rows split across lane groups (pipeline 3): within the oracle bound, deterministic."""
    shiro = gu.lib()
    flags, dt, acc, N, pers = 0, torch.float32, False, 64, 0
    A = synth.rmat(13, 12, 141)
    if case == "f32_n32":
        N = 32
    elif case.startswith("bf16"):
        dt = torch.bfloat16
        N = 64 if case.endswith("64") else 128
    elif case == "local_diag":
        flags = shiro.SHIRO_PLAN_LOCAL_DIAG
    elif case == "accumulate":
        acc = True
    elif case == "hub":
        A = synth.hub_matrix(64, 1 << 16, 5, 1 << 16, 2, 142)
    elif case == "empty_rows":
        A = synth.random_small(300, 300, 0.02, 143, empty_rows=150)
    elif case == "persistent":
        pers = 1
    B = synth.dense_normal(A.K, N, 144)
    if dt == torch.bfloat16:
        bits = synth.to_bf16_bits(B)
        B = synth.bf16_bits_to_f32(bits).reshape(B.shape)
        Bd = torch.from_numpy(bits.view(np.int16)).to(gu.dev()).view(torch.bfloat16)
    else:
        Bd = torch.from_numpy(B).to(gu.dev())
    opts = shiro.make_opts(pipeline=3, long_row_nnz=128, chunk_nnz=64, persistent=pers)
    P = gu.plan_of(A, 4, 4, flags, opts=opts)
    Bp = P.pack(Bd)
    C = P.spmm(Bp, B=Bd)
    C2 = P.spmm(Bp, B=Bd)
    if acc:
        P.spmm(Bp, B=Bd, out=C, accumulate=True)
    P.check()
    torch.cuda.synchronize()
    assert torch.equal(C2 * (2 if acc else 1), C), "grouped SpMM not deterministic"
    Ch = C.cpu().numpy() / (2.0 if acc else 1.0)
    err = gu.scaled_err(Ch, oracle.spmm(A, B), oracle.abs_scale(A, B))
    assert err <= gu.TOL, err
