"""shiro_pack_spmm: pack + SpMM in one call (one launch for FP32 rows of 512 bytes, and for BF16
ones with pipeline 6; BF16 rows of 512 bytes with the automatic pipeline take the pack and the
gather4 ring).

Bpack must equal shiro_pack's bit for bit and C must equal shiro_spmm's over those rows bit for bit
(the same work items, summed in the same order), on every row shape, on 1D plans with local
diagonal tiles, hub rows cut into chunks, empty and ragged matrices, batched (diagonal-only) plans,
with ACCUMULATE, twice in a row (the per-block counters are reset by every call), and C must be
within the scaled tolerance of the FP64 oracle.  Schedules and shapes the fused kernel does not
take (narrower rows, pipeline 5, FP64, masked N) go through the two launches and must give the same
results."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_20178_gb300 import synth
import gpu_util as gu

pytestmark = pytest.mark.gpu


def setup_module(_):
    gu.need_gpu()


def _run(P, A, B_host, dt, N, accumulate=False, B_dev=None, tol_check=True):
    d = gu.dev()
    Bd = B_dev if B_dev is not None else torch.from_numpy(B_host).to(d).to(dt)
    Bp1 = P.pack(Bd)
    C0 = torch.from_numpy(synth.dense_normal(A.M, N, 9)).to(d).to(
        torch.float64 if dt == torch.float64 else torch.float32)
    C1 = C0.clone()
    P.spmm(Bp1, B=Bd, out=C1, accumulate=accumulate)
    for _ in range(2):
        Bp2 = torch.full_like(Bp1, float("nan"))
        C2 = C0.clone()
        P.pack_spmm(Bd, Bpack=Bp2, out=C2, accumulate=accumulate)
        torch.cuda.synchronize()
        P.check()
        assert torch.equal(Bp2.view(torch.uint8) if dt == torch.bfloat16 else Bp2,
                           Bp1.view(torch.uint8) if dt == torch.bfloat16 else Bp1), "Bpack differs"
        assert torch.equal(C2, C1), "C differs from pack + spmm"
    if tol_check and not accumulate:
        Bq = Bd.to(torch.float64).cpu().numpy()
        gu.check_spmm(A, Bq, C2)


@pytest.mark.parametrize("dt,N", [(torch.float32, 128), (torch.float32, 64), (torch.float32, 32),
                                  (torch.bfloat16, 256), (torch.bfloat16, 128),
                                  (torch.bfloat16, 64)])
def test_pack_spmm_row_shapes(dt, N):
    A = synth.rmat(13, 12, 150)
    B = synth.dense_normal(A.K, N, 151)
    P = gu.plan_of(A, 4, 4)
    _run(P, A, B, dt, N)


@pytest.mark.parametrize("case", ["hub_chunks", "local_diag", "empty_rows", "ragged", "accumulate",
                                  "more_blocks_than_rows", "pipeline5", "f64", "masked_n100"])
def test_pack_spmm_cases(case):
    shiro = gu.lib()
    dt, N, flags, opts, Pr, Pc = torch.float32, 128, 0, None, 4, 4
    A = synth.rmat(13, 12, 152)
    vdt = torch.float32
    if case == "hub_chunks":
        A = synth.hub_matrix(300, 1 << 15, 7, 20000, 3, 153)
        opts = shiro.make_opts(long_row_nnz=128, chunk_nnz=64)
    elif case == "local_diag":
        flags = shiro.SHIRO_PLAN_LOCAL_DIAG
    elif case == "empty_rows":
        A = synth.random_small(900, 700, 0.02, 154, empty_rows=300)
    elif case == "ragged":
        A = synth.random_small(333, 517, 0.037, 155)
        Pr, Pc = 3, 5
    elif case == "more_blocks_than_rows":
        A = synth.random_small(5, 40, 0.3, 156)
        Pr, Pc = 8, 3
    elif case == "pipeline5":
        opts = shiro.make_opts(pipeline=5)
    elif case == "f64":
        dt, vdt, N = torch.float64, torch.float64, 64
    elif case == "masked_n100":
        N = 100
    B = synth.dense_normal(A.K, N, 157)
    P = gu.plan_of(A, Pr, Pc, flags, opts=opts, vdt=vdt)
    _run(P, A, B, dt, N, accumulate=(case == "accumulate"))


def test_pack_spmm_batched_plan():
    """Diagonal-only batch plan (BF16 N = 256, fused): one row block per graph, the pack of graph
    g + 1 among the items of graph g."""
    shiro = gu.lib()
    gb = synth.batch_graphs(40, 158, n_lo=50, n_hi=900)
    d = gu.dev()
    tens = [(torch.from_numpy(g.rowptr).to(d), torch.from_numpy(g.col).to(d),
             torch.from_numpy(g.val).to(d), g.M, g.K) for g in gb.graphs]
    P = shiro.Plan.create_batch(tens)
    N = 256
    Bh = np.concatenate([synth.dense_normal(g.K, N, 600 + i) for i, g in enumerate(gb.graphs)])
    bits = synth.to_bf16_bits(Bh)
    Bd = torch.from_numpy(bits.view(np.int16)).to(d).view(torch.bfloat16)
    Bp1 = P.pack(Bd)
    C1 = P.spmm(Bp1)
    Bp2 = torch.empty_like(Bp1)
    C2 = P.pack_spmm(Bd, Bpack=Bp2)
    torch.cuda.synchronize()
    P.check()
    assert torch.equal(Bp2.view(torch.int16), Bp1.view(torch.int16))
    assert torch.equal(C2, C1)
    off = 0
    Cg = C2.cpu().numpy()
    Bq = synth.bf16_bits_to_f32(bits).reshape(Bh.shape)
    for g in gb.graphs[:5]:
        err = gu.scaled_err(Cg[off:off + g.M], oracle.spmm(g, Bq[off:off + g.K]),
                            oracle.abs_scale(g, Bq[off:off + g.K]))
        assert err <= gu.TOL
        off += g.M


def test_pack_spmm_full_size_rmat20():
    """The default workload (R-MAT 2^20, avg degree 16, N = 128, FP32, 4x4 tiles): bit-identical
    to pack + SpMM, and sampled rows within the tolerance of the FP64 oracle."""
    A = synth.rmat(20, 16, 2)
    N = 128
    B = synth.dense_normal(A.K, N, 2)
    P = gu.plan_of(A, 4, 4)
    d = gu.dev()
    Bd = torch.from_numpy(B).to(d)
    Bp1 = P.pack(Bd)
    C1 = P.spmm(Bp1)
    Bp2 = torch.empty_like(Bp1)
    C2 = P.pack_spmm(Bd, Bpack=Bp2)
    torch.cuda.synchronize()
    P.check()
    assert torch.equal(Bp2, Bp1) and torch.equal(C2, C1)
    deg = np.diff(A.rowptr)
    rows = np.unique(np.concatenate([(synth.uniform_f64(159, synth.STREAM_PERM, 0, 500) * A.M)
                                     .astype(np.int64), np.argsort(deg)[-16:]]))
    err = gu.sampled_rows_error(A, B, C2[torch.from_numpy(rows).to(d)].cpu().numpy(), rows)
    assert err.max() <= gu.TOL


def test_pack_spmm_in_cuda_graph():
    """The one-launch call (its two memset nodes and the kernel) recorded in a CUDA graph and
    replayed three times gives the eager call's bits every time."""
    A = synth.rmat(14, 16, 160)
    N = 128
    B = synth.dense_normal(A.K, N, 161)
    P = gu.plan_of(A, 4, 4)
    d = gu.dev()
    Bd = torch.from_numpy(B).to(d)
    Bp = torch.empty((P.info.packed_rows, N), device=d)
    C = torch.empty((A.M, N), device=d)
    scr = P.new_scratch(N, torch.float32)
    ref = P.pack_spmm(Bd, Bpack=torch.empty_like(Bp), scratch=scr).clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        P.pack_spmm(Bd, Bpack=Bp, out=C, scratch=scr)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        P.pack_spmm(Bd, Bpack=Bp, out=C, scratch=scr)
    for _ in range(3):
        C.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        P.check()
        assert torch.equal(C, ref)
