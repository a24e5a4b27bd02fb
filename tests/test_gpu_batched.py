"""Batched form: many graphs of uneven size as one block-diagonal plan, one launch, CUDA graph."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_20178_gb300 import synth
import gpu_util as gu

pytestmark = pytest.mark.gpu


def setup_module(_):
    gu.need_gpu()


def batch_tensors(gb, dt=torch.float32):
    return [gu.to_dev(g) + (g.M, g.K) for g in gb.graphs]


def stacked(gb, N, seed, bf16=False):
    Bs = [synth.dense_normal(g.K, N, seed + i) for i, g in enumerate(gb.graphs)]
    if bf16:
        Bs = [synth.bf16_bits_to_f32(synth.to_bf16_bits(b)).reshape(b.shape) for b in Bs]
    return Bs, np.concatenate(Bs, axis=0)


def test_batch_plan_and_spmm_equal_single_graphs():
    shiro = gu.lib()
    gb = synth.batch_graphs(24, 7, 100, 1500)
    opts = shiro.make_opts(long_row_nnz=64, chunk_nnz=32)
    PB = shiro.Plan.create_batch(batch_tensors(gb), opts=opts)
    st = PB.tile_stats()
    ex = PB.export()
    torch.cuda.synchronize()
    off = 0
    for g_i, g in enumerate(gb.graphs):
        O = oracle.plan(g, 1, 1)
        assert st["tile_ncols"][g_i].item() == O.tile_ncols[0]
        got = ex["cols_sorted"][st["tile_cols_ptr"][g_i]:st["tile_cols_ptr"][g_i + 1]].cpu().numpy()
        assert np.array_equal(got - off, O.cols_sorted)
        off += g.K
    N = 64
    Bs, Bcat = stacked(gb, N, 100)
    d = gu.dev()
    Bd = torch.from_numpy(Bcat).to(d)
    C = PB.spmm(PB.pack(Bd))
    torch.cuda.synchronize()
    r = 0
    for g, Bg in zip(gb.graphs, Bs):
        P1 = gu.plan_of(g, 1, 1, opts=opts)
        Bg_d = torch.from_numpy(Bg).to(d)
        C1 = P1.spmm(P1.pack(Bg_d))
        torch.cuda.synchronize()
        assert torch.equal(C[r:r + g.M], C1), "batched result differs from the single-graph call"
        gu.check_spmm(g, Bg, C1)
        r += g.M


def test_cuda_graph_capture_replay_persistent():
    shiro = gu.lib()
    gb = synth.batch_graphs(32, 8, 100, 3000)
    PB = shiro.Plan.create_batch(batch_tensors(gb), opts=shiro.make_opts(persistent=1))
    N = 64
    d = gu.dev()
    _, Bcat = stacked(gb, N, 200, bf16=True)
    bits = synth.to_bf16_bits(Bcat)
    Bd = torch.from_numpy(bits.view(np.int16)).to(d).view(torch.bfloat16)
    Bp = torch.empty((PB.info.packed_rows, N), dtype=torch.bfloat16, device=d)
    C = torch.empty((PB.info.M, N), dtype=torch.float32, device=d)
    scratch = PB.new_scratch(N, torch.bfloat16)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        PB.pack(Bd, out=Bp)
        PB.spmm(Bp, out=C, scratch=scratch)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    eager = C.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        PB.pack(Bd, out=Bp)
        PB.spmm(Bp, out=C, scratch=scratch)
    C.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(C, eager), "graph replay differs from eager"
    # New inputs through the same captured buffers.
    _, B2 = stacked(gb, N, 300, bf16=True)
    bits2 = synth.to_bf16_bits(B2)
    Bd.copy_(torch.from_numpy(bits2.view(np.int16)).to(d).view(torch.bfloat16))
    g.replay()
    torch.cuda.synchronize()
    Bq2 = synth.bf16_bits_to_f32(bits2).reshape(B2.shape)
    off_r = np.concatenate([[0], np.cumsum([x.M for x in gb.graphs])])
    off_c = np.concatenate([[0], np.cumsum([x.K for x in gb.graphs])])
    for gi in range(0, len(gb.graphs), 5):
        gr = gb.graphs[gi]
        gu.check_spmm(gr, Bq2[off_c[gi]:off_c[gi + 1]], C[off_r[gi]:off_r[gi + 1]])


def test_full_batch_512_graphs():
    """512 R-MAT graphs, n ~ U{100..20000}, degree log-uniform [4, 40], B n x 64 in BF16: one
    persistent launch in a CUDA graph; sampled graphs against the oracle."""
    shiro = gu.lib()
    gb = synth.batch_graphs(512, 5)
    PB = shiro.Plan.create_batch(batch_tensors(gb), opts=shiro.make_opts(persistent=1))
    N = 64
    d = gu.dev()
    _, Bcat = stacked(gb, N, 500, bf16=True)
    bits = synth.to_bf16_bits(Bcat)
    Bq = synth.bf16_bits_to_f32(bits).reshape(Bcat.shape)
    Bd = torch.from_numpy(bits.view(np.int16)).to(d).view(torch.bfloat16)
    Bp = torch.empty((PB.info.packed_rows, N), dtype=torch.bfloat16, device=d)
    C = torch.empty((PB.info.M, N), dtype=torch.float32, device=d)
    scratch = PB.new_scratch(N, torch.bfloat16)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        PB.pack(Bd, out=Bp)
        PB.spmm(Bp, out=C, scratch=scratch)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        PB.pack(Bd, out=Bp)
        PB.spmm(Bp, out=C, scratch=scratch)
    C.zero_()
    g.replay()
    torch.cuda.synchronize()
    off_r = np.concatenate([[0], np.cumsum([x.M for x in gb.graphs])])
    off_c = np.concatenate([[0], np.cumsum([x.K for x in gb.graphs])])
    pick = np.unique((synth.uniform_f64(6, synth.STREAM_PERM, 0, 24) * 512).astype(np.int64))
    for gi in pick:
        gr = gb.graphs[gi]
        gu.check_spmm(gr, Bq[off_c[gi]:off_c[gi + 1]], C[off_r[gi]:off_r[gi + 1]])
    # Cols of every graph = its non-empty columns.
    st = PB.tile_stats()
    for gi in pick:
        assert st["tile_ncols"][gi].item() == len(np.unique(gb.graphs[gi].col))
