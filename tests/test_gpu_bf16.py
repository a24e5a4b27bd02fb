"""B stored in BF16, FP32 accumulation: pack bit-exact, SpMM within 1e-5 of the FP64 oracle on the
BF16-rounded B; the quantisation error against the FP32 B is reported."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_20178_gb300 import synth
import gpu_util as gu

pytestmark = pytest.mark.gpu


def setup_module(_):
    gu.need_gpu()


@pytest.mark.parametrize("N", [32, 64, 100, 128, 256, 512])
def test_bf16_spmm(N):
    shiro = gu.lib()
    A = synth.rmat(13, 16, 81)
    B = synth.dense_normal(A.K, N, 82)
    bits = synth.to_bf16_bits(B)
    Bq = synth.bf16_bits_to_f32(bits).reshape(B.shape)
    P = gu.plan_of(A, 4, 4, opts=shiro.make_opts(long_row_nnz=128, chunk_nnz=64))
    d = gu.dev()
    Bd = torch.from_numpy(bits.view(np.int16)).to(d).view(torch.bfloat16)
    Bp = P.pack(Bd)
    src = P.export()["pack_src"].cpu().numpy()
    assert np.array_equal(Bp.view(torch.int16).cpu().numpy().view(np.uint16), bits[src])
    C = P.spmm(Bp)
    torch.cuda.synchronize()
    err = gu.check_spmm(A, Bq, C)
    q = gu.scaled_err(C.cpu().numpy(), oracle.spmm(A, B), oracle.abs_scale(A, B))
    print(f"N={N}: scaled error vs FP64(bf16 B) {err:.2e}, vs FP64(fp32 B) {q:.2e}")
    assert q <= 2 ** -8, "quantisation error larger than BF16 rounding allows"


def test_bf16_rmat18_deg32_n256():
    """Scaled-down precision workload (R-MAT 2^18, avg degree 32, N = 256, 4x4): sampled rows,
    per-row maximum error reported."""
    A = synth.rmat(18, 32, 3)
    B = synth.dense_normal(A.K, 256, 3)
    bits = synth.to_bf16_bits(B)
    Bq = synth.bf16_bits_to_f32(bits).reshape(B.shape)
    P = gu.plan_of(A, 4, 4)
    d = gu.dev()
    Bd = torch.from_numpy(bits.view(np.int16)).to(d).view(torch.bfloat16)
    C = P.spmm(P.pack(Bd))
    torch.cuda.synchronize()
    deg = np.diff(A.rowptr)
    rows = np.unique(np.concatenate([(synth.uniform_f64(5, synth.STREAM_PERM, 0, 2000) * A.M).astype(np.int64),
                                     np.argsort(deg)[-32:]]))
    gu.check_spmm(A, Bq, C, rows=rows)


def test_full_size_precision_rmat22_deg32_n256():
    """The precision workload at full size: R-MAT 2^22, avg degree 32, FP32 values U(0,1), B
    2^22 x 256 stored in BF16, FP32 accumulation and C, 4x4 tiles.  Sampled rows (random, the 64
    longest, empty ones) against the FP64 oracle on the BF16-rounded B; the per-row maximum scaled
    error is reported, and the quantisation error against the FP32 B."""
    A = synth.rmat(22, 32, 3)
    B = synth.dense_normal(A.K, 256, 3)
    bits = synth.to_bf16_bits(B)
    P = gu.plan_of(A, 4, 4)
    d = gu.dev()
    Bd = torch.from_numpy(bits.view(np.int16)).to(d).view(torch.bfloat16)
    Bp = P.pack(Bd)
    C = P.spmm(Bp)
    # The one-launch pack + SpMM the bench times: the same bits.
    Bp2 = torch.empty_like(Bp)
    C2 = P.pack_spmm(Bd, Bpack=Bp2)
    torch.cuda.synchronize()
    P.check()
    assert torch.equal(Bp2.view(torch.int16), Bp.view(torch.int16)) and torch.equal(C2, C)
    del Bp, Bp2, C2
    deg = np.diff(A.rowptr)
    rows = np.unique(np.concatenate([
        (synth.uniform_f64(7, synth.STREAM_PERM, 0, 1500) * A.M).astype(np.int64),
        np.argsort(deg)[-64:], np.nonzero(deg == 0)[0][:32]]))
    Cr = C[torch.from_numpy(rows).to(d)].cpu().numpy()
    Bq_rows = lambda ix: synth.bf16_bits_to_f32(bits[ix]).reshape(len(ix), -1)

    class _View:  # rows of the BF16-rounded B on demand (the full FP32 copy would be 4 GB more)
        shape = B.shape
        def __getitem__(self, ix):
            return Bq_rows(ix)

    err = gu.sampled_rows_error(A, _View(), Cr, rows)
    q = gu.sampled_rows_error(A, B, Cr, rows)
    print(f"precision workload: nnz={A.nnz}, rows checked={len(rows)}, per-row max scaled error "
          f"vs FP64 on the BF16 B: max {err.max():.2e} median {np.median(err):.2e}; vs FP64 on the "
          f"FP32 B (quantisation): max {q.max():.2e} median {np.median(q):.2e}")
    assert err.max() <= gu.TOL
    assert q.max() <= 2 ** -8
