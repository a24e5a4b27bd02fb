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
