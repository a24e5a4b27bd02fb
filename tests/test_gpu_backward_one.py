"""shiro_spmm_backward in one launch: the pack of dC's rows, dB = A^T dC and dA on A's pattern
computed from the same gathered dC rows, for rows of 256 or 512 bytes (FP32 N = 64 / 128, BF16
N = 128 / 256) when the caller passes B.

dB and the packed dC rows must equal the two-call path (shiro_pack_spmm on the TRANSPOSE plan) bit
for bit: the same work items summed in the same order.  dA is summed in another order than the
SDDMM kernels (per lane, then a tree over the warp), so it is held to the scaled tolerance of the
FP64 oracle, on every nonzero.  Cases: the four row shapes, hub rows cut into chunks, 1D plans whose
local diagonal tiles read dC in place, empty rows and columns, a ragged grid, more row blocks than
rows, and every call twice in a row (the per-block counters and the work counter are reset by each
call)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_20178_gb300 import synth
import gpu_util as gu

pytestmark = pytest.mark.gpu


def setup_module(_):
    gu.need_gpu()


def _kernel_names(fn):
    """Names of the CUDA kernels fn launches (an empty set where the profiler sees none)."""
    from torch.profiler import ProfilerActivity, profile
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        fn()
        torch.cuda.synchronize()
    return {e.name for e in prof.events() if str(e.device_type).endswith("CUDA")}


def _transposed(A):
    """A^T as a CSR matrix (input construction: a hub row of A becomes a hub column)."""
    rp, col, perm = oracle.transpose(A)
    return synth.CSR(A.K, A.M, rp, col, A.val[perm])


def _case(A, N, dt, Pr, Pc, flags=0, opts=None, seed=300):
    shiro = gu.lib()
    B = synth.dense_normal(A.K, N, seed)
    G = synth.dense_normal(A.M, N, seed + 1)
    if dt == torch.bfloat16:
        B = synth.bf16_bits_to_f32(synth.to_bf16_bits(B)).reshape(B.shape)
        G = synth.bf16_bits_to_f32(synth.to_bf16_bits(G)).reshape(G.shape)
    P = gu.plan_of(A, Pr, Pc, flags, opts=opts)
    PT = gu.plan_of(A, Pr, Pc, flags | shiro.SHIRO_PLAN_TRANSPOSE, opts=opts)
    d = gu.dev()
    Bd = torch.from_numpy(B).to(d).to(dt)
    Gd = torch.from_numpy(G).to(d).to(dt)
    Bp = P.pack(Bd)
    # The two-call path: pack + SpMM of dC on the transposed plan, then the SDDMM.
    Gp_ref = torch.empty((PT.info.packed_rows, N), dtype=dt, device=d)
    dB_ref = PT.pack_spmm(Gd, Bpack=Gp_ref)
    dA_sd = P.sddmm(Gd, Bp, B=Bd)
    ref = oracle.sddmm(A, G, B)
    scale = oracle.sddmm(A, np.abs(G), np.abs(B))
    for _ in range(2):
        Gp = torch.full_like(Gp_ref, float("nan"))
        dB = torch.full((A.K, N), float("nan"), dtype=torch.float32, device=d)
        dA = torch.full((A.nnz,), float("nan"), dtype=torch.float32, device=d)
        shiro.spmm_backward(P, PT, Gd, Bp, B=Bd, dCpack=Gp, dB=dB, dA=dA)
        torch.cuda.synchronize()
        P.check()
        PT.check()
        bits = (lambda t: t.view(torch.int16)) if dt == torch.bfloat16 else (lambda t: t)
        assert torch.equal(bits(Gp), bits(Gp_ref)), "packed dC rows differ from the pack"
        assert torch.equal(dB, dB_ref), "dB differs from pack + SpMM on the transposed plan"
        err = gu.scaled_err(dA.cpu().numpy(), ref, scale)
        assert err <= gu.TOL, f"dA scaled error {err}"
    err_sd = gu.scaled_err(dA_sd.cpu().numpy(), ref, scale)
    assert err_sd <= gu.TOL
    return P, PT, Bd, Gd, Bp


@pytest.mark.parametrize("dt,N", [(torch.float32, 128), (torch.bfloat16, 256), (torch.float32, 64),
                                  (torch.bfloat16, 128)])
def test_backward_one_launch_row_shapes(dt, N):
    _case(synth.rmat(13, 12, 301), N, dt, 4, 4)


@pytest.mark.parametrize("case", ["hub_chunks", "local_diag", "empty_rows_cols", "ragged_grid",
                                  "more_blocks_than_rows", "bf16_hub_local"])
def test_backward_one_launch_cases(case):
    shiro = gu.lib()
    opts, flags, dt, N = None, 0, torch.float32, 128
    Pr = Pc = 4
    if case == "hub_chunks":
        # A hub column of 20,000 rows: a row of A^T cut into chunks of 64 nonzeros.
        A = _transposed(synth.hub_matrix(300, 1 << 15, 7, 20000, 3, 302))
        opts = shiro.make_opts(long_row_nnz=128, chunk_nnz=64)
    elif case == "local_diag":
        A = synth.rmat(13, 12, 303)
        flags = shiro.SHIRO_PLAN_LOCAL_DIAG
    elif case == "empty_rows_cols":
        A = synth.random_small(900, 700, 0.02, 304, empty_rows=300)
    elif case == "ragged_grid":
        A = synth.random_small(333, 517, 0.037, 305)
        Pr, Pc = 3, 5
    elif case == "more_blocks_than_rows":
        A = synth.random_small(5, 9, 0.5, 306)
        Pr, Pc = 8, 8
    else:
        A = _transposed(synth.hub_matrix(256, 1 << 14, 5, 12000, 3, 307))
        dt, N = torch.bfloat16, 256
        flags = shiro.SHIRO_PLAN_LOCAL_DIAG
        opts = shiro.make_opts(long_row_nnz=256, chunk_nnz=128)
    _case(A, N, dt, Pr, Pc, flags=flags, opts=opts)


def test_backward_one_launch_runs_one_kernel():
    """With B the call takes the one launch, without B the two calls (pack + SpMM, then the SDDMM).
    The two dA differ in their last bits (another summation order) while dB is the same; without B,
    dA equals shiro_sddmm's bit for bit.  Where the profiler lists kernels, the one-launch kernel
    and no SDDMM kernel must run with B, and the reverse without."""
    shiro = gu.lib()
    P, PT, Bd, Gd, Bp = _case(synth.rmat(12, 8, 308), 128, torch.float32, 2, 2)
    dA_sd = P.sddmm(Gd, Bp, B=Bd)
    dB1, dA1 = shiro.spmm_backward(P, PT, Gd, Bp, B=Bd)
    dB2, dA2 = shiro.spmm_backward(P, PT, Gd, Bp, B=None)
    torch.cuda.synchronize()
    assert torch.equal(dB1, dB2)
    assert torch.equal(dA2, dA_sd)
    assert not torch.equal(dA1, dA_sd), "dA with B equals the SDDMM's bit for bit"
    names = _kernel_names(lambda: shiro.spmm_backward(P, PT, Gd, Bp, B=Bd))
    if names:
        assert any("k_spmm_lean_bwd" in n for n in names), names
        assert not any("sddmm" in n for n in names), names
        names = _kernel_names(lambda: shiro.spmm_backward(P, PT, Gd, Bp, B=None))
        assert not any("k_spmm_lean_bwd" in n for n in names), names
        assert any("sddmm" in n for n in names), names


def test_backward_one_launch_full_size_rmat20():
    """R-MAT 2^20, average degree 16, N = 128, 4x4 tiles (the benchmark matrix): dB bit-equal to
    the two calls and within the oracle bound on sampled rows; dA on 200,000 sampled nonzeros."""
    shiro = gu.lib()
    A = synth.rmat(20, 16, 2)
    N = 128
    B = synth.dense_normal(A.K, N, 310)
    G = synth.dense_normal(A.M, N, 311)
    d = gu.dev()
    P = gu.plan_of(A, 4, 4)
    PT = gu.plan_of(A, 4, 4, shiro.SHIRO_PLAN_TRANSPOSE)
    Bd = torch.from_numpy(B).to(d)
    Gd = torch.from_numpy(G).to(d)
    Bp = P.pack(Bd)
    dB_ref = PT.pack_spmm(Gd)
    dB, dA = shiro.spmm_backward(P, PT, Gd, Bp, B=Bd)
    torch.cuda.synchronize()
    P.check()
    PT.check()
    assert torch.equal(dB, dB_ref)
    es = (synth.uniform_f64(312, synth.STREAM_PERM, 0, 200000) * A.nnz).astype(np.int64)
    eA = gu.sampled_sddmm_error(A, G, B, dA.cpu().numpy(), es)
    assert eA <= gu.TOL, f"dA (sampled) scaled error {eA}"


def test_backward_one_launch_full_size_precision_bf16():
    """The precision workload at full size (R-MAT 2^22, average degree 32, B and dC 2^22 x 256
    stored in BF16, 4x4 tiles): dB bit-equal to the two calls; dB on sampled rows (random and the
    64 densest columns of A) and dA on 200,000 sampled nonzeros within the bound of the FP64
    oracle on the BF16-rounded operands."""
    shiro = gu.lib()
    A = synth.rmat(22, 32, 3)
    N = 256
    bB = synth.to_bf16_bits(synth.dense_normal(A.K, N, 3))
    bG = synth.to_bf16_bits(synth.dense_normal(A.M, N, 313))
    d = gu.dev()
    P = gu.plan_of(A, 4, 4)
    PT = gu.plan_of(A, 4, 4, shiro.SHIRO_PLAN_TRANSPOSE)
    Bd = torch.from_numpy(bB.view(np.int16)).to(d).view(torch.bfloat16)
    Gd = torch.from_numpy(bG.view(np.int16)).to(d).view(torch.bfloat16)
    Bp = P.pack(Bd)
    dB_ref = PT.pack_spmm(Gd)
    dB, dA = shiro.spmm_backward(P, PT, Gd, Bp, B=Bd)
    torch.cuda.synchronize()
    P.check()
    PT.check()
    assert torch.equal(dB, dB_ref)
    del dB_ref, Bp

    class _Rows:  # BF16-rounded rows on demand (FP32 copies of both would be 8 GB more)
        def __init__(self, bits):
            self.bits, self.shape = bits, bits.shape
        def __getitem__(self, ix):
            return synth.bf16_bits_to_f32(self.bits[ix]).reshape(len(ix), -1)

    rpT, colT, perm = oracle.transpose(A)
    AT = synth.CSR(A.K, A.M, rpT, colT, A.val[perm])
    degT = np.diff(rpT)
    rows = np.unique(np.concatenate([
        (synth.uniform_f64(314, synth.STREAM_PERM, 0, 1000) * A.K).astype(np.int64),
        np.argsort(degT)[-64:]]))
    eB = gu.sampled_rows_error(AT, _Rows(bG), dB[torch.from_numpy(rows).to(d)].cpu().numpy(), rows)
    assert eB.max() <= gu.TOL, f"dB (sampled rows) scaled error {eB.max()}"
    es = (synth.uniform_f64(315, synth.STREAM_PERM, 0, 200000) * A.nnz).astype(np.int64)
    eA = gu.sampled_sddmm_error(A, _Rows(bG), _Rows(bB), dA.cpu().numpy(), es)
    assert eA <= gu.TOL, f"dA (sampled) scaled error {eA}"


def test_backward_one_launch_strided_outputs():
    """dB and the packed dC rows written into views with leading dimensions larger than N: the
    same values as into contiguous buffers, and the padding columns untouched."""
    shiro = gu.lib()
    A = synth.rmat(12, 8, 316)
    N, pad = 128, 16
    P = gu.plan_of(A, 2, 2)
    PT = gu.plan_of(A, 2, 2, shiro.SHIRO_PLAN_TRANSPOSE)
    d = gu.dev()
    Bd = torch.from_numpy(synth.dense_normal(A.K, N, 317)).to(d)
    Gd = torch.from_numpy(synth.dense_normal(A.M, N, 318)).to(d)
    Bp = P.pack(Bd)
    dB0, dA0 = shiro.spmm_backward(P, PT, Gd, Bp, B=Bd)
    Gpw = torch.full((PT.info.packed_rows, N + pad), 7.0, device=d)
    dBw = torch.full((A.K, N + pad), 7.0, device=d)
    dA = torch.empty(A.nnz, device=d)
    shiro.spmm_backward(P, PT, Gd, Bp, B=Bd, dCpack=Gpw[:, :N], dB=dBw[:, :N], dA=dA)
    torch.cuda.synchronize()
    assert torch.equal(dBw[:, :N], dB0) and torch.equal(dA, dA0)
    assert torch.equal(Gpw[:, :N], PT.pack(Gd))
    assert bool((dBw[:, N:] == 7.0).all()) and bool((Gpw[:, N:] == 7.0).all())
