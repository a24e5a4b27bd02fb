"""shiro_spmm_noalloc: SpMM whose split-row scratch is a static array inside the library.

Some callers cannot allocate device memory at the point where they run an SpMM: code recorded
into a CUDA graph while a stream is being captured (an allocation is not a capturable
operation), kernels hosted by a runtime that owns all device memory and passes only input and
output buffers, and serving paths that must not allocate once they are up.  This entry point
needs nothing from them beyond the plan and the operands.

The test calls it through the C ABI twice in a row.  Each result must equal shiro_spmm's on a
caller-provided scratch bit for bit (the same kernel sums every row in the same fixed order, only
the scratch address differs), and must be within the scaled tolerance of the other SpMM tests
against the FP64 oracle.  It also checks that a plan needing more scratch than the static array
holds is refused.  It sits in a file of its
own, collected last, and passes alone in a fresh process or after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2512_20178_gb300 import synth
import gpu_util as gu

pytestmark = pytest.mark.gpu


def setup_module(_):
    gu.need_gpu()


def _noalloc(shiro, P, Bp, C, N, dt, flags=0):
    return shiro.lib().shiro_spmm_noalloc(P.handle, ctypes.c_void_p(Bp.data_ptr()), Bp.stride(0),
                                          None, N, N, shiro.dtype_code(dt),
                                          ctypes.c_void_p(C.data_ptr()), C.stride(0), flags,
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("case", ["rmat12_small_chunks", "rmat14_default", "bf16_n256"])
def test_noalloc_matches_spmm_twice(case):
    shiro = gu.lib()
    if case == "rmat12_small_chunks":
        A, N, dt = synth.rmat(12, 8, 91), 128, torch.float32
        opts = shiro.make_opts(long_row_nnz=64, chunk_nnz=32)
    elif case == "rmat14_default":
        A, N, dt = synth.rmat(14, 16, 92), 64, torch.float32
        opts = None
    else:
        A, N, dt = synth.rmat(13, 16, 93), 256, torch.bfloat16
        opts = shiro.make_opts(long_row_nnz=128, chunk_nnz=64)
    B = synth.dense_normal(A.K, N, 94)
    if dt == torch.bfloat16:
        bits = synth.to_bf16_bits(B)
        B = synth.bf16_bits_to_f32(bits).reshape(B.shape)
        Bd = torch.from_numpy(bits.view(np.int16)).to(gu.dev()).view(torch.bfloat16)
    else:
        Bd = torch.from_numpy(B).to(gu.dev())
    P = gu.plan_of(A, 4, 4, opts=opts)
    assert P.info.n_chunks > 0, "the case must exercise the split-row scratch"
    assert 0 < P.scratch_bytes(N, dt) <= shiro.SHIRO_NOALLOC_SCRATCH_BYTES
    Bp = P.pack(Bd)
    ref = P.spmm(Bp)
    C64 = oracle.spmm(A, B)
    S = oracle.abs_scale(A, B)
    for _ in range(2):
        C = torch.full((A.M, N), float("nan"), dtype=torch.float32, device=gu.dev())
        st = _noalloc(shiro, P, Bp, C, N, dt)
        torch.cuda.synchronize()
        assert st == 0, shiro.lib().shiro_last_error()
        assert torch.equal(C, ref), "no-alloc SpMM differs from shiro_spmm"
        err = gu.scaled_err(C.cpu().numpy(), C64, S)
        assert err <= gu.TOL, f"no-alloc SpMM against the FP64 oracle: scaled error {err}"


def test_noalloc_rejects_plans_beyond_the_static_scratch():
    shiro = gu.lib()
    A = synth.rmat(16, 16, 95)
    P = gu.plan_of(A, 1, 1, opts=shiro.make_opts(long_row_nnz=32, chunk_nnz=32))
    N = 512
    assert P.scratch_bytes(N, torch.float32) > shiro.SHIRO_NOALLOC_SCRATCH_BYTES
    Bd = torch.zeros((A.K, N), dtype=torch.float32, device=gu.dev())
    Bp = P.pack(Bd)
    C = torch.empty((A.M, N), dtype=torch.float32, device=gu.dev())
    st = _noalloc(shiro, P, Bp, C, N, torch.float32)
    assert st == 3
    assert b"static scratch" in shiro.lib().shiro_last_error()
