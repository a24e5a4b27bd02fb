"""The TMA gather4 ring (pipeline 7, rows of 512 bytes): bit-identical to the 48-register gathers
(same summation order) and within the oracle bound, on the shapes its control flow branches on:
items longer than one staged segment of 256 pairs, chunked hub rows, empty rows, ragged grids,
ACCUMULATE, more blocks than rows."""
import numpy as np
import pytest
import torch

from paper_2512_20178_gb300 import synth
import gpu_util as gu

pytestmark = pytest.mark.gpu


def setup_module(_):
    gu.need_gpu()


def lengths_matrix(lengths, K, seed):
    """Row i holds lengths[i] distinct columns (i-dependent offsets, a stride coprime to K)."""
    keys = []
    for i, n in enumerate(lengths):
        c = np.unique((np.arange(n, dtype=np.int64) * 7919 + 131 * i) % K)
        keys.append(i * np.int64(K) + c)
    keys = np.concatenate(keys) if keys else np.zeros(0, np.int64)
    val = synth.uniform_f32(seed, synth.STREAM_VAL, 0, len(keys))
    return synth.csr_from_sorted_keys(keys, len(lengths), K, val)


def case_matrix(case):
    if case == "segments":
        # Rows around one staged segment (256) and the long-row cut (512): single-row items of
        # 255-512 nonzeros, chunked rows past 512, short and empty rows between them.
        lens = [0, 1, 3, 255, 256, 257, 300, 2, 511, 512, 513, 0, 0, 1000, 4, 7, 260] * 3
        lens += [5] * 200
        return lengths_matrix(lens, 4096, 51), 2, 2
    if case == "hub_chunks":
        return synth.hub_matrix(512, 4096, 7, 3000, 6, 41), 4, 4
    if case == "empty_and_ragged":
        return synth.random_small(999, 777, 0.02, 42, empty_rows=100), 3, 5
    if case == "more_blocks":
        return synth.random_small(5, 9, 0.5, 13), 8, 8
    return synth.rmat(12, 8, 43), 4, 4  # accumulate


@pytest.mark.parametrize("dt", ["f32", "bf16"])
@pytest.mark.parametrize("case", ["segments", "hub_chunks", "empty_and_ragged", "more_blocks",
                                  "accumulate"])
def test_gather4_matches_register_gathers(dt, case):
    shiro = gu.lib()
    A, Pr, Pc = case_matrix(case)
    N = 128 if dt == "f32" else 256
    B = synth.dense_normal(A.K, N, 52)
    d = gu.dev()
    if dt == "bf16":
        bits = synth.to_bf16_bits(B)
        B = synth.bf16_bits_to_f32(bits).reshape(B.shape)
        Bd = torch.from_numpy(bits.view(np.int16)).to(d).view(torch.bfloat16)
    else:
        Bd = torch.from_numpy(B).to(d)
    acc = case == "accumulate"
    C0 = torch.from_numpy(synth.dense_normal(A.M, N, 53)).to(d)
    P = gu.plan_of(A, Pr, Pc, opts=shiro.make_opts(pipeline=7))
    Bp = P.pack(Bd)
    outs = {}
    for pipe in (7, 6):
        P.reschedule(pipeline=pipe)
        C = C0.clone() if acc else torch.full((A.M, N), float("nan"), device=d)
        P.spmm(Bp, out=C, accumulate=acc)
        torch.cuda.synchronize()
        P.check()
        outs[pipe] = C
    assert torch.equal(outs[7], outs[6]), "gather4 ring differs from the register gathers"
    if not acc:
        gu.check_spmm(A, B, outs[7])
