"""The sampled parity checks of the GPU tests, run on the CPU against the full oracle metric.

The large-size GPU tests compare sampled rows (SpMM) or sampled nonzeros (SDDMM) on sub-problems
built from the samples.  Here a result with a known error -- the FP64 answer rounded to FP32, then
one element moved by a fixed multiple of its scale -- must give the same per-row and per-nonzero
errors through the sampled sub-problems as through the full oracle metric."""
import numpy as np

import gpu_util as gu
import oracle
from paper_2512_20178_gb300 import synth


def test_sampled_rows_error_matches_full_metric():
    A = synth.random_small(40, 50, 0.2, 31, empty_rows=3)
    B = synth.dense_normal(A.K, 8, 32)
    C64 = oracle.spmm(A, B)
    S = oracle.abs_scale(A, B)
    C = C64.astype(np.float32).astype(np.float64)
    i, k = 17, 5
    assert S[i, k] > 0
    C[i, k] = C64[i, k] + 3e-4 * S[i, k]
    full = oracle.scaled_error(C, C64, S, per_row=True)
    rows = np.array([0, 1, 17, 20, 39], np.int64)
    got = gu.sampled_rows_error(A, B, C[rows], rows)
    assert np.allclose(got, full[rows], rtol=1e-9, atol=1e-15)
    assert abs(got[2] - 3e-4) < 1e-9
    # An empty row (rows 0..2 are empty) with a nonzero value must fail.
    C[1, 0] = 1e-20
    assert gu.sampled_rows_error(A, B, C[rows], rows)[1] == np.inf


def test_sampled_sddmm_error_matches_full_metric():
    A = synth.random_small(30, 45, 0.25, 41)
    G = synth.dense_normal(A.M, 16, 42)
    B = synth.dense_normal(A.K, 16, 43)
    ref = oracle.sddmm(A, G, B)
    sc = oracle.sddmm(A, np.abs(G), np.abs(B))
    dA = ref.astype(np.float32).astype(np.float64)
    e = A.nnz // 2
    dA[e] = ref[e] - 2e-4 * sc[e]
    es = np.array([0, 3, e, A.nnz - 1], np.int64)
    got = gu.sampled_sddmm_error(A, G, B, dA, es)
    assert abs(got - oracle.scaled_error(dA[es], ref[es], sc[es])) < 1e-15
    assert abs(got - 2e-4) < 1e-9
