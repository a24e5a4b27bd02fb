"""Seeded input generators: determinism, published SplitMix64 outputs, structure (CPU only)."""
import numpy as np

from paper_2512_20178_gb300 import synth


def test_splitmix64_reference_vector():
    # First outputs of SplitMix64 (Steele et al. 2014; Vigna's splitmix64.c) from state 1234567.
    x = np.uint64(1234567)
    with np.errstate(over="ignore"):
        got = synth._mix(x + np.arange(1, 6, dtype=np.uint64) * synth.GAMMA)
    assert [int(v) for v in got] == [6457827717110365317, 3203168211198807973,
                                     9817491932198370423, 4593380528125082431,
                                     16408922859458223821]


def test_counter_based_chunk_independent():
    a = synth.draw_bits(9, 3, 0, 100)
    b = synth.draw_bits(9, 3, 40, 60)
    assert np.array_equal(a[40:], b)


def test_rmat_structure_and_determinism():
    A = synth.rmat(12, 8, 3)
    A2 = synth.rmat(12, 8, 3)
    assert np.array_equal(A.col, A2.col) and np.array_equal(A.val, A2.val)
    assert A.rowptr[0] == 0 and np.all(np.diff(A.rowptr) >= 0) and A.rowptr[-1] == len(A.col)
    rows = A.row_ids()
    key = rows * A.K + A.col
    assert np.all(np.diff(key) > 0), "CSR not sorted/unique"
    assert 0.8 * 8 * 4096 < A.nnz <= 8 * 4096
    deg = np.diff(A.rowptr)
    assert deg.max() > 20 * deg.mean(), "R-MAT should be power-law (hub rows)"
    assert np.all((A.val >= 0) & (A.val < 1))


def test_rmat_rejection_for_non_power_of_two():
    keys = synth.rmat_keys(1000, 10, 20000, 5)
    assert keys.max() < 1000 * 1000


def test_bf16_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7 + 2 ** -9, -2.5, 3.0e-39],
                 dtype=np.float32)
    back = synth.bf16_bits_to_f32(synth.to_bf16_bits(x))
    # 1+2^-8 is a tie -> even (1.0); 1+3*2^-8 tie -> even (1+2^-6); 1+2^-7+2^-9 rounds down.
    assert back[0] == 1.0 and back[1] == 1.0 and back[2] == np.float32(1.0 + 2 ** -6)
    assert back[3] == np.float32(1.0 + 2 ** -7) and back[4] == -2.5


def test_normal_moments():
    v = synth.normal_f32(1, 3, 200001)
    assert abs(v.mean()) < 0.01 and abs(v.std() - 1) < 0.01


def test_gcn_normalized_symmetric():
    A = synth.gcn_normalized(9, 4, 2)
    rows = A.row_ids()
    D = np.zeros((A.M, A.M))
    D[rows, A.col] = A.val
    assert np.allclose(D, D.T)
    assert np.all(np.diag(D) > 0)


def test_batch_graph_ranges():
    gb = synth.batch_graphs(6, 11, 100, 300)
    assert len(gb.graphs) == 6
    assert np.all((gb.node_counts >= 100) & (gb.node_counts <= 300))
    for g, n in zip(gb.graphs, gb.node_counts):
        assert g.M == n and g.K == n and (g.nnz == 0 or g.col.max() < n)
