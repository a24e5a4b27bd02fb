"""Per-tile volume matrices of the four strategies (Eq. 1-3 and 9) from the library against the
oracle's tile statistics and covers."""
import numpy as np
import pytest

import oracle
from paper_2512_20178_gb300 import synth, volumes
import gpu_util as gu

pytestmark = pytest.mark.gpu


def setup_module(_):
    gu.need_gpu()


@pytest.mark.parametrize("b_dtype", ["f32", "bf16"])
@pytest.mark.parametrize("local", [False, True])
def test_volume_matrices(b_dtype, local):
    shiro = gu.lib()
    A = synth.rmat(12, 8, 201)
    N = 32
    flags = shiro.SHIRO_PLAN_LOCAL_DIAG if local else 0
    P = gu.plan_of(A, 4, 4, flags)
    R = volumes.report(P, N, b_dtype, "f32")
    O = oracle.plan(A, 4, 4)
    szb = volumes.SIZES[b_dtype]
    ob, oc, orow = O.volumes(N, szb, 4, local)
    V = {k: np.array(v) for k, v in R["tiles"].items()}
    for t in range(O.T):
        p, q = O.tile_pq(t)
        if local and p == q:
            assert all(V[k][t] == 0 for k in ("V_block", "V_col", "V_row", "V_joint"))
            continue
        assert V["V_block"][t] == ob[t] and V["V_col"][t] == oc[t], "Eq. 1 / Eq. 2"
        assert V["V_row"][t] == orow[t], "Eq. 3 (FP32 partial C rows, also for BF16 B)"
        nL, nR, ptr, adj = oracle.tile_graph(A, O, t)
        if szb == 4:
            assert V["V_joint"][t] == oracle.max_matching(nL, nR, ptr, adj) * N * 4
        else:
            flow, _, _ = oracle.min_weight_cover(nL, nR, ptr, adj, np.full(nL, N * 4),
                                                 np.full(nR, N * szb))
            assert V["V_joint"][t] == flow
        assert V["V_joint"][t] <= min(V["V_col"][t], V["V_row"][t])
    assert "V_joint (MiB)" in R["text"] and R["reductions"]["joint_vs_col"] >= 0
