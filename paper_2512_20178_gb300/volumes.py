"""Per-tile communication volumes of the four strategies (the volume matrices of Sec. 6.2-6.3).

For every tile A^(p,q) of a plan this reports, in bytes for N columns:
  V_block  = (width of column block q) * N * sz_B       (Eq. 1, block-based: the whole B block)
  V_col    = |Cols(A^(p,q))| * N * sz_B                 (Eq. 2, column-based)
  V_row    = |Rows(A^(p,q))| * N * sz_C                 (Eq. 3, row-based)
  V_joint  = cost of the minimum weighted vertex cover  (Eq. 9 / Sec. 5.3.3, joint)
with sz_B the size of a B element and sz_C the size of a partial-C element (FP32 accumulators).
The joint cover is the min cut of Sec. 5.3.3 with costs N * sz_C per row and N * sz_B per
column (with sz_B == sz_C it is the uniform cover, mu * N * sz).  Local diagonal tiles of a
LOCAL_DIAG (1D) plan communicate nothing and report 0 everywhere.

Every number comes from the library (shiro_plan_volumes and the weighted cover solver); this
module only formats them.  ``--census 16,64,256`` instead prints, on the host, how often a
column repeats inside windows of consecutive rows (the evidence on tensor-core tiles).  Run as ``python -m paper_2512_20178_gb300.volumes --scale 20 --deg 16 --grid 4x4``
(needs a GPU: the plan is built on the device).
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

SIZES = {"f32": 4, "bf16": 2, "f64": 8}
DTYPES = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}


def tile_volumes(plan, N: int, b_dtype: str = "f32", c_dtype: str = "f32"):
    """Per-tile V_block, V_col, V_row (shiro_plan_volumes) and V_joint (the minimum weighted cover
    of shiro_plan_joint_weighted with a row priced at one partial C row, N * sz_C bytes, and a
    column at one B row, N * sz_B bytes), int64 arrays of n_tiles, plus the cover sizes.  Local
    diagonal tiles of a LOCAL_DIAG plan are reported as 0 by the library."""
    vb, vc, vr = plan.volumes(N, DTYPES[b_dtype], DTYPES[c_dtype])
    J = plan.joint_weighted(N * SIZES[c_dtype], N * SIZES[b_dtype])
    return {"V_block": vb.numpy(), "V_col": vc.numpy(), "V_row": vr.numpy(),
            "V_joint": J["cost"].numpy(), "cover_rows": J["cover_rows"].numpy(),
            "cover_cols": J["cover_cols"].numpy()}


def window_census(A, W: int, Pr: int = 4) -> dict:
    """Reuse of B rows inside windows of W consecutive rows of a row block (host only).

    For every window: nnz (gathers of a one-row-per-nonzero SpMM) and the number of distinct
    columns (the B rows an MMA tile over the window, or any kernel that stages each row of the
    window once, would read).  Reports sum(distinct) / nnz and the share of the nonzeros that sit
    in windows whose reuse nnz / distinct reaches 1.25, 2, 4 and 8."""
    rows = A.row_ids()
    rb = -(-A.M // Pr)
    p = rows // rb
    w = p * (-(-rb // W)) + (rows - p * rb) // W
    keys = w.astype(np.int64) * A.K + A.col.astype(np.int64)
    uw = np.unique(keys) // A.K
    nw = int(w.max()) + 1 if A.nnz else 1
    nnz_w = np.bincount(w, minlength=nw)
    dist_w = np.bincount(uw, minlength=nw)
    reuse = np.where(nnz_w > 0, nnz_w / np.maximum(dist_w, 1), 0.0)
    out = {"W": W, "windows_nonempty": int((nnz_w > 0).sum()),
           "distinct_over_nnz": float(dist_w.sum() / max(1, A.nnz)),
           "mma_density": float(A.nnz / max(1, W * dist_w.sum()))}
    for lo in (1.25, 2, 4, 8):
        out[f"nnz_share_reuse_ge_{lo}"] = float(nnz_w[reuse >= lo].sum() / max(1, A.nnz))
    return out


def format_matrix(name: str, v: np.ndarray, Pr: int, Pc: int, unit: float = 2**20) -> str:
    """One volume matrix as text, rows = receiving row block p, columns = sending block q (MiB)."""
    m = v.reshape(Pr, Pc) / unit
    w = max(8, max(len(f"{x:.1f}") for x in m.ravel()) + 1)
    lines = [f"{name} (MiB), row block p x column block q; total {v.sum() / unit:.1f} MiB"]
    lines.append(" " * 6 + "".join(f"q={q}".rjust(w) for q in range(Pc)))
    for p in range(Pr):
        lines.append(f"p={p}".ljust(6) + "".join(f"{x:.1f}".rjust(w) for x in m[p]))
    return "\n".join(lines)


def report(plan, N: int, b_dtype="f32", c_dtype="f32") -> dict:
    Pr, Pc = plan.info.P_r, plan.info.P_c
    V = tile_volumes(plan, N, b_dtype, c_dtype)
    tot = {k: int(V[k].sum()) for k in ("V_block", "V_col", "V_row", "V_joint")}
    text = "\n\n".join(format_matrix(k, V[k], Pr, Pc) for k in ("V_block", "V_col", "V_row", "V_joint"))
    red = {"joint_vs_col": 1 - tot["V_joint"] / max(1, tot["V_col"]),
           "joint_vs_row": 1 - tot["V_joint"] / max(1, tot["V_row"]),
           "col_vs_block": 1 - tot["V_col"] / max(1, tot["V_block"])}
    return {"totals": tot, "reductions": red, "text": text,
            "tiles": {k: V[k].tolist() for k in V}}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--graph", choices=["rmat", "er"], default="rmat")
    ap.add_argument("--scale", type=int, default=20)
    ap.add_argument("--deg", type=int, default=16)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--grid", default="4x4", help="P_r x P_c")
    ap.add_argument("--local-diag", action="store_true", help="1D: diagonal tiles are local")
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--b-dtype", choices=list(SIZES), default="f32")
    ap.add_argument("--c-dtype", choices=list(SIZES), default="f32")
    ap.add_argument("--json", action="store_true")
    ap.add_argument("--census", default="",
                    help="comma-separated window heights: print the row-window reuse census of "
                         "the matrix instead (host only, no GPU)")
    a = ap.parse_args(argv)
    from . import synth
    Pr, Pc = (int(x) for x in a.grid.lower().split("x"))
    A = synth.rmat(a.scale, a.deg, a.seed) if a.graph == "rmat" else \
        synth.er(1 << a.scale, a.deg, a.seed)
    if a.census:
        for W in (int(x) for x in a.census.split(",")):
            print(json.dumps({"graph": a.graph, "scale": a.scale, "deg": a.deg, "seed": a.seed,
                              "nnz": int(A.nnz), **window_census(A, W, Pr)}))
        return
    from . import shiro
    d = torch.device("cuda:0")
    rp = torch.from_numpy(A.rowptr).to(d)
    col = torch.from_numpy(A.col).to(d)
    val = torch.from_numpy(A.val).to(d)
    flags = shiro.SHIRO_PLAN_LOCAL_DIAG if a.local_diag else 0
    P = shiro.Plan.create(rp, col, val, A.M, A.K, Pr, Pc, flags=flags)
    R = report(P, a.N, a.b_dtype, a.c_dtype)
    head = {"graph": a.graph, "scale": a.scale, "deg": a.deg, "nnz": int(A.nnz), "grid": a.grid,
            "local_diag": a.local_diag, "N": a.N, "b_dtype": a.b_dtype, "c_dtype": a.c_dtype}
    if a.json:
        print(json.dumps({**head, **{k: R[k] for k in ("totals", "reductions", "tiles")}}))
    else:
        print(json.dumps(head))
        print(R["text"])
        print(json.dumps({"totals_bytes": R["totals"],
                          "reductions": {k: round(v, 4) for k, v in R["reductions"].items()}}))


if __name__ == "__main__":
    main()
