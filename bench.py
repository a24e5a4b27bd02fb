"""Benchmark of the sparsity-aware SpMM hot path on one GB300 (or N independent replicas).

Workload (the JSON line's step): R-MAT CSR A 2^20 x 2^20, avg degree 16 (a,b,c,d =
.57,.19,.19,.05, duplicates merged), FP32 values U(0,1), dense B 2^20 x 128 FP32 N(0,1), 4x4
logical tiles.  One step = pack the B rows named by every tile's unique columns (Sec. 5.1 stage 3)
+ SpMM over the packed rows summed over the tiles of each row block (stage 5).  The plan (stage 1)
is built once per pattern, as in the paper, and timed on its own.

Bytes are algorithmic, each counted once:
  SpMM  (M+1)*8 + nnz*(4 col + 4 val) + R*N*sz (packed rows) + M*N*4 (C);
  pack  2*R*N*sz + R*4 (gather read + packed write + index), R = packed rows.
The step runs through the public call shiro_pack_spmm: one launch (k_spmm_lean_fused) for rows of
512 bytes, else the pack then the SpMM.  The JSON line reports:
  value     -- SpMM bytes / step time (pack + SpMM): the SpMM's numerator over the whole step,
               the conservative reading of the headline; GB/s;
  roofline  -- the step's kernel: for the one-launch step its pack + SpMM bytes / its mean launch
               time (CUDA events on its stream) vs the measured HBM copy bandwidth; under
               `spmm_kernel` the SpMM kernel alone over pre-packed rows (SpMM bytes / its launch
               time), with two ceilings: the HBM time of those bytes, and the same kernel,
               schedule and gather count on a matrix whose columns are folded so that every
               packed row stays in L2 (the gather-rate bound);
  e2e       -- the same SpMM bytes over steps that also copy B from pinned host memory and C back;
  forms     -- every other configuration, each with its time, algorithmic GB/s and fraction of
               the HBM peak: the backward (dB = A^T dC, dA by SDDMM), BF16-stored B, an N sweep,
               the precision workload (R-MAT 2^22, BF16 N = 256), the GCN layer fwd + bwd, 512
               batched graphs in one CUDA graph (tuned and default schedules), the small 1D ER
               case; clocks are sampled over all of them;
  cpu_baseline -- the FP64 C oracle on a strided row sample, on this host's cores.
Inputs are larger than L2 (B 512 MB, packed B 650 MB, C 512 MB), so no L2 flush is needed.

--impl reference times the FP64 CPU oracle (the reference arm here; the paper ships no kernels).
With N > 1 (torchrun) every rank runs its own replica (weak scaling, no collective on the path).
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMM GB/s & GFLOP/s (2*nnz*N) vs HBM roofline; fwd+bwd ms, FP32 vs BF16"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
# Every source of the library: a stored DRAM-traffic figure is used only while all are unchanged.
KERNEL_SOURCE_GLOBS = ["paper_2512_20178_gb300/csrc/*.cu", "paper_2512_20178_gb300/csrc/*.cuh",
                       "include/shiro.h"]
FORMS = ("backward", "bf16", "nsweep", "autotune", "cusparse", "precision", "gcn", "batch", "er")


def fused_step(N, sz):
    """Whether shiro_pack_spmm runs as one launch (k_spmm_lean_fused) with the default schedule:
    FP32 rows of 512 bytes (N = 128).  BF16 rows of 512 bytes take the pack and then the TMA
    gather4 ring, two launches."""
    return N * sz == 512 and sz == 4


def spmm_kernel(N, sz):
    """The SpMM kernel the automatic pipeline picks for N columns of sz-byte elements."""
    row = N * sz
    if sz == 2 and row == 512:
        return "k_spmm_g4"
    if row in (128, 256, 512):
        return "k_spmm_lean" if (sz == 2 and row == 256) else "k_spmm_lean_dyn"
    if row in (1024, 2048):
        return "k_spmm_lring"
    return "k_spmm"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=20)
    ap.add_argument("--deg", type=int, default=16)
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--tiles", type=int, default=4)
    ap.add_argument("--seed", type=int, default=None,
                    help="generator seed (default: 3 for the R-MAT 2^22 degree-32 precision "
                         "workload, else 2)")
    ap.add_argument("--forms", default="all",
                    help="comma-separated subset of " + ",".join(FORMS) + ", or all / none")
    ap.add_argument("--no-forms", action="store_true", help="same as --forms none")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16"],
                    help="storage of B (and of the packed rows); accumulation is FP32 either way")
    ap.add_argument("--er", action="store_true",
                    help="time only the small 1D case: Erdos-Renyi 4096 x 4096, avg degree 8, "
                         "values U(-1, 1), B 4096 x 32, P = 4 row blocks with local diagonal tiles")
    ap.add_argument("--gcn", action="store_true",
                    help="time only the GCN layer: Y = A_hat (X W), A_hat the symmetric-normalised "
                         "R-MAT 2^scale graph with self loops, X n x 256, W 256 x N, fwd + bwd")
    ap.add_argument("--batch", type=int, default=0,
                    help="time only the batched form: this many R-MAT graphs, n ~ U{100..20000}, "
                         "degree log-uniform [4, 40], B n x N in BF16, one CUDA-graph replay per step")
    ap.add_argument("--traffic-from", default=None, metavar="CSV",
                    help="write the DRAM-traffic record of profiles/traffic.json from an ncu "
                         "'--page raw --csv' export (with --kernel and --workload) and exit")
    ap.add_argument("--kernel", default=None, help="kernel instantiation of --traffic-from")
    ap.add_argument("--workload", default=None, help="workload name of --traffic-from")
    ap.add_argument("--command", default=None, help="the ncu command of --traffic-from")
    a = ap.parse_args(argv)
    if a.no_forms:
        a.forms = "none"
    if a.seed is None:
        a.seed = 3 if (a.scale, a.deg) == (22, 32) else 2
    return a


def forms_of(args):
    if args.forms in ("all", ""):
        return set(FORMS)
    if args.forms == "none":
        return set()
    s = {f.strip() for f in args.forms.split(",") if f.strip()}
    bad = s - set(FORMS)
    if bad:
        raise SystemExit(f"unknown forms {sorted(bad)}")
    return s


def workload(args):
    from paper_2512_20178_gb300 import synth
    A = synth.rmat(args.scale, args.deg, args.seed)
    B = synth.dense_normal(A.K, args.N, args.seed)
    return A, B


def workload_name(scale, deg, N, tiles, dtype):
    return f"rmat{scale}_deg{deg}_N{N}_{tiles}x{tiles}_{dtype}"


def config(args, A):
    """The workload, identical on both arms (no measured or plan-dependent keys)."""
    return {"workload": workload_name(args.scale, args.deg, args.N, args.tiles, args.dtype),
            "M": A.M, "K": A.K, "nnz": A.nnz, "N": args.N, "tiles": f"{args.tiles}x{args.tiles}",
            "rmat": [0.57, 0.19, 0.19, 0.05], "seed": args.seed, "storage": args.dtype,
            "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas"}


def spmm_bytes(M, nnz, R, N, sz):
    """Algorithmic bytes of one SpMM over R packed rows of N sz-byte elements (FP32 C)."""
    return (M + 1) * 8 + nnz * 8 + R * N * sz + M * N * 4


def pack_bytes(R, N, sz):
    """Algorithmic bytes of one pack of R rows: gather read, packed write, source index."""
    return 2 * R * N * sz + R * 4


def sddmm_bytes(M, nnz, R, N, sz):
    """Algorithmic bytes of one SDDMM: A's pattern, dC rows, packed B rows, dA values."""
    return nnz * 8 + M * N * sz + R * N * sz + nnz * 4


def bwd_bytes(K, nnz, RT, N, sz, nzc):
    """Algorithmic bytes of the one-launch backward over A^T (K rows, RT packed dC rows): the pack
    of dC, the SpMM of A^T over the packed rows (writing dB), one B row per non-empty row of A^T
    (nzc of them) and the dA values."""
    return pack_bytes(RT, N, sz) + spmm_bytes(K, nnz, RT, N, sz) + nzc * N * sz + nnz * 4


def step_bytes(M, nnz, R, N, sz):
    return spmm_bytes(M, nnz, R, N, sz), pack_bytes(R, N, sz)


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def reduce_max(value: float, world: int, device=None) -> float:
    """Max over ranks (the slowest replica sets the job time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return
        time.sleep(0.1)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 10:
                continue
            try:
                sm.append(float(f[2]))
                mx = float(f[3])
            except ValueError:
                continue
            for n, v in zip(names, f[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        # Under load: samples above half the maximum (drops the idle edges of the window).
        load = [s for s in sm if mx is None or s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def sources_sha256() -> str:
    h = hashlib.sha256()
    for pat in KERNEL_SOURCE_GLOBS:
        for f in sorted(glob.glob(os.path.join(ROOT, pat))):
            h.update(os.path.relpath(f, ROOT).encode())
            h.update(open(f, "rb").read())
    return h.hexdigest()


def traffic_from_profile(kernel: str, workload_name_: str):
    """DRAM bytes per launch of `kernel` on `workload_name_` from the committed ncu record, if
    the library's sources are those the counters were taken on (else None)."""
    try:
        recs = json.load(open(PROFILE_TRAFFIC))
    except (OSError, ValueError):
        return None
    sha = sources_sha256()
    for r in recs.get("records", []):
        if (r.get("kernel_name") == kernel and r.get("workload") == workload_name_
                and r.get("sources_sha256") == sha):
            return r.get("dram_bytes_per_launch")
    return None


def write_traffic_record(csv_path, instantiation, workload_name_, command):
    """Adds (or replaces) the record of one kernel on one workload: the mean over the captured
    launches of dram__bytes_read.sum + dram__bytes_write.sum, from an ncu raw CSV export."""
    import csv
    rows = [r for r in csv.reader(open(csv_path)) if r and not r[0].startswith("==")]
    head = rows[0]
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    name = instantiation.split("<")[0]
    want = ("dram__bytes_read.sum", "dram__bytes_write.sum")
    tot = []
    strip = lambda k: k.replace("void ", "").replace("shiro::", "")
    if "Metric Name" in head:
        # One row per (launch, metric): the --metrics --csv log.
        ci = {k: head.index(k) for k in ("ID", "Kernel Name", "Metric Name", "Metric Unit",
                                         "Metric Value")}
        per = {}
        for r in rows[1:]:
            if not strip(r[ci["Kernel Name"]]).startswith(name) or r[ci["Metric Name"]] not in want:
                continue
            v = float(r[ci["Metric Value"]].replace(",", "")) * scale.get(r[ci["Metric Unit"]], 1)
            per[r[ci["ID"]]] = per.get(r[ci["ID"]], 0.0) + v
        tot = list(per.values())
    else:
        # One row per launch with a units row below the header: the --page raw --csv export.
        ci = {k: head.index(k) for k in ("Kernel Name",) + want}
        units = rows[1] if len(rows) > 1 and not rows[1][ci["Kernel Name"]] else None
        for r in rows[1 + (units is not None):]:
            if not strip(r[ci["Kernel Name"]]).startswith(name):
                continue
            b = 0.0
            for k in want:
                u = units[ci[k]] if units else "byte"
                b += float(r[ci[k]].replace(",", "")) * scale.get(u, 1)
            tot.append(b)
    if not tot:
        raise SystemExit(f"no launch of {name} in {csv_path}")
    try:
        recs = json.load(open(PROFILE_TRAFFIC))
    except (OSError, ValueError):
        recs = {"records": []}
    recs["note"] = ("DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, ncu, "
                    "--clock-control none), mean over the captured launches; valid while the "
                    "library sources hash to sources_sha256")
    recs["records"] = [r for r in recs.get("records", [])
                       if not (r.get("kernel") == instantiation and r.get("workload") == workload_name_)]
    recs["records"].append({"kernel": instantiation, "kernel_name": name, "workload": workload_name_,
                            "dram_bytes_per_launch": int(round(sum(tot) / len(tot))),
                            "launches": len(tot), "sources_sha256": sources_sha256(),
                            "command": command})
    with open(PROFILE_TRAFFIC, "w") as f:
        json.dump(recs, f, indent=1)
        f.write("\n")


def cpu_model() -> str:
    """Host CPU model as lscpu reports it (empty if unavailable)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
    except (OSError, subprocess.SubprocessError):
        return ""
    for line in out.splitlines():
        if line.strip().lower().startswith("model name"):
            return line.split(":", 1)[1].strip()
    return ""


def hbm_peak():
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        peaks = {}
    if peaks.get("hbm_gbs"):
        return float(peaks["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def cpu_baseline(A, B, args, stride=8):
    """The FP64 oracle (pack + SpMM through the packed rows) on every stride-th row of A."""
    import oracle
    from paper_2512_20178_gb300 import synth
    rows = np.arange(0, A.M, stride)
    cnt = np.diff(A.rowptr)[rows]
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(cnt, out=rp[1:])
    idx = np.concatenate([np.arange(A.rowptr[r], A.rowptr[r + 1]) for r in rows]) if len(rows) else np.zeros(0, np.int64)
    S = synth.CSR(len(rows), A.K, rp, A.col[idx], A.val[idx])
    t0 = time.perf_counter()
    P = oracle.plan(S, args.tiles, args.tiles)
    t1 = time.perf_counter()
    _, src = P.pack_layout(False)
    Bp = oracle.pack(B, src)
    oracle.spmm_packed(S, P, Bp, B)
    t2 = time.perf_counter()
    sp = spmm_bytes(S.M, S.nnz, len(src), args.N, 4)
    return {"value": sp / (t2 - t1) / 1e9, "unit": "GB/s", "cores": oracle.threads(),
            "kind": "oracle", "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "sample": f"every {stride}th row ({S.M} rows, {S.nnz} nnz), pack + SpMM via packed "
                      f"rows in FP64 (SpMM bytes over pack + SpMM time); plan {t1 - t0:.2f} s "
                      f"not counted",
            "seconds": t2 - t1}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    A, B = workload(args)
    oracle.build()
    # Size the per-step row sample so that warmup + steps take about two minutes in total.
    probe = cpu_baseline(A, B, args, 256)
    per_step = 120.0 / max(1, args.warmup + args.steps)
    stride = 256
    while stride > 8 and probe["seconds"] * 256 / (stride // 2) <= per_step:
        stride //= 2
    res = None
    ts = []
    for k in range(args.warmup + args.steps):
        r = cpu_baseline(A, B, args, stride)
        if k >= args.warmup:
            ts.append(r["seconds"])
        res = r
    ms = 1e3 * sum(ts) / max(len(ts), 1)
    line = {"impl": "reference", "metric": METRIC, "value": res["value"], "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded R-MAT, counter-based SplitMix64)", "config": config(args, A),
            "cpu_baseline": {k: res[k] for k in ("value", "unit", "cores", "kind", "sample", "cpu_model", "nproc")},
            "e2e": {"value": res["value"], "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def timed(fn, stream, reps=20, warm=3):
    """Mean device time of fn() in ms (CUDA events on `stream`, after `warm` untimed calls)."""
    import torch
    for _ in range(warm):
        fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def gbps(nbytes, ms):
    return nbytes / (ms * 1e-3) / 1e9


def frac_entry(nbytes, ms, peak):
    g = gbps(nbytes, ms)
    return {"ms": ms, "bytes": int(nbytes), "GBps": g, "frac": g / peak}


def measure_l2_ceiling(A, args, dev, stream, sz, tdt, reps):
    """The same SpMM kernel, schedule and gather count with every packed row L2-resident: A's
    columns are divided by a power of two so that the packed set is at most 32 MB (row structure,
    nonzeros per row and their order unchanged; duplicates are summed), B is random."""
    import torch
    from paper_2512_20178_gb300 import shiro
    N = args.N
    row = N * sz
    # Each row block's tiles together name at most K2 packed rows: K2 <= 32 MB / row / P_r.
    target = max(args.tiles, (32 << 20) // row // args.tiles)
    shift = max(0, int(np.ceil(np.log2(max(1.0, A.K / target)))))
    K2 = ((A.K - 1) >> shift) + 1
    rp = torch.from_numpy(A.rowptr).to(dev)
    colf = torch.from_numpy((A.col >> shift).astype(np.int32)).to(dev)
    val = torch.from_numpy(A.val).to(dev)
    P = shiro.Plan.create(rp, colf, val, A.M, K2, args.tiles, args.tiles)
    R = P.info.packed_rows
    Bp = torch.randn((R, N), device=dev).to(tdt)
    C = torch.empty((A.M, N), dtype=torch.float32, device=dev)
    scr = P.new_scratch(N, tdt)
    ms = timed(lambda: P.spmm(Bp, out=C, scratch=scr), stream, reps)
    gather_bytes = A.nnz * N * sz
    return {"ms": ms, "packed_rows": R, "packed_MB": R * row / 1e6, "column_shift": shift,
            "gather_bytes": gather_bytes, "gather_GBps": gbps(gather_bytes, ms),
            "what": "same kernel and schedule, columns >> shift so the packed rows fit in L2"}


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", torch.cuda.current_device())
    import __graft_entry__ as g
    g.build()
    from paper_2512_20178_gb300 import shiro, synth

    A, B = workload(args)
    N = args.N
    rp = torch.from_numpy(A.rowptr).to(dev)
    col = torch.from_numpy(A.col).to(dev)
    val = torch.from_numpy(A.val).to(dev)
    bf16 = args.dtype == "bf16"
    tdt = torch.bfloat16 if bf16 else torch.float32
    sz = 2 if bf16 else 4
    if bf16:
        Bh = torch.from_numpy(synth.to_bf16_bits(B).view(np.int16)).view(torch.bfloat16)
    else:
        Bh = torch.from_numpy(B)
    Bd = Bh.to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P = shiro.Plan.create(rp, col, val, A.M, A.K, args.tiles, args.tiles)
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    R = P.info.packed_rows
    Bp = torch.empty((R, N), dtype=tdt, device=dev)
    C = torch.empty((A.M, N), dtype=torch.float32, device=dev)
    tuned = None
    if args.autotune:
        P.pack(Bd, out=Bp)
        tuned = P.autotune(Bp, B=Bd, C=C)
    scratch = P.new_scratch(N, tdt)
    stream = torch.cuda.current_stream()
    fused = fused_step(N, sz) and not args.autotune

    def step():
        # One step of the hot path through the public API: pack (stage 3) + SpMM (stage 5).
        P.pack_spmm(Bd, Bpack=Bp, out=C, scratch=scratch)

    for _ in range(args.warmup):
        step()
    K = args.steps
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(K):
        step()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks.stop()
    ms = ev[0].elapsed_time(ev[K]) / K
    step_ms = sorted(ev[k].elapsed_time(ev[k + 1]) for k in range(K))
    pct = lambda xs, q: xs[min(len(xs) - 1, int(q * (len(xs) - 1) + 0.5))]
    step_stats = {"mean": ms, "median": pct(step_ms, 0.5), "p10": pct(step_ms, 0.1),
                  "p90": pct(step_ms, 0.9)}
    ms_max = reduce_max(ms, world, dev)
    sp_bytes, pk_bytes = step_bytes(A.M, A.nnz, R, N, sz)
    value = world * sp_bytes / (ms_max * 1e-3) / 1e9
    gflops = world * 2.0 * A.nnz * N / (ms_max * 1e-3) / 1e9
    peak, peak_src = hbm_peak()
    wname = workload_name(args.scale, args.deg, N, args.tiles, args.dtype)

    # The SpMM kernel alone over pre-packed rows (events around each launch) and the pack alone.
    P.pack(Bd, out=Bp)
    torch.cuda.synchronize()
    Ks = max(10, min(K, 100))
    ea = [torch.cuda.Event(enable_timing=True) for _ in range(Ks)]
    eb = [torch.cuda.Event(enable_timing=True) for _ in range(Ks)]
    for k in range(3):
        P.spmm(Bp, out=C, scratch=scratch)
    for k in range(Ks):
        ea[k].record(stream)
        P.spmm(Bp, out=C, scratch=scratch)
        eb[k].record(stream)
    torch.cuda.synchronize()
    launch_ms = sorted(a.elapsed_time(b) for a, b in zip(ea, eb))
    spmm_ms = sum(launch_ms) / Ks
    spmm_stats = {"mean": spmm_ms, "median": pct(launch_ms, 0.5), "p10": pct(launch_ms, 0.1),
                  "p90": pct(launch_ms, 0.9)}
    pack_ms = timed(lambda: P.pack(Bd, out=Bp), stream, Ks)

    ceiling = measure_l2_ceiling(A, args, dev, stream, sz, tdt, reps=max(10, min(K, 50)))
    achieved_spmm = gbps(sp_bytes, spmm_ms)
    kname = spmm_kernel(N, sz)
    spmm_roof = {"bound": "hbm", "kernel": kname, "achieved": achieved_spmm, "peak": peak,
                 "peak_source": peak_src, "unit": "GB/s", "frac": achieved_spmm / peak,
                 "traffic": traffic_from_profile(kname, wname), "algorithmic_bytes": sp_bytes,
                 "ms_per_launch": spmm_ms, "launch_ms": spmm_stats,
                 "ceilings": {
                     "hbm_ms": sp_bytes / (peak * 1e9) * 1e3,
                     "l2_gather_ms": ceiling["ms"],
                     "l2_gather_frac": gbps(sp_bytes, ceiling["ms"]) / peak,
                     "kernel_vs_l2_gather": ceiling["ms"] / spmm_ms,
                     "l2_gather": ceiling}}
    if fused:
        # The step is one launch of the fused kernel: its algorithmic bytes are the pack's and
        # the SpMM's, each counted once.
        ach = gbps(sp_bytes + pk_bytes, ms)
        roofline = {"bound": "hbm", "kernel": "k_spmm_lean_fused", "achieved": ach, "peak": peak,
                    "peak_source": peak_src, "unit": "GB/s", "frac": ach / peak,
                    "traffic": traffic_from_profile("k_spmm_lean_fused", wname),
                    "algorithmic_bytes": sp_bytes + pk_bytes,
                    "bytes_definition": "pack 2*R*N*sz + R*4 plus SpMM (M+1)*8 + nnz*8 + R*N*sz + M*N*4",
                    "ms_per_launch": ms, "launch_ms": step_stats,
                    "spmm_kernel": spmm_roof}
    else:
        roofline = dict(spmm_roof)

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(args, P, Bh, Bd, Bp, C, scratch, stream, dev, sp_bytes, sz, world, K)

    forms = None
    fset = forms_of(args)
    if fset and rank == 0:
        fclocks = ClockSampler(dev.index if dev.index is not None else 0)
        fclocks.start()
        forms = measure_forms(args, fset, A, B, P, Bd, Bp, C, scratch, rp, col, val, dev, stream,
                              peak, bf16)
        fclocks.stop()
        forms["clocks"] = fclocks.summary()

    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "storage": args.dtype,
            "data": "synthetic (seeded R-MAT, counter-based SplitMix64)",
            "config": config(args, A),
            "value_definition": "SpMM algorithmic bytes / (pack + SpMM) step time",
            "step_ms": step_stats,
            "plan": {"packed_rows": R, "plan_ms": plan_ms, "schedule": P.info.opts.as_dict(),
                     "autotuned": tuned},
            "gflops": gflops, "step": "shiro_pack_spmm" + (" (one launch)" if fused else
                                                            " (pack, then SpMM)"),
            "spmm_ms": spmm_ms, "pack_ms": pack_ms, "two_launch_ms": spmm_ms + pack_ms,
            "spmm_over_packed_GBps": achieved_spmm,
            "pack_GBps": gbps(pk_bytes, pack_ms), "pack_bytes": pk_bytes,
            "gpu_launches": (1 if fused else 2) * K, "roofline": roofline,
            "clocks": clocks.summary()}
    if e2e:
        line["e2e"] = e2e
    if forms:
        line["forms"] = forms
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        line["cpu_baseline"] = {k: v for k, v in cpu_baseline(A, B, args).items() if k != "seconds"}
        cores = oracle.threads()
        oracle.set_threads(1)
        one = cpu_baseline(A, B, args, stride=128)
        oracle.set_threads(cores)
        line["cpu_baseline"]["one_thread"] = {"value": one["value"], "unit": "GB/s", "cores": 1,
                                              "sample": one["sample"]}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def measure_e2e(args, P, Bh, Bd, Bp, C, scratch, stream, dev, sp_bytes, sz, world, K):
    """End to end through the public API: every step copies its B from pinned host memory and
    reads its C back into pinned host memory.  Steps are pipelined as a serving loop would run
    them: step k+1's upload and step k-1's download overlap step k's pack + SpMM (two device
    buffers each for B and C, one stream per direction).  The serial figure (one stream, no
    overlap) is reported beside it."""
    import torch
    N = args.N
    Bh = Bh.pin_memory()
    Ch = [torch.empty(tuple(C.shape), dtype=torch.float32).pin_memory() for _ in range(2)]
    Bdd = [Bd, torch.empty_like(Bd)]
    Cd = [C, torch.empty_like(C)]
    s_up, s_down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev = lambda: torch.cuda.Event()
    up_done, comp_done, down_done = [ev(), ev()], [ev(), ev()], [ev(), ev()]
    for e in comp_done + down_done:
        e.record(stream)

    def e2e_step(k):
        j = k % 2
        with torch.cuda.stream(s_up):
            s_up.wait_event(comp_done[j])          # B buffer j free again
            Bdd[j].copy_(Bh, non_blocking=True)
            up_done[j].record(s_up)
        stream.wait_event(up_done[j])
        stream.wait_event(down_done[j])            # C buffer j read back
        P.pack_spmm(Bdd[j], Bpack=Bp, out=Cd[j], scratch=scratch)
        comp_done[j].record(stream)
        with torch.cuda.stream(s_down):
            s_down.wait_event(comp_done[j])
            Ch[j].copy_(Cd[j], non_blocking=True)
            down_done[j].record(s_down)

    Ke = max(2, min(K, 100))
    for k in range(min(args.warmup, 3) + 1):
        e2e_step(k)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s_up.wait_event(e0)                            # the first upload starts inside the region
    for k in range(Ke):
        e2e_step(k)
    stream.wait_event(down_done[(Ke - 1) % 2])
    stream.wait_event(down_done[Ke % 2])
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = reduce_max(e0.elapsed_time(e1) / Ke, world, dev)
    # Serial: upload, step and download on one stream.
    for _ in range(2):
        Bd.copy_(Bh, non_blocking=True)
        P.pack_spmm(Bd, Bpack=Bp, out=C, scratch=scratch)
        Ch[0].copy_(C, non_blocking=True)
    torch.cuda.synchronize()
    e0.record(stream)
    Ks = max(1, min(K, 30))
    for _ in range(Ks):
        Bd.copy_(Bh, non_blocking=True)
        P.pack_spmm(Bd, Bpack=Bp, out=C, scratch=scratch)
        Ch[0].copy_(C, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    serial_ms = reduce_max(e0.elapsed_time(e1) / Ks, world, dev)
    return {"value": world * gbps(sp_bytes, e2e_ms), "unit": "GB/s",
            "h2d_bytes_per_step": int(Bh.numel() * sz), "d2h_bytes_per_step": int(Ch[0].numel() * 4),
            "ms_per_step": e2e_ms, "pipelined": "upload k+1 / compute k / download k-1",
            "serial_ms_per_step": serial_ms}


def measure_forms(args, fset, A, B, P, Bd, Bp, C, scratch, rp, col, val, dev, stream, peak,
                  bf16, reps=20):
    """Every other configuration on this GPU (device times, algorithmic bytes, frac of peak)."""
    import torch
    from paper_2512_20178_gb300 import shiro, synth
    N = args.N
    R = P.info.packed_rows
    out = {"peak_GBps": peak}
    run = lambda fn: timed(fn, stream, reps)
    fwd_ms = run(lambda: P.pack_spmm(Bd, Bpack=Bp, out=C, scratch=scratch))
    if "backward" in fset and not bf16:
        PT = shiro.Plan.create(rp, col, val, A.M, A.K, args.tiles, args.tiles,
                               flags=shiro.SHIRO_PLAN_TRANSPOSE)
        G = torch.randn((A.M, N), device=dev, generator=torch.Generator(device=dev).manual_seed(5))
        RT = PT.info.packed_rows
        Gp = torch.empty((RT, N), dtype=torch.float32, device=dev)
        dB = torch.empty((A.K, N), dtype=torch.float32, device=dev)
        dA = torch.empty(A.nnz, dtype=torch.float32, device=dev)
        sT = PT.new_scratch(N, torch.float32)
        PT.pack(G, out=Gp)
        db_spmm = run(lambda: PT.spmm(Gp, out=dB, scratch=sT))
        db_pack = run(lambda: PT.pack(G, out=Gp))
        db_ms = run(lambda: PT.pack_spmm(G, Bpack=Gp, out=dB, scratch=sT))
        da_ms = run(lambda: P.sddmm(G, Bp, out=dA))
        # The backward as the autograd wrapper runs it: one launch for dB and dA (B given).
        bwd_ms = run(lambda: shiro.spmm_backward(P, PT, G, Bp, B=Bd, scratch=sT, dCpack=Gp,
                                                 dB=dB, dA=dA))
        wname = workload_name(args.scale, args.deg, N, args.tiles, "f32")
        sd = frac_entry(sddmm_bytes(A.M, A.nnz, R, N, 4), da_ms, peak)
        sd["kernel"] = "k_sddmm_grp"
        sd["traffic"] = traffic_from_profile("k_sddmm_grp", wname)
        nzc = int(np.count_nonzero(np.bincount(A.col, minlength=A.K)))
        one = frac_entry(bwd_bytes(A.K, A.nnz, RT, N, 4, nzc), bwd_ms, peak)
        one["kernel"] = "k_spmm_lean_bwd"
        one["traffic"] = traffic_from_profile("k_spmm_lean_bwd", wname)
        one["bytes_definition"] = ("pack 2*RT*N*4 + RT*4, SpMM of A^T (K+1)*8 + nnz*8 + RT*N*4 + "
                                   "K*N*4, B rows nzc*N*4, dA nnz*4")
        # Rows of 256 bytes (N = 64): the one launch against the two calls.
        narrow = {}
        for n in (64,):
            Bn = torch.from_numpy(synth.dense_normal(A.K, n, 12)).to(dev)
            Gn = torch.randn((A.M, n), device=dev, generator=torch.Generator(device=dev).manual_seed(6))
            Bpn = P.pack(Bn)
            Gpn = torch.empty((RT, n), dtype=torch.float32, device=dev)
            dBn = torch.empty((A.K, n), dtype=torch.float32, device=dev)
            sTn = PT.new_scratch(n, torch.float32)
            one_n = run(lambda: shiro.spmm_backward(P, PT, Gn, Bpn, B=Bn, scratch=sTn, dCpack=Gpn,
                                                    dB=dBn, dA=dA))
            two_n = run(lambda: (PT.pack_spmm(Gn, Bpack=Gpn, out=dBn, scratch=sTn),
                                 P.sddmm(Gn, Bpn, out=dA)))
            narrow[str(n)] = {"one_launch": frac_entry(bwd_bytes(A.K, A.nnz, RT, n, 4, nzc), one_n,
                                                       peak),
                              "two_calls_ms": two_n}
            del Bn, Gn, Bpn, Gpn, dBn, sTn
        out["backward"] = {
            "workload": wname, "fwd_ms": fwd_ms, "fwd_bwd_ms": fwd_ms + bwd_ms,
            "bwd_one_launch": one, "narrow_rows_fp32": narrow,
            "two_calls": {"fwd_bwd_ms": fwd_ms + db_ms + da_ms, "bwd_ms": db_ms + da_ms,
                          "what": "shiro_pack_spmm on the transposed plan, then shiro_sddmm"},
            "dB_step_ms": db_ms, "dB_spmm": frac_entry(spmm_bytes(A.K, A.nnz, RT, N, 4), db_spmm, peak),
            "dB_pack": frac_entry(pack_bytes(RT, N, 4), db_pack, peak),
            "dB_step_GBps_spmm_bytes": gbps(spmm_bytes(A.K, A.nnz, RT, N, 4), db_ms),
            "dA_sddmm": sd, "transpose_packed_rows": RT}
        del PT, G, Gp, dB, dA, sT
    if "bf16" in fset and not bf16:
        Bh16 = torch.from_numpy(synth.to_bf16_bits(B).view(np.int16)).to(dev).view(torch.bfloat16)
        Bp16 = torch.empty((R, N), dtype=torch.bfloat16, device=dev)
        s16 = P.new_scratch(N, torch.bfloat16)
        P.pack(Bh16, out=Bp16)
        sp16 = run(lambda: P.spmm(Bp16, out=C, scratch=s16))
        st16 = run(lambda: P.pack_spmm(Bh16, Bpack=Bp16, out=C, scratch=s16))
        e = frac_entry(spmm_bytes(A.M, A.nnz, R, N, 2), sp16, peak)
        out["bf16_B"] = {"spmm": e, "step_ms": st16,
                         "step_GBps_spmm_bytes": gbps(spmm_bytes(A.M, A.nnz, R, N, 2), st16),
                         "vs_fp32_step_speedup": fwd_ms / st16}
        del Bh16, Bp16, s16
    if "nsweep" in fset:
        n_sweep = {}
        for n in (32, 64, 128, 256):
            Bn = torch.from_numpy(synth.dense_normal(A.K, n, 7)).to(dev)
            Bpn = torch.empty((R, n), dtype=torch.float32, device=dev)
            Cn = torch.empty((A.M, n), dtype=torch.float32, device=dev)
            sn = P.new_scratch(n, torch.float32)
            P.pack(Bn, out=Bpn)
            spmm_n = run(lambda: P.spmm(Bpn, out=Cn, scratch=sn))
            step_n = run(lambda: P.pack_spmm(Bn, Bpack=Bpn, out=Cn, scratch=sn))
            e = frac_entry(spmm_bytes(A.M, A.nnz, R, n, 4), spmm_n, peak)
            e["step_ms"] = step_n
            e["step_GBps_spmm_bytes"] = gbps(spmm_bytes(A.M, A.nnz, R, n, 4), step_n)
            n_sweep[str(n)] = e
            del Bn, Bpn, Cn, sn
        out["n_sweep_fp32"] = n_sweep
    if "autotune" in fset and not bf16:
        # The schedule the autotuner picks per N on this matrix, against the default schedule
        # (SpMM alone over pre-packed rows, FP32).  The plan's schedule is restored afterwards.
        tunes = {}
        default = P.info.opts.as_dict()
        for n in (32, 64, 128, 256):
            Bn = torch.from_numpy(synth.dense_normal(A.K, n, 11)).to(dev)
            Bpn = torch.empty((R, n), dtype=torch.float32, device=dev)
            Cn = torch.empty((A.M, n), dtype=torch.float32, device=dev)
            P.pack(Bn, out=Bpn)
            sn = P.new_scratch(n, torch.float32)
            d_ms = run(lambda: P.spmm(Bpn, out=Cn, scratch=sn))
            pick = P.autotune(Bpn, C=Cn, reps=3)
            sn = P.new_scratch(n, torch.float32)
            t_ms = run(lambda: P.spmm(Bpn, out=Cn, scratch=sn))
            tunes[str(n)] = {"default_ms": d_ms, "tuned_ms": t_ms, "speedup": d_ms / t_ms,
                             "pick": pick}
            P.reschedule(**default)
            del Bn, Bpn, Cn, sn
        out["autotune_fp32"] = tunes
    if "cusparse" in fset and not bf16:
        # Comparator (not on the path): cuSPARSE CSR SpMM through torch.sparse.mm, unpacked B.
        try:
            At = torch.sparse_csr_tensor(rp.to(torch.int32), col, val, size=(A.M, A.K))
            Cc = torch.sparse.mm(At, Bd)
            cus_ms = run(lambda: torch.sparse.mm(At, Bd))
            P.pack(Bd, out=Bp)
            P.spmm(Bp, out=C, scratch=scratch)
            torch.cuda.synchronize()
            out["cusparse"] = {"ms": cus_ms, "ours_spmm_ms": run(lambda: P.spmm(Bp, out=C, scratch=scratch)),
                               "ours_step_ms": fwd_ms, "max_abs_diff": float((Cc - C).abs().max()),
                               "what": "torch.sparse.mm (cuSPARSE CSR SpMM) on the original B, same A, N"}
            del At, Cc
        except Exception as e:  # the comparator is optional context
            out["cusparse"] = {"unavailable": str(e).splitlines()[0][:200]}
    torch.cuda.empty_cache()
    if "precision" in fset:
        out["precision"] = form_precision(dev, stream, peak, reps)
        torch.cuda.empty_cache()
    if "gcn" in fset:
        out["gcn"] = form_gcn(dev, stream, peak, reps)
        torch.cuda.empty_cache()
    if "batch" in fset:
        out["batch"] = form_batch(dev, stream, peak, reps)
        torch.cuda.empty_cache()
    if "er" in fset:
        out["er"] = form_er(dev, stream, peak, max(reps, 100))
    return out


def form_precision(dev, stream, peak, reps, scale=22, deg=32, N=256, seed=3):
    """The precision workload: R-MAT 2^22, avg degree 32, B 2^22 x 256 stored in BF16, FP32
    accumulation and C, 4x4 tiles (the same matrix and B as its parity test)."""
    import torch
    from paper_2512_20178_gb300 import shiro, synth
    A = synth.rmat(scale, deg, seed)
    B = synth.dense_normal(A.K, N, seed)
    Bd = torch.from_numpy(synth.to_bf16_bits(B).view(np.int16)).to(dev).view(torch.bfloat16)
    del B
    rp = torch.from_numpy(A.rowptr).to(dev)
    col = torch.from_numpy(A.col).to(dev)
    val = torch.from_numpy(A.val).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P = shiro.Plan.create(rp, col, val, A.M, A.K, 4, 4)
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    R = P.info.packed_rows
    Bp = torch.empty((R, N), dtype=torch.bfloat16, device=dev)
    C = torch.empty((A.M, N), dtype=torch.float32, device=dev)
    scr = P.new_scratch(N, torch.bfloat16)
    P.pack(Bd, out=Bp)
    sp_ms = timed(lambda: P.spmm(Bp, out=C, scratch=scr), stream, reps)
    pk_ms = timed(lambda: P.pack(Bd, out=Bp), stream, reps)
    st_ms = timed(lambda: P.pack_spmm(Bd, Bpack=Bp, out=C, scratch=scr), stream, reps)
    spb = spmm_bytes(A.M, A.nnz, R, N, 2)
    wname = workload_name(scale, deg, N, 4, "bf16")
    e = frac_entry(spb, sp_ms, peak)
    e["kernel"] = spmm_kernel(N, 2)
    e["traffic"] = traffic_from_profile(spmm_kernel(N, 2), wname)
    stp = frac_entry(spb + pack_bytes(R, N, 2), st_ms, peak)
    stp["kernel"] = "k_spmm_lean_fused" if fused_step(N, 2) else "pack + " + spmm_kernel(N, 2)
    stp["traffic"] = traffic_from_profile("k_spmm_lean_fused", wname) if fused_step(N, 2) else None
    # The backward with dC stored in BF16 too: dB and dA in one launch over the transposed plan,
    # and the two calls beside it.
    PT = shiro.Plan.create(rp, col, val, A.M, A.K, 4, 4, flags=shiro.SHIRO_PLAN_TRANSPOSE)
    RT = PT.info.packed_rows
    G = torch.randn((A.M, N), device=dev,
                    generator=torch.Generator(device=dev).manual_seed(seed)).to(torch.bfloat16)
    Gp = torch.empty((RT, N), dtype=torch.bfloat16, device=dev)
    dB = torch.empty((A.K, N), dtype=torch.float32, device=dev)
    dA = torch.empty(A.nnz, dtype=torch.float32, device=dev)
    sT = PT.new_scratch(N, torch.bfloat16)
    bwd_ms = timed(lambda: shiro.spmm_backward(P, PT, G, Bp, B=Bd, scratch=sT, dCpack=Gp, dB=dB,
                                               dA=dA), stream, reps)
    two_ms = timed(lambda: (PT.pack_spmm(G, Bpack=Gp, out=dB, scratch=sT),
                            P.sddmm(G, Bp, B=Bd, out=dA)), stream, reps)
    nzc = int(np.count_nonzero(np.bincount(A.col, minlength=A.K)))
    one = frac_entry(bwd_bytes(A.K, A.nnz, RT, N, 2, nzc), bwd_ms, peak)
    one["kernel"] = "k_spmm_lean_bwd"
    one["traffic"] = traffic_from_profile("k_spmm_lean_bwd", wname)
    del PT, G, Gp, dB, dA, sT
    return {"workload": wname, "seed": seed, "M": A.M, "nnz": A.nnz, "packed_rows": R,
            "plan_ms": plan_ms, "spmm": e, "pack": frac_entry(pack_bytes(R, N, 2), pk_ms, peak),
            "step": stp, "step_ms": st_ms, "step_GBps_spmm_bytes": gbps(spb, st_ms),
            "gather_bytes": A.nnz * N * 2, "gather_GBps": gbps(A.nnz * N * 2, sp_ms),
            "gflops": 2.0 * A.nnz * N / (st_ms * 1e-3) / 1e9,
            "backward": {"bwd_one_launch": one, "two_calls_ms": two_ms,
                         "fwd_bwd_ms": st_ms + bwd_ms, "transpose_packed_rows": RT,
                         "what": "dC stored in BF16 (FP32 accumulation, FP32 dB and dA)"}}


def form_gcn(dev, stream, peak, reps, scale=20, deg=16, N=128, F=256, seed=4, tiles=4):
    """GCN layer Y = A_hat (X W) through the public autograd wrapper: the dense product X W is
    torch's (glue, timed on its own), A_hat times it is the library's pack + SpMM, and the backward
    gives dX and dW through torch and dH (A_hat^T dY: pack + SpMM on the transposed plan) and the
    gradient of A_hat's values (SDDMM) through the library.  Loss <G, Y> with a fixed G."""
    import torch
    from paper_2512_20178_gb300 import autograd, shiro, synth
    A = synth.gcn_normalized(scale, deg, seed)
    rp = torch.from_numpy(A.rowptr).to(dev)
    col = torch.from_numpy(A.col).to(dev)
    val = torch.from_numpy(A.val).to(dev).requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S = autograd.SparseMatrix(rp, col, val, A.M, A.K, tiles, tiles)
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    X = torch.from_numpy(synth.dense_normal(A.M, F, seed, std=0.02)).to(dev).requires_grad_(True)
    W = torch.from_numpy(synth.dense_normal(F, N, seed + 1, std=0.02)).to(dev).requires_grad_(True)
    G = torch.from_numpy(synth.dense_normal(A.M, N, seed + 2)).to(dev)

    def fwd():
        return autograd.spmm(S, torch.matmul(X, W))

    def fwd_bwd():
        X.grad = W.grad = val.grad = None
        fwd().backward(G)

    P, PT = S.plan, S.planT
    R, RT = P.info.packed_rows, PT.info.packed_rows
    with torch.no_grad():
        H = torch.matmul(X, W)
        glue_ms = timed(lambda: torch.matmul(X, W, out=H), stream, reps)
        Hp = torch.empty((R, N), device=dev)
        Y = torch.empty((A.M, N), device=dev)
        sc = P.new_scratch(N, torch.float32)
        P.pack(H, out=Hp)
        spmm_ms = timed(lambda: P.spmm(Hp, out=Y, scratch=sc), stream, reps)
        pack_ms = timed(lambda: P.pack(H, out=Hp), stream, reps)
        Gp = torch.empty((RT, N), device=dev)
        dH = torch.empty((A.K, N), device=dev)
        scT = PT.new_scratch(N, torch.float32)
        PT.pack(G, out=Gp)
        dh_spmm = timed(lambda: PT.spmm(Gp, out=dH, scratch=scT), stream, reps)
        dh_pack = timed(lambda: PT.pack(G, out=Gp), stream, reps)
        dA = torch.empty(A.nnz, device=dev)
        da_ms = timed(lambda: P.sddmm(G, Hp, out=dA), stream, reps)
        bwd_ms = timed(lambda: shiro.spmm_backward(P, PT, G, Hp, B=H, scratch=scT, dCpack=Gp,
                                                   dB=dH, dA=dA), stream, reps)
        nzc = int(np.count_nonzero(np.bincount(A.col, minlength=A.K)))
    fwd_ms = timed(fwd, stream, reps)
    ms = timed(fwd_bwd, stream, reps)
    return {"workload": f"gcn_rmat{scale}_deg{deg}_F{F}_N{N}_{tiles}x{tiles}_f32", "M": A.M,
            "nnz": A.nnz, "F": F, "N": N, "plan_ms": plan_ms, "packed_rows": R,
            "packed_rows_transpose": RT, "fwd_bwd_ms": ms, "fwd_ms": fwd_ms,
            "dense_xw_ms": glue_ms,
            "sparse_fwd": {"spmm": frac_entry(spmm_bytes(A.M, A.nnz, R, N, 4), spmm_ms, peak),
                           "pack": frac_entry(pack_bytes(R, N, 4), pack_ms, peak)},
            "sparse_bwd": {"dH_spmm": frac_entry(spmm_bytes(A.K, A.nnz, RT, N, 4), dh_spmm, peak),
                           "dH_pack": frac_entry(pack_bytes(RT, N, 4), dh_pack, peak),
                           "dA_sddmm": frac_entry(sddmm_bytes(A.M, A.nnz, R, N, 4), da_ms, peak),
                           "dH_dA_one_launch": frac_entry(bwd_bytes(A.K, A.nnz, RT, N, 4, nzc),
                                                          bwd_ms, peak)},
            "sparse_ms": spmm_ms + pack_ms + bwd_ms,
            "sparse_fwd_gflops": 2.0 * A.nnz * N / (spmm_ms * 1e-3) / 1e9,
            "what": "fwd + bwd through torch.autograd: X W and the dense gradients in torch (FP32), "
                    "pack + SpMM, dH and dA_hat in the library"}


def form_batch(dev, stream, peak, reps, G=512, N=64, seed=5):
    """Batched form: G graphs as one block-diagonal plan; each step replays one CUDA graph that
    holds the pack and one SpMM launch over every graph.  Timed with the library's default
    schedule and with the schedule the autotuner picks for this batch and N."""
    import torch
    from paper_2512_20178_gb300 import shiro, synth
    gb = synth.batch_graphs(G, seed)
    tens = [(torch.from_numpy(gr.rowptr).to(dev), torch.from_numpy(gr.col).to(dev),
             torch.from_numpy(gr.val).to(dev), gr.M, gr.K) for gr in gb.graphs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P = shiro.Plan.create_batch(tens, opts=shiro.make_opts())
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    M, nnz, R = P.info.M, P.info.nnz, P.info.packed_rows
    Bh = np.concatenate([synth.dense_normal(gr.K, N, 500 + i) for i, gr in enumerate(gb.graphs)])
    Bd = torch.from_numpy(synth.to_bf16_bits(Bh).view(np.int16)).to(dev).view(torch.bfloat16)
    Bp = torch.empty((R, N), dtype=torch.bfloat16, device=dev)
    C = torch.empty((M, N), dtype=torch.float32, device=dev)
    spb = spmm_bytes(M, nnz, R, N, 2)

    def graph_ms():
        scratch = P.new_scratch(N, torch.bfloat16)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                P.pack_spmm(Bd, Bpack=Bp, out=C, scratch=scratch)
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            P.pack_spmm(Bd, Bpack=Bp, out=C, scratch=scratch)
        ms = timed(graph.replay, stream, reps)
        del graph
        return ms

    default_opts = P.info.opts.as_dict()
    default_ms = graph_ms()
    P.pack(Bd, out=Bp)
    tune_scr = torch.empty(64 << 20, dtype=torch.uint8, device=dev)
    tuned = P.autotune(Bp, C=C, scratch=tune_scr, reps=3)
    del tune_scr
    tuned_ms = graph_ms()
    e = frac_entry(spb, tuned_ms, peak)
    e["bytes_note"] = "SpMM bytes over the pack + SpMM graph replay"
    return {"workload": f"batch{G}_rmat_n100-20000_deg4-40_N{N}_bf16_cudagraph", "graphs": G,
            "rows": M, "nnz": nnz, "packed_rows": R, "plan_ms": plan_ms,
            "default": {"schedule": default_opts, "ms": default_ms,
                        "GBps": gbps(spb, default_ms), "frac": gbps(spb, default_ms) / peak},
            "tuned": {"schedule": tuned, **e}, "tuned_speedup": default_ms / tuned_ms,
            "gflops": 2.0 * nnz * N / (tuned_ms * 1e-3) / 1e9}


def form_er(dev, stream, peak, reps, n=4096, N=32, P_=4, seed=1):
    """The small 1D configuration: ER G(4096, 8/4096), N = 32, P = 4 row blocks whose diagonal
    tiles read B in place (LOCAL_DIAG) and whose off-diagonal tiles are packed (L2-resident and
    launch-bound: reported, not roofline-judged)."""
    import torch
    from paper_2512_20178_gb300 import shiro, synth
    A = synth.er(n, 8, seed)
    Bd = torch.from_numpy(synth.dense_normal(n, N, seed)).to(dev)
    rp = torch.from_numpy(A.rowptr).to(dev)
    col = torch.from_numpy(A.col).to(dev)
    val = torch.from_numpy(A.val).to(dev)
    P = shiro.Plan.create(rp, col, val, A.M, A.K, P_, P_, flags=shiro.SHIRO_PLAN_LOCAL_DIAG)
    R = P.info.packed_rows
    Bp = torch.empty((max(R, 1), N), dtype=torch.float32, device=dev)
    C = torch.empty((A.M, N), dtype=torch.float32, device=dev)
    scratch = P.new_scratch(N, torch.float32)
    step = lambda: (P.pack(Bd, out=Bp), P.spmm(Bp, B=Bd, out=C, scratch=scratch))
    ms = timed(step, stream, reps)
    # The same step replayed from a CUDA graph: the device time without the host's per-call cost.
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    ms_graph = timed(graph.replay, stream, reps)
    del graph
    # SpMM reads the packed rows of off-diagonal tiles and, in place, the B rows named by the
    # diagonal tiles' Cols.
    ncols = P.tile_stats()["tile_ncols"].numpy()
    diag_cols = int(sum(ncols[p * P_ + p] for p in range(P_)))
    nbytes = spmm_bytes(A.M, A.nnz, R + diag_cols, N, 4)
    e = frac_entry(nbytes, ms, peak)
    e["note"] = ("two launches of a few microseconds, called from Python: L2-resident and bound by "
                 "the host's per-call cost, not roofline-judged")
    g = frac_entry(nbytes, ms_graph, peak)
    g["note"] = "the same pack + SpMM replayed from a CUDA graph"
    return {"workload": "er4096_deg8_N32_1d_p4_local_diag", "M": A.M, "nnz": A.nnz,
            "packed_rows_offdiag": R, "diag_cols": diag_cols, "step": e, "step_graph": g}


def run_single_form(args, which):
    """--gcn / --batch / --er: one JSON line for that configuration alone."""
    import torch
    import __graft_entry__ as g
    g.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    peak, _ = hbm_peak()
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    clocks.start()
    if which == "gcn":
        r = form_gcn(dev, stream, peak, args.steps, scale=args.scale, deg=args.deg, N=args.N)
        value, unit, hib, ms = r["fwd_bwd_ms"], "ms", False, r["fwd_bwd_ms"]
    elif which == "batch":
        r = form_batch(dev, stream, peak, args.steps, G=args.batch, N=args.N)
        value, unit, hib, ms = r["tuned"]["GBps"], "GB/s", True, r["tuned"]["ms"]
    else:
        r = form_er(dev, stream, peak, max(args.steps, 100))
        value, unit, hib, ms = r["step"]["GBps"], "GB/s", True, r["step"]["ms"]
    clocks.stop()
    print(json.dumps({"metric": METRIC, "value": value, "unit": unit, "n_gpus": 1,
                      "steps": args.steps, "warmup": 3, "ms_per_step": ms,
                      "higher_is_better": hib, "scaling": "weak", "vs_baseline": None,
                      "dtype": "f32", "data": "synthetic (seeded)",
                      "config": {"workload": r["workload"]}, "detail": r,
                      "clocks": clocks.summary()}))


def main():
    args = parse()
    if args.traffic_from:
        if not (args.kernel and args.workload):
            raise SystemExit("--traffic-from needs --kernel and --workload")
        write_traffic_record(args.traffic_from, args.kernel, args.workload, args.command or "")
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.gcn:
        run_single_form(args, "gcn")
    elif args.er:
        run_single_form(args, "er")
    elif args.batch:
        run_single_form(args, "batch")
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
