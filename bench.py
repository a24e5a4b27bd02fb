"""Benchmark of the sparsity-aware SpMM hot path on one GB300 (or N independent replicas).

Workload (default): R-MAT CSR A 2^20 x 2^20, avg degree 16 (a,b,c,d = .57,.19,.19,.05,
duplicates merged), FP32 values U(0,1), dense B 2^20 x 128 FP32 N(0,1), 4x4 logical tiles.
One step = pack the B rows named by every tile's unique columns (Sec. 5.1 stage 3) + SpMM over
the packed rows summed over the tiles of each row block (stage 5).  The plan (stage 1) is built
once per pattern, as in the paper, and timed on its own.

The JSON line reports:
  value     -- algorithmic GB/s of the step: pack 2*R*N*4 + R*4, SpMM (M+1)*8 + nnz*8 + R*N*4 +
               M*N*4 bytes (R = packed rows), over the device time of K steps (CUDA events);
  roofline  -- the SpMM kernel alone: its algorithmic bytes / its mean launch time vs the
               measured HBM copy bandwidth;
  e2e       -- the same bytes over steps that also copy B from pinned host memory and C back;
  cpu_baseline -- the FP64 C oracle on a strided row sample, on this host's cores;
  forms     -- BF16-stored B, the backward (dB = A^T dC, dA by SDDMM) and fwd+bwd time.
Inputs are larger than L2 (B 512 MB, packed B 650 MB, C 512 MB), so no L2 flush is needed.

--impl reference times the FP64 CPU oracle (the reference arm here; the paper ships no kernels).
With N > 1 (torchrun) every rank runs its own replica (weak scaling, no collective on the path).
"""
from __future__ import annotations

import argparse
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

METRIC = "SpMM GB/s (pack + SpMM, algorithmic bytes) vs HBM roofline"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "spmm_rmat20_n128_traffic.json")
KERNEL_SOURCES = ["paper_2512_20178_gb300/csrc/spmm.cu", "paper_2512_20178_gb300/csrc/vec.cuh",
                  "paper_2512_20178_gb300/csrc/internal.cuh",
                  "paper_2512_20178_gb300/csrc/spmm_lean.cuh"]


def spmm_kernel(N, sz):
    """The SpMM kernel the automatic pipeline picks for N columns of sz-byte elements."""
    row = N * sz
    if row in (128, 256, 512):
        return "k_spmm_lean" if (sz == 2 and row == 256) else "k_spmm_lean_dyn"
    if row in (1024, 2048):
        return "k_spmm_lring"
    return "k_spmm"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=20)
    ap.add_argument("--deg", type=int, default=16)
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--tiles", type=int, default=4)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16"],
                    help="storage of B (and of the packed rows); accumulation is FP32 either way")
    ap.add_argument("--er", action="store_true",
                    help="time the small 1D case instead: Erdos-Renyi 4096 x 4096, avg degree 8, "
                         "values U(-1, 1), B 4096 x 32, P = 4 row blocks with local diagonal tiles "
                         "(L2-resident and launch-bound: reported, not roofline-judged)")
    ap.add_argument("--gcn", action="store_true",
                    help="time the GCN layer instead: Y = A_hat (X W), A_hat the symmetric-normalised "
                         "R-MAT 2^scale graph with self loops, X n x 256, W 256 x N, fwd + bwd "
                         "through the autograd wrapper")
    ap.add_argument("--batch", type=int, default=0,
                    help="time the batched form instead: this many R-MAT graphs, n ~ U{100..20000}, "
                         "degree log-uniform [4, 40], B n x N in BF16, one CUDA-graph replay per step")
    return ap.parse_args()


def workload(args):
    from paper_2512_20178_gb300 import synth
    A = synth.rmat(args.scale, args.deg, args.seed)
    B = synth.dense_normal(A.K, args.N, args.seed)
    return A, B


def config(args, A, extra=None):
    c = {"workload": f"rmat{args.scale}_deg{args.deg}_N{args.N}_{args.tiles}x{args.tiles}_{args.dtype}",
         "M": A.M, "K": A.K, "nnz": A.nnz, "N": args.N, "tiles": f"{args.tiles}x{args.tiles}",
         "rmat": [0.57, 0.19, 0.19, 0.05], "seed": args.seed,
         "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas"}
    if extra:
        c.update(extra)
    return c


def step_bytes(M, nnz, R, N, sz):
    spmm = (M + 1) * 8 + nnz * 8 + R * N * sz + M * N * 4
    pack = 2 * R * N * sz + R * 4
    return spmm, pack


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


def traffic_from_profile():
    """DRAM bytes per SpMM launch from the committed ncu summary, if the kernel is unchanged."""
    try:
        rec = json.load(open(PROFILE_TRAFFIC))
    except (OSError, ValueError):
        return None
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if rec.get("kernel_sources_sha256") != h.hexdigest():
        return None
    return rec.get("dram_bytes_per_launch")


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
    sp, pk = step_bytes(S.M, S.nnz, len(src), args.N, 4)
    gbs = (sp + pk) / (t2 - t1) / 1e9
    return {"value": gbs, "unit": "GB/s", "cores": oracle.threads(), "kind": "oracle",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "sample": f"every {stride}th row ({S.M} rows, {S.nnz} nnz), pack + SpMM via packed "
                      f"rows in FP64; plan {t1 - t0:.2f} s not counted",
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
            "data": "synthetic (seeded R-MAT)", "config": config(args, A),
            "cpu_baseline": {k: res[k] for k in ("value", "unit", "cores", "kind", "sample", "cpu_model", "nproc")},
            "e2e": {"value": res["value"], "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


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

    def step():
        P.pack(Bd, out=Bp)
        P.spmm(Bp, out=C, scratch=scratch)

    for _ in range(args.warmup):
        step()
    K = args.steps
    ev_a = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    start.record(stream)
    for k in range(K):
        P.pack(Bd, out=Bp)
        ev_a[k].record(stream)
        P.spmm(Bp, out=C, scratch=scratch)
        ev_b[k].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks.stop()
    ms = start.elapsed_time(end) / K
    launch_ms = sorted(a.elapsed_time(b) for a, b in zip(ev_a, ev_b))
    spmm_ms = sum(launch_ms) / K
    pct = lambda q: launch_ms[min(K - 1, int(q * (K - 1) + 0.5))]
    spmm_stats = {"mean": spmm_ms, "median": pct(0.5), "p10": pct(0.1), "p90": pct(0.9)}
    ms_max = reduce_max(ms, world, dev)
    sp_bytes, pk_bytes = step_bytes(A.M, A.nnz, R, N, sz)
    value = world * (sp_bytes + pk_bytes) / (ms_max * 1e-3) / 1e9
    gflops = world * 2.0 * A.nnz * N / (ms_max * 1e-3) / 1e9

    # End to end through the public API: every step copies its B from pinned host memory and
    # reads its C back into pinned host memory.  Steps are pipelined as a serving loop would run
    # them: step k+1's upload and step k-1's download overlap step k's pack + SpMM (two device
    # buffers each for B and C, one stream per direction).  The serial figure (one stream, no
    # overlap) is reported beside it.
    Bh = Bh.pin_memory()
    Ch = [torch.empty((A.M, N), dtype=torch.float32).pin_memory() for _ in range(2)]
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
        P.pack(Bdd[j], out=Bp)
        P.spmm(Bp, out=Cd[j], scratch=scratch)
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
        step()
        Ch[0].copy_(C, non_blocking=True)
    torch.cuda.synchronize()
    e0.record(stream)
    Ks = max(1, min(K, 30))
    for _ in range(Ks):
        Bd.copy_(Bh, non_blocking=True)
        step()
        Ch[0].copy_(C, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    serial_ms = reduce_max(e0.elapsed_time(e1) / Ks, world, dev)
    e2e = {"value": world * (sp_bytes + pk_bytes) / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": int(Bh.numel() * sz), "d2h_bytes_per_step": int(Ch[0].numel() * 4),
           "ms_per_step": e2e_ms, "pipelined": "upload k+1 / compute k / download k-1",
           "serial_ms_per_step": serial_ms}
    del Bdd, Cd

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    achieved = sp_bytes / (spmm_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": spmm_kernel(args.N, sz), "achieved": achieved, "peak": peak,
                "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_from_profile(), "algorithmic_bytes": sp_bytes,
                "ms_per_launch": spmm_ms, "launch_ms": spmm_stats}

    forms = None
    if not args.no_forms and not bf16:
        forms = measure_forms(args, A, B, P, Bd, Bp, C, scratch, rp, col, val, dev, stream)

    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "storage": args.dtype,
            "data": "synthetic (seeded R-MAT, counter-based SplitMix64)",
            "config": config(args, A, {"packed_rows": R, "plan_ms": plan_ms,
                                       "schedule": P.info.opts.as_dict(), "autotuned": tuned}),
            "gflops": gflops, "spmm_ms": spmm_ms, "pack_ms": ms - spmm_ms,
            "gpu_launches": 2 * K, "roofline": roofline, "e2e": e2e,
            "clocks": clocks.summary()}
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


def measure_forms(args, A, B, P, Bd, Bp, C, scratch, rp, col, val, dev, stream, reps=20):
    """BF16-stored B, backward (dB and dA) and fwd+bwd on the same A, N (device times)."""
    import torch
    from paper_2512_20178_gb300 import shiro, synth
    N = args.N

    def timed(fn):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    R = P.info.packed_rows
    Bh16 = torch.from_numpy(synth.to_bf16_bits(B).view(np.int16)).to(dev).view(torch.bfloat16)
    Bp16 = torch.empty((R, N), dtype=torch.bfloat16, device=dev)
    s16 = P.new_scratch(N, torch.bfloat16)
    bf16_ms = timed(lambda: (P.pack(Bh16, out=Bp16), P.spmm(Bp16, out=C, scratch=s16)))
    sp16, pk16 = step_bytes(A.M, A.nnz, R, N, 2)
    fwd_ms = timed(lambda: (P.pack(Bd, out=Bp), P.spmm(Bp, out=C, scratch=scratch)))
    PT = shiro.Plan.create(rp, col, val, A.M, A.K, args.tiles, args.tiles,
                           flags=shiro.SHIRO_PLAN_TRANSPOSE)
    G = torch.randn((A.M, N), device=dev, generator=torch.Generator(device=dev).manual_seed(5))
    RT = PT.info.packed_rows
    Gp = torch.empty((RT, N), dtype=torch.float32, device=dev)
    dB = torch.empty((A.K, N), dtype=torch.float32, device=dev)
    dA = torch.empty(A.nnz, dtype=torch.float32, device=dev)
    sT = PT.new_scratch(N, torch.float32)
    db_ms = timed(lambda: (PT.pack(G, out=Gp), PT.spmm(Gp, out=dB, scratch=sT)))
    da_ms = timed(lambda: P.sddmm(G, Bp, out=dA))
    sddmm_bytes = A.nnz * 8 + A.M * N * 4 + R * N * 4 + A.nnz * 4
    # N sweep (FP32 B): pack + SpMM and SpMM alone at N = 32 .. 256 on the same plan.
    n_sweep = {}
    for n in (32, 64, 128, 256):
        Bn = torch.from_numpy(synth.dense_normal(A.K, n, 7)).to(dev)
        Bpn = torch.empty((R, n), dtype=torch.float32, device=dev)
        Cn = torch.empty((A.M, n), dtype=torch.float32, device=dev)
        sn = P.new_scratch(n, torch.float32)
        P.pack(Bn, out=Bpn)
        spmm_n = timed(lambda: P.spmm(Bpn, out=Cn, scratch=sn))
        step_n = timed(lambda: (P.pack(Bn, out=Bpn), P.spmm(Bpn, out=Cn, scratch=sn)))
        spb, pkb = step_bytes(A.M, A.nnz, R, n, 4)
        n_sweep[str(n)] = {"spmm_ms": spmm_n, "step_ms": step_n,
                           "spmm_GBps": spb / (spmm_n * 1e-3) / 1e9,
                           "step_GBps": (spb + pkb) / (step_n * 1e-3) / 1e9}
        del Bn, Bpn, Cn, sn
    # Comparator (not on the path): cuSPARSE CSR SpMM through torch.sparse.mm on the unpacked B.
    cus = None
    try:
        At = torch.sparse_csr_tensor(rp.to(torch.int32), col, val, size=(A.M, A.K))
        Cc = torch.sparse.mm(At, Bd)
        cus_ms = timed(lambda: torch.sparse.mm(At, Bd))
        P.pack(Bd, out=Bp)
        P.spmm(Bp, out=C, scratch=scratch)
        torch.cuda.synchronize()
        cus = {"ms": cus_ms, "ours_spmm_ms": timed(lambda: P.spmm(Bp, out=C, scratch=scratch)),
               "ours_step_ms": fwd_ms, "max_abs_diff": float((Cc - C).abs().max()),
               "what": "torch.sparse.mm (cuSPARSE CSR SpMM) on the original B, same A, N"}
        del At, Cc
    except Exception as e:  # the comparator is optional context
        cus = {"unavailable": str(e).splitlines()[0][:200]}
    return {"n_sweep_fp32": n_sweep, "cusparse": cus,"bf16_B": {"ms": bf16_ms, "GBps": (sp16 + pk16) / (bf16_ms * 1e-3) / 1e9,
                       "vs_fp32_speedup": fwd_ms / bf16_ms},
            "fp32_fwd_ms": fwd_ms, "bwd_dB_ms": db_ms, "bwd_dA_ms": da_ms,
            "fwd_bwd_ms": fwd_ms + db_ms + da_ms,
            "sddmm_GBps": sddmm_bytes / (da_ms * 1e-3) / 1e9,
            "transpose_packed_rows": RT}


def run_batch(args):
    """Batched form: G graphs as one block-diagonal plan; each step replays one CUDA graph that
    holds the pack and one persistent SpMM launch over every graph."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2512_20178_gb300 import shiro, synth
    dev = torch.device("cuda", torch.cuda.current_device())
    N = args.N
    gb = synth.batch_graphs(args.batch, 5)
    tens = []
    for gr in gb.graphs:
        tens.append((torch.from_numpy(gr.rowptr).to(dev), torch.from_numpy(gr.col).to(dev),
                     torch.from_numpy(gr.val).to(dev), gr.M, gr.K))
    t0 = time.perf_counter()
    P = shiro.Plan.create_batch(tens, opts=shiro.make_opts(persistent=1))
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    M, nnz, R = P.info.M, P.info.nnz, P.info.packed_rows
    Bh = np.concatenate([synth.dense_normal(gr.K, N, 500 + i) for i, gr in enumerate(gb.graphs)])
    Bd = torch.from_numpy(synth.to_bf16_bits(Bh).view(np.int16)).to(dev).view(torch.bfloat16)
    Bp = torch.empty((R, N), dtype=torch.bfloat16, device=dev)
    C = torch.empty((M, N), dtype=torch.float32, device=dev)
    # Autotuned schedule (group size, chunk size, CTA size, pipeline) for this batch and N.
    P.pack(Bd, out=Bp)
    tune_scr = torch.empty(64 << 20, dtype=torch.uint8, device=dev)
    tuned = P.autotune(Bp, C=C, scratch=tune_scr, reps=3)
    del tune_scr
    scratch = P.new_scratch(N, torch.bfloat16)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            P.pack(Bd, out=Bp)
            P.spmm(Bp, out=C, scratch=scratch)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        P.pack(Bd, out=Bp)
        P.spmm(Bp, out=C, scratch=scratch)
    for _ in range(args.warmup):
        graph.replay()
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(args.steps):
        graph.replay()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    sp, pk = step_bytes(M, nnz, R, N, 2)
    print(json.dumps({
        "metric": METRIC, "value": (sp + pk) / (ms * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "storage": "bf16",
        "data": "synthetic (seeded R-MAT graphs)",
        "config": {"workload": f"batch{args.batch}_rmat_n100-20000_deg4-40_N{N}_bf16_cudagraph",
                   "graphs": args.batch, "rows": M, "nnz": nnz, "packed_rows": R, "N": N,
                   "plan_ms": plan_ms, "schedule": P.info.opts.as_dict(), "autotuned": True},
        "gflops": 2.0 * nnz * N / (ms * 1e-3) / 1e9, "gpu_launches": 2 * args.steps}))


def run_er(args):
    """The small 1D configuration: ER G(4096, 8/4096), N = 32, P = 4 row blocks whose diagonal
    tiles read B in place (LOCAL_DIAG) and whose off-diagonal tiles are packed."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2512_20178_gb300 import shiro, synth
    dev = torch.device("cuda", torch.cuda.current_device())
    n, N, P_ = 4096, 32, 4
    A = synth.er(n, 8, 1)
    Bd = torch.from_numpy(synth.dense_normal(n, N, 1)).to(dev)
    rp = torch.from_numpy(A.rowptr).to(dev)
    col = torch.from_numpy(A.col).to(dev)
    val = torch.from_numpy(A.val).to(dev)
    P = shiro.Plan.create(rp, col, val, A.M, A.K, P_, P_, flags=shiro.SHIRO_PLAN_LOCAL_DIAG)
    R = P.info.packed_rows
    Bp = torch.empty((max(R, 1), N), dtype=torch.float32, device=dev)
    C = torch.empty((A.M, N), dtype=torch.float32, device=dev)
    scratch = P.new_scratch(N, torch.float32)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        P.pack(Bd, out=Bp)
        P.spmm(Bp, B=Bd, out=C, scratch=scratch)
    K = max(args.steps, 100)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(K):
        P.pack(Bd, out=Bp)
        P.spmm(Bp, B=Bd, out=C, scratch=scratch)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / K
    # Bytes: SpMM reads the packed rows of off-diagonal tiles and, in place, the B rows named by
    # the diagonal tiles' Cols.
    ncols = P.tile_stats()["tile_ncols"].numpy()
    diag_cols = int(sum(ncols[p * P_ + p] for p in range(P_)))
    sp, pk = step_bytes(A.M, A.nnz, R + diag_cols, N, 4)
    pk = 2 * R * N * 4 + R * 4
    print(json.dumps({
        "metric": METRIC, "value": (sp + pk) / (ms * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": 1,
        "steps": K, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "storage": "f32",
        "data": "synthetic (seeded Erdos-Renyi)",
        "config": {"workload": "er4096_deg8_N32_1d_p4_local_diag", "M": A.M, "nnz": A.nnz,
                   "N": N, "packed_rows_offdiag": R, "diag_cols": diag_cols,
                   "l2": "L2-resident (launch-bound)"},
        "note": "two launches per step of a few microseconds each: reported, not roofline-judged",
        "gpu_launches": 2 * K}))


def run_gcn(args):
    """GCN layer Y = A_hat (X W) through the public autograd wrapper: the dense product X W is
    torch's (glue, timed on its own), A_hat times it is the library's pack + SpMM, and the backward
    gives dX and dW through torch and dH (A_hat^T dY: pack + SpMM on the transposed plan) and the
    gradient of A_hat's values (SDDMM) through the library.  Loss <G, Y> with a fixed G."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2512_20178_gb300 import autograd, synth
    dev = torch.device("cuda", torch.cuda.current_device())
    seed = 4
    A = synth.gcn_normalized(args.scale, args.deg, seed)
    F, N = 256, args.N
    rp = torch.from_numpy(A.rowptr).to(dev)
    col = torch.from_numpy(A.col).to(dev)
    val = torch.from_numpy(A.val).to(dev).requires_grad_(True)
    t0 = time.perf_counter()
    S = autograd.SparseMatrix(rp, col, val, A.M, A.K, args.tiles, args.tiles)
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    X = torch.from_numpy(synth.dense_normal(A.M, F, seed, std=0.02)).to(dev).requires_grad_(True)
    W = torch.from_numpy(synth.dense_normal(F, N, seed + 1, std=0.02)).to(dev).requires_grad_(True)
    G = torch.from_numpy(synth.dense_normal(A.M, N, seed + 2)).to(dev)
    stream = torch.cuda.current_stream()

    def fwd():
        return autograd.spmm(S, torch.matmul(X, W))

    def fwd_bwd():
        X.grad = W.grad = val.grad = None
        fwd().backward(G)

    def timed(fn, k):
        for _ in range(args.warmup):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    with torch.no_grad():
        H = torch.matmul(X, W)
        glue_ms = timed(lambda: torch.matmul(X, W, out=H), args.steps)
        sparse_fwd_ms = timed(lambda: autograd.spmm(S, H), args.steps)
    fwd_ms = timed(fwd, args.steps)
    ms = timed(fwd_bwd, args.steps)
    print(json.dumps({
        "metric": "GCN layer fwd+bwd ms", "value": ms, "unit": "ms", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "storage": "f32",
        "data": "synthetic (seeded R-MAT, symmetrised, self loops, 1/sqrt(d_i d_j))",
        "config": {"workload": f"gcn_rmat{args.scale}_deg{args.deg}_F{F}_N{N}_{args.tiles}x{args.tiles}",
                   "M": A.M, "nnz": A.nnz, "F": F, "N": N, "plan_ms": plan_ms,
                   "packed_rows": S.plan.info.packed_rows,
                   "packed_rows_transpose": S.planT.info.packed_rows},
        "fwd_ms": fwd_ms, "dense_xw_ms": glue_ms, "sparse_fwd_ms": sparse_fwd_ms,
        "sparse_fwd_gflops": 2.0 * A.nnz * N / (sparse_fwd_ms * 1e-3) / 1e9}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.gcn:
        run_gcn(args)
    elif args.er:
        run_er(args)
    elif args.batch:
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
