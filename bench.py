"""Benchmark: RS(10,4) Cauchy encode over 256 stripes x 10 x 1 MiB on one GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload encode|batched|served|codes] [--executor auto|interp|compiled|dense]

One step = one pass of the hot path over one batch: a single
ec_encode_strided() launch over the 256 stripes (2.5 GiB in, 1 GiB out;
inputs larger than L2, so no flush is needed between steps).  `value` is
GB/s (1e9 B) of input data, whole job; `e2e` is the same metric through the
C ABI with the inputs in pinned host memory and the host<->device copies
inside the timed region.  Prints one JSON line.  On one GPU the default run
adds, as keys of the same line: `decode` (RS(10,4) decode of 256 stripes,
erasure sets uniform over all 1470 patterns, one batch run, against one
launch per stripe), `batched` (8192 mixed-code stripes in one batch run
replayed as a CUDA graph, against one launch per stripe) and `served`
(Poisson request streams through the continuous-batching server at 20k and
100k requests/s, p50/p99 latency, against a one-request-at-a-time server);
each with its bit-exact status against the oracle.

With --impl reference the CPU oracle (test infrastructure, plain C) is
timed on this host's cores on a bounded sample of the same workload.
Under torchrun every rank encodes its own 256 stripes (weak scaling, no
collective on the data path); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

K_DATA, M_PAR, BLOCK, N_STRIPES = 10, 4, 1 << 20, 256
ENCODE_WORKLOAD_ID = 2       # seed namespace of the encode inputs
WORKLOAD = "RS(10,4) Cauchy GF(2^8)/0x11d encode, 256 stripes x 10 x 1 MiB"
METRIC = "RS(10,4) encode/decode GB/s & % HBM peak; batched vs plain; served p50/p99"
DECODE_WORKLOAD_ID = 3       # seed namespace of the decode inputs


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="encode", choices=["encode", "batched", "served", "codes"])
    ap.add_argument("--matrix", default="cauchy", choices=["cauchy", "cauchy_min", "power"],
                    help="coding matrix (default: Cauchy)")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-rate", type=float, default=20000.0)
    ap.add_argument("--serve-rates", default="",
                    help="comma-separated arrival rates (req/s) of a served load sweep")
    ap.add_argument("--serve-obj", default="4096,16777216",
                    help="MIN,MAX object bytes of the served requests (log-uniform)")
    ap.add_argument("--no-batched", action="store_true",
                    help="default run: skip the batched (mixed-code) leg")
    ap.add_argument("--no-served", action="store_true",
                    help="default run: skip the served leg")
    ap.add_argument("--serve-idle-spin-us", type=int, default=0,
                    help="scheduler polling window before it sleeps (0 = library default "
                         "1000 us, -1 = sleep at once)")
    ap.add_argument("--batched-stripes", type=int, default=8192)
    ap.add_argument("--executor", default="auto", choices=["auto", "interp", "compiled", "dense"])
    ap.add_argument("--opt", default="xorrepair", choices=["raw", "repair", "xorrepair", "triple"],
                    help="optimiser level of the encoding program")
    ap.add_argument("--max-temps", type=int, default=-2,
                    help="RePair temporaries budget (-1 = unlimited, -2 = automatic)")
    ap.add_argument("--stripes", type=int, default=N_STRIPES,
                    help="stripes per step (profiling runs use fewer)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-decode", action="store_true")
    ap.add_argument("--no-dense", action="store_true",
                    help="skip the dense executor's encode (the tier without a compiled kernel)")
    ap.add_argument("--decode-stripes", type=int, default=N_STRIPES,
                    help="stripes of the decode measurement")
    ap.add_argument("--decode-patterns", type=int, default=0,
                    help="0: erasure sets uniform over all patterns; N > 0: the stripes cycle "
                         "through N distinct sets of m erasures (profiling program diversity)")
    ap.add_argument("--decode-erasures", default="",
                    help="comma-separated block ids erased in every decode stripe (e.g. 2,4,5,6, "
                         "the paper's P_dec)")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner")
    ap.add_argument("--decode-launch", default="",
                    help="THREADS,REG_BUDGET launch shape of the decode plan (default: the "
                         "plan's default shape)")
    ap.add_argument("--stream-temps", type=int, default=0,
                    help="codes with more than 12 data blocks: XorRePair temporals per input "
                         "window of the two-level program (0 = automatic, -1 = none)")
    ap.add_argument("--codes", default="",
                    help="--workload codes: comma-separated KxM list in place of the paper's "
                         "RS(8..10, 2..4), e.g. 16x4,20x4,32x4")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, dist, device) -> float:
    """Largest value over all ranks (time of the slowest rank); identity
    without a process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbps(per_rank_bytes_per_step: int, world: int, steps: int, ms_total: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank processes its own stripes)."""
    return world * per_rank_bytes_per_step * steps / (ms_total / 1e3) / 1e9


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ cpu baseline

def oracle_sample_gbs(n_threads: int, stripes_per_thread: int = 1, decode: bool = False):
    """Time the oracle on whole stripes of the headline workloads on host
    threads: encode of C2 stripes (10 x 1 MiB), or decode of C3-shaped
    stripes (10 x 1 MiB survivors, 4 erasures, one pattern per stripe)."""
    import oracle
    from paper_2108_02692_gb300 import synth

    P = oracle.cauchy(K_DATA, M_PAR)
    n = n_threads * stripes_per_thread
    if decode:
        pats = [p for p in synth.decode_patterns(K_DATA, M_PAR, 4 * n) if len(p) == M_PAR][:n]
        work = []
        for s, er in enumerate(pats):
            avail = [None if i in er else synth.block_bytes(DECODE_WORKLOAD_ID, s, i, BLOCK)
                     for i in range(K_DATA + M_PAR)]
            work.append((list(er), avail))
        fn = lambda w: oracle.decode(P, w[0], w[1])
    else:
        work = [[synth.block_bytes(ENCODE_WORKLOAD_ID, s, j, BLOCK) for j in range(K_DATA)]
                for s in range(n)]
        fn = lambda d: oracle.encode(P, d)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=n_threads) as ex:
        list(ex.map(fn, work))
    dt = time.perf_counter() - t0
    return n * K_DATA * BLOCK / dt / 1e9, dt, n


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline_obj():
    """The oracle on this host: encode over all cores (the reported value),
    encode on one core, and decode over all cores."""
    cores = os.cpu_count() or 1
    gbs, dt, n = oracle_sample_gbs(cores, 2)
    g1, dt1, _ = oracle_sample_gbs(1, 1)
    gd, dtd, nd = oracle_sample_gbs(cores, 1, decode=True)
    return {"value": round(gbs, 5), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"encode of {n} of the 256 stripes (10 x 1 MiB each), two per host thread, "
                      f"{dt:.2f} s wall ({dt * cores:.1f} s of CPU work)",
            "cpu_model": cpu_model(),
            "single_thread": {"value": round(g1, 5), "unit": "GB/s",
                              "sample": f"encode of 1 stripe on 1 thread, {dt1:.2f} s"},
            "decode": {"value": round(gd, 5), "unit": "GB/s",
                       "sample": f"decode of {nd} stripes (10 x 1 MiB survivors, 4 erasures), one "
                                 f"per host thread, {dtd:.2f} s wall"}}


# Sources that determine each kernel kind's code (the planner's programs,
# the shared pipeline and the kernel body).
KERNEL_SOURCES = {
    "compiled": ("tile_pipeline.cuh", "jit.cc", "slp.cc", "plan.cc"),
    "interp": ("tile_pipeline.cuh", "executor.cu", "slp.cc", "plan.cc"),
    "dense": ("tile_pipeline.cuh", "executor.cu", "plan.cc"),
}


def kernel_source_hash(kind: str = "compiled") -> str:
    """Fingerprint of the code (comments and blank lines removed) of the
    sources that determine a kernel kind."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kind]:
        text = open(os.path.join(ROOT, "paper_2108_02692_gb300", "csrc", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        lines = [re.sub(r"(^|\s)//.*$", "", ln).rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()[:16]


def traffic_from_profiles(kind: str):
    """dram bytes per launch recorded by an ncu capture of the same kernel
    sources (profiles/*.md line 'traffic_per_launch: <bytes> source_hash:
    <hash> kind: <kind>'); null when the kernel changed since."""
    want = kernel_source_hash(kind)
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    pat = re.compile(r"traffic_per_launch:\s*(\d+)\s+source_hash:\s*([0-9a-f]+)\s+kind:\s*(\w+)")
    for f in sorted(os.listdir(pdir)):
        try:
            for line in open(os.path.join(pdir, f)):
                mm = pat.search(line)
                if mm and mm.group(2) == want and mm.group(3) == kind:
                    return int(mm.group(1))
        except Exception:
            pass
    return None


# ------------------------------------------------------------------ ours

def run_ours(args):
    import torch
    import paper_2108_02692_gb300 as xo
    from paper_2108_02692_gb300 import synth

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    executor = {"auto": xo.EC_EXEC_AUTO, "interp": xo.EC_EXEC_INTERP,
                "compiled": xo.EC_EXEC_COMPILED, "dense": xo.EC_EXEC_DENSE}[args.executor]
    k, m, B, n = K_DATA, M_PAR, BLOCK, args.stripes
    S = B // 8
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    opt = {"raw": xo.EC_OPT_RAW, "repair": xo.EC_OPT_REPAIR,
           "xorrepair": xo.EC_OPT_XORREPAIR, "triple": xo.EC_OPT_TRIPLE}[args.opt]
    plan = xo.ec_plan_create_ex(k, m, matrix_kind=matrix_kind(xo, args.matrix), executor=executor,
                                opt_level=opt, max_temps=args.max_temps)
    data = torch.empty((n, k, B), dtype=torch.uint8, device="cuda")
    par = torch.empty((n, m, B), dtype=torch.uint8, device="cuda")
    for s in range(n):
        for j in range(k):
            xo.ec_synth_fill(data[s, j].data_ptr(), B, synth.block_seed(ENCODE_WORKLOAD_ID, s, j), 0, sp)
    stream.synchronize()
    tune = None
    if not args.no_tune and executor in (xo.EC_EXEC_AUTO, xo.EC_EXEC_COMPILED) and args.max_temps == -2 and args.opt == "xorrepair":
        tune = xo.ec_plan_autotune(plan, B, 32, sp)

    def step(st):
        xo.ec_encode_strided(plan, data.data_ptr(), k * B, B, par.data_ptr(), m * B, B, n, B, st)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(sp)
    stream.synchronize()
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    with torch.cuda.stream(stream):
        t_start.record(stream)
        for i in range(K):
            ev[i][0].record(stream)
            step(sp)
            ev[i][1].record(stream)
        t_end.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms_total = t_start.elapsed_time(t_end)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    ms_total = max_over_ranks(ms_total, dist, "cuda")

    # sampled bit-exact check of the timed output against the oracle
    parity_status = "not-checked"
    if rank == 0:
        import numpy as np
        import oracle
        P = oracle_matrix(oracle, args.matrix, k, m)
        ok = True
        rng = np.random.default_rng(7)
        for s in rng.choice(n, 4, replace=False):
            w0 = int(rng.integers(0, (S - 64) // 16)) * 16
            mini = [synth.strip_slice(ENCODE_WORKLOAD_ID, int(s), j, B, w0, 64) for j in range(k)]
            ref = oracle.encode(P, mini)
            got = par[int(s)].view(m, 8, S)[:, :, w0:w0 + 64].cpu().numpy()
            ok &= all(np.array_equal(got[i].reshape(-1), ref[i]) for i in range(m))
        # and one whole stripe (10 x 1 MiB in, 4 x 1 MiB out)
        s = int(rng.integers(0, n))
        full = [synth.block_bytes(ENCODE_WORKLOAD_ID, s, j, B) for j in range(k)]
        ref = oracle.encode(P, full)
        got = par[s].cpu().numpy()
        ok &= all(np.array_equal(got[i], ref[i]) for i in range(m))
        parity_status = ("bit-exact on sampled windows of 4 stripes and on all of stripe "
                         f"{s}") if ok else "MISMATCH"

    info = xo.ec_plan_info(plan)
    in_bytes = n * k * B
    moved = (k + m) * B * n
    value = whole_job_gbps(in_bytes, ws, K, ms_total)
    peak, peak_kind = measured_peaks()
    mean_launch_ms = statistics.mean(launch_ms)
    achieved = moved / (mean_launch_ms / 1e3) / 1e9
    if args.executor in ("interp", "dense"):
        kind = args.executor
    else:
        kind = "compiled" if info["compiled"] else "dense"

    e2e = None
    if not args.no_e2e and n == N_STRIPES:
        e2e = run_e2e(args, xo, plan, data, par, stream, torch)
    dense = None
    if not args.no_dense and n == N_STRIPES and kind == "compiled":
        dense = run_dense(args, xo, data, par, stream, torch, peak)
    decode = None
    if not args.no_decode and (n == N_STRIPES or args.decode_patterns > 0 or args.decode_erasures
                               or args.decode_stripes != N_STRIPES):
        del data, par
        torch.cuda.empty_cache()
        decode = run_decode(args, xo, torch, stream, peak)
    batched = served = None
    if ws == 1 and n == N_STRIPES and not args.no_batched:
        torch.cuda.empty_cache()
        batched = batched_leg(args)
    if ws == 1 and n == N_STRIPES and not args.no_served:
        torch.cuda.empty_cache()
        served = served_leg(args, [args.serve_rate, 100000.0])
    status = xo.ec_device_status()

    out = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "GB/s",
        "n_gpus": ws,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": round(ms_total / K, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic (SplitMix64 bytes generated on the device)",
        "config": {"workload": WORKLOAD if n == N_STRIPES else WORKLOAD.replace("256", str(n)),
                   "k": k, "m": m, "n_stripes": n, "block_bytes": B,
                   "matrix": args.matrix, "executor": kind, "opt": args.opt,
                   "max_temps": args.max_temps, "autotune": tune,
                   "l2": "inputs (2.5 GiB) larger than L2 (129 MB); no flush",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "bytes_per_launch": moved,
                     "traffic": traffic_from_profiles(kind)},
        "e2e": e2e,
        "decode": decode,
        "dense": dense,
        "batched": batched,
        "served": served,
        "gpu_launches": K,
        "clocks": clk,
        "parity": parity_status,
        "device_status": status,
        "program": {"slots": info["slots"], "stmts": info["stmts"],
                    "xors": info["fused"]["xors"], "mem": info["fused"]["mem"],
                    "raw_xors": info["raw"]["xors"], "regs": info["regs"],
                    "temps": info["temps"], "max_live": info["max_live"]},
    }
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline_obj()
    xo.ec_plan_destroy(plan)
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def run_decode(args, xo, torch, stream, peak):
    """RS(10,4) decode, 256 stripes x 1 MiB blocks, one erasure set per stripe
    drawn uniformly from all C(14,<=4) = 1470 patterns.  The survivors are
    synthetic bytes (the decode map is linear; validity of the codeword does
    not change the work).  Timed: one ec_batch_run over the 256 stripes,
    against a loop of plain single-stripe ec_decode calls on the same data."""
    import numpy as np
    import oracle
    from paper_2108_02692_gb300 import synth

    k, m, B, n = K_DATA, M_PAR, BLOCK, args.decode_stripes
    S = B // 8
    sp = stream.cuda_stream
    if args.decode_erasures:
        fixed = tuple(int(x) for x in args.decode_erasures.split(","))
        pats = [fixed] * n
        what = f"RS(10,4) decode, {n} stripes x 1 MiB, erased blocks {list(fixed)} in every stripe"
    elif args.decode_patterns > 0:
        full = list(dict.fromkeys(p for p in synth.decode_patterns(k, m, 4096) if len(p) == m))
        pats = [full[s % min(args.decode_patterns, len(full))] for s in range(n)]
        what = (f"RS(10,4) decode, {n} stripes x 1 MiB, {m} erasures per stripe, cycling "
                f"through {min(args.decode_patterns, len(full))} erasure sets")
    else:
        pats = synth.decode_patterns(k, m, n)
        what = (f"RS(10,4) decode, {n} stripes x 1 MiB, erasure sets uniform over all "
                "1470 patterns of 1-4 blocks")
    surv = torch.empty((n, k, B), dtype=torch.uint8, device="cuda")
    outs = torch.zeros((n, m, B), dtype=torch.uint8, device="cuda")
    for s in range(n):
        for j in range(k):
            xo.ec_synth_fill(surv[s, j].data_ptr(), B, synth.block_seed(DECODE_WORKLOAD_ID, s, j),
                             0, sp)
    stream.synchronize()
    plan = xo.ec_plan_create_ex(k, m, matrix_kind=matrix_kind(xo, args.matrix))
    tune = None
    if args.decode_launch:
        th, rb = (int(x) for x in args.decode_launch.split(","))
        xo.ec_plan_set_launch(plan, th, rb)
    elif not args.no_tune:
        # the plan's launch shape from the autotuner (timed on the encoder);
        # the decoders and their batch modules are built with it
        tune = xo.ec_plan_autotune(plan, B, 32, sp)
    jobs, calls = [], []
    for s, er in enumerate(pats):
        ids = [i for i in range(k + m) if i not in er][:k]
        ptrs = [None] * (k + m)
        for j, bid in enumerate(ids):
            ptrs[bid] = surv[s, j].data_ptr()
        o = [outs[s, i].data_ptr() for i in range(len(er))]
        jobs.append({"plan": plan, "op": xo.EC_OP_DECODE, "erasures": list(er), "blocks": ptrs,
                     "out": o, "block_bytes": B})
        calls.append((list(er), ptrs, o))
    t0 = time.perf_counter()
    batch = xo.ec_batch_create(jobs)
    prep_s = time.perf_counter() - t0
    binfo = xo.ec_batch_info_get(batch)
    moved = sum((k + len(er)) * B for er in pats)
    in_bytes = n * k * B

    def timed(fn, reps):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    with torch.cuda.stream(stream):
        for _ in range(max(1, args.warmup)):
            xo.ec_batch_run(batch, sp)
        ms_batch = timed(lambda: xo.ec_batch_run(batch, sp), max(3, args.steps))
    # sampled bit-exact check against the oracle's decode map
    P = oracle_matrix(oracle, args.matrix, k, m)
    rng = np.random.default_rng(11)
    ok = True
    for s in rng.choice(n, min(n, 6), replace=False):
        er = list(pats[int(s)])
        R = oracle.decode_matrix(P, er)
        w0 = int(rng.integers(0, (S - 32) // 16)) * 16
        mini = [synth.strip_slice(DECODE_WORKLOAD_ID, int(s), j, B, w0, 32) for j in range(k)]
        ref = oracle.apply(R, mini)
        got = outs[int(s), :len(er)].view(len(er), 8, S)[:, :, w0:w0 + 32].cpu().numpy()
        ok &= all(np.array_equal(got[i].reshape(-1), ref[i]) for i in range(len(er)))
    # one whole stripe of each erasure count (1..4 blocks lost)
    whole = []
    for ne in range(1, m + 1):
        cand = [s for s, er in enumerate(pats) if len(er) == ne]
        if not cand:
            continue
        s = cand[0]
        er = list(pats[s])
        R = oracle.decode_matrix(P, er)
        full = [synth.block_bytes(DECODE_WORKLOAD_ID, s, j, B) for j in range(k)]
        ref = oracle.apply(R, full)
        got = outs[s, :len(er)].cpu().numpy()
        ok &= all(np.array_equal(got[i], ref[i]) for i in range(len(er)))
        whole.append(s)
    # plain single-stripe launches (compiled tier, kernels compiled beforehand)
    t0 = time.perf_counter()
    xo.ec_plan_compile(plan, sorted(set(pats)))
    compile_s = time.perf_counter() - t0

    def plain():
        for er, ptrs, o in calls:
            xo.ec_decode(plan, er, ptrs, o, B, sp)

    with torch.cuda.stream(stream):
        plain()
        ms_plain = timed(plain, 2)
    xo.ec_batch_destroy(batch)
    xo.ec_plan_destroy(plan)
    del surv, outs
    torch.cuda.empty_cache()
    return {
        "workload": what,
        "value": round(in_bytes / (ms_batch / 1e3) / 1e9, 2), "unit": "GB/s",
        "ms_per_step": round(ms_batch, 4),
        "roofline": {"bound": "hbm", "achieved": round(moved / (ms_batch / 1e3) / 1e9, 1),
                     "peak": peak, "unit": "GB/s",
                     "frac": round(moved / (ms_batch / 1e3) / 1e9 / peak, 4),
                     "bytes_per_step": moved},
        "plain": {"value": round(in_bytes / (ms_plain / 1e3) / 1e9, 2), "unit": "GB/s",
                  "ms_per_step": round(ms_plain, 3), "launches_per_step": n},
        "batched_over_plain": round(ms_plain / ms_batch, 2),
        "distinct_patterns": len(set(pats)),
        "launches_per_step": binfo["launches"],
        "autotune": tune,
        "prepare_s": round(prep_s, 2), "plain_compile_s": round(compile_s, 2),
        "parity": (f"bit-exact on sampled windows of 6 stripes and on all of stripes {whole} "
                   "(one per erasure count)") if ok else "MISMATCH",
    }


def matrix_kind(xo, name):
    return {"cauchy": xo.EC_MATRIX_CAUCHY, "cauchy_min": xo.EC_MATRIX_CAUCHY_MIN,
            "power": xo.EC_MATRIX_POWER}[name]


def oracle_matrix(oracle, name, k, m):
    return {"cauchy": oracle.cauchy, "cauchy_min": oracle.cauchy_min,
            "power": oracle.power}[name](k, m)


CODES = [(8, 2), (9, 2), (10, 2), (8, 3), (9, 3), (10, 3), (8, 4), (9, 4), (10, 4)]


def run_codes(args):
    """The codes of the paper's throughput comparison (Sec. 7.6): RS(d,p)
    for d = 8..10 and p = 2..4, each with the Cauchy matrix and the scaled
    Cauchy matrix.  Per code: encode of 256 stripes x d x 1 MiB in one
    launch, and decode of the same stripes with data blocks 0..p-1 erased
    (every parity block is a survivor) in one batched launch; XOR counts of
    the programs; sampled bit-exact check against the oracle."""
    import numpy as np
    import torch
    import oracle
    import paper_2108_02692_gb300 as xo
    from paper_2108_02692_gb300 import synth

    torch.cuda.set_device(0)
    B, n = BLOCK, args.stripes
    S = B // 8
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    peak, _ = measured_peaks()
    reps = max(3, args.steps)

    def timed(fn):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for _ in range(max(1, args.warmup)):
                fn()
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(reps):
                fn()
            ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    codes = [tuple(int(x) for x in c.split("x")) for c in args.codes.split(",")] if args.codes \
        else CODES
    rows, all_ok = [], True
    for (k, m) in codes:
        data = torch.empty((n, k, B), dtype=torch.uint8, device="cuda")
        par = torch.empty((n, m, B), dtype=torch.uint8, device="cuda")
        rec = torch.empty((n, m, B), dtype=torch.uint8, device="cuda")
        for s in range(n):
            for j in range(k):
                xo.ec_synth_fill(data[s, j].data_ptr(), B, synth.block_seed(6, s, j), 0, sp)
        er = list(range(m))
        for name in ("cauchy", "cauchy_min"):
            plan = xo.ec_plan_create_ex(k, m, matrix_kind=matrix_kind(xo, name),
                                        stream_temps=args.stream_temps)
            ms_enc = timed(lambda: xo.ec_encode_strided(plan, data.data_ptr(), k * B, B, par.data_ptr(),
                                                        m * B, B, n, B, sp))
            jobs = []
            for s in range(n):
                blocks = [None] * m + [data[s, j].data_ptr() for j in range(m, k)] + \
                         [par[s, i].data_ptr() for i in range(m)]
                jobs.append({"plan": plan, "op": xo.EC_OP_DECODE, "erasures": er, "blocks": blocks,
                             "out": [rec[s, i].data_ptr() for i in range(m)], "block_bytes": B})
            batch = xo.ec_batch_create(jobs)
            ms_dec = timed(lambda: xo.ec_batch_run(batch, sp))
            xo.ec_batch_destroy(batch)
            # sampled windows: parity against the oracle, recovered blocks
            # against the original data
            P = oracle_matrix(oracle, name, k, m)
            rng = np.random.default_rng(17)
            ok = True
            for s in rng.choice(n, 3, replace=False):
                w0 = int(rng.integers(0, (S - 64) // 16)) * 16
                mini = [synth.strip_slice(6, int(s), j, B, w0, 64) for j in range(k)]
                ref = oracle.encode(P, mini)
                got = par[int(s)].view(m, 8, S)[:, :, w0:w0 + 64].cpu().numpy()
                ok &= all(np.array_equal(got[i].reshape(-1), ref[i]) for i in range(m))
                got = rec[int(s)].view(m, 8, S)[:, :, w0:w0 + 64].cpu().numpy()
                ok &= all(np.array_equal(got[i].reshape(-1), mini[i]) for i in range(m))
            all_ok &= ok
            ie, idd = xo.ec_plan_info(plan), xo.ec_plan_info(plan, er)
            rows.append({
                "code": f"RS({k},{m})", "matrix": name,
                "encode_GBps": round(n * k * B / (ms_enc / 1e3) / 1e9, 1),
                "encode_frac": round(n * (k + m) * B / (ms_enc / 1e3) / 1e9 / peak, 4),
                "decode_GBps": round(n * k * B / (ms_dec / 1e3) / 1e9, 1),
                "decode_frac": round(n * (k + m) * B / (ms_dec / 1e3) / 1e9 / peak, 4),
                "enc_xors_raw": ie["raw"]["xors"], "enc_xors_fused": ie["fused"]["xors"],
                "dec_xors_raw": idd["raw"]["xors"], "dec_xors_fused": idd["fused"]["xors"],
                "enc_lop3": ie["lop3"], "enc_compiled": ie["compiled"], "enc_regs": ie["regs"],
                "enc_threads": ie["threads"], "enc_window_temps": ie["window_temps"],
                "parity": "bit-exact on sampled windows" if ok else "MISMATCH"})
            xo.ec_plan_destroy(plan)
        del data, par, rec
        torch.cuda.empty_cache()
    head = next((r for r in rows if r["code"] == "RS(10,4)" and r["matrix"] == "cauchy"), rows[0])
    print(json.dumps({
        "metric": METRIC, "value": head["encode_GBps"], "unit": "GB/s", "n_gpus": 1,
        "steps": reps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (SplitMix64 bytes generated on the device)",
        "config": {"workload": f"codes {', '.join(f'RS({k},{m})' for k, m in codes)}, {n} stripes "
                               "x d x 1 MiB, Cauchy and scaled Cauchy; decode erases data blocks "
                               "0..p-1",
                   "l2": "inputs larger than L2 (129 MB); no flush"},
        "codes": rows,
        "parity": "bit-exact on sampled windows" if all_ok else "MISMATCH",
        "device_status": xo.ec_device_status(),
    }))


def percentile(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs), q)) if xs else None


def serve_stream(xo, torch, reqs, plans, data_arena, out_arena, max_batch, slots, warm_s,
                 budget=32 << 30, idle_spin_us=0, check=0):
    """Replay a request trace against a server; returns latencies (µs) of the
    requests that arrived after warm_s, throughput and server stats.  With
    check > 0 the last `check` requests are verified against the oracle
    (sampled windows) right after the run."""
    import numpy as np
    rng = np.random.default_rng(13)
    dbase, dsize = data_arena.data_ptr(), data_arena.numel()
    obase, osize = out_arena.data_ptr(), out_arena.numel()
    jobs, in_bytes, where = [], [], []
    opos = 0
    for r in reqs:
        k, m, B = r["k"], r["m"], r["B"]
        nblk = k + m
        off = int(rng.integers(0, (dsize - nblk * B) // 128)) * 128
        blocks = [dbase + off + j * B for j in range(nblk)]
        nout = len(r["erasures"]) if r["erasures"] else m
        if opos + nout * B > osize:
            opos = 0
        outs = [obase + opos + i * B for i in range(nout)]
        opos += nout * B
        if r["erasures"]:
            er = list(r["erasures"])
            jobs.append({"plan": plans[(k, m)], "op": xo.EC_OP_DECODE, "erasures": er,
                         "blocks": [None if i in er else blocks[i] for i in range(nblk)],
                         "out": outs, "block_bytes": B})
        else:
            jobs.append({"plan": plans[(k, m)], "op": xo.EC_OP_ENCODE, "blocks": blocks[:k],
                         "out": outs, "block_bytes": B})
        in_bytes.append(k * B)
        where.append((blocks, outs))
    arr, keep = xo.make_jobs(jobs)
    server = xo.ec_server_create(hbm_budget=budget, max_batch=max_batch, slots=slots,
                                 idle_spin_us=idle_spin_us)
    t_ticket, lat, t_sub, failed = {}, {}, {}, 0
    n = len(reqs)

    def drain():
        nonlocal failed
        for tk, us, st in xo.ec_server_poll_ex(server):
            lat[t_ticket[tk]] = us
            failed += st != xo.EC_OK

    t0 = time.perf_counter()
    next_poll = t0
    i = 0
    while i < n:
        now = time.perf_counter()
        target = t0 + reqs[i]["t"]
        if now >= target:
            tk = xo.ec_server_submit_raw(server, arr[i])
            if tk:
                t_ticket[tk] = i
                t_sub[i] = now
                i += 1
                continue
        if now >= next_poll or now < target:
            drain()
            next_poll = now + 0.001
    while len(lat) < n:
        drain()
        time.sleep(0.0005)
    t_end = time.perf_counter()
    stats = xo.ec_server_stats_get(server)
    xo.ec_server_destroy(server)
    measured = [j for j in range(n) if reqs[j]["t"] >= warm_s]
    span = reqs[-1]["t"] - warm_s if n else 0.0
    done_at = [t_sub[j] + lat[j] / 1e6 for j in measured]
    wall = (max(done_at) - min(t_sub[j] for j in measured)) if measured else 0.0
    mbytes = sum(in_bytes[j] for j in measured)
    out = {
        "p50_us": round(percentile([lat[j] for j in measured], 50), 1),
        "p99_us": round(percentile([lat[j] for j in measured], 99), 1),
        "p999_us": round(percentile([lat[j] for j in measured], 99.9), 1),
        "requests": len(measured),
        "offered_GBps": round(mbytes / span / 1e9, 2) if span > 0 else None,
        "GBps_in": round(mbytes / wall / 1e9, 2) if wall > 0 else None,
        "req_per_s": round(len(measured) / wall, 1) if wall > 0 else None,
        "batches": stats["batches"], "mean_batch": round(stats["completed"] / max(1, stats["batches"]), 2),
        "max_batch_seen": stats["max_batch_seen"], "rejected_retries": stats["rejected"],
        "failed": failed, "wall_s": round(t_end - t0, 2),
    }
    if check:
        out["parity"] = served_parity(xo, torch, reqs, where, data_arena, out_arena,
                                      range(max(0, n - check), n))
    return out


def served_parity(xo, torch, reqs, where, data_arena, out_arena, idx, L=64):
    """Bit-exact check of served requests against the oracle on sampled
    windows: encode outputs against the oracle's encode of the data window,
    decode outputs against the oracle's decode map applied to the survivor
    window (the survivors are arbitrary bytes; the map is linear)."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(23)
    dbase, obase = data_arena.data_ptr(), out_arena.data_ptr()

    def window(arena, base, ptr, B, w0, Lw):
        S = B // 8
        o = ptr - base
        return np.concatenate([arena[o + t * S + w0:o + t * S + w0 + Lw].cpu().numpy()
                               for t in range(8)])

    ok, n = True, 0
    for j in idx:
        r = reqs[j]
        k, m, B = r["k"], r["m"], r["B"]
        S = B // 8
        Lw = min(L, S)
        w0 = int(rng.integers(0, (S - Lw) // 16 + 1)) * 16
        blocks, outs = where[j]
        P = oracle.cauchy(k, m)
        got = [window(out_arena, obase, o, B, w0, Lw) for o in outs]
        if r["erasures"]:
            er = list(r["erasures"])
            surv = [i for i in range(k + m) if i not in er][:k]
            ref = oracle.apply(oracle.decode_matrix(P, er),
                               [window(data_arena, dbase, blocks[i], B, w0, Lw) for i in surv])
        else:
            ref = oracle.encode(P, [window(data_arena, dbase, blocks[i], B, w0, Lw)
                                    for i in range(k)])
        ok &= all(np.array_equal(a, b) for a, b in zip(got, ref))
        n += 1
    return ("bit-exact on sampled windows" if ok else "MISMATCH") + f" ({n} requests)"


def served_leg(args, rates):
    """Served workload: Poisson arrivals, RS(10,4)/RS(6,3), objects log-uniform
    4 KiB-16 MiB (B = roundup(ceil(L/k), 128)), half of them decodes with
    1..m random erasures; 32 GiB admission budget.  For every arrival rate,
    the continuous-batching server (512 requests per batch, 4 slots) and the
    plain form (one request at a time on one slot) replay the same trace."""
    import torch
    import paper_2108_02692_gb300 as xo
    from paper_2108_02692_gb300 import synth

    torch.cuda.set_device(0)
    warm_s = 1.0
    plans = {c: xo.ec_plan_create(*c) for c in ((10, 4), (6, 3))}
    tuned = {}
    if not args.no_tune:
        for c, h in plans.items():
            r = xo.ec_plan_autotune(h, 1 << 20, 16, torch.cuda.current_stream().cuda_stream)
            tuned[f"RS{c}"] = {"threads": r["threads"], "reg_budget": r["reg_budget"]}
    t0 = time.perf_counter()
    probe = xo.ec_server_create()
    for c, p in plans.items():
        xo.ec_server_warm(probe, p, c[1])
    xo.ec_server_destroy(probe)
    warm_time = time.perf_counter() - t0
    data_arena = torch.empty(8 << 30, dtype=torch.uint8, device="cuda")
    xo.ec_synth_fill(data_arena.data_ptr(), data_arena.numel(), synth.block_seed(5, 0, 0), 0, 0)
    out_arena = torch.empty(48 << 30, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    spin = args.serve_idle_spin_us
    points = []
    for rate in rates:
        # long enough for config 5's rate; ~200k requests at higher rates
        secs = args.serve_seconds if rate <= args.serve_rate else \
            max(1.0, min(args.serve_seconds, 2e5 / rate))
        lo, hi = (int(x) for x in args.serve_obj.split(","))
        reqs = synth.served_requests(secs + warm_s, rate, min_obj=lo, max_obj=hi)
        served = serve_stream(xo, torch, reqs, plans, data_arena, out_arena, 512, 4, warm_s,
                              idle_spin_us=spin, check=16)
        plain = serve_stream(xo, torch, reqs, plans, data_arena, out_arena, 1, 1, warm_s,
                             idle_spin_us=spin, check=16)
        points.append({"rate": rate, "seconds": secs, "served": served, "plain": plain,
                       "p99_plain_over_served": round(plain["p99_us"] / served["p99_us"], 2)})
    for p in plans.values():
        xo.ec_plan_destroy(p)
    del data_arena, out_arena
    torch.cuda.empty_cache()
    ok = all(pt[f]["parity"].startswith("bit-exact") and pt[f]["failed"] == 0
             for pt in points for f in ("served", "plain"))
    lo, hi = (int(x) for x in args.serve_obj.split(","))
    return {
        "workload": "served: Poisson arrivals, RS(10,4)/RS(6,3), objects log-uniform "
                    f"{lo} B-{hi} B, 50% decodes with 1..m erasures, 32 GiB admission budget; "
                    "served = continuous batching (512 per batch, 4 slots), plain = one request "
                    "at a time on one slot",
        "autotune": tuned or None, "warm_s": round(warm_time, 1),
        "points": points,
        "parity": "bit-exact on sampled windows" if ok else "MISMATCH",
        "device_status": xo.ec_device_status(),
    }


def run_served(args):
    rates = [float(x) for x in args.serve_rates.split(",")] if args.serve_rates \
        else [args.serve_rate]
    leg = served_leg(args, rates)
    head = leg["points"][0]
    out = {
        "metric": METRIC, "value": head["served"]["GBps_in"], "unit": "GB/s", "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (SplitMix64 bytes generated on the device)",
        "config": {"workload": f"served: Poisson {head['rate']:.0f} req/s for "
                               f"{head['seconds']:.0f} s (+1 s warm-up); " + leg["workload"]},
        "served": leg,
    }
    print(json.dumps(out))


def batched_leg(args):
    """Batched workload: mixed codes RS(6,3)/(8,4)/(10,4)/(12,4), block sizes
    log-uniform 4 KiB-8 MiB, half of the stripes decoded with random
    erasures, all in one batch run (replayed as a CUDA graph), against one
    launch per stripe."""
    import numpy as np
    import torch
    import paper_2108_02692_gb300 as xo
    from paper_2108_02692_gb300 import synth

    torch.cuda.set_device(0)
    mix = synth.batched_mix(args.batched_stripes)
    need = sum((s["k"] + s["m"]) * s["B"] for s in mix)
    free, _ = torch.cuda.mem_get_info()
    n = len(mix)
    while need > 0.85 * free and n > 16:
        n //= 2
        need = sum((s["k"] + s["m"]) * s["B"] for s in mix[:n])
    mix = mix[:n]
    arena = torch.empty(int(need), dtype=torch.uint8, device="cuda")
    plans = {c: xo.ec_plan_create(*c) for c in synth.BATCH_CODES}
    sp0 = torch.cuda.current_stream().cuda_stream
    tuned = {}
    if not args.no_tune:
        # per-code launch shape (strip tile = 4 x threads bytes) and register
        # budget; the batch compiles each code's modules with its own shape
        for c, h in plans.items():
            r = xo.ec_plan_autotune(h, 1 << 20, 16, sp0)
            tuned[f"RS{c}"] = {"threads": r["threads"], "reg_budget": r["reg_budget"]}
    jobs, pos, bytes_in, moved, where = [], 0, 0, 0, []
    base = arena.data_ptr()
    sp = torch.cuda.current_stream().cuda_stream
    for si, s in enumerate(mix):
        k, m, B = s["k"], s["m"], s["B"]
        blocks = [base + pos + j * B for j in range(k + m)]
        for j in range(k):
            xo.ec_synth_fill(blocks[j], B, synth.block_seed(4, si, j), 0, sp)
        where.append(pos)
        pos += (k + m) * B
        if s["erasures"]:
            er = list(s["erasures"])
            outs = [blocks[e] for e in er]            # recovered in place of the erased blocks
            jobs.append({"plan": plans[(k, m)], "op": xo.EC_OP_DECODE, "erasures": er,
                         "blocks": [None if i in er else blocks[i] for i in range(k + m)],
                         "out": outs, "block_bytes": B})
            moved += (k + len(er)) * B
        else:
            jobs.append({"plan": plans[(k, m)], "op": xo.EC_OP_ENCODE, "blocks": blocks[:k],
                         "out": blocks[k:], "block_bytes": B})
            moved += (k + m) * B
        bytes_in += k * B
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch = xo.ec_batch_create(jobs)
    prep = time.perf_counter() - t0
    info = xo.ec_batch_info_get(batch)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(max(1, args.warmup)):
        xo.ec_batch_run(batch, sp)
    torch.cuda.synchronize()
    ev0.record()
    reps = max(3, min(args.steps, 10))
    for _ in range(reps):
        xo.ec_batch_run(batch, sp)
    ev1.record()
    torch.cuda.synchronize()
    ms_eager = ev0.elapsed_time(ev1) / reps
    # the same run captured once in a CUDA graph and replayed
    gs = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gs):
        xo.ec_batch_run(batch, gs.cuda_stream)
    torch.cuda.synchronize()
    with torch.cuda.stream(gs):
        for _ in range(max(1, args.warmup)):
            graph.replay()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(gs)
        for _ in range(reps):
            graph.replay()
        g1.record(gs)
    torch.cuda.synchronize()
    ms = g0.elapsed_time(g1) / reps
    del graph
    batch_status = xo.ec_batch_status(batch)
    # plain: one launch per stripe with the same compiled programs
    singles = [xo.ec_batch_create([j]) for j in jobs]
    for b in singles[:64]:
        xo.ec_batch_run(b, sp)
    torch.cuda.synchronize()
    ev0.record()
    for b in singles:
        xo.ec_batch_run(b, sp)
    ev1.record()
    torch.cuda.synchronize()
    ms_plain = ev0.elapsed_time(ev1)
    for b in singles:
        xo.ec_batch_destroy(b)
    xo.ec_batch_destroy(batch)
    parity = batched_parity(mix, where, arena, n)
    peak, _ = measured_peaks()
    for p in plans.values():
        xo.ec_plan_destroy(p)
    del arena
    torch.cuda.empty_cache()
    return {
        "workload": f"batched: {n} stripes, RS(6,3)/(8,4)/(10,4)/(12,4), blocks log-uniform "
                    "4 KiB-8 MiB, ~50% decodes with 1..m erasures; one ec_batch_run replayed "
                    "as a CUDA graph",
        "value": round(bytes_in / (ms / 1e3) / 1e9, 2), "unit": "GB/s",
        "ms_per_step": round(ms, 3), "steps": reps,
        "input_bytes": bytes_in, "moved_bytes": moved, "autotune": tuned or None,
        "eager": {"value": round(bytes_in / (ms_eager / 1e3) / 1e9, 2),
                  "ms_per_step": round(ms_eager, 3)},
        "roofline": {"bound": "hbm", "achieved": round(moved / (ms / 1e3) / 1e9, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(moved / (ms / 1e3) / 1e9 / peak, 4),
                     "bytes_per_step": moved},
        "plain": {"value": round(bytes_in / (ms_plain / 1e3) / 1e9, 2),
                  "ms_per_step": round(ms_plain, 2), "launches_per_step": n},
        "batched_over_plain": round(ms_plain / ms, 2),
        "batch": info, "prepare_s": round(prep, 1),
        "parity": parity, "batch_status": batch_status,
        "device_status": xo.ec_device_status(),
    }


def run_batched(args):
    leg = batched_leg(args)
    print(json.dumps({
        "metric": METRIC, "value": leg["value"], "unit": "GB/s",
        "n_gpus": 1, "steps": leg["steps"], "warmup": args.warmup,
        "ms_per_step": leg["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (SplitMix64 bytes generated on the device)",
        "config": {"workload": leg["workload"]},
        "batched": leg,
    }))


def batched_parity(mix, where, arena, n, samples=24, L=64):
    """Sampled bit-exact check of a batched run against the oracle: for a
    few stripes, a window of L bytes of every strip of the stripe's inputs
    and outputs is read back; encode outputs must equal the oracle's encode
    of the data window, decode outputs the oracle's decode map applied to
    the survivor window."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(19)

    def window(off, B, w0):
        S = B // 8
        return np.concatenate([arena[off + t * S + w0:off + t * S + w0 + L].cpu().numpy()
                               for t in range(8)])

    ok = True
    for si in rng.choice(n, min(samples, n), replace=False):
        s = mix[int(si)]
        k, m, B = s["k"], s["m"], s["B"]
        S = B // 8
        w0 = int(rng.integers(0, max(1, (S - L) // 16 + 1))) * 16 if S >= L else 0
        Lw = min(L, S)
        if Lw != L:
            continue
        P = oracle.cauchy(k, m)
        blk = [window(where[int(si)] + j * B, B, w0) for j in range(k + m)]
        if s["erasures"]:
            er = list(s["erasures"])
            surv = [i for i in range(k + m) if i not in er][:k]
            ref = oracle.apply(oracle.decode_matrix(P, er), [blk[i] for i in surv])
            got = [blk[e] for e in er]
        else:
            ref = oracle.encode(P, blk[:k])
            got = blk[k:]
        ok &= all(np.array_equal(a, b) for a, b in zip(got, ref))
    return "bit-exact on sampled windows" if ok else "MISMATCH"


def run_dense(args, xo, data, par, stream, torch, peak):
    """The same encode on the dense bitmatrix executor (the tier that runs
    programs without a compiled kernel): one launch over the 256 stripes,
    timed with CUDA events on the launching stream; its parity is compared
    byte for byte with the compiled kernel's, which the headline checks
    against the oracle."""
    k, m, B, n = K_DATA, M_PAR, BLOCK, N_STRIPES
    plan = xo.ec_plan_create_ex(k, m, matrix_kind=matrix_kind(xo, args.matrix),
                                executor=xo.EC_EXEC_DENSE)
    try:
        out = torch.empty_like(par)
        sp = stream.cuda_stream

        def launch():
            xo.ec_encode_strided(plan, data.data_ptr(), k * B, B, out.data_ptr(), m * B, B, n, B, sp)

        with torch.cuda.stream(stream):
            for _ in range(3):
                launch()
            torch.cuda.synchronize()
            reps = 5
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(reps):
                launch()
            ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / reps
        same = bool(torch.equal(out, par))
        del out
        return {"value": round(n * k * B / (ms / 1e3) / 1e9, 1), "unit": "GB/s",
                "frac": round(n * (k + m) * B / (ms / 1e3) / 1e9 / peak, 4),
                "ms_per_launch": round(ms, 4), "launches": reps,
                "kernel": "dense_kernel (%s form)" % os.environ.get("EC_DENSE_KIND", "table"),
                "parity": "identical to the compiled kernel's parity, all 256 stripes" if same
                          else "MISMATCH"}
    finally:
        xo.ec_plan_destroy(plan)


def run_e2e(args, xo, plan, data, par, stream, torch):
    """Same metric from pinned host buffers, through ec_encode_host_strided:
    per step the 256 stripes go host -> device in chunks, are encoded and
    their parity comes back, with copies and kernels overlapped on the
    library's internal lanes."""
    k, m, B, n = K_DATA, M_PAR, BLOCK, N_STRIPES
    chunk = int(os.environ.get("EC_E2E_CHUNK", "16"))
    h_data = torch.empty((n, k, B), dtype=torch.uint8, pin_memory=True)
    h_par = torch.empty((n, m, B), dtype=torch.uint8, pin_memory=True)
    h_data.copy_(data, non_blocking=False)
    sp = stream.cuda_stream

    def one_step():
        xo.ec_encode_host_strided(plan, h_data.data_ptr(), k * B, B, h_par.data_ptr(), m * B, B,
                                  n, B, chunk, sp)

    for _ in range(2):
        one_step()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(steps):
        one_step()
    stream.synchronize()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ok = bool(torch.equal(h_par[n - 1, :, :4096].cuda(), par[n - 1, :, :4096]))
    return {"value": round(n * k * B * steps / dt / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": n * k * B, "d2h_bytes_per_step": n * m * B,
            "steps": steps, "launches_per_step": (n + chunk - 1) // chunk,
            "matches_device_result": ok}


# ------------------------------------------------------------- reference

def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_sample_gbs(cores, 1)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g, _, _ = oracle_sample_gbs(cores, 1)
        vals.append(g)
    wall = time.perf_counter() - t0
    value = statistics.mean(vals)
    sample = f"{cores} of the 256 stripes per step (10 x 1 MiB each), one per host thread"
    print(json.dumps({
        "impl": "reference",
        "metric": METRIC, "value": round(value, 5), "unit": "GB/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(wall / args.steps * 1e3, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (SplitMix64 bytes)",
        "config": {"workload": WORKLOAD, "k": K_DATA, "m": M_PAR, "n_stripes": N_STRIPES,
                   "block_bytes": BLOCK, "matrix": "cauchy"},
        "cpu_baseline": {"value": round(value, 5), "unit": "GB/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 5), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    import __graft_entry__
    __graft_entry__.build()
    if args.workload == "served":
        run_served(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "codes":
        run_codes(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
