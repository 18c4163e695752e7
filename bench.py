"""Benchmark: BLS12-377 G1 MSM points/s at n = 2^20 (one step = one msm_g1 call).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n N] [--c C]
                [--mode best|xyzz|edwards|glv|edwards+glv|edwards+precomputed|edwards+glv+precomputed]
                [--no-extras]

Our arm. The headline (`value`) is the single MSM over n = 2^20 resident points
(prepared once, outside the timed region) with fresh seeded scalars per step already
in HBM, signed digits and the window width c chosen by the autotuner from 12..17:
the fastest of the four variable-base schedules (XYZZ; the paper's twisted Edwards
model; the GLV split; Edwards + GLV), each autotuned and timed. L2 is flushed (a
256 MB write) between timed steps; per-step CUDA events on the launch stream. Every
timed mode's result is checked against the closed form ((sum a_i s_i) mod r) G of the
workload (points P_i = s_i G) and the line says so ("verified").
Extras (rank 0): fixed-base resident sets (per-window shifted copies made once per
set, labelled with their size and setup time), n = 2^22, the 2^12 / c = 8 unsigned
MSM on standard-form points, 2^24 Fq multiplications and 2^24 mixed PADDs with 1 %
each of P + P, P + (-P), acc = O and Q = O, the dependent-chain latency, 64 batched
MSMs, the serving loop, the end-to-end host-buffer call and the CPU oracle baseline.
Reference arm (--impl reference): the CPU oracle's Pippenger (plain C, all host
cores) on a bounded sample of the same workload; rank 0 only.
For N > 1 (torchrun) every rank runs its own MSMs on its own GPU (replicas, no
collective on the data path); value = all ranks' points / max-over-ranks time.
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

import synth  # noqa: E402

METRIC = "BLS12-377 MSM points/s & PADD/s at n=2^20; batched vs sequential speedup"
PRODUCTS = {"fq_mul": 276, "fq_sqr": 210}
PRODUCTS["madd"] = 8 * PRODUCTS["fq_mul"] + 2 * PRODUCTS["fq_sqr"]     # 2628
PRODUCTS["add"] = 12 * PRODUCTS["fq_mul"] + 2 * PRODUCTS["fq_sqr"]     # 3732
PRODUCTS["dbl"] = 6 * PRODUCTS["fq_mul"] + 3 * PRODUCTS["fq_sqr"]      # 2286
# twisted Edwards, extended coordinates (a = -1): madd 7M, add 9M (with k T2), dbl 4M + 4S
PRODUCTS["ed_madd"] = 7 * PRODUCTS["fq_mul"]                            # 1932
PRODUCTS["ed_add"] = 9 * PRODUCTS["fq_mul"]                             # 2484
PRODUCTS["ed_dbl"] = 4 * PRODUCTS["fq_mul"] + 4 * PRODUCTS["fq_sqr"]    # 1944
# mode -> (edwards, glv, precomputed)
MODES = {"xyzz": (False, False, False), "edwards": (True, False, False), "glv": (False, True, False),
         "edwards+glv": (True, True, False), "edwards+precomputed": (True, False, True),
         "edwards+glv+precomputed": (True, True, True)}
VARIABLE_MODES = ("xyzz", "edwards", "glv", "edwards+glv")
FIXED_MODES = ("edwards+precomputed", "edwards+glv+precomputed")
X0 = 0x8508C00000000001
R_ORDER = X0 ** 4 - X0 ** 2 + 1
GLV_LAMBDA = X0 * X0 - 1
BITS = 253
PROFILE_DIR = os.path.join(ROOT, "profiles")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--c", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=0,
                    help="with --c: items per accumulation thread for the run (0 = the built-in rule)")
    ap.add_argument("--mode", default="best", choices=["best"] + list(MODES))
    ap.add_argument("--no-extras", action="store_true", help="skip every extra beyond the headline")
    ap.add_argument("--only", default="", choices=["", "batch_ops"],
                    help="run one extra alone (no headline): batch_ops = the Fq multiplications, their variants, "
                         "the mixed PADDs and the integer-multiply probe")
    ap.add_argument("--batch-ops-n", type=int, default=1 << 24, help="elements of the batch_ops workloads")
    return ap.parse_args()


def agree_on(value, world: int):
    """Rank 0's value on every rank (the headline mode, so every rank times the same work)."""
    if world == 1:
        return value
    import torch.distributed as dist
    obj = [value]
    dist.broadcast_object_list(obj, src=0)
    return obj[0]


def max_over_ranks(x: float, world: int, device) -> float:
    """The slowest rank's time: the whole job finishes when its last rank does."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_points_per_s(n: int, world: int, ms: float) -> float:
    """Weak scaling: every rank runs its own n-point MSM per step."""
    return world * n / (ms / 1e3)


def rank_workload(n: int, rank: int, nsets: int):
    """Seeds of rank `rank`'s resident point set and its per-step scalar sets (disjoint streams per rank)."""
    seeds = synth.scalars(synth.stream_seed(2, n, 2 + 1000 * rank), n)
    scal = [synth.scalars(synth.stream_seed(2, n, 100 + j + 1000 * rank), n) for j in range(nsets)]
    return seeds, scal


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- result checks

def dot_mod_r(a: np.ndarray, s: np.ndarray) -> int:
    """sum_i a_i s_i mod r for (n, 8) u32 scalar arrays, exactly: the 16-bit halves of
    the limbs give 16 x 16 dot products whose terms are below 2^32; over chunks of
    2^18 rows every partial sum is below 2^50, so float64 matrix products are exact."""
    total = 0
    n = a.shape[0]
    step = 1 << 18
    for lo in range(0, n, step):
        a16 = np.ascontiguousarray(a[lo:lo + step]).view(np.uint16).astype(np.float64)
        s16 = np.ascontiguousarray(s[lo:lo + step]).view(np.uint16).astype(np.float64)
        m = a16.T @ s16
        for u in range(16):
            for v in range(16):
                total += int(m[u, v]) << (16 * (u + v))
    return total % R_ORDER


def on_curve(pt: np.ndarray) -> bool:
    x = synth.limbs_to_int(pt[:12])
    y = synth.limbs_to_int(pt[12:24])
    p = synth.P_INT
    if x == 0 and y == 0:
        return True          # the identity's encoding
    return x < p and y < p and (y * y - x * x * x - 1) % p == 0


def expected_points(pkg, dev, ks) -> np.ndarray:
    """k * G for each k (affine standard form, (0, 0) for O), computed on the device by
    g1_generator_mul, the library's double-and-add kernel."""
    arr = np.stack([synth.int_to_limbs(int(k) % R_ORDER, 8) for k in ks])
    return pkg.to_host(pkg.g1_generator_mul(pkg.to_device(arr, dev))).reshape(len(ks), 24)


def verify_msm(pkg, dev, out, k: int) -> bool:
    """The MSM output equals the closed form k G, k = (sum a_i s_i) mod r."""
    got = pkg.to_host(out).reshape(24)
    want = expected_points(pkg, dev, [k])[0]
    return bool(np.array_equal(got, want) and on_curve(got))


# ---------------------------------------------------------------- op counts

def glv_halves(scalars: np.ndarray) -> np.ndarray:
    """(n, 8) scalars -> (2n, 8): rows 2i, 2i + 1 = k1, k2 of k mod r = k1 + lambda k2
    (the split the library makes; used here only to count the work)."""
    k = np.zeros(scalars.shape[0], dtype=object)
    for w in range(8):
        k += scalars[:, w].astype(object) << (32 * w)
    k %= R_ORDER
    k2 = k // GLV_LAMBDA
    k1 = k - k2 * GLV_LAMBDA
    out = np.zeros((2 * scalars.shape[0], 8), dtype=np.uint32)
    for w in range(4):
        out[0::2, w] = ((k1 >> (32 * w)) & 0xFFFFFFFF).astype(np.uint64).astype(np.uint32)
        out[1::2, w] = ((k2 >> (32 * w)) & 0xFFFFFFFF).astype(np.uint64).astype(np.uint32)
    return out


def digit_counts(scalars: np.ndarray, c: int, signed: bool, bits: int, shared: bool = False):
    """Nonzero digits and distinct nonzero buckets, per window or (shared) over one
    bucket set for all windows (host numpy, for op counts)."""
    words = scalars.astype(np.uint64)
    W = -(-(bits + (1 if signed else 0)) // c)
    carry = np.zeros(scalars.shape[0], dtype=np.int64)
    nonzero = 0
    runs = 0
    seen = np.zeros(1 << c, dtype=bool)
    half = 1 << (c - 1)
    for j in range(W):
        b0 = j * c
        raw = np.zeros(scalars.shape[0], dtype=np.int64)
        for b in range(c):
            bit = b0 + b
            if bit >= 256:
                break
            raw |= ((words[:, bit // 32] >> np.uint64(bit % 32)) & np.uint64(1)).astype(np.int64) << b
        if signed:
            v = raw + carry
            neg = v > half
            key = np.where(neg, (1 << c) - v, v)
            carry = neg.astype(np.int64)
        else:
            key = raw
        nz = key[key != 0]
        nonzero += nz.size
        if shared:
            seen[np.unique(nz)] = True
        else:
            runs += np.unique(nz).size
    if shared:
        runs = int(seen.sum())
    return W, nonzero, runs


def op_counts(sc_host: np.ndarray, c: int, bits: int, edwards: bool, glv: bool, pre: bool = False,
              signed: bool = True):
    """Additions and doublings of one MSM, and the textbook products and algorithmic
    bytes of its bucket accumulation."""
    sc = glv_halves(sc_host) if glv else sc_host
    W, nonzero, runs = digit_counts(sc, c, signed, 127 if glv else bits, shared=pre)
    madds = nonzero - runs            # the first point of each run is an assignment
    sets = 1 if pre else W            # bucket sets
    buckets = (1 << (c - 1)) if signed else (1 << c) - 1
    full_adds = 2 * sets * buckets    # running sums of the bucket reduction
    dbls = 0 if pre else (W - 1) * c
    pm = PRODUCTS["ed_madd" if edwards else "madd"]
    stored = 144 if edwards else 96
    return {"windows": W, "madd": madds, "bucket_running_sum_adds": full_adds, "window_dbls": dbls,
            "products_per_madd": pm, "accumulate_products": madds * pm,
            "accumulate_bytes": nonzero * (stored + 8),
            "bytes_per_madd": f"{stored} B gathered stored point + 8 B sorted (key, value) pair"}


# ---------------------------------------------------------------- clocks, traffic

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# The source the bucket-accumulation kernel is compiled from: the field and curve
# headers and three sections of msm.cu (memory I/O, curve models, stages 4-5).
ACC_SECTIONS = (("// ---------------------------------------------------------------- memory I/O",
                 "// Second operand of ec::add_q()"),
                ("// ---------------------------------------------------------------- curve models",
                 "// ---------------------------------------------------------------- stage 1"),
                ("// ---------------------------------------------------------------- stages 4-5",
                 "// Batched MSMs:"))


def kernel_hash(edwards: bool = True) -> str:
    """Source hash of the accumulation kernel of one curve model: the field header,
    that model's header and the msm.cu sections the kernel is compiled from."""
    csrc = os.path.join(ROOT, "paper_2502_11660_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("fq.cuh", "ed.cuh" if edwards else "ec.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    src = open(os.path.join(csrc, "msm.cu")).read()
    for start, end in ACC_SECTIONS:
        a = src.index(start)
        h.update(src[a:src.index(end, a)].encode())
    return h.hexdigest()[:16]


def recorded_traffic(mode: str, c: int):
    """DRAM bytes per accumulate launch of `mode` at window c from the committed ncu
    summary, if it was taken from this kernel source; else None."""
    path = os.path.join(PROFILE_DIR, "accumulate_traffic.json")
    if not os.path.exists(path):
        return None
    recs = json.load(open(path))
    rec = recs.get(mode) if isinstance(recs, dict) else None
    if not rec or rec.get("kernel_hash") != kernel_hash(MODES[mode][0] or MODES[mode][2]) or rec.get("c") != c:
        return None
    return rec


# ---------------------------------------------------------------- reference arm, CPU baseline

def cpu_baseline(n: int, reps_budget_s: float = 12.0):
    """The oracle's C Pippenger (as it stands) on a bounded sample, all host cores and one core."""
    from oracle import coracle
    a, s = synth.workloads.msm(n, tag=2)
    pts = coracle.gen_points(s)
    c = max(4, min(16, int(np.log2(max(n, 2))) - 3))
    cores = os.cpu_count() or 1

    def rate(nthreads, budget):
        t0 = time.perf_counter()
        runs = 0
        while True:
            coracle.msm(pts, a, c=c, nthreads=nthreads)
            runs += 1
            if time.perf_counter() - t0 > budget or runs >= 20:
                break
        return n / ((time.perf_counter() - t0) / runs), runs

    v_all, runs = rate(0, reps_budget_s)
    v_one, runs1 = rate(1, reps_budget_s / 2)
    return {"value": v_all, "unit": "points/s", "cores": cores, "kind": "oracle",
            "sample": f"textbook Pippenger (plain C, unsigned c={c}), n={n} points of the workload, "
                      f"{runs} run(s), {cores} threads over windows",
            "single_thread": {"value": v_one, "unit": "points/s", "cores": 1, "runs": runs1}}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    n = min(args.n, 1 << 16)
    from oracle import coracle
    a, s = synth.workloads.msm(n, tag=2)
    pts = coracle.gen_points(s)
    c = max(4, min(16, int(np.log2(max(n, 2))) - 3))
    for _ in range(args.warmup):
        coracle.msm(pts, a, c=c)
    times = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        coracle.msm(pts, a, c=c)
        times.append(time.perf_counter() - t0)
    wall = time.perf_counter() - t_all
    ms = 1e3 * sum(times) / len(times)
    val = n / (ms / 1e3)
    cores = os.cpu_count() or 1
    out = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "points/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64 (C big-integer)", "data": "synthetic",
        "config": {"workload": f"msm_g1 BLS12-377 G1, bounded CPU sample n={n} of the n=2^20 workload",
                   "n": n, "c": c},
        "cpu_baseline": {"value": val, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "sample": f"textbook Pippenger (plain C, unsigned c={c}), n={n} points per step"},
        "e2e": {"value": val, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- our arm

class Harness:
    """Device buffers and timing helpers shared by the headline and the extras."""

    def __init__(self, pkg, torch, dev, stream):
        self.pkg, self.torch, self.dev, self.stream = pkg, torch, dev, stream
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        self.out = torch.empty(24, dtype=torch.int32, device=dev)

    def steps(self, fn, steps, profile=False):
        """Per-step event times (ms) of fn(j), L2 flushed between steps outside the events."""
        torch = self.torch
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        stages = []
        for j in range(steps):
            self.flush.fill_(j & 0xFF)
            ev[j][0].record(self.stream)
            fn(j)
            ev[j][1].record(self.stream)
            if profile:
                stages.append(self.pkg.profile_last())   # synchronises on the step's last event
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev], stages


def tuned_c(pkg, autotune, dev, log2n, edw, gl, pre, forced=0, chunk=0):
    """c for (mode, 2^log2n): the autotuner's measured choice (installed into the
    library's tables for that mode; variable-base modes also tune the chunk size, the
    sort, the reduction threads and the window groups), or `forced` (with `chunk`
    items per accumulation thread when nonzero)."""
    if forced:
        if chunk and not pre:
            autotune.install_schedule({log2n: [forced, chunk, 0, 0, 0]}, edwards=edw, glv=gl)
            return forced, f"given, chunk {chunk}", None
        return forced, "given", None
    if pre:
        tuning = autotune.tune(log2_sizes=[log2n], reps=3, device=dev, edwards=edw, glv=gl, precomputed=pre)
        autotune.install(tuning["table"], edwards=edw, glv=gl, precomputed=pre)
        c = pkg.msm_g1_default_c(1 << log2n, True, edw, gl, pre)
        return c, {str(cc): round(v, 3) for cc, v in tuning["timings"][log2n].items()}, None
    tuning = autotune.tune_schedule(log2_sizes=[log2n], reps=3, device=dev, edwards=edw, glv=gl)
    entry = tuning["schedule"][log2n]
    ms = tuning["ms"][log2n]
    return entry[0], {f: {str(v): round(t, 3) for v, t in d.items()} for f, d in ms.items()}, list(entry)


def survey_mode(h, autotune, name, n, pts_std, sc_dev, ks, warmup, forced_c=0, chunk=0):
    """Autotune, prepare and time one mode for 10 steps; check one result against the closed form."""
    pkg, torch, dev = h.pkg, h.torch, h.dev
    edw, gl, pre = MODES[name]
    c, timings, entry = tuned_c(pkg, autotune, dev, int(np.log2(n)), edw, gl, pre, forced_c, chunk)
    t0 = time.perf_counter()
    if pre:
        prep = pkg.msm_points_precompute(pts_std, c=c, scalar_bits=BITS, glv=gl)
    else:
        prep = pkg.msm_points_prepare(pts_std, edwards=edw, glv=gl)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    ws = pkg.msm_g1_workspace(n, c=c, scalar_bits=BITS, prepared=True, device=dev, edwards=edw, glv=gl,
                              precomputed=pre)
    kw = dict(out=h.out, workspace=ws, c=c, scalar_bits=BITS, prepared=True, stream=h.stream, edwards=edw,
              glv=gl, precomputed=pre)
    nsets = len(sc_dev)
    for j in range(warmup):
        pkg.msm_g1(prep, sc_dev[j % nsets], **kw)
    ms, st = h.steps(lambda j: pkg.msm_g1(prep, sc_dev[(warmup + j) % nsets], profile=True, **kw), 10, True)
    j = (warmup + 9) % nsets
    ok = verify_msm(pkg, dev, h.out, ks[j]) and pkg.msm_g1_status(ws, h.stream) == 0
    sched = pkg.msm_g1_schedule(n, c=c, scalar_bits=BITS, edwards=edw, glv=gl, precomputed=pre)
    rec = {"c": c, "ms_per_step": statistics.mean(ms), "points_per_s": n / (statistics.mean(ms) / 1e3),
           "schedule": sched, "schedule_entry": entry,
           "stages_ms": {s2: statistics.mean(x[s2] for x in st) for s2 in st[0]},
           "resident_set": {"GB": prep.numel() * 4 / 1e9, "setup_s": setup_s},
           "c_by_autotuner": timings, "verified": bool(ok)}
    return rec, (prep, ws, c, edw, gl, pre)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2502_11660_gb300 as pkg
    from paper_2502_11660_gb300 import autotune

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    h = Harness(pkg, torch, dev, stream)
    n = args.n
    k = int(np.log2(n))

    # resident point set P_i = s_i G, built on the device and prepared per mode (not timed);
    # nsets scalar sets, one per step, with their closed-form k = sum a_i s_i mod r
    nsets = max(4, min(args.steps + args.warmup, 24))
    seeds, sc_host = rank_workload(n, rank, nsets)
    pts_std = pkg.g1_generator_mul(pkg.to_device(seeds, dev))
    sc_dev = [pkg.to_device(x, dev) for x in sc_host]
    ks = [dot_mod_r(x, seeds) for x in sc_host]

    # every variable-base mode: c from the autotuner (12..17) unless --c, 10 timed steps, checked
    survey, preps = {}, {}
    wanted = VARIABLE_MODES if args.mode == "best" else (args.mode,)
    for name in wanted:
        survey[name], preps[name] = survey_mode(h, autotune, name, n, pts_std, sc_dev, ks, args.warmup, args.c,
                                                args.chunk)
    mode = agree_on(min(survey, key=lambda m: survey[m]["ms_per_step"]), world)
    prep, ws, c, edw, gl, pre = preps[mode]
    for other in list(preps):
        if other != mode:
            del preps[other]
    peak = pkg.imad_probe(20000, stream=stream)   # measured limb-product peak (products/s)
    kw = dict(out=h.out, workspace=ws, c=c, scalar_bits=BITS, prepared=True, stream=stream, edwards=edw,
              glv=gl, precomputed=pre)

    # the timed region: K steps of the headline mode
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for j in range(args.warmup):
        pkg.msm_g1(prep, sc_dev[j % nsets], **kw)
    torch.cuda.synchronize()
    launches0 = pkg.launch_count()
    t_wall = time.perf_counter()
    step_ms, stage_ms = h.steps(lambda j: pkg.msm_g1(prep, sc_dev[j % nsets], profile=True, **kw), args.steps,
                                True)
    wall = time.perf_counter() - t_wall
    launches = pkg.launch_count() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    last = (args.steps - 1) % nsets
    verified = verify_msm(pkg, dev, h.out, ks[last]) and pkg.msm_g1_status(ws, stream) == 0
    ms = max_over_ranks(sum(step_ms) / len(step_ms), world, dev)
    value = job_points_per_s(n, world, ms)

    ops = op_counts(sc_host[last], c, BITS, edw, gl, pre)
    # the accumulation kernel alone for the roofline: with window groups the
    # "accumulate" stage also holds the overlapped tails of earlier groups, so a few
    # profiled steps run with one group (same c, chunk, sort, reduction)
    sched = pkg.msm_g1_schedule(n, c=c, scalar_bits=BITS, edwards=edw, glv=gl, precomputed=pre)
    acc_ms = statistics.mean(x["accumulate"] for x in stage_ms)
    entry = survey[mode].get("schedule_entry") or [c, 0, 0, 0, 0]
    if sched["groups"] > 1:
        pkg.msm_g1_set_schedule(k, *entry[:4], 1, edwards=edw, glv=gl)
        ws1 = pkg.msm_g1_workspace(n, c=c, scalar_bits=BITS, prepared=True, device=dev, edwards=edw, glv=gl)
        kw1 = dict(kw, workspace=ws1)
        _, st1 = h.steps(lambda j: pkg.msm_g1(prep, sc_dev[j % nsets], profile=True, **kw1), 5, True)
        acc_ms = statistics.mean(x["accumulate"] for x in st1)
        pkg.msm_g1_set_schedule(k, *entry, edwards=edw, glv=gl)
        del ws1
    achieved = ops["accumulate_products"] / (acc_ms / 1e3)
    hbm_peak = measured_hbm_peak()
    kname = "k_accumulate<%s>" % ("ModelEdwards" if edw else "ModelXyzz")
    rec = recorded_traffic(mode, c)
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved / 1e12, "peak": peak / 1e12,
                "unit": "Tprod/s", "frac": achieved / peak,
                "peak_source": "of measured: msm377_imad_probe (even/odd mad.lo.cc/madc.hi.cc chains, all SMs), "
                               "in this run",
                "algorithmic_products_per_launch": ops["accumulate_products"],
                "kernel_ms": acc_ms,
                "kernel_ms_source": ("events around the accumulation launch in 5 profiled steps with one window group "
                                     "(the timed steps overlap later groups' accumulation with earlier groups' tails)"
                                     if sched["groups"] > 1 else "the timed steps' accumulate stage"),
                "traffic": (rec["bytes_per_launch"] if rec else None),
                "traffic_source": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of this kernel source "
                                   f"(hash {rec['kernel_hash']}), {rec['date']}, carried from "
                                   f"profiles/accumulate_traffic.json" if rec else
                                   "null: no ncu capture of this kernel source at this c"),
                "hbm": {"algorithmic_bytes_per_launch": ops["accumulate_bytes"],
                        "achieved_GBps": ops["accumulate_bytes"] / (acc_ms / 1e3) / 1e9,
                        "peak_GBps": hbm_peak, "frac": ops["accumulate_bytes"] / (acc_ms / 1e3) / 1e9 / hbm_peak,
                        "peak_source": "of measured: MEASURED_PEAKS.json hbm_gbs (copy)"}}
    padds = ops["madd"] + ops["bucket_running_sum_adds"] + ops["window_dbls"]

    result = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32 (12x32-bit limb Montgomery integer arithmetic)", "data": "synthetic",
        "config": {"workload": f"msm_g1 BLS12-377 G1 n={n}, mode {mode} (signed digits, c={c} by the autotuner "
                               f"from 12..17), resident prepared points, fresh scalars per step", "n": n, "c": c,
                   "mode": mode, "windows": ops["windows"],
                   "l2": "flushed between steps (256 MB write, outside the timed events)",
                   "parallelism": f"replicas x{world}"},
        "verified": bool(verified),
        "verified_how": "the last timed step's output equals ((sum_i a_i s_i) mod r) G (points P_i = s_i G; k from "
                        "the host, k G by g1_generator_mul) and lies on y^2 = x^3 + 1; device status 0",
        "padd_per_s": world * padds / (ms / 1e3),
        "op_counts": ops,
        "stages_ms": {k2: statistics.mean(x[k2] for x in stage_ms) for k2 in stage_ms[0]},
        "modes": survey,
        "roofline": roofline,
        "gpu_launches": launches,
        "clocks": clk,
        "wall_s_timed_region": wall,
    }
    del preps, prep, ws

    if rank == 0 and not args.no_extras:
        plain = sorted(survey, key=lambda m: survey[m]["ms_per_step"])
        hm_edw, hm_gl, _ = MODES[mode]
        result["fixed_base"] = fixed_base(h, autotune, n, pts_std, sc_dev, ks, args.warmup)
        # window widths measured for every size 2^10 .. 2^22 of the headline mode, installed
        # before the 2^22, batched and serving runs
        tuning = autotune.tune_schedule(log2_sizes=range(10, 23), reps=3, device=dev, edwards=hm_edw, glv=hm_gl)
        result["autotune"] = {"mode": mode,
                              "schedule_by_log2n (c, chunk, sort, reduce_log2, groups; 0 = built-in rule)":
                                  {str(q): list(v) for q, v in tuning["schedule"].items()},
                              "ms": {str(q): {f: {str(v): round(t, 3) for v, t in d.items()} for f, d in rec.items()}
                                     for q, rec in tuning["ms"].items()}}
        autotune.clear_cache()
        result["n_2e22"] = msm_2e22(h, autotune, mode)
        result["config0_2e12_c8_unsigned"] = msm_small(h)
        result["e2e"] = end_to_end(h, n, pts_std, sc_host, ks, survey, plain[:2], args.steps)
        result["batch_ops"] = batch_ops(h, peak, hbm_peak)
        result["latency"] = latency_chain(h, pts_std)
        result["batched_msm"] = batched_msm(h, autotune, hm_edw, hm_gl)
        result["serving"] = serve(h, hm_edw, hm_gl)
        result["cpu_baseline"] = cpu_baseline(1 << 16)

    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


def measured_hbm_peak() -> float:
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def fixed_base(h, autotune, n, pts_std, sc_dev, ks, warmup):
    """Fixed-base resident sets (per-window shifted copies 2^(cj) P_i, built once per set
    outside the timing; c from 15..20): labelled with their size and setup time."""
    res = {"note": "not the headline: resident sets holding every window's shifted copy of each point"}
    for name in FIXED_MODES:
        rec, keep = survey_mode(h, autotune, name, n, pts_std, sc_dev, ks, warmup)
        res[name] = rec
        del keep
    h.torch.cuda.empty_cache()
    return res


def msm_2e22(h, autotune, mode):
    """The headline mode at n = 2^22 (c from the autotuned table, 12..17 at that size), checked."""
    pkg, torch, dev = h.pkg, h.torch, h.dev
    n = 1 << 22
    seeds = synth.scalars(synth.stream_seed(2, n, 2), n)
    scs = [synth.scalars(synth.stream_seed(2, n, 100 + j), n) for j in range(3)]
    ks = [dot_mod_r(x, seeds) for x in scs]
    std = pkg.g1_generator_mul(pkg.to_device(seeds, dev))
    edw, gl, pre = MODES[mode]
    c = pkg.msm_g1_default_c(n, True, edw, gl, pre)   # the installed (tuned) table
    rec, keep = survey_mode(h, autotune, mode, n, std, [pkg.to_device(x, dev) for x in scs], ks, 3, forced_c=c)
    rec["c_by_autotuner"] = "installed table"
    del keep, std
    torch.cuda.empty_cache()
    rec["mode"] = mode
    return rec


def msm_small(h, n=1 << 12, c=8, steps=50):
    """2^12 points in standard (non-Montgomery) form, c = 8 unsigned digits, XYZZ: the
    preparation runs inside every call. Checked against the closed form."""
    pkg, torch, dev = h.pkg, h.torch, h.dev
    seeds = synth.scalars(synth.stream_seed(0, n, 2), n)
    scs = [synth.scalars(synth.stream_seed(0, n, 100 + j), n) for j in range(4)]
    ks = [dot_mod_r(x, seeds) for x in scs]
    pts = pkg.g1_generator_mul(pkg.to_device(seeds, dev))
    sc_dev = [pkg.to_device(x, dev) for x in scs]
    ws = pkg.msm_g1_workspace(n, c=c, signed=False, scalar_bits=BITS, device=dev)
    kw = dict(out=h.out, workspace=ws, c=c, signed=False, scalar_bits=BITS, stream=h.stream)
    for j in range(5):
        pkg.msm_g1(pts, sc_dev[j % 4], **kw)
    ms, _ = h.steps(lambda j: pkg.msm_g1(pts, sc_dev[j % 4], **kw), steps)
    ok = verify_msm(pkg, dev, h.out, ks[(steps - 1) % 4])
    return {"n": n, "c": c, "digits": "unsigned", "mode": "xyzz, standard-form points prepared inside the call",
            "ms_per_step": statistics.mean(ms), "points_per_s": n / (statistics.mean(ms) / 1e3),
            "verified": bool(ok), "l2": "flushed between steps"}


def end_to_end(h, n, pts_std, sc_host, ks, survey, modes, steps):
    """msm_g1_host: pinned host points and scalars copied in, the points prepared, the MSM
    and the result copied out, every step; the faster of the two fastest modes."""
    pkg, torch, dev = h.pkg, h.torch, h.dev
    pinned_pts = torch.from_numpy(pkg.to_host(pts_std).view(np.int32)).pin_memory()
    hp = pinned_pts.numpy().view(np.uint32)
    nh = min(4, len(sc_host))
    hsc = [torch.from_numpy(x.view(np.int32)).pin_memory().numpy().view(np.uint32) for x in sc_host[:nh]]
    runs = {}
    for m in modes:
        e_edw, e_gl, _ = MODES[m]
        hkw = dict(c=survey[m]["c"], scalar_bits=BITS, edwards=e_edw, glv=e_gl)
        hws = torch.empty(pkg.msm_g1_host_workspace_bytes(n, **hkw), dtype=torch.uint8, device=dev)
        pkg.msm_g1_host(hp, hsc[0], workspace=hws, **hkw)
        et, outs = [], None
        for j in range(steps):
            t0 = time.perf_counter()
            outs = pkg.msm_g1_host(hp, hsc[j % nh], workspace=hws, **hkw)
            et.append(time.perf_counter() - t0)
        ok = np.array_equal(outs, expected_points(pkg, dev, [ks[(steps - 1) % nh]])[0])
        runs[m] = (sum(et) / len(et), survey[m]["c"], ok)
        del hws
    best = min(runs, key=lambda m: runs[m][0])
    e2e_s, c, ok = runs[best]
    # the prover's step: the points (committed bases) stay resident, every step brings
    # fresh scalars from the host and reads the result back
    e_edw, e_gl, _ = MODES[best]
    rs = pkg.ResidentSet(pts_std, edwards=e_edw, glv=e_gl)
    rws = rs.host_workspace(n)
    rs.msm_host(hsc[0], workspace=rws)
    rt, rout = [], None
    for j in range(steps):
        t0 = time.perf_counter()
        rout = rs.msm_host(hsc[j % nh], workspace=rws)
        rt.append(time.perf_counter() - t0)
    rok = np.array_equal(rout, expected_points(pkg, dev, [ks[(steps - 1) % nh]])[0])
    rs.close()
    del rws
    r_s = sum(rt) / len(rt)
    return {"value": n / e2e_s, "unit": "points/s", "h2d_bytes_per_step": n * (96 + 32),
            "d2h_bytes_per_step": 96, "ms_per_step": 1e3 * e2e_s, "c": c, "verified": bool(ok),
            "call": f"msm_g1_host (pinned host points + scalars, synchronous; mode {best}, "
                    f"points prepared inside the call)",
            "ms_by_mode": {m: round(1e3 * v[0], 3) for m, v in runs.items()},
            "resident_points": {"value": n / r_s, "unit": "points/s", "ms_per_step": 1e3 * r_s,
                                "h2d_bytes_per_step": n * 32, "d2h_bytes_per_step": 96, "verified": bool(rok),
                                "call": f"msm_g1_resident_host (points resident in a library-owned set, "
                                        f"pinned host scalars copied in and the result copied out every step; "
                                        f"mode {best})"}}


def padd_inputs(h, n, edge_rate=0.01, pool_log2=16, tag=1):
    """2^24 mixed additions acc + Q in Montgomery form: acc a pool point in a random XYZZ
    scaling (l^2 x, l^3 y, l^2, l^3), Q a pool point; 1 % each of Q = acc, Q = -acc,
    acc = O and Q = O. Returns the device operands and, per op, the pool indices."""
    pkg, torch, dev = h.pkg, h.torch, h.dev
    m = 1 << pool_log2
    pool_seeds = synth.scalars(synth.stream_seed(tag, n, 20), m)
    std = pkg.to_host(pkg.g1_generator_mul(pkg.to_device(pool_seeds, dev))).reshape(m, 24)
    neg = std.copy()
    p = synth.P_INT
    for i in range(m):   # -P = (x, p - y); no pool point is O
        neg[i, 12:] = synth.int_to_limbs(p - synth.limbs_to_int(std[i, 12:]), 12)
    pool = pkg.msm_points_prepare(pkg.to_device(np.concatenate([std, neg]), dev))   # (2m, 24) Montgomery
    case = torch.from_numpy(synth.workloads.padd_cases(n, tag, edge_rate)).to(dev)
    g = torch.Generator(device=dev).manual_seed(tag)
    i1 = torch.randint(0, m, (n,), device=dev, generator=g)
    i2 = torch.randint(0, m, (n,), device=dev, generator=g)
    i2 = torch.where(case == 1, i1, i2)
    i2 = torch.where(case == 2, i1 + m, i2)
    A, Q = pool[i1], pool[i2]
    lam = torch.randint(-(2 ** 31), 2 ** 31, (12, n), dtype=torch.int32, device=dev, generator=g)
    lam[11] &= 0x00FFFFFF          # below 2^376 < p
    lam[0] |= 1                    # nonzero
    M = pkg.FORM_MONTGOMERY
    l2 = pkg.fq_mul_batch(lam, lam, form=M)
    l3 = pkg.fq_mul_batch(l2, lam, form=M)
    del lam
    acc = torch.empty((4, 12, n), dtype=torch.int32, device=dev)
    pkg.fq_mul_batch(A[:, :12].T.contiguous(), l2, out=acc[0], form=M)
    pkg.fq_mul_batch(A[:, 12:].T.contiguous(), l3, out=acc[1], form=M)
    acc[2] = l2
    acc[3] = l3
    del A, l2, l3
    q = torch.stack([Q[:, :12].T.contiguous(), Q[:, 12:].T.contiguous()])
    del Q
    acc[:, :, case == 3] = 0
    q[:, :, case == 4] = 0
    return acc, q, case, i1, i2, pool_seeds


def padd_expected(h, out, case, i1, i2, pool_seeds, m, samples):
    """Sampled results of the PADD batch against k G from the pool seeds (k = s1 + s2,
    2 s1, 0, s2 or s1 by case)."""
    pkg, torch = h.pkg, h.torch
    idx = torch.tensor(samples, dtype=torch.int64, device=h.dev)
    sub = out[:, :, idx].contiguous()
    aff = pkg.xyzz_to_affine_batch(sub, form=pkg.FORM_MONTGOMERY)
    got = np.stack([pkg.to_host(pkg.fq_from_montgomery(aff[cc].contiguous())) for cc in range(2)])
    cs, a1, a2 = (pkg.to_host(t[idx]).astype(np.int64) for t in (case.to(torch.int32), i1.to(torch.int32),
                                                                      i2.to(torch.int32)))
    ks = []
    for cc, x, y in zip(cs.tolist(), a1.tolist(), a2.tolist()):
        s1 = synth.limbs_to_int(pool_seeds[x])
        s2 = synth.limbs_to_int(pool_seeds[y % m])
        ks.append({0: s1 + s2, 1: 2 * s1, 2: 0, 3: s2, 4: s1}[cc])
    want = expected_points(pkg, h.dev, ks)
    got_rows = np.concatenate([got[0].T, got[1].T], axis=1)
    return bool(np.array_equal(got_rows, want)), {k2: int((cs == k2).sum()) for k2 in range(5)}


def batch_ops(h, peak, hbm_peak, n=1 << 24):
    """2^24 independent Fq multiplications and 2^24 mixed PADDs (1 % edge cases each)."""
    pkg, torch, dev, stream = h.pkg, h.torch, h.dev, h.stream
    a, b = synth.workloads.fq_pairs(n, tag=1)
    mA = pkg.fq_to_montgomery(pkg.to_device(a.T.copy(), dev))
    mB = pkg.fq_to_montgomery(pkg.to_device(b.T.copy(), dev))
    out = torch.empty_like(mA)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_mul = timed(lambda: pkg.fq_mul_batch(mA, mB, out=out, form=pkg.FORM_MONTGOMERY))
    # a sample against Python integers: the product of a R and b R in Montgomery form is (a b) R
    got = pkg.to_host(pkg.fq_from_montgomery(out[:, :4096].contiguous()))
    mul_ok = all(synth.limbs_to_int(got[:, i]) == synth.limbs_to_int(a[i]) * synth.limbs_to_int(b[i]) % synth.P_INT
                 for i in range(0, 4096, 37))
    variants = {}
    for name, v in (("cios", pkg.FQMUL_CIOS), ("barrett", pkg.FQMUL_BARRETT),
                    ("karatsuba", pkg.FQMUL_KARATSUBA), ("carrysave", pkg.FQMUL_CARRYSAVE),
                    ("cios_twopass", pkg.FQMUL_CIOS_TWOPASS), ("cios_doublerow", pkg.FQMUL_CIOS_DOUBLEROW),
                    ("warp_per_product", pkg.FQMUL_WARP), ("paper_25bit_loose_barrett", pkg.FQMUL_PAPER),
                    ("fips", pkg.FQMUL_FIPS), ("cios_singlerow", pkg.FQMUL_CIOS_SINGLEROW)):
        ms_v = timed(lambda v=v: pkg.fq_mul_batch_variant(mA, mB, v, out=out))
        variants[name] = {"ms_2^24": ms_v, "mul_per_s": n / (ms_v / 1e3)}
    del mA, mB, out
    torch.cuda.empty_cache()
    acc, q, case, i1, i2, pool_seeds = padd_inputs(h, n)
    outp = torch.empty_like(acc)
    ms_padd = timed(lambda: pkg.padd_batch(acc, q, out=outp, form=pkg.FORM_MONTGOMERY), reps=3)
    step = max(1, n // 4096)
    samples = sorted(set(range(0, n, step)) | set(torch.nonzero(case != 0)[:512, 0].tolist()))
    padd_ok, counts = padd_expected(h, outp, case, i1, i2, pool_seeds, 1 << 16, samples)
    edge = {nm: float((case == cc).float().mean().item()) for cc, nm in
            ((1, "P+P"), (2, "P+(-P)"), (3, "acc=O"), (4, "Q=O"))}
    del acc, q, outp, case, i1, i2
    torch.cuda.empty_cache()
    mul_rate = n / (ms_mul / 1e3)
    padd_rate = n / (ms_padd / 1e3)
    return {"fq_mul": {"n": n, "ms": ms_mul, "per_s": mul_rate, "verified_sample": bool(mul_ok),
                       "imad_frac": mul_rate * PRODUCTS["fq_mul"] / peak,
                       "hbm_GBps": mul_rate * 144 / 1e9, "hbm_frac": mul_rate * 144 / 1e9 / hbm_peak,
                       "layout": "SoA [12][n], Montgomery form, 144 B per product (two operands + result)"},
            "fq_mul_variants": variants,
            "padd": {"n": n, "ms": ms_padd, "per_s": padd_rate, "edge_case_rates": edge,
                     "verified_sample": bool(padd_ok), "sample_cases": counts,
                     "imad_frac": padd_rate * PRODUCTS["madd"] / peak,
                     "hbm_GBps": padd_rate * 480 / 1e9, "hbm_frac": padd_rate * 480 / 1e9 / hbm_peak,
                     "layout": "XYZZ [4][12][n] + affine [2][12][n] in, XYZZ out, Montgomery form; 480 B per op"},
            "peak_products_per_s": peak}


def latency_chain(h, pts_std, n=1 << 18):
    """Microseconds per mixed PADD of a dependent chain (each addition waits for the
    previous one) over the first n resident points, per model and lane count."""
    pkg, torch, dev, stream = h.pkg, h.torch, h.dev, h.stream
    src = pts_std[:n]
    res = {"n": n, "paper_context_us": {"AIE med-ind (VCK190)": 1.05, "VCK190 CPU (GMP)": 9.69}}
    for name, edw, lanes in (("xyzz_1_lane", False, 1), ("edwards_1_lane", True, 1), ("edwards_4_lanes", True, 4),
                             ("edwards_4_warps", True, 128)):
        st = pkg.msm_points_prepare(src, edwards=edw)
        out = torch.empty(24, dtype=torch.int32, device=dev)
        pkg.padd_chain(st[:1024], 1024, edwards=edw, lanes=lanes, out=out, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pkg.padd_chain(st, n, edwards=edw, lanes=lanes, out=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        res[name + "_us_per_padd"] = 1e3 * e0.elapsed_time(e1) / n
    return res


def batched_msm(h, autotune, edw=False, gl=False, njobs=64, reps=3):
    pkg, torch, dev = h.pkg, h.torch, h.dev
    sizes = synth.workloads.batch_sizes(njobs=njobs, lo_log2=10, hi_log2=20, tag=3).tolist()
    pts, scs, ks = [], [], []
    for i, n in enumerate(sizes):
        seeds = synth.scalars(synth.stream_seed(3, n, 1000 + i), n)
        sc = synth.scalars(synth.stream_seed(3, n, 2000 + i), n)
        pts.append(pkg.msm_points_prepare(pkg.g1_generator_mul(pkg.to_device(seeds, dev)), edwards=edw, glv=gl))
        scs.append(pkg.to_device(sc, dev))
        ks.append(dot_mod_r(sc, seeds))
    mk = dict(edwards=edw, glv=gl)
    cs = [pkg.msm_g1_default_c(n, True, edw, gl) for n in sizes]
    s = torch.cuda.Stream(dev)
    ws = pkg.msm_g1_batched_workspace(pts, scalar_bits=BITS, prepared=True, device=dev, **mk)
    outs = [torch.empty(24, dtype=torch.int32, device=dev) for _ in sizes]
    with torch.cuda.stream(s):
        pkg.msm_g1_batched(pts, scs, outs=outs, workspace=ws, scalar_bits=BITS, prepared=True, stream=s, **mk)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pkg.msm_g1_batched(pts, scs, outs=outs, workspace=ws, scalar_bits=BITS, prepared=True, stream=s, **mk)
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        g.replay()
    e1.record(s)
    torch.cuda.synchronize()
    batched_ms = e0.elapsed_time(e1) / reps
    batched_out = [pkg.to_host(o).copy() for o in outs]
    want = expected_points(pkg, dev, ks)
    ok = all(np.array_equal(o, w) for o, w in zip(batched_out, want))
    del g, ws
    # the same 64 MSMs as 64 msm_g1 calls on one stream (one shared workspace), same table
    wseq = torch.empty(max(_ws_bytes(pkg, n, edw, gl) for n in sizes), dtype=torch.uint8, device=dev)
    seq_outs = [torch.empty(24, dtype=torch.int32, device=dev) for _ in sizes]

    def sequential():
        for i in range(len(sizes)):
            pkg.msm_g1(pts[i], scs[i], out=seq_outs[i], workspace=wseq, scalar_bits=BITS, prepared=True,
                       stream=s, **mk)

    sequential()
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        sequential()
    e1.record(s)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1) / reps
    same = all((pkg.to_host(o) == b).all() for o, b in zip(seq_outs, batched_out))
    total = int(sum(sizes))
    return {"jobs": len(sizes), "points": total, "min_n": int(min(sizes)), "max_n": int(max(sizes)),
            "batched_graph_ms": batched_ms, "sequential_ms": seq_ms, "speedup": seq_ms / batched_ms,
            "batched_points_per_s": total / (batched_ms / 1e3), "results_identical": bool(same),
            "verified": bool(ok), "c_per_job": cs,
            "form": "msm_g1_batched captured in one CUDA graph (persistent accumulation kernel over all "
                    "jobs) vs 64 msm_g1 calls on one stream, both with the installed window tables",
            "mode": ("edwards" if edw else "xyzz") + ("+glv" if gl else "")}


def _ws_bytes(pkg, n, edw, gl):
    import ctypes
    o = pkg._opts(0, True, BITS, True, edwards=edw, glv=gl)
    return int(pkg.lib().msm_g1_workspace_bytes(n, ctypes.byref(o)))


def serve(h, edw=False, gl=False, nreq=2000, nsets=8, set_size=1 << 22, load=0.8):
    pkg, torch, dev = h.pkg, h.torch, h.dev
    from paper_2502_11660_gb300 import serving
    seeds = [synth.scalars(synth.stream_seed(4, set_size, 700 + k), set_size) for k in range(nsets)]
    t0 = time.perf_counter()
    rs = serving.ResidentSets(seeds, device=dev, edwards=edw, glv=gl)
    setup_s = time.perf_counter() - t0
    srv = serving.MsmServer(rs, slots=8, device=dev)
    # capacity from the run's own first 128 requests served back to back, then arrivals
    # at `load` of it in points/s over the whole run's size mix
    unit = serving.poisson_requests(nreq, rate=1.0, nsets=nsets, set_size=set_size, lo_log2=12, hi_log2=22, tag=4)
    calib = unit[:128]
    srv.run(calib[:8], realtime=False)
    cap = srv.run(calib, realtime=False)
    mean_n = float(np.mean([r.n for r in unit]))
    rate = load * cap["points_per_s"] / mean_n
    reqs = serving.poisson_requests(nreq, rate=rate, nsets=nsets, set_size=set_size, lo_log2=12, hi_log2=22, tag=4)
    rep = srv.run(reqs, realtime=True)
    # a few served results against their closed forms (scalars redrawn from the request seeds)
    checks = []
    for r in reqs[:: max(1, nreq // 8)]:
        sc = pkg.to_host(serving.device_scalars(r.n, r.seed, dev)).reshape(r.n, 8)
        k = dot_mod_r(sc, seeds[r.set_id][r.offset:r.offset + r.n])
        checks.append(np.array_equal(rep["results"][r.rid], expected_points(pkg, dev, [k])[0]))
    return {"requests": rep["requests"], "points": rep["points"], "rate_req_per_s": rate,
            "offered_load": rate * mean_n / cap["points_per_s"], "capacity_points_per_s": cap["points_per_s"],
            "capacity_from": "the run's first 128 requests back to back",
            "sustained_points_per_s": rep["points_per_s"], "p50_ms": rep["p50_ms"], "p99_ms": rep["p99_ms"],
            "mean_ms": rep["mean_ms"], "max_inflight": rep["max_inflight"], "slots": 8,
            "verified_sample": bool(all(checks)), "checked": len(checks),
            "mem_budget_GB": rep["mem_budget_bytes"] / 1e9, "max_footprint_GB": rep["max_footprint_bytes"] / 1e9,
            "resident_sets": f"{nsets} x {set_size} points "
                             f"({nsets * pkg.msm_points_prepared_bytes(set_size, edw, gl) / 1e9:.1f} GB stored)",
            "mode": ("edwards" if edw else "xyzz") + ("+glv" if gl else ""),
            "setup_s": setup_s, "n": "log-uniform [2^12, 2^22]",
            "scalars": "fresh per request, drawn on the device from the request seed"}


def run_only(args):
    """One extra alone on cuda:0 (small captures of its kernels); prints its JSON."""
    import torch

    import paper_2502_11660_gb300 as pkg
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    h = Harness(pkg, torch, dev, torch.cuda.current_stream(dev))
    peak = pkg.imad_probe(20000, stream=h.stream)
    print(json.dumps({"batch_ops": batch_ops(h, peak, measured_hbm_peak(), n=args.batch_ops_n)}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        run_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
