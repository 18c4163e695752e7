"""Benchmark: BLS12-377 G1 MSM points/s at n = 2^20 (one step = one msm_g1 call).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n N] [--c C]
                [--mode xyzz|edwards|glv|edwards+glv|edwards+precomputed|edwards+glv+precomputed|best]

Our arm: resident prepared points (prepared once), fresh seeded scalars per
step already in HBM, L2 flushed (256 MB write) between timed steps, per-step
CUDA events on the launch stream. Every curve-model / GLV / fixed-base mode is
autotuned and timed; the headline (`value`) is the fastest mode unless --mode
names one (the workload's points P_i = s_i G lie in the order-r subgroup, which
the Edwards and GLV modes require; the fixed-base modes store 2^(cj) P_i for every
window once per resident set, outside the timed region). Prints one JSON line
(rank 0).
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
X0 = 0x8508C00000000001
R_ORDER = X0 ** 4 - X0 ** 2 + 1
GLV_LAMBDA = X0 * X0 - 1
PROFILE_DIR = os.path.join(ROOT, "profiles")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--c", type=int, default=0)
    ap.add_argument("--mode", default="best", choices=["best"] + list(MODES))
    ap.add_argument("--no-extras", action="store_true", help="skip the e2e, cpu and batch-op extras")
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
                 "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
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


def recorded_traffic(mode: str):
    """DRAM bytes per accumulate launch of `mode` from the committed ncu summary, if it
    matches this source."""
    path = os.path.join(PROFILE_DIR, "accumulate_traffic.json")
    if not os.path.exists(path):
        return None, None
    recs = json.load(open(path))
    rec = recs.get(mode) if isinstance(recs, dict) and "kernel_hash" not in recs else None
    if rec is None or rec.get("kernel_hash") != kernel_hash(MODES[mode][0] or MODES[mode][2]):
        return None, rec
    return rec, rec


def cpu_baseline(n: int, reps_budget_s: float = 12.0):
    """The oracle's C Pippenger (as it stands) on a bounded sample, all host cores."""
    from oracle import coracle
    a, s = synth.workloads.msm(n, tag=2)
    pts = coracle.gen_points(s)
    c = max(4, min(16, int(np.log2(max(n, 2))) - 3))
    t0 = time.perf_counter()
    runs = 0
    while True:
        coracle.msm(pts, a, c=c)
        runs += 1
        if time.perf_counter() - t0 > reps_budget_s or runs >= 20:
            break
    dt = (time.perf_counter() - t0) / runs
    cores = os.cpu_count() or 1
    return {"value": n / dt, "unit": "points/s", "cores": cores, "kind": "oracle",
            "sample": f"textbook Pippenger (plain C, unsigned c={c}), n={n} points, {runs} run(s), "
                      f"{cores} threads over windows"}


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


def op_counts(sc_host: np.ndarray, c: int, bits: int, edwards: bool, glv: bool, pre: bool = False):
    """Additions and doublings of one MSM, and the textbook products of its accumulation."""
    sc = glv_halves(sc_host) if glv else sc_host
    W, nonzero, runs = digit_counts(sc, c, True, 127 if glv else bits, shared=pre)
    madds = nonzero - runs            # the first point of each run is an assignment
    sets = 1 if pre else W            # bucket sets
    full_adds = 2 * sets * (1 << (c - 1))  # running sums of the bucket reduction
    dbls = 0 if pre else (W - 1) * c
    pm = PRODUCTS["ed_madd" if edwards else "madd"]
    return {"windows": W, "madd": madds, "bucket_running_sum_adds": full_adds, "window_dbls": dbls,
            "products_per_madd": pm, "accumulate_products": madds * pm}


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
    n = args.n
    bits = 253
    k = int(np.log2(n))

    # resident point set P_i = s_i G, built on the device and prepared per mode (not timed)
    nsets = args.steps + args.warmup
    seeds, sc_host = rank_workload(n, rank, nsets)
    pts_std = pkg.g1_generator_mul(pkg.to_device(seeds, dev))
    sc_dev = [pkg.to_device(x, dev) for x in sc_host]
    out = torch.empty(24, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed_steps(prep, ws, c, edw, gl, pre, steps, offset, profile):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        stages = []
        for j in range(steps):
            flush.fill_(j & 0xFF)                 # L2 flush between timed steps (outside the events)
            ev[j][0].record(stream)
            pkg.msm_g1(prep, sc_dev[(offset + j) % nsets], out=out, workspace=ws, c=c, scalar_bits=bits,
                       prepared=True, stream=stream, profile=profile, edwards=edw, glv=gl, precomputed=pre)
            ev[j][1].record(stream)
            if profile:
                stages.append(pkg.profile_last())   # synchronises on the step's last event
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev], stages

    # every mode: window width measured on this GPU (the autotuner) unless --c, then a short timing
    survey = {}
    preps = {}
    for name, (edw, gl, pre) in MODES.items():
        if args.mode != "best" and name != args.mode:
            continue
        tuning = None
        if args.c:
            c = args.c
        else:
            tuning = autotune.tune(log2_sizes=[k], reps=3, device=dev, edwards=edw, glv=gl, precomputed=pre)
            autotune.install(tuning["table"], edwards=edw, glv=gl, precomputed=pre)
            c = pkg.msm_g1_default_c(n, True, edw, gl, pre)
        t_prep = time.perf_counter()
        if pre:
            prep = pkg.msm_points_precompute(pts_std, c=c, scalar_bits=bits, glv=gl)
        else:
            prep = pkg.msm_points_prepare(pts_std, edwards=edw, glv=gl)
        torch.cuda.synchronize()
        t_prep = time.perf_counter() - t_prep
        ws = pkg.msm_g1_workspace(n, c=c, scalar_bits=bits, prepared=True, device=dev, edwards=edw, glv=gl,
                                  precomputed=pre)
        for j in range(args.warmup):
            pkg.msm_g1(prep, sc_dev[j], out=out, workspace=ws, c=c, scalar_bits=bits, prepared=True,
                       stream=stream, edwards=edw, glv=gl, precomputed=pre)
        torch.cuda.synchronize()
        ms, st = timed_steps(prep, ws, c, edw, gl, pre, 10, args.warmup, True)
        survey[name] = {"c": c, "ms_per_step": statistics.mean(ms),
                        "points_per_s": world * n / (statistics.mean(ms) / 1e3),
                        "resident_set": {"GB": prep.numel() * 4 / 1e9, "setup_s": t_prep},
                        "stages_ms": {s2: statistics.mean(x[s2] for x in st) for s2 in st[0]},
                        "c_by_autotuner": ({str(cc): round(v, 3) for cc, v in tuning["timings"][k].items()}
                                           if tuning else "given")}
        preps[name] = (prep, ws, c, edw, gl, pre)
    mode = agree_on(min(survey, key=lambda m: survey[m]["ms_per_step"]), world)
    prep, ws, c, edw, gl, pre = preps[mode]
    for other in list(preps):
        if other != mode:
            del preps[other]
    peak = pkg.imad_probe(20000, stream=stream)   # measured limb-product peak (products/s)

    # the timed region: K steps of the headline mode
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = pkg.launch_count()
    t_wall = time.perf_counter()
    step_ms, stage_ms = timed_steps(prep, ws, c, edw, gl, pre, args.steps, args.warmup, True)
    wall = time.perf_counter() - t_wall
    launches = pkg.launch_count() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(sum(step_ms) / len(step_ms), world, dev)
    value = job_points_per_s(n, world, ms)

    ops = op_counts(sc_host[args.warmup], c, bits, edw, gl, pre)
    acc_ms = statistics.mean(x["accumulate"] for x in stage_ms)
    achieved = ops["accumulate_products"] / (acc_ms / 1e3)
    rec, rec_any = recorded_traffic(mode)
    kname = "k_accumulate<%s>" % ("ModelEdwards" if edw else "ModelXyzz")
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved / 1e12, "peak": peak / 1e12,
                "unit": "Tprod/s", "frac": achieved / peak,
                "peak_source": "of measured: msm377_imad_probe (even/odd mad.lo.cc/madc.hi.cc chains, all SMs)",
                "algorithmic_products_per_launch": ops["accumulate_products"],
                "traffic": (rec["bytes_per_launch_full"] if rec else None)}
    padds = ops["madd"] + ops["bucket_running_sum_adds"] + ops["window_dbls"]

    result = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32 (12x32-bit limb Montgomery integer arithmetic)", "data": "synthetic",
        "config": {"workload": f"msm_g1 BLS12-377 G1 n={n}, mode {mode} (signed digits c={c}), resident "
                               f"prepared points{' with per-window shifted copies made once per set' if pre else ''}, "
                               f"fresh scalars per step", "n": n, "c": c, "mode": mode,
                   "windows": ops["windows"],
                   "l2": "flushed between steps (256 MB write, outside the timed events)",
                   "parallelism": f"replicas x{world}"},
        "padd_per_s": world * padds / (ms / 1e3),
        "op_counts": ops,
        "stages_ms": {k2: statistics.mean(x[k2] for x in stage_ms) for k2 in stage_ms[0]},
        "modes": survey,
        "roofline": roofline,
        "gpu_launches": launches,
        "clocks": clk,
        "wall_s_timed_region": wall,
    }

    if rank == 0 and not args.no_extras:
        # End to end through the host-buffer C-ABI call: H2D of points and scalars, the
        # points' preparation, the MSM and the D2H of the result, every step. Each call
        # prepares its points, so the precomputed modes do not apply; the two fastest
        # other modes are timed and the faster end to end is reported.
        pinned_pts = torch.from_numpy(pkg.to_host(pts_std).view(np.int32)).pin_memory()
        hp = pinned_pts.numpy().view(np.uint32)
        hsc = [torch.from_numpy(x.view(np.int32)).pin_memory().numpy().view(np.uint32)
               for x in sc_host[: min(4, nsets)]]
        plain = sorted((m for m in survey if not MODES[m][2]), key=lambda m: survey[m]["ms_per_step"])[:2]
        e2e_runs = {}
        for m in plain or ["edwards+glv"]:
            e_edw, e_gl, _ = MODES[m]
            e_c = survey[m]["c"] if m in survey else pkg.msm_g1_default_c(n, True, e_edw, e_gl)
            hkw = dict(c=e_c, scalar_bits=bits, edwards=e_edw, glv=e_gl)
            hws = torch.empty(pkg.msm_g1_host_workspace_bytes(n, **hkw), dtype=torch.uint8, device=dev)
            pkg.msm_g1_host(hp, hsc[0], workspace=hws, **hkw)
            et = []
            for j in range(args.steps):
                t0 = time.perf_counter()
                pkg.msm_g1_host(hp, hsc[j % len(hsc)], workspace=hws, **hkw)
                et.append(time.perf_counter() - t0)
            e2e_runs[m] = (sum(et) / len(et), e_c)
            del hws
        e2e_mode = min(e2e_runs, key=lambda m: e2e_runs[m][0])
        e2e_s, c = e2e_runs[e2e_mode]
        # batched and serving: the fastest mode without precomputation on the device
        edw, gl, _ = MODES[plain[0] if plain else "edwards+glv"]
        result["e2e"] = {"value": n / e2e_s, "unit": "points/s", "h2d_bytes_per_step": n * (96 + 32),
                         "d2h_bytes_per_step": 96, "ms_per_step": 1e3 * e2e_s,
                         "call": f"msm_g1_host (pinned host points + scalars, synchronous; mode {e2e_mode}, "
                                 f"points prepared inside the call)",
                         "ms_by_mode": {m: round(1e3 * v[0], 3) for m, v in e2e_runs.items()}}
        # standalone batched arithmetic at 2^24 (Fq Montgomery multiplications, mixed PADDs)
        result["batch_ops"] = batch_ops(pkg, torch, dev, stream)
        # the paper's dependent-chain experiment: 2^18 points summed in order
        result["latency"] = latency_chain(pkg, torch, dev, stream, pts_std)
        # 64 MSMs of log-uniform n in [2^10, 2^20]: one graph launch vs 64 sequential calls
        result["batched_msm"] = batched_msm(pkg, torch, dev, edw, gl)
        # 2000 Poisson requests over 8 resident sets of 2^22 points
        result["serving"] = serve(pkg, torch, dev, edw, gl)
        result["cpu_baseline"] = cpu_baseline(1 << 16)

    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


def batched_msm(pkg, torch, dev, edw=False, gl=False, njobs=64, reps=3):
    sizes = synth.workloads.batch_sizes(njobs=njobs, lo_log2=10, hi_log2=20, tag=3).tolist()
    pts, scs = [], []
    for i, n in enumerate(sizes):
        seeds = synth.scalars(synth.stream_seed(3, n, 1000 + i), n)
        pts.append(pkg.msm_points_prepare(pkg.g1_generator_mul(pkg.to_device(seeds, dev)), edwards=edw, glv=gl))
        scs.append(pkg.to_device(synth.scalars(synth.stream_seed(3, n, 2000 + i), n), dev))
    bits = 253
    mk = dict(edwards=edw, glv=gl)
    s = torch.cuda.Stream(dev)
    ws = pkg.msm_g1_batched_workspace(pts, scalar_bits=bits, prepared=True, device=dev, **mk)
    outs = [torch.empty(24, dtype=torch.int32, device=dev) for _ in sizes]
    with torch.cuda.stream(s):
        pkg.msm_g1_batched(pts, scs, outs=outs, workspace=ws, scalar_bits=bits, prepared=True, stream=s, **mk)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pkg.msm_g1_batched(pts, scs, outs=outs, workspace=ws, scalar_bits=bits, prepared=True, stream=s, **mk)
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
    del g, ws
    # the same 64 MSMs as 64 msm_g1 calls on one stream (one shared workspace)
    wseq = pkg.msm_g1_workspace(max(sizes), scalar_bits=bits, prepared=True, device=dev, **mk)
    seq_outs = [torch.empty(24, dtype=torch.int32, device=dev) for _ in sizes]

    def sequential():
        for i in range(len(sizes)):
            pkg.msm_g1(pts[i], scs[i], out=seq_outs[i], workspace=wseq, scalar_bits=bits, prepared=True,
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
            "form": "msm_g1_batched captured in one CUDA graph (persistent accumulation kernel over all "
                    "jobs) vs 64 msm_g1 calls on one stream",
            "mode": ("edwards" if edw else "xyzz") + ("+glv" if gl else "")}


def serve(pkg, torch, dev, edw=False, gl=False, nreq=2000, nsets=8, set_size=1 << 22, load=0.8):
    from paper_2502_11660_gb300 import serving
    seeds = [synth.scalars(synth.stream_seed(4, set_size, 700 + k), set_size) for k in range(nsets)]
    t0 = time.perf_counter()
    rs = serving.ResidentSets(seeds, device=dev, edwards=edw, glv=gl)
    setup_s = time.perf_counter() - t0
    srv = serving.MsmServer(rs, slots=8, device=dev)
    # sustained capacity from a back-to-back burst of the same size mix, then 0.8 of it
    calib = serving.poisson_requests(48, rate=1.0, nsets=nsets, set_size=set_size, lo_log2=12, hi_log2=22, tag=5)
    srv.run(calib[:8], realtime=False)
    cap = srv.run(calib, realtime=False)
    mean_n = float(np.mean([r.n for r in calib]))
    rate = load * cap["points_per_s"] / mean_n
    reqs = serving.poisson_requests(nreq, rate=rate, nsets=nsets, set_size=set_size, lo_log2=12, hi_log2=22, tag=4)
    rep = srv.run(reqs, realtime=True)
    return {"requests": rep["requests"], "points": rep["points"], "rate_req_per_s": rate,
            "offered_load": load, "capacity_points_per_s": cap["points_per_s"],
            "sustained_points_per_s": rep["points_per_s"], "p50_ms": rep["p50_ms"], "p99_ms": rep["p99_ms"],
            "mean_ms": rep["mean_ms"], "max_inflight": rep["max_inflight"], "slots": 8,
            "mem_budget_GB": rep["mem_budget_bytes"] / 1e9, "max_footprint_GB": rep["max_footprint_bytes"] / 1e9,
            "resident_sets": f"{nsets} x {set_size} points "
                             f"({nsets * pkg.msm_points_prepared_bytes(set_size, edw, gl) / 1e9:.1f} GB stored)",
            "mode": ("edwards" if edw else "xyzz") + ("+glv" if gl else ""),
            "setup_s": setup_s, "n": "log-uniform [2^12, 2^22]",
            "scalars": "fresh per request, drawn on the device from the request seed"}


def latency_chain(pkg, torch, dev, stream, pts_std, n=1 << 18):
    """Microseconds per mixed PADD of a dependent chain (each addition waits for the
    previous one) over the first n resident points, per model and lane count."""
    src = pts_std[:n]
    res = {"n": n, "paper_context_us": {"AIE med-ind (VCK190)": 1.05, "VCK190 CPU (GMP)": 9.69}}
    for name, edw, lanes in (("xyzz_1_lane", False, 1), ("edwards_1_lane", True, 1), ("edwards_4_lanes", True, 4)):
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


def batch_ops(pkg, torch, dev, stream):
    n = 1 << 24
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
    # the alternative multiplications on the same operands (variants: Sec. III-C Barrett,
    # Karatsuba top level, radix-2^24 carry-save, two-pass CIOS rows), one kernel each
    variants = {}
    for name, v in (("cios", pkg.FQMUL_CIOS), ("barrett", pkg.FQMUL_BARRETT),
                    ("karatsuba", pkg.FQMUL_KARATSUBA), ("carrysave", pkg.FQMUL_CARRYSAVE),
                    ("cios_twopass", pkg.FQMUL_CIOS_TWOPASS), ("cios_doublerow", pkg.FQMUL_CIOS_DOUBLEROW)):
        ms_v = timed(lambda v=v: pkg.fq_mul_batch_variant(mA, mB, v, out=out))
        variants[name] = {"ms_2^24": ms_v, "mul_per_s": n / (ms_v / 1e3)}
    del mA, mB, out
    # mixed PADDs on a pool of 2^16 device-generated points, XYZZ accumulators with ZZ = ZZZ = R
    pool = pkg.g1_generator_mul(pkg.to_device(synth.scalars(3, 1 << 16), dev))
    mpool = pkg.msm_points_prepare(pool)
    g = torch.Generator(device=dev).manual_seed(7)
    i1 = torch.randint(0, 1 << 16, (n,), device=dev, generator=g)
    i2 = torch.randint(0, 1 << 16, (n,), device=dev, generator=g)
    P, Q = mpool[i1], mpool[i2]
    one = pkg.fq_to_montgomery(pkg.to_device(np.eye(12, 1, dtype=np.uint32).reshape(12, 1), dev))
    acc = torch.empty((4, 12, n), dtype=torch.int32, device=dev)
    acc[0] = P[:, :12].T
    acc[1] = P[:, 12:].T
    acc[2] = one.expand(12, n)
    acc[3] = one.expand(12, n)
    q = torch.stack([Q[:, :12].T.contiguous(), Q[:, 12:].T.contiguous()])
    del P, Q, i1, i2
    outp = torch.empty_like(acc)
    ms_padd = timed(lambda: pkg.padd_batch(acc, q, out=outp, form=pkg.FORM_MONTGOMERY), reps=3)
    return {"fq_mul_per_s": n / (ms_mul / 1e3), "fq_mul_ms_2^24": ms_mul, "fq_mul_variants": variants,
            "fq_mul_hbm_GBps": n * 144 / (ms_mul / 1e3) / 1e9,
            "padd_per_s": n / (ms_padd / 1e3), "padd_ms_2^24": ms_padd,
            "padd_products_per_s": n * PRODUCTS["madd"] / (ms_padd / 1e3)}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
