"""Window-width autotuner for msm_g1 (signed digits).

For each size n = 2^k it times msm_g1 on the device (resident prepared points,
fresh scalars) for every candidate c, keeps the fastest, and installs the table
into the library (msm_g1_set_window_table), so every later call with c = 0 --
single, batched or served -- uses the measured choice. The library keeps one
table per curve model / GLV combination; tune and install the one you run.
Tables can be saved to and loaded from a JSON file keyed by the device name.

One synthetic point set of the largest size tuned is generated on the device and
prepared once per curve model; smaller sizes time a prefix of it. tune_schedule()
also searches, per size, the accumulation chunk size, the sort and the bucket
reduction's parallelism (msm_g1_set_schedule), one coordinate at a time.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np
import torch

from . import (PRECOMPUTED, _model_flags, g1_generator_mul, lib, msm_g1, msm_g1_default_c, msm_g1_workspace,
               msm_points_precompute, msm_points_prepare, to_device)
from ._lib import check

# variable-base window widths searched at large n (the BLS12-377 MSM configuration
# of 2^20 and 2^22 points: c from 12 to 17)
LARGE_C = tuple(range(12, 18))
# fixed-base sets: every window adds into one bucket set, so wider windows pay
PRECOMPUTED_C = tuple(range(15, 21))

_SETS: dict = {}


def _point_set(n: int, device, seed: int, edwards: bool, glv: bool):
    """Stored points for n (a prefix of one cached set per model and device)."""
    dev = torch.device(device)
    key = (str(dev), seed, bool(edwards), bool(glv))
    have = _SETS.get(key)
    if have is None or have[0] < n:
        import synth
        std = g1_generator_mul(to_device(synth.scalars(seed, n), dev))
        _SETS[key] = (n, std, msm_points_prepare(std, edwards=edwards, glv=glv))
    _, std, prep = _SETS[key]
    rows = prep.shape[0] // std.shape[0]
    return std[:n], prep[:rows * n]


def clear_cache() -> None:
    _SETS.clear()


def time_msm(n: int, c: int, reps: int = 3, device="cuda", seed: int = 11, edwards: bool = False,
             glv: bool = False, precomputed: bool = False) -> float:
    """Median milliseconds of one msm_g1 call with window c at size n (a precomputed
    set is built for each c, outside the timing)."""
    import synth
    std, prep = _point_set(n, device, seed, edwards or precomputed, glv)
    if precomputed:
        pts = msm_points_precompute(std, c=c, scalar_bits=253, glv=glv)
    else:
        pts = prep
    sc = to_device(synth.scalars(seed + 1, n), device)
    kw = dict(c=c, scalar_bits=253, prepared=True, edwards=edwards or precomputed, glv=glv,
              precomputed=precomputed)
    ws = msm_g1_workspace(n, device=device, **kw)
    out = torch.empty(24, dtype=torch.int32, device=device)
    msm_g1(pts, sc, out=out, workspace=ws, **kw)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        msm_g1(pts, sc, out=out, workspace=ws, **kw)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    del ws, pts
    return float(np.median(times))


def candidates(log2n: int, glv: bool = False, precomputed: bool = False) -> list[int]:
    """Window widths to time at n = 2^log2n: 12..17 for the large sizes (15..20 for
    fixed-base sets); around the built-in rule below 2^16."""
    if log2n >= 16:
        return list(PRECOMPUTED_C if precomputed else LARGE_C)
    base = max(4, log2n - 4 + (1 if glv else 0))
    return sorted({max(3, base - 2), max(3, base - 1), base, base + 1, base + 2})


# Window widths timed within this fraction of the fastest count as a tie (about the
# run-to-run spread of these timings on GB300: at n = 2^16, c = 12 and c = 16 came out
# 0.4 % apart in one run and 1.4 % apart, either way, in two others), and the widest is
# kept: fewer windows mean fewer mixed additions, which is what counts when several MSMs
# share the GPU (batched calls, serving).
C_TIE = 0.01


def pick_c(t: dict) -> int:
    """The widest window among those timed within C_TIE of the fastest."""
    best = min(t.values())
    return max(c for c, ms in t.items() if ms <= best * (1 + C_TIE))


def tune(log2_sizes=range(10, 23, 2), reps: int = 3, device="cuda", edwards: bool = False,
         glv: bool = False, precomputed: bool = False) -> dict:
    """Returns {"table": [c by log2 n], "timings": {k: {c: ms}}}; fills gaps from neighbours."""
    timings = {}
    best = {}
    for k in log2_sizes:
        n = 1 << k
        t = {c: time_msm(n, c, reps, device, edwards=edwards, glv=glv, precomputed=precomputed)
             for c in candidates(k, glv, precomputed)}
        timings[k] = t
        best[k] = pick_c(t)
    table = [0] * 32
    keys = sorted(best)
    for k in range(32):
        if keys:
            near = min(keys, key=lambda q: (abs(q - k), q))
            if abs(near - k) <= 2:
                table[k] = best[near]
    return {"table": table, "timings": timings, "device": torch.cuda.get_device_name(device),
            "edwards": edwards, "glv": glv, "precomputed": precomputed}


def time_schedule(n: int, c: int, chunk: int, sort: int, reduce_log2: int, groups: int = 0, reps: int = 3,
                  device="cuda", seed: int = 11, edwards: bool = False, glv: bool = False) -> float:
    """Median milliseconds of msm_g1 at size n with one schedule entry installed for 2^floor(log2 n)."""
    from . import msm_g1_set_schedule
    k = int(np.log2(n))
    msm_g1_set_schedule(k, c, chunk, sort, reduce_log2, groups, edwards=edwards, glv=glv)
    return time_msm(n, 0, reps, device, seed, edwards=edwards, glv=glv)


# chunk sizes (items per accumulation thread), sorts (1 counting, 2 radix), level-1
# reduction thread counts and window groups searched after the window width
CHUNKS = (0, 16, 32, 48, 64, 96, 128)
SORTS = (1, 2)
REDUCE_LOG2 = (0, 13, 14, 16, 17)
GROUPS = (1, 2, 4)


def tune_schedule(log2_sizes=range(10, 23), reps: int = 3, device="cuda", edwards: bool = False,
                  glv: bool = False) -> dict:
    """Per size: the window width c (candidates as in tune(), ties to the widest), then, at that c, the chunk
    size, the sort, the number of level-1 reduction threads and the window groups, one
    coordinate at a time (each step keeps the fastest value; 0 = the built-in rule).
    Installs every entry as it goes and returns {"schedule": {k: (c, chunk, sort,
    reduce_log2, groups)}, "ms": {k: {field: {value: ms}}}}."""
    sched, ms = {}, {}
    for k in log2_sizes:
        n = 1 << k
        cur = [0, 0, 0, 0, 0]
        rec = {}
        t = {c: time_schedule(n, c, 0, 0, 0, 0, reps, device, edwards=edwards, glv=glv)
             for c in candidates(k, glv)}
        cur[0] = pick_c(t)
        rec["c"] = t
        for field, values in ((1, CHUNKS), (2, SORTS), (3, REDUCE_LOG2), (4, GROUPS)):
            t = {}
            for v in values:
                trial = list(cur)
                trial[field] = v
                t[v] = time_schedule(n, *trial, reps=reps, device=device, edwards=edwards, glv=glv)
            cur[field] = min(t, key=t.get)
            rec[("c", "chunk", "sort", "reduce_log2", "groups")[field]] = t
        from . import msm_g1_set_schedule
        msm_g1_set_schedule(k, *cur, edwards=edwards, glv=glv)
        sched[k] = tuple(cur)
        ms[k] = rec
    return {"schedule": sched, "ms": ms, "device": torch.cuda.get_device_name(device), "edwards": edwards,
            "glv": glv}


def install_schedule(schedule: dict, edwards: bool = False, glv: bool = False) -> None:
    from . import msm_g1_set_schedule
    for k, entry in schedule.items():
        msm_g1_set_schedule(int(k), *[int(x) for x in entry], edwards=edwards, glv=glv)


def clear_schedule(edwards: bool = False, glv: bool = False, precomputed: bool = False) -> None:
    from . import msm_g1_set_schedule
    for k in range(32):
        msm_g1_set_schedule(k, 0, 0, 0, 0, 0, edwards=edwards, glv=glv, precomputed=precomputed)


def save_schedule(result: dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump({"device": result.get("device"), "edwards": result.get("edwards"), "glv": result.get("glv"),
                   "schedule": {str(k): list(v) for k, v in result["schedule"].items()}}, f, indent=1)


def load_schedule(path: str) -> dict | None:
    """A saved schedule table, if it was measured on this device model."""
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    if torch.cuda.is_available() and rec.get("device") != torch.cuda.get_device_name():
        return None
    return rec


def _flags(edwards: bool, glv: bool, precomputed: bool) -> int:
    return _model_flags(edwards or precomputed, glv) | (PRECOMPUTED if precomputed else 0)


def install(table, edwards: bool = False, glv: bool = False, precomputed: bool = False) -> None:
    arr = (ctypes.c_int32 * len(table))(*[int(x) for x in table])
    check(lib().msm_g1_set_window_table(arr, len(table), _flags(edwards, glv, precomputed)))


def clear(edwards: bool = False, glv: bool = False, precomputed: bool = False) -> None:
    check(lib().msm_g1_set_window_table(None, 0, _flags(edwards, glv, precomputed)))


def save(result: dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump({"table": result["table"], "device": result.get("device"),
                   "timings": {str(k): {str(c): v for c, v in t.items()} for k, t in result["timings"].items()}},
                  f, indent=1)


def load(path: str) -> dict | None:
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def current_choice(n: int, edwards: bool = False, glv: bool = False, precomputed: bool = False) -> int:
    return msm_g1_default_c(n, True, edwards or precomputed, glv, precomputed)
