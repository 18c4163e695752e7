"""Continuous-batching MSM server over resident point sets (one GPU).

Requests name a resident point set, an offset into it and a length n; each
brings fresh scalars. The host loop admits arrived requests while a slot (a CUDA
stream) is free and the HBM footprint of everything in flight (workspace +
scalars) stays within a budget, enqueues msm_g1_resident on the slot's stream over
the resident set, and retires requests whose completion event has
fired. Requests that arrive while others run are admitted as soon as a slot and
memory free up, so their work overlaps on the device. Latency is measured from
a request's arrival to the host seeing its completion event.

Scalars are drawn on the device per request from the request's own seed (like
witness-derived scalars that already live on the GPU in a prover); every GPU
step is a call into libmsm377. Each slot keeps its own device buffers (workspace,
scalars, result), grown to the largest request it has served and reused by the
next request on the same stream, so a warm server allocates nothing per request
(the memory budget still admits requests by their own footprint). With GLV the stored set interleaves P_i and
phi(P_i), so a request's slice is still one contiguous range of rows.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np
import torch

from . import ResidentSet, g1_generator_mul, to_device, to_host


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float   # seconds after the start of the run
    set_id: int
    offset: int
    n: int
    seed: int


@dataclasses.dataclass
class Done:
    rid: int
    latency: float
    start_delay: float
    result: np.ndarray


def device_scalars(n: int, seed: int, device, out: torch.Tensor | None = None) -> torch.Tensor:
    """n scalars uniform in [0, 2^252) (below r), drawn on the device from `seed`
    (into `out`, an (n, 8) int32 view, when given)."""
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    if out is None:
        sc = torch.randint(-(2 ** 31), 2 ** 31, (n, 8), dtype=torch.int32, device=device, generator=g)
    else:
        sc = torch.randint(-(2 ** 31), 2 ** 31, (n, 8), dtype=torch.int32, device=device, generator=g, out=out)
    sc[:, 7] &= 0x0FFFFFFF
    return sc


class ResidentSets:
    """Resident point sets P_i = s_i G held by the library (msm_points_create): the
    stored form for one curve model (XYZZ Montgomery affine, or the Edwards stored form;
    with GLV interleaved with phi(P_i); or fixed-base copies for one window width)."""

    def __init__(self, seeds: list[np.ndarray], device="cuda", edwards: bool = False, glv: bool = False,
                 precompute_c: int = 0, validate: bool = False):
        """precompute_c > 0: fixed-base sets (Edwards, 2^(c j) P_i for every window j) made for
        that window width, which every request then uses."""
        self.edwards, self.glv, self.c = edwards or precompute_c > 0, glv, precompute_c
        self.sets: list[ResidentSet] = []
        for s in seeds:
            pts = g1_generator_mul(to_device(s, device))
            self.sets.append(ResidentSet(pts, edwards=edwards, glv=glv, precompute_c=precompute_c,
                                         scalar_bits=253, validate=validate))
            del pts
        torch.cuda.synchronize(device)

    def set(self, set_id: int) -> ResidentSet:
        return self.sets[set_id]

    def close(self) -> None:
        for s in self.sets:
            s.close()
        self.sets = []


class MsmServer:
    def __init__(self, sets: ResidentSets, slots: int = 8, mem_budget: int | None = None, device="cuda"):
        self.sets = sets
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        # per slot: workspace bytes, scalar words and the 24-word result, grown on demand
        self.arenas: list[dict] = [{"ws": None, "sc": None, "out": None} for _ in range(slots)]
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            mem_budget = int(free * 0.5)
        self.mem_budget = mem_budget

    def footprint(self, n: int) -> int:
        """Device bytes a request of n points holds while in flight: its workspace, its
        scalars and its result."""
        return self.sets.set(0).workspace_bytes(n) + 32 * n + 96

    def _buffers(self, slot: int, rs: ResidentSet, n: int):
        """The slot's buffers, grown to hold a request of n points. The slot's previous
        request has completed (a slot is reused only after its event fired), so
        replacing or reusing them is safe."""
        a = self.arenas[slot]
        need = rs.workspace_bytes(n)
        if a["ws"] is None or a["ws"].numel() < need:
            a["ws"] = torch.empty(need, dtype=torch.uint8, device=self.device)
        if a["sc"] is None or a["sc"].shape[0] < n:
            a["sc"] = torch.empty((n, 8), dtype=torch.int32, device=self.device)
        if a["out"] is None:
            a["out"] = torch.empty(24, dtype=torch.int32, device=self.device)
        return a["ws"], a["sc"][:n], a["out"]

    def _launch(self, req: Request, slot: int):
        st = self.streams[slot]
        with torch.cuda.stream(st):
            rs = self.sets.set(req.set_id)
            ws, sc_buf, out = self._buffers(slot, rs, req.n)
            sc = device_scalars(req.n, req.seed, self.device, out=sc_buf)
            rs.msm(sc, offset=req.offset, out=out, workspace=ws, stream=st)
            ev = torch.cuda.Event()
            ev.record(st)
        return {"req": req, "slot": slot, "event": ev, "out": out, "tensors": (sc, ws),
                "need": self.footprint(req.n)}

    def run(self, requests: list[Request], realtime: bool = True) -> dict:
        """Serves `requests` (arrival times relative to the start); returns a report."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        inflight = []
        free = list(range(len(self.streams)))
        used = 0
        done: list[Done] = []
        max_inflight = 0
        max_used = 0
        t0 = time.perf_counter()
        while pending or inflight:
            now = time.perf_counter() - t0
            progressed = False
            while pending and free and (not realtime or pending[0].arrival <= now):
                need = self.footprint(pending[0].n)
                if used + need > self.mem_budget and inflight:
                    break                      # wait for memory to free up
                req = pending.popleft()
                item = self._launch(req, free.pop())
                item["t_start"] = time.perf_counter() - t0
                used += item["need"]
                inflight.append(item)
                progressed = True
            max_inflight = max(max_inflight, len(inflight))
            max_used = max(max_used, used)
            for item in list(inflight):
                if item["event"].query():
                    t = time.perf_counter() - t0
                    req = item["req"]
                    arrival = req.arrival if realtime else 0.0
                    done.append(Done(req.rid, t - arrival, item["t_start"] - arrival,
                                     to_host(item["out"]).copy()))
                    free.append(item["slot"])
                    used -= item["need"]
                    inflight.remove(item)
                    progressed = True
            if not progressed:
                if pending and realtime and not inflight:
                    time.sleep(max(0.0, min(0.001, pending[0].arrival - (time.perf_counter() - t0))))
                else:
                    time.sleep(20e-6)
        makespan = time.perf_counter() - t0
        lat = np.array([d.latency for d in done])
        points = int(sum(r.n for r in requests))
        return {
            "requests": len(done),
            "points": points,
            "makespan_s": makespan,
            "points_per_s": points / makespan if makespan > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
            "mean_ms": float(lat.mean() * 1e3) if len(lat) else None,
            "max_inflight": max_inflight,
            "max_footprint_bytes": max_used,
            "mem_budget_bytes": self.mem_budget,
            "results": {d.rid: d.result for d in done},
            "latencies": {d.rid: d.latency for d in done},
        }


def poisson_requests(nreq: int, rate: float, nsets: int, set_size: int, lo_log2: float, hi_log2: float,
                     tag: int = 4) -> list[Request]:
    """Poisson arrivals at `rate` per second; n log-uniform in [2^lo, 2^hi]; 256-aligned offsets."""
    import synth
    gaps, n, sets, offs = synth.workloads.requests(nreq, lo_log2, hi_log2, nsets, set_size, tag)
    arrival = np.cumsum(gaps) / rate
    seeds = synth.splitmix64(synth.stream_seed(tag, nreq, 99), nreq)
    return [Request(i, float(arrival[i]), int(sets[i]), int(offs[i]), int(n[i]), int(seeds[i]))
            for i in range(nreq)]
