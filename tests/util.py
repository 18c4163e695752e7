"""Test helpers: limb conversions, oracle-side normalisation, cached oracle point sets."""
from __future__ import annotations

import numpy as np

import synth
from oracle import coracle, fq, g1

_POINTS: dict = {}


def ints_of_soa(arr: np.ndarray) -> list[int]:
    """[12][n] u32 -> list of n ints."""
    a = np.asarray(arr, dtype=np.uint64)
    out = [0] * a.shape[1]
    for k in range(a.shape[0]):
        col = a[k].tolist()
        for i, w in enumerate(col):
            out[i] |= int(w) << (32 * k)
    return out


def soa_of_ints(vals, nlimbs: int = 12) -> np.ndarray:
    out = np.zeros((nlimbs, len(vals)), dtype=np.uint32)
    for i, v in enumerate(vals):
        for k in range(nlimbs):
            out[k, i] = (v >> (32 * k)) & 0xFFFFFFFF
    return out


def xyzz_to_affine_int(X: int, Y: int, ZZ: int, ZZZ: int):
    """Oracle-side normalisation x = X/ZZ, y = Y/ZZZ; ZZ = 0 is O."""
    if ZZ % fq.P == 0:
        return None
    return (X * fq.inv(ZZ) % fq.P, Y * fq.inv(ZZZ) % fq.P)


def oracle_points(seeds: np.ndarray, key=None) -> np.ndarray:
    """P_i = seeds_i * G from the C oracle, cached per key within the session."""
    if key is not None and key in _POINTS:
        return _POINTS[key]
    pts = coracle.gen_points(seeds)
    if key is not None:
        _POINTS[key] = pts
    return pts


def msm_inputs(n: int, tag: int):
    a, s = synth.workloads.msm(n, tag)
    return a, s, oracle_points(s, key=("msm", n, tag))


def dot_plain(scalars: np.ndarray, seeds: np.ndarray) -> int:
    """sum_i a_i s_i over Python integers, term by term."""
    k = 0
    for a, s in zip(scalars, seeds):
        k += synth.limbs_to_int(a) * synth.limbs_to_int(s)
    return k


def dot_fast(scalars: np.ndarray, seeds: np.ndarray) -> int:
    """The same sum, exactly, for large n: the 16-bit halves of the limbs give 16 x 16
    dot products of terms below 2^32; over chunks of 2^18 rows each partial sum stays
    below 2^50, so float64 matrix products carry it without rounding."""
    total = 0
    for lo in range(0, scalars.shape[0], 1 << 18):
        a16 = np.ascontiguousarray(scalars[lo:lo + (1 << 18)], dtype=np.uint32).view(np.uint16).astype(np.float64)
        s16 = np.ascontiguousarray(seeds[lo:lo + (1 << 18)], dtype=np.uint32).view(np.uint16).astype(np.float64)
        m = a16.T @ s16
        for u in range(16):
            for v in range(16):
                total += int(m[u, v]) << (16 * (u + v))
    return total


_CLOSED: dict = {}


def closed_form_limbs(seeds: np.ndarray, scalars: np.ndarray, key=None):
    """Expected MSM result sum a_i (s_i G) = ((sum a_i s_i) mod r) G, as an affine point
    (cached per key within the session when a key is given)."""
    if key is not None and key in _CLOSED:
        return _CLOSED[key]
    k = dot_plain(scalars, seeds) if len(seeds) <= 4096 else dot_fast(scalars, seeds)
    pt = g1.mul(k % fq.R, g1.G)
    if key is not None:
        _CLOSED[key] = pt
    return pt
