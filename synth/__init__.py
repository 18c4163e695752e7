"""Seeded synthetic inputs shared by the CUDA path's tests, the bench and the oracle.

This module draws random numbers and nothing else: it holds none of the field or
curve arithmetic of the method (no modular multiplication, no point operations).
Curve points P_i = s_i*G are therefore NOT produced here; only their seeds s_i are.
Each side computes the points from those seeds with its own arithmetic.

Generator: splitmix64 used as a counter-based stream (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): word i of stream
`seed` is mix64(seed + (i + 1) * 0x9E3779B97F4A7C15) with the published
finaliser constants. It vectorises in numpy, so 2^22 scalars take well under a
second.

Workload recipes (sizes and distributions of the MSM workloads: a single MSM of
n = 2^12 with c = 8 unsigned digits, independent Fq multiplications and mixed
point additions at 2^24, single MSMs at 2^20 and 2^22, a batch of 64 MSMs with
log-uniform n in [2^10, 2^20], and a Poisson request stream with log-uniform n in
[2^12, 2^22]) live in `workloads` below.
"""
from __future__ import annotations

import numpy as np

# Public BLS12-377 parameters, used here only as rejection bounds for uniform
# draws (no arithmetic modulo them happens in this module).
P_HEX = ("01ae3a4617c510eac63b05c06ca1493b1a22d9f300f5138f"
         "1ef3622fba094800170b5d44300000008508c00000000001")
R_HEX = "12ab655e9a2ca55660b44d1e5c37b00159aa76fed00000010a11800000000001"
P_INT = int(P_HEX, 16)
R_INT = int(R_HEX, 16)

BASE_SEED = 0x250211660

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def stream_seed(*tags: int) -> int:
    """Derive a 64-bit stream seed from the base seed and integer tags."""
    s = BASE_SEED
    for t in tags:
        s = int(splitmix64(s ^ (int(t) * 0x632BE59BD9B4E019 & 0xFFFFFFFFFFFFFFFF), 1)[0])
    return s


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Words start..start+count-1 of the counter-based splitmix64 stream `seed`."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _words_of(value: int, nwords: int) -> np.ndarray:
    return np.array([(value >> (64 * k)) & 0xFFFFFFFFFFFFFFFF for k in range(nwords)],
                    dtype=np.uint64)


def _below(cand: np.ndarray, bound_words: np.ndarray) -> np.ndarray:
    """Row-wise cand < bound for little-endian u64 words (lexicographic from the top)."""
    n, w = cand.shape
    less = np.zeros(n, dtype=bool)
    decided = np.zeros(n, dtype=bool)
    for k in range(w - 1, -1, -1):
        lt = cand[:, k] < bound_words[k]
        gt = cand[:, k] > bound_words[k]
        less |= ~decided & lt
        decided |= lt | gt
    return less


def _uniform_below(seed: int, n: int, bound: int, nwords: int, topbits: int) -> np.ndarray:
    """n uniform integers in [0, bound) as (n, nwords) little-endian u64 words."""
    bw = _words_of(bound, nwords)
    mask = np.uint64((1 << topbits) - 1)
    out = np.empty((0, nwords), dtype=np.uint64)
    drawn = 0
    while out.shape[0] < n:
        want = max(1024, int((n - out.shape[0]) * 1.8))
        raw = splitmix64(seed, want * nwords, start=drawn * nwords).reshape(want, nwords)
        drawn += want
        raw[:, nwords - 1] &= mask
        out = np.concatenate([out, raw[_below(raw, bw)]], axis=0)
    return np.ascontiguousarray(out[:n])


def scalars(seed: int, n: int) -> np.ndarray:
    """n scalars uniform in [0, r) as (n, 8) little-endian u32 limbs."""
    w = _uniform_below(seed, n, R_INT, 4, 253 - 192)
    return w.view(np.uint32).reshape(n, 8)


def scalars_full(seed: int, n: int) -> np.ndarray:
    """n scalars uniform in [0, 2^256) as (n, 8) u32 limbs (accepted, not reduced mod r)."""
    return splitmix64(seed, 4 * n).view(np.uint32).reshape(n, 8).copy()


def field_elems(seed: int, n: int) -> np.ndarray:
    """n elements uniform in [0, p) as (n, 12) little-endian u32 limbs."""
    w = _uniform_below(seed, n, P_INT, 6, 377 - 320)
    return w.view(np.uint32).reshape(n, 12)


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles uniform in [0, 1) from the top 53 bits of the stream."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def small_ints(seed: int, n: int, hi: int) -> np.ndarray:
    """n integers uniform in [0, hi) (hi small; modulo bias below 2^-40)."""
    return (splitmix64(seed, n) % np.uint64(hi)).astype(np.int64)


def limbs_to_int(row) -> int:
    """Little-endian u32 limbs to a Python int (a format helper, no arithmetic mod p)."""
    v = 0
    for k, w in enumerate(np.asarray(row, dtype=np.uint64).tolist()):
        v |= int(w) << (32 * k)
    return v


def int_to_limbs(v: int, nlimbs: int) -> np.ndarray:
    return np.array([(v >> (32 * k)) & 0xFFFFFFFF for k in range(nlimbs)], dtype=np.uint32)


class workloads:
    """Seeded recipes for each workload. Every recipe returns plain arrays."""

    @staticmethod
    def msm(n: int, tag: int):
        """Single MSM: scalars a_i uniform in [0, r) and point seeds s_i uniform in [0, r).

        The points are P_i = s_i * G; knowing s_i gives the closed form
        sum_i a_i P_i = ((sum_i a_i s_i) mod r) * G.
        """
        a = scalars(stream_seed(tag, n, 1), n)
        s = scalars(stream_seed(tag, n, 2), n)
        return a, s

    @staticmethod
    def fq_pairs(n: int, tag: int):
        """Independent Fq multiplications: a, b uniform in [0, p)."""
        return field_elems(stream_seed(tag, n, 3), n), field_elems(stream_seed(tag, n, 4), n)

    @staticmethod
    def padd_plan(n: int, tag: int, edge_rate: float = 0.01):
        """Mixed point additions acc + Q with edge cases at `edge_rate` each.

        Returns point seeds for acc and Q, the XYZZ scaling factors lambda (acc is
        handed over as (l^2 X, l^3 Y, l^2, l^3)), and a case code per op:
        0 generic, 1 Q = acc (doubling), 2 Q = -acc, 3 acc = O, 4 Q = O.
        """
        sa = scalars(stream_seed(tag, n, 5), n)
        sq = scalars(stream_seed(tag, n, 6), n)
        lam = field_elems(stream_seed(tag, n, 7), n)
        return sa, sq, lam, workloads.padd_cases(n, tag, edge_rate)

    @staticmethod
    def padd_cases(n: int, tag: int, edge_rate: float = 0.01):
        """The case code of each of n mixed additions: 0 generic, 1 Q = acc (doubling),
        2 Q = -acc, 3 acc = O, 4 Q = O; each special case at `edge_rate`."""
        u = uniform01(stream_seed(tag, n, 8), n)
        case = np.zeros(n, dtype=np.int8)
        for k in range(4):
            lo, hi = k * edge_rate, (k + 1) * edge_rate
            case[(u >= lo) & (u < hi)] = k + 1
        return case

    @staticmethod
    def batch_sizes(njobs: int = 64, lo_log2: float = 10.0, hi_log2: float = 20.0, tag: int = 3):
        u = uniform01(stream_seed(tag, njobs, 9), njobs)
        return np.floor(2.0 ** (lo_log2 + u * (hi_log2 - lo_log2))).astype(np.int64)

    @staticmethod
    def requests(nreq: int = 2000, lo_log2: float = 12.0, hi_log2: float = 22.0,
                 nsets: int = 8, set_size: int = 1 << 22, tag: int = 4):
        """Poisson request stream: unit-rate exponential gaps (scaled by the caller),
        log-uniform n, a resident set id and a 256-aligned offset per request."""
        u = uniform01(stream_seed(tag, nreq, 10), nreq)
        gaps = -np.log1p(-uniform01(stream_seed(tag, nreq, 11), nreq))
        n = np.floor(2.0 ** (lo_log2 + u * (hi_log2 - lo_log2))).astype(np.int64)
        sets = small_ints(stream_seed(tag, nreq, 12), nreq, nsets)
        room = (set_size - n) // 256
        offs = (small_ints(stream_seed(tag, nreq, 13), nreq, 1 << 30) % (room + 1)) * 256
        return gaps, n, sets, offs
