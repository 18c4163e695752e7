"""ctypes binding of oracle.c (plain C big-integer oracle) — test infrastructure only.

`build()` compiles oracle.c with gcc into oracle/_build/liboracle.so; `lib()`
loads it (building on first use) and hands it the modulus, the Barrett constant
floor(2^754 / p) and the generator, all derived in `oracle.fq` / `oracle.g1`.
Arrays cross the boundary as little-endian u32 limbs: 24 per affine point
(x then y, standard form, (0, 0) = O) and 8 per scalar.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import fq, g1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _words64(v: int, n: int):
    return (ctypes.c_uint64 * n)(*[(v >> (64 * k)) & 0xFFFFFFFFFFFFFFFF for k in range(n)])


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            L.orc_init.argtypes = [u64p, u64p, u64p, u64p]
            L.orc_fq_mul.argtypes = [u64p, u64p, u64p]
            L.orc_fq_inv.argtypes = [u64p, u64p]
            L.orc_scalar_mul.argtypes = [u32p, u32p, u32p]
            L.orc_padd.argtypes = [u32p, u32p, u32p]
            L.orc_gen_points.argtypes = [u32p, ctypes.c_size_t, u32p, ctypes.c_int]
            L.orc_msm.argtypes = [u32p, u32p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, u32p]
            L.orc_msm_naive.argtypes = [u32p, u32p, ctypes.c_size_t, u32p]
            L.orc_padd_stream.argtypes = [u32p, u32p, ctypes.c_size_t, u32p]
            mu = (1 << (2 * fq.P.bit_length())) // fq.P
            L.orc_init(_words64(fq.P, 6), _words64(mu, 7), _words64(g1.GX, 6), _words64(g1.GY, 6))
            _lib = L
    return _lib


def _u32(a: np.ndarray):
    assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def fq_mul(a: int, b: int) -> int:
    out = (ctypes.c_uint64 * 6)()
    rc = lib().orc_fq_mul(_words64(a, 6), _words64(b, 6), out)
    assert rc == 0
    return sum(int(out[k]) << (64 * k) for k in range(6))


def fq_inv(a: int) -> int:
    out = (ctypes.c_uint64 * 6)()
    rc = lib().orc_fq_inv(_words64(a, 6), out)
    assert rc == 0
    return sum(int(out[k]) << (64 * k) for k in range(6))


def gen_points(seeds: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """P_i = seeds_i * G as (n, 24) u32 limbs (affine, standard form)."""
    seeds = np.ascontiguousarray(seeds, dtype=np.uint32)
    n = seeds.shape[0]
    out = np.zeros((n, 24), dtype=np.uint32)
    if n:
        rc = lib().orc_gen_points(_u32(seeds), n, _u32(out), nthreads)
        assert rc == 0
    return out


def msm(points: np.ndarray, scalars: np.ndarray, c: int = 0, nthreads: int = 0) -> np.ndarray:
    """Textbook Pippenger; returns 24 u32 limbs (affine, (0,0) = O)."""
    points = np.ascontiguousarray(points, dtype=np.uint32)
    scalars = np.ascontiguousarray(scalars, dtype=np.uint32)
    n = points.shape[0]
    if c <= 0:
        c = max(4, min(16, int(np.log2(max(n, 2))) - 3))
    out = np.zeros(24, dtype=np.uint32)
    rc = lib().orc_msm(_u32(points), _u32(scalars), n, c, nthreads, _u32(out))
    assert rc == 0
    return out


def msm_naive(points: np.ndarray, scalars: np.ndarray) -> np.ndarray:
    points = np.ascontiguousarray(points, dtype=np.uint32)
    scalars = np.ascontiguousarray(scalars, dtype=np.uint32)
    out = np.zeros(24, dtype=np.uint32)
    rc = lib().orc_msm_naive(_u32(points), _u32(scalars), points.shape[0], _u32(out))
    assert rc == 0
    return out


def scalar_mul(pt_limbs: np.ndarray, k: int) -> np.ndarray:
    pt = np.ascontiguousarray(pt_limbs, dtype=np.uint32)
    ks = np.array([(k >> (32 * i)) & 0xFFFFFFFF for i in range(8)], dtype=np.uint32)
    out = np.zeros(24, dtype=np.uint32)
    rc = lib().orc_scalar_mul(_u32(pt), _u32(ks), _u32(out))
    assert rc == 0
    return out


def padd(p1: np.ndarray, p2: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(p1, dtype=np.uint32)
    b = np.ascontiguousarray(p2, dtype=np.uint32)
    out = np.zeros(24, dtype=np.uint32)
    assert lib().orc_padd(_u32(a), _u32(b), _u32(out)) == 0
    return out


def padd_stream(acc: np.ndarray, q: np.ndarray) -> np.ndarray:
    acc = np.ascontiguousarray(acc, dtype=np.uint32)
    q = np.ascontiguousarray(q, dtype=np.uint32)
    out = np.zeros_like(acc)
    assert lib().orc_padd_stream(_u32(acc), _u32(q), acc.shape[0], _u32(out)) == 0
    return out
