"""BLS12-377 G1 multi-scalar multiplication on sm_103a — Python binding of libmsm377.

Argument marshalling only: every call goes straight to the C-ABI in
include/msm377.h with device pointers taken from torch tensors (torch provides
device memory and streams). Arrays of 32-bit limbs are carried in torch.int32
tensors holding the u32 bit patterns.

Layouts (see the header): field batches are structure-of-arrays [12][n];
XYZZ batches [4][12][n]; affine batches [2][12][n]; MSM points are
array-of-structures (n, 24) and scalars (n, 8).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from ._lib import MsmError, MsmJob, MsmOpts, check, last_error, lib

FORM_STANDARD = 0
FORM_MONTGOMERY = 1
POINTS_PREPARED = 1
PROFILE = 2
EDWARDS = 4   # the paper's twisted Edwards model; points of the order-r subgroup
GLV = 8       # endomorphism split, half the windows; points of the order-r subgroup
PRECOMPUTED = 16  # fixed-base shifted copies 2^(cj) P (Edwards resident sets, explicit c)
RADIX_SORT = 32   # 8-bit LSD radix passes instead of the default counting sort (comparison)
VALIDATE = 64     # check input points (on the curve; in the subgroup for Edwards / GLV)
MSM_STAGES = ("head", "accumulate", "tail")
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTONCURVE, ERANGE = 0, -1, -2, -3, -4, -5, -6

__all__ = [
    "MsmError", "MsmOpts", "FORM_STANDARD", "FORM_MONTGOMERY", "POINTS_PREPARED",
    "to_device", "to_host", "fq_mul_batch", "fq_to_montgomery", "fq_from_montgomery",
    "padd_batch", "xyzz_to_affine_batch", "g1_generator_mul", "msm_points_prepare",
    "msm_g1", "msm_g1_workspace", "msm_g1_host", "msm_g1_status", "msm_g1_default_c",
    "imad_probe", "lib", "last_error", "profile_last", "launch_count", "MSM_STAGES", "PROFILE",
    "MsmJob", "msm_g1_batched", "msm_g1_batched_workspace", "EDWARDS", "GLV",
    "msm_points_prepared_bytes", "padd_chain", "fq_mul_batch_variant", "FQMUL_CIOS", "FQMUL_BARRETT",
    "FQMUL_KARATSUBA", "FQMUL_CARRYSAVE", "FQMUL_CIOS_TWOPASS", "FQMUL_CIOS_DOUBLEROW", "FQMUL_WARP", "FQMUL_PAPER", "FQMUL_FIPS", "FQMUL_CIOS_SINGLEROW", "PRECOMPUTED", "RADIX_SORT", "msm_points_precompute",
    "msm_points_precomputed_bytes", "VALIDATE", "ENOTONCURVE", "ERANGE", "ResidentSet", "msm_points_validate",
]


def to_device(arr: np.ndarray, device="cuda") -> torch.Tensor:
    """u32 numpy array -> int32 torch tensor on the device (same bits)."""
    a = np.ascontiguousarray(arr, dtype=np.uint32)
    return torch.from_numpy(a.view(np.int32)).to(device)


def to_host(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().contiguous().numpy().view(np.uint32)


def _p(t: torch.Tensor | None):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _s(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _check_dev(*ts):
    for t in ts:
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError("expected contiguous CUDA tensors")


def fq_mul_batch(a: torch.Tensor, b: torch.Tensor, out: torch.Tensor | None = None,
                 form: int = FORM_STANDARD, stream=None) -> torch.Tensor:
    n = a.shape[-1]
    out = torch.empty_like(a) if out is None else out
    _check_dev(a, b, out)
    check(lib().fq_mul_batch(_p(a), _p(b), _p(out), n, form, _s(stream)))
    return out


FQMUL_CIOS, FQMUL_BARRETT, FQMUL_KARATSUBA, FQMUL_CARRYSAVE, FQMUL_CIOS_TWOPASS, FQMUL_CIOS_DOUBLEROW = (
    0, 1, 2, 3, 4, 5)
FQMUL_WARP = 6
FQMUL_PAPER = 7
FQMUL_FIPS = 8
FQMUL_CIOS_SINGLEROW = 9


def fq_mul_batch_variant(a: torch.Tensor, b: torch.Tensor, variant: int, out: torch.Tensor | None = None,
                         stream=None) -> torch.Tensor:
    """[12][n] operands in [0, p): BARRETT gives a b mod p, the others a b 2^-384 mod p."""
    n = a.shape[-1]
    out = torch.empty_like(a) if out is None else out
    _check_dev(a, b, out)
    check(lib().fq_mul_batch_variant(_p(a), _p(b), _p(out), n, int(variant), _s(stream)))
    return out


def fq_to_montgomery(x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    out = torch.empty_like(x) if out is None else out
    _check_dev(x, out)
    check(lib().fq_to_montgomery(_p(x), _p(out), x.shape[-1], _s(stream)))
    return out


def fq_from_montgomery(x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    out = torch.empty_like(x) if out is None else out
    _check_dev(x, out)
    check(lib().fq_from_montgomery(_p(x), _p(out), x.shape[-1], _s(stream)))
    return out


def padd_batch(acc: torch.Tensor, q: torch.Tensor, out: torch.Tensor | None = None,
               form: int = FORM_STANDARD, stream=None) -> torch.Tensor:
    n = acc.shape[-1]
    out = torch.empty_like(acc) if out is None else out
    _check_dev(acc, q, out)
    check(lib().padd_batch(_p(acc), _p(q), _p(out), n, form, _s(stream)))
    return out


def xyzz_to_affine_batch(xyzz: torch.Tensor, form: int = FORM_STANDARD, stream=None) -> torch.Tensor:
    n = xyzz.shape[-1]
    out = torch.empty((2, 12, n), dtype=torch.int32, device=xyzz.device)
    _check_dev(xyzz)
    check(lib().xyzz_to_affine_batch(_p(xyzz), _p(out), n, form, _s(stream)))
    return out


def g1_generator_mul(seeds: torch.Tensor, stream=None) -> torch.Tensor:
    """seeds (n, 8) -> points (n, 24), P_i = seeds_i * G."""
    n = seeds.shape[0]
    out = torch.empty((n, 24), dtype=torch.int32, device=seeds.device)
    _check_dev(seeds)
    check(lib().g1_generator_mul(_p(seeds), n, _p(out), _s(stream)))
    return out


def _model_flags(edwards: bool, glv: bool) -> int:
    return (EDWARDS if edwards else 0) | (GLV if glv else 0)


def msm_points_prepared_bytes(n: int, edwards: bool = False, glv: bool = False) -> int:
    return int(lib().msm_points_prepared_bytes(n, _model_flags(edwards, glv)))


def msm_points_prepare(points: torch.Tensor, out: torch.Tensor | None = None, stream=None,
                       edwards: bool = False, glv: bool = False) -> torch.Tensor:
    """Stored form of (n, 24) standard points for msm_g1(..., prepared=True) with the same
    edwards / glv choice: (n', 24) int32 for XYZZ, (n', 36) for Edwards; n' = 2n with GLV."""
    flags = _model_flags(edwards, glv)
    n = points.shape[0]
    words = lib().msm_points_prepared_bytes(n, flags) // 4
    rows = 2 * n if glv else n
    if out is None:
        out = torch.empty((rows, words // rows if rows else 24), dtype=torch.int32, device=points.device)
    _check_dev(points, out)
    check(lib().msm_points_prepare_ex(_p(points), n, _p(out), flags, _s(stream)))
    return out


def _opts(c=0, signed=True, scalar_bits=0, prepared=False, stream=0, profile=False, edwards=False,
          glv=False, precomputed=False, radix_sort=False, validate=False) -> MsmOpts:
    """stream=0 for size queries (no CUDA context needed); None = torch's current stream."""
    sv = 0 if (isinstance(stream, int) and stream == 0) else _s(stream).value
    flags = (POINTS_PREPARED if prepared else 0) | (PROFILE if profile else 0) | _model_flags(edwards, glv)
    flags |= (PRECOMPUTED if precomputed else 0) | (RADIX_SORT if radix_sort else 0)
    flags |= VALIDATE if validate else 0
    return MsmOpts(int(c), 1 if signed else 0, int(scalar_bits), flags, sv)


def msm_points_precomputed_bytes(n: int, c: int, scalar_bits: int = 0, signed: bool = True,
                                 glv: bool = False) -> int:
    o = _opts(c, signed, scalar_bits, True, edwards=True, glv=glv, precomputed=True)
    return int(lib().msm_points_precomputed_bytes(n, ctypes.byref(o)))


def msm_points_precompute(points: torch.Tensor, c: int, scalar_bits: int = 0, signed: bool = True,
                          glv: bool = False, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Fixed-base set for msm_g1(..., edwards=True, precomputed=True) with the same c, scalar_bits,
    signed and glv: rows j n' + i = stored 2^(c j) P'_i, as an (rows, 36) int32 tensor."""
    n = points.shape[0]
    nbytes = msm_points_precomputed_bytes(n, c, scalar_bits, signed, glv)
    if msm_points_precomputed_bytes(max(n, 1), c, scalar_bits, signed, glv) == 0:
        raise MsmError(-1, "bad precompute options (explicit c needed)")
    if out is None:
        out = torch.empty((nbytes // 144, 36), dtype=torch.int32, device=points.device)
    _check_dev(points, out)
    o = _opts(c, signed, scalar_bits, True, None if stream is None else stream, edwards=True, glv=glv,
              precomputed=True)
    check(lib().msm_points_precompute(_p(points), n, _p(out), ctypes.byref(o)))
    return out


def msm_g1_default_c(n: int, signed: bool = True, edwards: bool = False, glv: bool = False,
                     precomputed: bool = False) -> int:
    return lib().msm_g1_default_c(n, 1 if signed else 0,
                                  _model_flags(edwards, glv) | (PRECOMPUTED if precomputed else 0))


def msm_g1_workspace(n: int, c=0, signed=True, scalar_bits=0, prepared=False, device="cuda",
                     edwards: bool = False, glv: bool = False, precomputed: bool = False,
                     radix_sort: bool = False) -> torch.Tensor:
    o = _opts(c, signed, scalar_bits, prepared or precomputed, edwards=edwards, glv=glv, precomputed=precomputed,
              radix_sort=radix_sort)
    nbytes = lib().msm_g1_workspace_bytes(n, ctypes.byref(o))
    if nbytes == 0:
        raise MsmError(-1, "bad MSM options")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def msm_g1(points: torch.Tensor, scalars: torch.Tensor, out: torch.Tensor | None = None,
           workspace: torch.Tensor | None = None, c: int = 0, signed: bool = True,
           scalar_bits: int = 0, prepared: bool = False, stream=None, profile: bool = False,
           edwards: bool = False, glv: bool = False, precomputed: bool = False,
           radix_sort: bool = False, validate: bool = False) -> torch.Tensor:
    """Enqueues sum_i scalars_i * points_i; returns the (24,) int32 device tensor it writes.
    With prepared=True, points is msm_points_prepare(..., edwards=, glv=) output; with
    precomputed=True (Edwards, explicit c) msm_points_precompute output for the same options.
    radix_sort=True sorts by LSD radix passes instead of the counting sort (same result;
    the workspace must be sized with the same choice)."""
    n = scalars.shape[0]
    o = _opts(c, signed, scalar_bits, prepared or precomputed, None if stream is None else stream, profile,
              edwards, glv, precomputed, radix_sort, validate)
    _check_points(points, n, prepared or precomputed, edwards, glv, o)
    if workspace is None:
        workspace = msm_g1_workspace(n, c, signed, scalar_bits, prepared or precomputed, points.device, edwards,
                                     glv, precomputed, radix_sort)
    out = torch.empty(24, dtype=torch.int32, device=points.device) if out is None else out
    _check_dev(points, scalars, out, workspace)
    check(lib().msm_g1(_p(points), _p(scalars), n, _p(out), _p(workspace), workspace.numel(),
                       ctypes.byref(o)))
    return out


def _check_points(points: torch.Tensor, n: int, prepared: bool, edwards: bool, glv: bool, o=None) -> None:
    """The points tensor must hold exactly what the call will read for n scalars."""
    if o is not None and o.flags & PRECOMPUTED:
        want = lib().msm_points_precomputed_bytes(n, ctypes.byref(o))
    else:
        want = lib().msm_points_prepared_bytes(n, _model_flags(edwards, glv)) if prepared else 96 * n
    if points.numel() * points.element_size() != want:
        raise ValueError(f"points tensor holds {points.numel() * points.element_size()} bytes; "
                         f"{want} expected for n = {n} ({'prepared' if prepared else 'standard'} form)")


def _rows(pt: torch.Tensor, prepared: bool, glv: bool) -> int:
    return pt.shape[0] // 2 if (prepared and glv) else pt.shape[0]


def _jobs_array(points_list, scalars_list, outs, cs):
    arr = (MsmJob * len(points_list))()
    for i, (pt, sc, o) in enumerate(zip(points_list, scalars_list, outs)):
        arr[i].points = pt.data_ptr() if pt.shape[0] else 0
        arr[i].scalars = sc.data_ptr() if sc.shape[0] else 0
        arr[i].n = sc.shape[0]
        arr[i].out = o.data_ptr()
        arr[i].c = int(cs[i]) if cs is not None else 0
    return arr


def msm_g1_batched_workspace(points_list, c_list=None, signed=True, scalar_bits=0, prepared=False,
                             device="cuda", edwards: bool = False, glv: bool = False, precomputed: bool = False,
                             n_list=None) -> torch.Tensor:
    arr = (MsmJob * len(points_list))()
    for i, pt in enumerate(points_list):
        arr[i].n = int(n_list[i]) if n_list is not None else _rows(pt, prepared, glv)
        arr[i].c = int(c_list[i]) if c_list is not None else 0
    o = _opts(0, signed, scalar_bits, prepared or precomputed, edwards=edwards, glv=glv, precomputed=precomputed)
    nbytes = lib().msm_g1_batched_workspace_bytes(arr, len(points_list), ctypes.byref(o))
    if nbytes == 0:
        raise MsmError(-1, "bad batched MSM options")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def msm_g1_batched(points_list, scalars_list, outs=None, workspace: torch.Tensor | None = None,
                   c_list=None, signed: bool = True, scalar_bits: int = 0, prepared: bool = False,
                   stream=None, edwards: bool = False, glv: bool = False, precomputed: bool = False):
    """Enqueues len(points_list) <= 128 independent MSMs; returns their (24,) output tensors."""
    if len(points_list) != len(scalars_list):
        raise ValueError("points and scalars lists differ in length")
    dev = points_list[0].device
    if outs is None:
        outs = [torch.empty(24, dtype=torch.int32, device=dev) for _ in points_list]
    if workspace is None:
        workspace = msm_g1_batched_workspace(points_list, c_list, signed, scalar_bits, prepared, dev,
                                             edwards, glv, precomputed, [sc.shape[0] for sc in scalars_list])
    for i, (pt, sc) in enumerate(zip(points_list, scalars_list)):
        oj = _opts(int(c_list[i]) if c_list is not None else 0, signed, scalar_bits, prepared or precomputed,
                   edwards=edwards, glv=glv, precomputed=precomputed)
        _check_points(pt, sc.shape[0], prepared or precomputed, edwards, glv, oj)
        _check_dev(pt, sc)
    arr = _jobs_array(points_list, scalars_list, outs, c_list)
    o = _opts(0, signed, scalar_bits, prepared or precomputed, None if stream is None else stream,
              edwards=edwards, glv=glv, precomputed=precomputed)
    check(lib().msm_g1_batched(arr, len(points_list), _p(workspace), workspace.numel(), ctypes.byref(o)))
    return outs


def msm_g1_status(workspace: torch.Tensor, stream=None) -> int:
    o = _opts(stream=None if stream is None else stream)
    return lib().msm_g1_status(_p(workspace), ctypes.byref(o))


def msm_g1_host(points: np.ndarray, scalars: np.ndarray, workspace: torch.Tensor | None = None,
                c: int = 0, signed: bool = True, scalar_bits: int = 0, stream=None, edwards: bool = False,
                glv: bool = False, validate: bool = False) -> np.ndarray:
    """Synchronous MSM on host arrays (copies in and out inside the call)."""
    pts = np.ascontiguousarray(points, dtype=np.uint32)
    sc = np.ascontiguousarray(scalars, dtype=np.uint32)
    n = pts.shape[0]
    o = _opts(c, signed, scalar_bits, False, None if stream is None else stream, edwards=edwards, glv=glv,
              validate=validate)
    need = lib().msm_g1_host_workspace_bytes(n, ctypes.byref(o))
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
    out = np.zeros(24, dtype=np.uint32)
    check(lib().msm_g1_host(pts.ctypes.data_as(ctypes.c_void_p), sc.ctypes.data_as(ctypes.c_void_p), n,
                            out.ctypes.data_as(ctypes.c_void_p), _p(workspace), workspace.numel(),
                            ctypes.byref(o)))
    return out


def msm_g1_host_workspace_bytes(n: int, c=0, signed=True, scalar_bits=0, edwards=False, glv=False) -> int:
    o = _opts(c, signed, scalar_bits, edwards=edwards, glv=glv)
    return lib().msm_g1_host_workspace_bytes(n, ctypes.byref(o))


def profile_last() -> dict:
    """Stage times (ms) of the last msm_g1 call made with profile=True (synchronises)."""
    buf = (ctypes.c_float * 8)()
    k = lib().msm377_profile_last(buf, 8)
    if k < 0:
        raise MsmError(k, last_error())
    return {name: float(buf[i]) for i, name in enumerate(MSM_STAGES[:k])}


def launch_count() -> int:
    return int(lib().msm377_launch_count())


def padd_chain(stored: torch.Tensor, n: int, edwards: bool = False, lanes: int = 1, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """P_0 + ... + P_{n-1} as one dependent chain of mixed PADDs over stored points
    (msm_points_prepare(..., edwards=edwards)); lanes = 4 spreads each Edwards PADD over four lanes."""
    out = torch.empty(24, dtype=torch.int32, device=stored.device) if out is None else out
    _check_points(stored, n, True, edwards, False)
    _check_dev(stored, out)
    check(lib().padd_chain(_p(stored), n, _p(out), EDWARDS if edwards else 0, int(lanes), _s(stream)))
    return out


def imad_probe(iters: int = 20000, stream=None) -> float:
    """Measured 32x32->64 limb products per second over all SMs."""
    v = ctypes.c_double(0.0)
    check(lib().msm377_imad_probe(iters, ctypes.byref(v), _s(stream)))
    return v.value


def msm_points_validate(points: torch.Tensor, edwards: bool = False, glv: bool = False, subgroup: bool = False,
                        stream=None) -> int:
    """0 if every (n, 24) standard-form point is on the curve (and in the order-r subgroup
    when edwards, glv or subgroup asks for it), else ENOTONCURVE. Synchronous."""
    _check_dev(points)
    flags = _model_flags(edwards, glv) | (PRECOMPUTED if subgroup else 0)
    rc = lib().msm_points_validate(_p(points), points.shape[0], flags, _s(stream))
    if rc not in (OK, ENOTONCURVE):
        check(rc)
    return rc


class ResidentSet:
    """A resident point set owned by the library (msm_points_create / msm_points_destroy):
    the stored form of n standard-form points for one curve model (Edwards, GLV, or a
    fixed-base set for one window width c), reused by many msm() calls over slices."""

    def __init__(self, points: torch.Tensor, edwards: bool = False, glv: bool = False, precompute_c: int = 0,
                 scalar_bits: int = 0, signed: bool = True, validate: bool = False, stream=None):
        _check_dev(points)
        self.device = points.device
        self.n = points.shape[0]
        self.edwards, self.glv, self.c = edwards or precompute_c > 0, glv, precompute_c
        self.scalar_bits, self.signed = scalar_bits, signed
        o = _opts(precompute_c, signed, scalar_bits, False, None if stream is None else stream,
                  edwards=self.edwards, glv=glv, precomputed=precompute_c > 0, validate=validate)
        h = ctypes.c_void_p(0)
        self._h = None
        check(lib().msm_points_create(_p(points), self.n, ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def data_ptr(self, offset: int = 0) -> int:
        return int(lib().msm_points_data(self._h, offset) or 0)

    def _opts(self, stream, profile=False, radix_sort=False) -> MsmOpts:
        return _opts(0, self.signed, self.scalar_bits, True, stream, profile, self.edwards, self.glv, self.c > 0,
                     radix_sort)

    def workspace(self, n: int) -> torch.Tensor:
        nbytes = lib().msm_g1_resident_workspace_bytes(self._h, n, ctypes.byref(self._opts(0)))
        if nbytes == 0:
            raise MsmError(EINVAL, "bad resident MSM options")
        return torch.empty(nbytes, dtype=torch.uint8, device=self.device)

    def workspace_bytes(self, n: int) -> int:
        return int(lib().msm_g1_resident_workspace_bytes(self._h, n, ctypes.byref(self._opts(0))))

    def msm(self, scalars: torch.Tensor, offset: int = 0, out: torch.Tensor | None = None,
            workspace: torch.Tensor | None = None, stream=None, profile: bool = False,
            radix_sort: bool = False) -> torch.Tensor:
        """Enqueues sum_i scalars_i P_{offset + i} over the set (msm_g1_resident)."""
        n = scalars.shape[0]
        if workspace is None:
            workspace = self.workspace(n)
        out = torch.empty(24, dtype=torch.int32, device=self.device) if out is None else out
        _check_dev(scalars, out, workspace)
        o = self._opts(None if stream is None else stream, profile, radix_sort)
        check(lib().msm_g1_resident(self._h, offset, n, _p(scalars), _p(out), _p(workspace), workspace.numel(),
                                    ctypes.byref(o)))
        return out

    def host_workspace(self, n: int) -> torch.Tensor:
        nbytes = lib().msm_g1_resident_host_workspace_bytes(self._h, n, ctypes.byref(self._opts(0)))
        if nbytes == 0:
            raise MsmError(EINVAL, "bad resident MSM options")
        return torch.empty(nbytes, dtype=torch.uint8, device=self.device)

    def msm_host(self, scalars: np.ndarray, offset: int = 0, workspace: torch.Tensor | None = None,
                 stream=None) -> np.ndarray:
        """Synchronous MSM over the set with host scalars (msm_g1_resident_host): the scalars
        are copied in, the affine result (24 u32) copied out."""
        sc = np.ascontiguousarray(scalars, dtype=np.uint32)
        n = sc.shape[0]
        if workspace is None:
            workspace = self.host_workspace(n)
        out = np.zeros(24, dtype=np.uint32)
        o = self._opts(None if stream is None else stream)
        check(lib().msm_g1_resident_host(self._h, offset, n, sc.ctypes.data_as(ctypes.c_void_p),
                                         out.ctypes.data_as(ctypes.c_void_p), _p(workspace), workspace.numel(),
                                         ctypes.byref(o)))
        return out

    def close(self) -> None:
        if self._h is not None and self._h.value:
            check(lib().msm_points_destroy(self._h))
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def msm_g1_set_schedule(log2n: int, c: int = 0, chunk: int = 0, sort: int = 0, reduce_log2: int = 0,
                        groups: int = 0, edwards: bool = False, glv: bool = False,
                        precomputed: bool = False) -> None:
    """Installs one schedule entry (0 = built-in rule) for signed digits at n in [2^log2n, 2^(log2n+1))."""
    flags = _model_flags(edwards or precomputed, glv) | (PRECOMPUTED if precomputed else 0)
    check(lib().msm_g1_set_schedule(flags, int(log2n), int(c), int(chunk), int(sort), int(reduce_log2),
                                    int(groups)))


def msm_g1_schedule(n: int, c: int = 0, signed: bool = True, scalar_bits: int = 0, prepared: bool = True,
                    edwards: bool = False, glv: bool = False, precomputed: bool = False) -> dict:
    """The schedule msm_g1 uses for these options: window c, chunk K, sort, level-1 reduction threads."""
    o = _opts(c, signed, scalar_bits, prepared or precomputed, edwards=edwards, glv=glv, precomputed=precomputed)
    out = (ctypes.c_int32 * 5)()
    check(lib().msm_g1_schedule(n, ctypes.byref(o), out))
    return {"c": int(out[0]), "chunk": int(out[1]), "sort": "counting" if out[2] == 1 else "radix",
            "reduce_threads_log2": int(out[3]), "groups": int(out[4])}
