// Resident point sets (library-owned device memory holding the stored form of a
// caller's points, reused by many MSMs with fresh scalars) and input validation.
//
// The problem the paper accelerates is sum_i s_i P_i over points of BLS12-377 G1
// (Sec. I, II-C); its points are curve points of the prime-order subgroup. The
// validation kernel checks exactly that precondition for a batch of affine
// standard-form inputs: coordinates below p, y^2 = x^3 + 1 (the identity O is
// encoded (0, 0)), and, where the caller's curve model needs it (the twisted
// Edwards map and the GLV endomorphism are exact on the order-r subgroup only),
// r P = O by double-and-add.
#include <cuda_runtime.h>

#include <new>

#include "common.cuh"
#include "ec.cuh"

namespace {

using ec::affine;
using ec::xyzz;
using fq::fe;

// r, the order of G1, little-endian 32-bit limbs (253 bits).
__device__ __constant__ static const uint32_t kOrderR[8] = {0x00000001u, 0x0a118000u, 0xd0000001u, 0x59aa76feu,
                                                            0x5c37b001u, 0x60b44d1eu, 0x9a2ca556u, 0x12ab655eu};

// One thread per point: the first failing point sets *status (first error wins).
__global__ void k_validate(const uint4* __restrict__ pts, size_t n, int subgroup, int* __restrict__ status) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        affine Q;
        const uint4* p = pts + 6 * i;
        const uint4 a = p[0], b = p[1], c = p[2], d = p[3], e = p[4], f = p[5];
        const uint32_t w[24] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w,
                                d.x, d.y, d.z, d.w, e.x, e.y, e.z, e.w, f.x, f.y, f.z, f.w};
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            Q.x.v[k] = w[k];
            Q.y.v[k] = w[12 + k];
        }
        if (fq::is_zero_raw(Q.x) && fq::is_zero_raw(Q.y)) continue;   // O
        bool ok = fq::lt_p(Q.x) && fq::lt_p(Q.y);
        if (ok) {
            fq::to_mont(Q.x, Q.x);
            fq::to_mont(Q.y, Q.y);
            fe y2, x3, one;
            fq::mul(y2, Q.y, Q.y);
            fq::mul(x3, Q.x, Q.x);
            fq::mul(x3, x3, Q.x);
            fq::set_one(one);
            fq::add(x3, x3, one);
            ok = fq::equal(y2, x3);                   // y^2 = x^3 + 1
        }
        if (ok && subgroup) {                         // r P = O, left to right
            xyzz R;
            ec::set_inf(R);
            bool inf = true;
            for (int bit = 252; bit >= 0; --bit) {
                if (!inf) ec::dbl(R);
                if ((kOrderR[bit >> 5] >> (bit & 31)) & 1u) ec::madd(R, inf, Q);
            }
            ok = inf || ec::is_inf(R);
        }
        if (!ok) atomicCAS(status, 0, MSM377_ENOTONCURVE);
    }
}

struct PointSet {
    void* base = nullptr;      // 256-byte status header, then the stored rows
    size_t n = 0;
    size_t bytes = 0;          // stored rows
    size_t per_point = 0;      // bytes of stored rows per input point
    uint32_t model = 0;        // MSM377_EDWARDS | MSM377_GLV | MSM377_PRECOMPUTED
    int c = 0, scalar_bits = 0, signed_digits = 1;
    int device = 0;
};

constexpr size_t kHeader = 256;
constexpr uint32_t kModelBits = MSM377_EDWARDS | MSM377_GLV | MSM377_PRECOMPUTED;

PointSet* as_set(msm_points_t h) { return reinterpret_cast<PointSet*>(h); }

}  // namespace

namespace msm377 {

int launch_validate(const uint32_t* points_std, size_t n, bool subgroup, int* status, cudaStream_t s) {
    if (n == 0) return MSM377_OK;
    int dev = 0, sms = 152;
    MSM_CUDA_TRY(cudaGetDevice(&dev));
    MSM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t want = (n + 127) / 128, cap = (size_t)sms * 16;
    k_validate<<<(unsigned)(want < cap ? want : cap), 128, 0, s>>>(reinterpret_cast<const uint4*>(points_std), n,
                                                                  subgroup ? 1 : 0, status);
    note_launches(1);
    return check_launch("validate points");
}

}  // namespace msm377

using namespace msm377;

extern "C" int msm_points_validate(const uint32_t* points_std, size_t n, uint32_t flags, void* stream) {
    if (flags & ~(MSM377_EDWARDS | MSM377_GLV | MSM377_PRECOMPUTED | MSM377_VALIDATE))
        return set_error(MSM377_EINVAL, "msm_points_validate: flags 0x%x", flags);
    if (n == 0) return MSM377_OK;
    if (!points_std || !aligned(points_std, 16))
        return set_error(MSM377_EINVAL, "msm_points_validate: points NULL or not 16-byte aligned");
    cudaStream_t s = as_stream(stream);
    int* status = nullptr;
    MSM_CUDA_TRY(cudaMallocAsync(&status, sizeof(int), s));
    int st = 0;
    int r = MSM377_OK;
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        r = launch_validate(points_std, n, (flags & (MSM377_EDWARDS | MSM377_GLV | MSM377_PRECOMPUTED)) != 0,
                            status, s);
        if (r == MSM377_OK) e = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (r == MSM377_OK && e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFreeAsync(status, s);
    if (r) return r;
    if (e != cudaSuccess) return set_error(MSM377_ECUDA, "msm_points_validate: %s", cudaGetErrorString(e));
    if (st == MSM377_ENOTONCURVE)
        return set_error(MSM377_ENOTONCURVE, "msm_points_validate: a point is not on the curve%s",
                         (flags & (MSM377_EDWARDS | MSM377_GLV | MSM377_PRECOMPUTED)) ? " or not in the order-r subgroup"
                                                                                     : "");
    return st;
}

extern "C" int msm_points_create(const uint32_t* points_std, size_t n, const msm_opts* opts, msm_points_t* handle) {
    if (!opts || !handle) return set_error(MSM377_EINVAL, "msm_points_create: NULL argument");
    *handle = nullptr;
    const uint32_t extra = opts->flags & ~(kModelBits | MSM377_VALIDATE);
    if (extra) return set_error(MSM377_EINVAL, "msm_points_create: flags 0x%x not allowed here", extra);
    const uint32_t model = opts->flags & kModelBits;
    if (n == 0 || n >= (1ull << 30)) return set_error(MSM377_EINVAL, "msm_points_create: n = %zu", n);
    if (!points_std || !aligned(points_std, 16))
        return set_error(MSM377_EINVAL, "msm_points_create: points NULL or not 16-byte aligned");
    size_t bytes = 0;
    msm_opts o = *opts;
    o.flags = model | MSM377_POINTS_PREPARED;
    if (model & MSM377_PRECOMPUTED) {
        if (!(model & MSM377_EDWARDS) || o.c == 0)
            return set_error(MSM377_EINVAL, "msm_points_create: PRECOMPUTED needs EDWARDS and an explicit c");
        bytes = msm_points_precomputed_bytes(n, &o);
    } else {
        bytes = msm_points_prepared_bytes(n, model);
    }
    if (bytes == 0)
        return set_error(MSM377_EINVAL, "msm_points_create: bad options (c=%d scalar_bits=%d flags=0x%x)", o.c,
                         o.scalar_bits, opts->flags);
    cudaStream_t s = as_stream(opts->stream);
    PointSet* set = new (std::nothrow) PointSet;
    if (!set) return set_error(MSM377_EINVAL, "msm_points_create: host allocation failed");
    MSM_CUDA_TRY(cudaGetDevice(&set->device));
    cudaError_t e = cudaMalloc(&set->base, kHeader + bytes);
    if (e != cudaSuccess) {
        delete set;
        return set_error(MSM377_ENOMEM, "msm_points_create: cudaMalloc(%zu): %s", kHeader + bytes,
                         cudaGetErrorString(e));
    }
    set->n = n;
    set->bytes = bytes;
    set->per_point = bytes / n;
    set->model = model;
    set->c = o.c;
    set->scalar_bits = o.scalar_bits;
    set->signed_digits = o.signed_digits;
    auto fail = [&](int code) {
        cudaStreamSynchronize(s);
        cudaFree(set->base);
        delete set;
        return code;
    };
    int* status = static_cast<int*>(set->base);
    uint32_t* rows = reinterpret_cast<uint32_t*>(static_cast<char*>(set->base) + kHeader);
    if (cudaMemsetAsync(status, 0, kHeader, s) != cudaSuccess) return fail(set_error(MSM377_ECUDA, "memset"));
    if (opts->flags & MSM377_VALIDATE) {
        int r = launch_validate(points_std, n, model != 0, status, s);
        if (r) return fail(r);
        int st = 0;
        if (cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(set_error(MSM377_ECUDA, "msm_points_create: validation status"));
        if (st)
            return fail(set_error(MSM377_ENOTONCURVE,
                                  "msm_points_create: a point is not on the curve%s",
                                  model ? " or not in the order-r subgroup" : ""));
    }
    int r = (model & MSM377_PRECOMPUTED) ? msm_points_precompute(points_std, n, rows, &o)
                                         : msm_points_prepare_ex(points_std, n, rows, model & ~MSM377_PRECOMPUTED,
                                                                 opts->stream);
    if (r) return fail(r);
    *handle = reinterpret_cast<msm_points_t>(set);
    return MSM377_OK;
}

extern "C" int msm_points_destroy(msm_points_t handle) {
    if (!handle) return MSM377_OK;
    PointSet* set = as_set(handle);
    int cur = 0;
    MSM_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != set->device) MSM_CUDA_TRY(cudaSetDevice(set->device));
    cudaError_t e = cudaFree(set->base);   // waits for work that still reads the set
    if (cur != set->device) cudaSetDevice(cur);
    delete set;
    if (e != cudaSuccess) return set_error(MSM377_ECUDA, "msm_points_destroy: %s", cudaGetErrorString(e));
    return MSM377_OK;
}

extern "C" size_t msm_points_count(msm_points_t handle) { return handle ? as_set(handle)->n : 0; }

extern "C" const uint32_t* msm_points_data(msm_points_t handle, size_t offset) {
    if (!handle || offset > as_set(handle)->n) return nullptr;
    const PointSet* set = as_set(handle);
    return reinterpret_cast<const uint32_t*>(static_cast<const char*>(set->base) + kHeader +
                                             offset * set->per_point);
}

namespace {
// The options msm_g1 receives for a slice of a resident set: the set's curve model,
// and for a fixed-base set its window width, digit kind and scalar bound.
int resident_opts(const PointSet* set, const msm_opts* opts, msm_opts* o) {
    if (opts->flags & ~(MSM377_PROFILE | MSM377_RADIX_SORT | kModelBits | MSM377_POINTS_PREPARED))
        return set_error(MSM377_EINVAL, "msm_g1_resident: flags 0x%x not allowed", opts->flags);
    if ((opts->flags & kModelBits) && (opts->flags & kModelBits) != set->model)
        return set_error(MSM377_EINVAL, "msm_g1_resident: flags name another curve model than the set's");
    *o = *opts;
    o->flags = (opts->flags & (MSM377_PROFILE | MSM377_RADIX_SORT)) | set->model | MSM377_POINTS_PREPARED;
    if (set->model & MSM377_PRECOMPUTED) {
        if ((opts->c && opts->c != set->c) || (opts->scalar_bits && opts->scalar_bits != set->scalar_bits) ||
            (opts->signed_digits ? 1 : 0) != (set->signed_digits ? 1 : 0))
            return set_error(MSM377_EINVAL, "msm_g1_resident: a fixed-base set fixes c = %d, scalar_bits = %d "
                             "and its digit kind", set->c, set->scalar_bits);
        o->c = set->c;
        o->scalar_bits = set->scalar_bits;
    }
    return MSM377_OK;
}
}  // namespace

extern "C" size_t msm_g1_resident_workspace_bytes(msm_points_t handle, size_t n, const msm_opts* opts) {
    if (!handle || !opts) return 0;
    msm_opts o;
    if (resident_opts(as_set(handle), opts, &o)) return 0;
    return msm_g1_workspace_bytes(n, &o);
}

extern "C" int msm_g1_resident(msm_points_t handle, size_t offset, size_t n, const uint32_t* scalars, uint32_t* out,
                               void* workspace, size_t workspace_bytes, const msm_opts* opts) {
    if (!handle || !opts) return set_error(MSM377_EINVAL, "msm_g1_resident: NULL argument");
    const PointSet* set = as_set(handle);
    if (offset > set->n || n > set->n - offset)
        return set_error(MSM377_EINVAL, "msm_g1_resident: points [%zu, %zu) outside the set of %zu", offset,
                         offset + n, set->n);
    msm_opts o;
    int r = resident_opts(set, opts, &o);
    if (r) return r;
    return msm_g1(msm_points_data(handle, offset), scalars, n, out, workspace, workspace_bytes, &o);
}

extern "C" size_t msm_g1_resident_host_workspace_bytes(msm_points_t handle, size_t n, const msm_opts* opts) {
    const size_t core = msm_g1_resident_workspace_bytes(handle, n, opts);
    if (!core) return 0;
    return align_up(core, 256) + align_up(n * 32, 256) + 256;
}

extern "C" int msm_g1_resident_host(msm_points_t handle, size_t offset, size_t n, const uint32_t* scalars_host,
                                    uint32_t* out_host, void* workspace, size_t workspace_bytes,
                                    const msm_opts* opts) {
    if (!handle || !opts || !out_host || !workspace)
        return set_error(MSM377_EINVAL, "msm_g1_resident_host: NULL argument");
    if (n && !scalars_host) return set_error(MSM377_EINVAL, "msm_g1_resident_host: scalars_host is NULL");
    if (opts->flags & MSM377_PROFILE)
        return set_error(MSM377_EINVAL, "msm_g1_resident_host: MSM377_PROFILE is not available here");
    const size_t need = msm_g1_resident_host_workspace_bytes(handle, n, opts);
    if (!need) return set_error(MSM377_EINVAL, "msm_g1_resident_host: bad options");
    if (workspace_bytes < need)
        return set_error(MSM377_ENOMEM, "msm_g1_resident_host: workspace %zu bytes, need %zu", workspace_bytes, need);
    if (!aligned(workspace, 256)) return set_error(MSM377_EINVAL, "msm_g1_resident_host: workspace not 256-byte aligned");
    const size_t core = align_up(msm_g1_resident_workspace_bytes(handle, n, opts), 256);
    char* base = static_cast<char*>(workspace);
    uint32_t* d_sc = reinterpret_cast<uint32_t*>(base + core);
    uint32_t* d_out = reinterpret_cast<uint32_t*>(base + core + align_up(n * 32, 256));
    cudaStream_t s = as_stream(opts->stream);
    if (n) MSM_CUDA_TRY(cudaMemcpyAsync(d_sc, scalars_host, n * 32, cudaMemcpyHostToDevice, s));
    int r = msm_g1_resident(handle, offset, n, d_sc, d_out, workspace, core, opts);
    if (r) return r;
    MSM_CUDA_TRY(cudaMemcpyAsync(out_host, d_out, 24 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    return msm_g1_status(workspace, opts);
}
