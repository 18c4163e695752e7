// Batched field and point kernels behind fq_mul_batch, padd_batch and friends.
//
// One thread owns one independent operation (the GPU form of the paper's
// `single` mapping, a whole PADD per processing element, Sec. IV Table I); the
// batch is spread across threads and SMs. Operands are structure-of-arrays
// ([limb][element]) so each limb load of a warp is one 128-byte coalesced line.
#include <cuda_runtime.h>

#include "common.cuh"
#include "ec.cuh"

namespace {

using ec::affine;
using ec::xyzz;
using fq::fe;

constexpr unsigned kBlock = 256;

__device__ __forceinline__ void load_xyzz_soa(xyzz& P, const uint32_t* base, size_t i, size_t n) {
    fq::load_soa(P.X, base + 0 * 12 * n, i, n);
    fq::load_soa(P.Y, base + 1 * 12 * n, i, n);
    fq::load_soa(P.ZZ, base + 2 * 12 * n, i, n);
    fq::load_soa(P.ZZZ, base + 3 * 12 * n, i, n);
}

__device__ __forceinline__ void store_xyzz_soa(uint32_t* base, size_t i, size_t n, const xyzz& P) {
    fq::store_soa(base + 0 * 12 * n, i, n, P.X);
    fq::store_soa(base + 1 * 12 * n, i, n, P.Y);
    fq::store_soa(base + 2 * 12 * n, i, n, P.ZZ);
    fq::store_soa(base + 3 * 12 * n, i, n, P.ZZZ);
}

__global__ void k_fq_mul(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b,
                         uint32_t* __restrict__ out, size_t n, int form) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        fe x, y, r;
        fq::load_soa(x, a, i, n);
        fq::load_soa(y, b, i, n);
        if (form == MSM377_FORM_STANDARD) {
            // mont(x * R^2) = x R; mont(x R * y) = x y: the standard product.
            fe r2;
#pragma unroll
            for (int k = 0; k < 12; ++k) r2.v[k] = fq::kR2[k];
            fq::mul_inl(x, x, r2);
        }
        fq::mul_inl(r, x, y);
        fq::canon(r, r);
        fq::store_soa(out, i, n, r);
    }
}

__global__ void k_fq_convert(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, size_t n,
                             int to_mont) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        fe x;
        fq::load_soa(x, in, i, n);
        if (to_mont)
            fq::to_mont(x, x);
        else
            fq::from_mont(x, x);
        fq::store_soa(out, i, n, x);
    }
}

__global__ void k_padd(const uint32_t* __restrict__ acc, const uint32_t* __restrict__ q,
                       uint32_t* __restrict__ out, size_t n, int form) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        xyzz P;
        affine Q;
        load_xyzz_soa(P, acc, i, n);
        fq::load_soa(Q.x, q, i, n);
        fq::load_soa(Q.y, q + 12 * n, i, n);
        if (form == MSM377_FORM_STANDARD) {
            fq::to_mont(P.X, P.X);
            fq::to_mont(P.Y, P.Y);
            fq::to_mont(P.ZZ, P.ZZ);
            fq::to_mont(P.ZZZ, P.ZZZ);
            fq::to_mont(Q.x, Q.x);
            fq::to_mont(Q.y, Q.y);
        }
        ec::madd(P, Q);
        if (form == MSM377_FORM_STANDARD) {
            fq::from_mont(P.X, P.X);
            fq::from_mont(P.Y, P.Y);
            fq::from_mont(P.ZZ, P.ZZ);
            fq::from_mont(P.ZZZ, P.ZZZ);
        } else {
            fq::canon(P.X, P.X);
            fq::canon(P.Y, P.Y);
            fq::canon(P.ZZ, P.ZZ);
            fq::canon(P.ZZZ, P.ZZZ);
        }
        store_xyzz_soa(out, i, n, P);
    }
}

__global__ void k_xyzz_to_affine(const uint32_t* __restrict__ in, uint32_t* __restrict__ aff,
                                 size_t n, int form) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        xyzz P;
        load_xyzz_soa(P, in, i, n);
        if (form == MSM377_FORM_STANDARD) {
            fq::to_mont(P.X, P.X);
            fq::to_mont(P.Y, P.Y);
            fq::to_mont(P.ZZ, P.ZZ);
            fq::to_mont(P.ZZZ, P.ZZZ);
        }
        affine A;
        ec::to_affine(A, P);
        if (form == MSM377_FORM_STANDARD) {
            fq::from_mont(A.x, A.x);
            fq::from_mont(A.y, A.y);
        }
        fq::store_soa(aff, i, n, A.x);
        fq::store_soa(aff + 12 * n, i, n, A.y);
    }
}

// Standard BLS12-377 G1 generator, standard form limbs.
__device__ __constant__ uint32_t kGx[12] = {
    0xb21be9efu, 0xeab9b16eu, 0xffcd394eu, 0xd5481512u, 0xbd37cb5cu, 0x188282c8u,
    0xaa9d41bbu, 0x85951e2cu, 0xbf87ff54u, 0xc8fc6225u, 0xfe740a67u, 0x008848deu};
__device__ __constant__ uint32_t kGy[12] = {
    0x559c8ea6u, 0xfd82de55u, 0x34a9591au, 0xc2fe3d36u, 0x4fb82305u, 0x6d182ad4u,
    0xca3e52d9u, 0xbd7fb348u, 0x30afeec4u, 0x1f674f5du, 0xc5102effu, 0x01914a69u};

// out_i = seeds_i * G by left-to-right double-and-add, then affine.
__global__ void k_gen_mul(const uint32_t* __restrict__ seeds, size_t n, uint32_t* __restrict__ out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        affine G;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            G.x.v[k] = kGx[k];
            G.y.v[k] = kGy[k];
        }
        fq::to_mont(G.x, G.x);
        fq::to_mont(G.y, G.y);
        uint32_t s[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) s[k] = seeds[8 * i + k];
        xyzz P;
        ec::set_inf(P);
        bool inf = true;
        for (int bit = 255; bit >= 0; --bit) {
            if (!inf) ec::dbl(P);
            if ((s[bit >> 5] >> (bit & 31)) & 1u) ec::madd(P, inf, G);
        }
        affine A;
        ec::to_affine(A, P);
        if (!ec::is_inf(A)) {
            fq::from_mont(A.x, A.x);
            fq::from_mont(A.y, A.y);
        }
        fq::store(out + 24 * i, A.x);
        fq::store(out + 24 * i + 12, A.y);
    }
}

// Roofline probe: two independent 12-product rows per iteration, each in the shape
// of a Montgomery multiplication row: two carry chains (the products with the
// even- and the odd-indexed limbs), the low and high halves of one product
// adjacent in a chain, which the compiler turns into one wide multiply-add per
// product -- the cheapest form a 32 x 32 -> 64 product takes on the integer
// pipe. Every operand differs from thread to thread: values equal across a warp
// would be computed once per warp on the uniform datapath and overstate the rate.
// Where the probe stores its (never true) "keep the work observable" result.
__device__ uint32_t g_probe_sink[1];

__global__ void k_imad_probe(int iters, uint32_t seed, uint32_t* sink) {
    uint32_t t[13], u[13], v[13], w[13], b[12];
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int k = 0; k < 13; ++k) {
        t[k] = seed + k + tid;
        u[k] = (seed * 3 + k) ^ (tid * 0x85ebca6bu);
        v[k] = (seed * 5 + k) ^ (tid * 0xc2b2ae35u);
        w[k] = (seed * 7 + k) ^ (tid * 0x27d4eb2fu);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) b[k] = seed ^ (0x9e3779b9u * (k + 1)) ^ (tid * 0x165667b1u);
    uint32_t x = tid | 1u, y = (tid * 0x9e3779b9u) | 3u;
    for (int it = 0; it < iters; ++it) {
#define PROBE_CHAIN(T, A, B0, B1, B2, B3, B4, B5)                                                  \
    asm("mad.lo.cc.u32 %0, %13, %14, %0;\n\t"                                                     \
        "madc.hi.cc.u32 %1, %13, %14, %1;\n\t"                                                    \
        "madc.lo.cc.u32 %2, %13, %15, %2;\n\t"                                                    \
        "madc.hi.cc.u32 %3, %13, %15, %3;\n\t"                                                    \
        "madc.lo.cc.u32 %4, %13, %16, %4;\n\t"                                                    \
        "madc.hi.cc.u32 %5, %13, %16, %5;\n\t"                                                    \
        "madc.lo.cc.u32 %6, %13, %17, %6;\n\t"                                                    \
        "madc.hi.cc.u32 %7, %13, %17, %7;\n\t"                                                    \
        "madc.lo.cc.u32 %8, %13, %18, %8;\n\t"                                                    \
        "madc.hi.cc.u32 %9, %13, %18, %9;\n\t"                                                    \
        "madc.lo.cc.u32 %10, %13, %19, %10;\n\t"                                                  \
        "madc.hi.cc.u32 %11, %13, %19, %11;\n\t"                                                  \
        "addc.u32 %12, %12, 0;"                                                                   \
        : "+r"(T[0]), "+r"(T[1]), "+r"(T[2]), "+r"(T[3]), "+r"(T[4]), "+r"(T[5]), "+r"(T[6]),     \
          "+r"(T[7]), "+r"(T[8]), "+r"(T[9]), "+r"(T[10]), "+r"(T[11]), "+r"(T[12])               \
        : "r"(A), "r"(B0), "r"(B1), "r"(B2), "r"(B3), "r"(B4), "r"(B5))
        PROBE_CHAIN(t, x, b[0], b[2], b[4], b[6], b[8], b[10]);
        PROBE_CHAIN(u, x, b[1], b[3], b[5], b[7], b[9], b[11]);
        PROBE_CHAIN(v, y, b[0], b[2], b[4], b[6], b[8], b[10]);
        PROBE_CHAIN(w, y, b[1], b[3], b[5], b[7], b[9], b[11]);
#undef PROBE_CHAIN
        x = t[0] | 1u;
        y = v[1] | 1u;
    }
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < 13; ++k) acc ^= t[k] ^ u[k] ^ v[k] ^ w[k];
    if (acc == 0x12345678u) sink[0] = acc;  // keeps the work observable
}

unsigned batch_grid(size_t n) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t want = (n + kBlock - 1) / kBlock;
    size_t cap = (size_t)sms * 16;  // grid-stride beyond this
    return (unsigned)(want < cap ? (want ? want : 1) : cap);
}

}  // namespace

using namespace msm377;

extern "C" int fq_mul_batch(const uint32_t* a, const uint32_t* b, uint32_t* out, size_t n,
                            int form, void* stream) {
    if (n == 0) return MSM377_OK;
    if (!a || !b || !out || !aligned(a, 4) || !aligned(b, 4) || !aligned(out, 4))
        return set_error(MSM377_EINVAL, "fq_mul_batch: null or misaligned pointer");
    if (form != MSM377_FORM_STANDARD && form != MSM377_FORM_MONTGOMERY)
        return set_error(MSM377_EINVAL, "fq_mul_batch: bad form %d", form);
    k_fq_mul<<<batch_grid(n), kBlock, 0, as_stream(stream)>>>(a, b, out, n, form);
    note_launches(1);
    return check_launch("fq_mul_batch");
}

extern "C" int fq_to_montgomery(const uint32_t* in, uint32_t* out, size_t n, void* stream) {
    if (n == 0) return MSM377_OK;
    if (!in || !out) return set_error(MSM377_EINVAL, "fq_to_montgomery: null pointer");
    k_fq_convert<<<batch_grid(n), kBlock, 0, as_stream(stream)>>>(in, out, n, 1);
    note_launches(1);
    return check_launch("fq_to_montgomery");
}

extern "C" int fq_from_montgomery(const uint32_t* in, uint32_t* out, size_t n, void* stream) {
    if (n == 0) return MSM377_OK;
    if (!in || !out) return set_error(MSM377_EINVAL, "fq_from_montgomery: null pointer");
    k_fq_convert<<<batch_grid(n), kBlock, 0, as_stream(stream)>>>(in, out, n, 0);
    note_launches(1);
    return check_launch("fq_from_montgomery");
}

extern "C" int padd_batch(const uint32_t* acc, const uint32_t* q, uint32_t* out, size_t n, int form,
                          void* stream) {
    if (n == 0) return MSM377_OK;
    if (!acc || !q || !out) return set_error(MSM377_EINVAL, "padd_batch: null pointer");
    if (form != MSM377_FORM_STANDARD && form != MSM377_FORM_MONTGOMERY)
        return set_error(MSM377_EINVAL, "padd_batch: bad form %d", form);
    k_padd<<<batch_grid(n), kBlock, 0, as_stream(stream)>>>(acc, q, out, n, form);
    note_launches(1);
    return check_launch("padd_batch");
}

extern "C" int xyzz_to_affine_batch(const uint32_t* xyzz_in, uint32_t* aff, size_t n, int form,
                                    void* stream) {
    if (n == 0) return MSM377_OK;
    if (!xyzz_in || !aff) return set_error(MSM377_EINVAL, "xyzz_to_affine_batch: null pointer");
    if (form != MSM377_FORM_STANDARD && form != MSM377_FORM_MONTGOMERY)
        return set_error(MSM377_EINVAL, "xyzz_to_affine_batch: bad form %d", form);
    k_xyzz_to_affine<<<batch_grid(n), kBlock, 0, as_stream(stream)>>>(xyzz_in, aff, n, form);
    note_launches(1);
    return check_launch("xyzz_to_affine_batch");
}

extern "C" int g1_generator_mul(const uint32_t* seeds, size_t n, uint32_t* out, void* stream) {
    if (n == 0) return MSM377_OK;
    if (!seeds || !out) return set_error(MSM377_EINVAL, "g1_generator_mul: null pointer");
    k_gen_mul<<<batch_grid(n), kBlock, 0, as_stream(stream)>>>(seeds, n, out);
    note_launches(1);
    return check_launch("g1_generator_mul");
}

extern "C" int msm377_imad_probe(int iters, double* products_per_s, void* stream) {
    if (iters <= 0 || !products_per_s) return set_error(MSM377_EINVAL, "msm377_imad_probe: bad args");
    int dev = 0, sms = 0;
    MSM_CUDA_TRY(cudaGetDevice(&dev));
    MSM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s = as_stream(stream);
    uint32_t* sink = nullptr;
    MSM_CUDA_TRY(cudaGetSymbolAddress(reinterpret_cast<void**>(&sink), g_probe_sink));
    const unsigned block = 256, blocks_per_sm = 8;
    const unsigned grid = (unsigned)sms * blocks_per_sm;
    cudaEvent_t e[2] = {nullptr, nullptr};
    float ms = 0.f;
    cudaError_t err = cudaEventCreate(&e[0]);
    if (err == cudaSuccess) err = cudaEventCreate(&e[1]);
    if (err == cudaSuccess) {
        k_imad_probe<<<grid, block, 0, s>>>(iters / 10 + 1, 1u, sink);  // warm-up
        err = cudaEventRecord(e[0], s);
    }
    if (err == cudaSuccess) {
        k_imad_probe<<<grid, block, 0, s>>>(iters, 7u, sink);
        note_launches(2);
        err = cudaEventRecord(e[1], s);
    }
    if (err == cudaSuccess) err = cudaEventSynchronize(e[1]);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e[0], e[1]);
    for (cudaEvent_t ev : e)
        if (ev) cudaEventDestroy(ev);
    if (err != cudaSuccess) return set_error(MSM377_ECUDA, "msm377_imad_probe: %s", cudaGetErrorString(err));
    double products = (double)grid * block * (double)iters * 2.0 * 12.0;
    *products_per_s = products / ((double)ms * 1e-3);
    return MSM377_OK;
}
