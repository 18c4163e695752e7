// msm_g1_noalloc: the MSM entry point for callers that cannot allocate device
// memory. It runs the ordinary msm_g1 with a workspace carved out of one fixed
// array that lives in this file, so the call itself never allocates.
//
// The array is a file-scope __device__ variable: every GPU on which this module
// is loaded holds MSM377_NOALLOC_SCRATCH_BYTES of it until the process exits.
// In host code its name is only a host-side stand-in, never a device address,
// so the address is looked up with cudaGetSymbolAddress, once per device and CUDA
// context, by the first call made there, and cached together with that context.
// A module's globals live in each context that loads the module: a call made from
// another context (a driver-API context, or the primary context re-created after
// cudaDeviceReset) looks the address up again instead of using a stale one.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

static __device__ __align__(256) unsigned char g_msm_noalloc_scratch[MSM377_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 256;
std::mutex g_scratch_mu;
struct Scratch {
    CUcontext ctx = nullptr;  // context the address belongs to
    void* ptr = nullptr;
};
Scratch g_scratch[kMaxDevices];

// cuCtxGetCurrent through the runtime's driver entry-point lookup (no link
// dependency on the driver library).
typedef CUresult (*CtxGetCurrent)(CUcontext*);
CtxGetCurrent g_ctx_get = nullptr;

int current_context(CUcontext* ctx) {
    if (!g_ctx_get) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return msm377::set_error(MSM377_ECUDA, "msm_g1_noalloc: cuCtxGetCurrent not available");
        g_ctx_get = reinterpret_cast<CtxGetCurrent>(fn);
    }
    if (g_ctx_get(ctx) != CUDA_SUCCESS) return msm377::set_error(MSM377_ECUDA, "msm_g1_noalloc: cuCtxGetCurrent failed");
    return MSM377_OK;
}
}  // namespace

using namespace msm377;

extern "C" int msm_g1_noalloc(const uint32_t* points, const uint32_t* scalars, size_t n, uint32_t* out,
                              const msm_opts* opts) {
    if (!opts) return set_error(MSM377_EINVAL, "msm_g1_noalloc: opts is NULL");
    if (opts->flags & (MSM377_PROFILE | MSM377_VALIDATE))
        return set_error(MSM377_EINVAL, "msm_g1_noalloc: MSM377_PROFILE and MSM377_VALIDATE are not available on "
                         "this entry point (it reports no device status)");
    const size_t need = msm_g1_workspace_bytes(n, opts);
    if (need == 0)
        return set_error(MSM377_EINVAL, "msm_g1_noalloc: bad options (c=%d scalar_bits=%d) or n too large",
                         opts->c, opts->scalar_bits);
    if (need > (size_t)MSM377_NOALLOC_SCRATCH_BYTES)
        return set_error(MSM377_EINVAL,
                         "msm_g1_noalloc: n = %zu with these options needs %zu bytes of scratch, more than "
                         "the fixed %zu bytes this entry point has; use msm_g1 with a caller workspace",
                         n, need, (size_t)MSM377_NOALLOC_SCRATCH_BYTES);
    int dev = 0;
    MSM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(MSM377_EINVAL, "msm_g1_noalloc: device ordinal %d out of range", dev);
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        CUcontext ctx = nullptr;
        int r = current_context(&ctx);
        if (r) return r;
        Scratch& sc = g_scratch[dev];
        if (!sc.ptr || !ctx || ctx != sc.ctx) {
            // set-up for this device and context (the lookup also makes the
            // device's primary context current when no context is yet)
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_msm_noalloc_scratch);
            if (e != cudaSuccess)
                return set_error(MSM377_ECUDA, "msm_g1_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            r = current_context(&ctx);
            if (r) return r;
            sc.ctx = ctx;
            sc.ptr = p;
        }
        scratch = sc.ptr;
    }
    // no overlap helper: this entry point creates no stream or event either
    return msm_g1_run(points, scalars, n, out, scratch, (size_t)MSM377_NOALLOC_SCRATCH_BYTES, opts, false);
}
