// msm_g1_noalloc: the MSM entry point for callers that cannot allocate device
// memory. It runs the ordinary msm_g1 with a workspace carved out of one fixed
// array that lives in this file, so the call itself never allocates.
//
// The array is a file-scope __device__ variable: every GPU on which this module
// is loaded holds MSM377_NOALLOC_SCRATCH_BYTES of it until the process exits.
// In host code its name is only a host-side stand-in, never a device address,
// so the address is looked up once per device with cudaGetSymbolAddress (the
// first call on a device does that lookup) and cached.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

static __device__ __align__(256) unsigned char g_msm_noalloc_scratch[MSM377_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 256;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
}  // namespace

using namespace msm377;

extern "C" int msm_g1_noalloc(const uint32_t* points, const uint32_t* scalars, size_t n, uint32_t* out,
                              const msm_opts* opts) {
    if (!opts) return set_error(MSM377_EINVAL, "msm_g1_noalloc: opts is NULL");
    if (opts->flags & MSM377_PROFILE)
        return set_error(MSM377_EINVAL, "msm_g1_noalloc: MSM377_PROFILE is not available on this entry point");
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
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_msm_noalloc_scratch);
            if (e != cudaSuccess)
                return set_error(MSM377_ECUDA, "msm_g1_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_scratch_ptr[dev] = p;
        }
        scratch = g_scratch_ptr[dev];
    }
    return msm_g1(points, scalars, n, out, scratch, (size_t)MSM377_NOALLOC_SCRATCH_BYTES, opts);
}
