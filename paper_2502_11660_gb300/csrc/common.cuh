// Shared host-side helpers of the msm377 library: error reporting, status
// codes, alignment and stream casting.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/msm377.h"

namespace msm377 {

// Records a message for msm377_last_error (thread-local) and returns `code`.
int set_error(int code, const char* fmt, ...);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Checks the launch that was just enqueued.
int check_launch(const char* what);

// Host-side count of kernel launches (msm377_launch_count).
void note_launches(unsigned k);

// Stage events of a profiled msm_g1 call: reset, then record after each stage.
int profile_begin(cudaStream_t s);
int profile_mark(cudaStream_t s);

// Enqueues the check of n affine standard-form points (24 u32 each, 16-byte
// aligned) on s: coordinates below p and on y^2 = x^3 + 1 ((0, 0) is O), and with
// `subgroup` also r P = O. The first failing point stores MSM377_ENOTONCURVE into
// *status (device memory) unless it already holds an error.
int launch_validate(const uint32_t* points_std, size_t n, bool subgroup, int* status, cudaStream_t s);

// msm_g1 with the tails of window groups overlapped on a helper stream (overlap)
// or run in order on the caller's stream (no stream or event is created).
int msm_g1_run(const uint32_t* points, const uint32_t* scalars, size_t n, uint32_t* out, void* workspace,
               size_t workspace_bytes, const msm_opts* opts, bool overlap);

inline unsigned grid_for(size_t n, unsigned block) {
    return static_cast<unsigned>((n + block - 1) / block);
}

}  // namespace msm377

#define MSM_CUDA_TRY(expr)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return ::msm377::set_error(MSM377_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)
