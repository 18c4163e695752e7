// Error state and version of the msm377 C-ABI.
#include <cuda_runtime.h>
#include <stdarg.h>

#include <atomic>
#include <stdio.h>
#include <string.h>

#include "common.cuh"

namespace {
thread_local char g_err[512] = {0};
std::atomic<uint64_t> g_launches{0};
constexpr int kMaxEvents = 16;
cudaEvent_t g_ev[kMaxEvents];
bool g_ev_ready = false;
int g_ev_used = 0;
}

namespace msm377 {

int set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(MSM377_ECUDA, "%s: launch failed: %s", what, cudaGetErrorString(e));
    return MSM377_OK;
}

void note_launches(unsigned k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int profile_begin(cudaStream_t s) {
    if (!g_ev_ready) {
        for (int i = 0; i < kMaxEvents; ++i) MSM_CUDA_TRY(cudaEventCreate(&g_ev[i]));
        g_ev_ready = true;
    }
    g_ev_used = 0;
    return profile_mark(s);
}

int profile_mark(cudaStream_t s) {
    if (!g_ev_ready || g_ev_used >= kMaxEvents) return MSM377_OK;
    MSM_CUDA_TRY(cudaEventRecord(g_ev[g_ev_used], s));
    ++g_ev_used;
    return MSM377_OK;
}

}  // namespace msm377

extern "C" int msm377_profile_last(float* ms, int cap) {
    if (!g_ev_ready || g_ev_used < 2) return msm377::set_error(MSM377_EINVAL, "no profiled call recorded");
    MSM_CUDA_TRY(cudaEventSynchronize(g_ev[g_ev_used - 1]));
    int stages = g_ev_used - 1;
    for (int i = 0; i < stages && i < cap; ++i) {
        float t = 0.f;
        MSM_CUDA_TRY(cudaEventElapsedTime(&t, g_ev[i], g_ev[i + 1]));
        ms[i] = t;
    }
    return stages;
}

extern "C" uint64_t msm377_launch_count(void) { return g_launches.load(); }

extern "C" int msm377_last_error(char* buf, size_t len) {
    size_t n = strlen(g_err);
    if (buf && len) {
        size_t c = n < len - 1 ? n : len - 1;
        memcpy(buf, g_err, c);
        buf[c] = 0;
    }
    return (int)n;
}

extern "C" int msm377_version(void) { return 100; }
