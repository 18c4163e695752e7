// Error state and version of the msm377 C-ABI.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "common.cuh"

namespace {
thread_local char g_err[512] = {0};
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

}  // namespace msm377

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
