// Status strings, thread-local error messages and shared host-side validation
// for the C ABI declared in include/pmf.h.
#include <stdarg.h>
#include <stdio.h>

#include "pmf_common.cuh"

namespace pmf {

static thread_local char g_msg[512] = "";

pmf_status set_error(pmf_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return st;
}

pmf_status check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(PMF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return PMF_OK;
}

pmf_status validate_grid(const pmf_grid* g) {
    PMF_REQUIRE(g != nullptr, "grid is null");
    PMF_REQUIRE(g->nx > 0 && g->ny > 0 && g->nz > 0, "grid sizes must be positive (%d,%d,%d)", g->nx, g->ny, g->nz);
    PMF_REQUIRE(g->vx > 0.f && g->vy > 0.f && g->vz > 0.f, "voxel sizes must be positive");
    PMF_REQUIRE(isfinite(g->vx) && isfinite(g->vy) && isfinite(g->vz), "voxel sizes must be finite");
    int64_t n = (int64_t)g->nx * g->ny * g->nz;
    PMF_REQUIRE(n < ((int64_t)1 << 40), "grid too large");
    PMF_REQUIRE(g->nx < (1 << 24) && g->ny < (1 << 24) && g->nz < (1 << 24), "grid axis too long");
    return PMF_OK;
}

pmf_status validate_dtype(pmf_dtype dt) {
    PMF_REQUIRE(dt == PMF_F32 || dt == PMF_BF16 || dt == PMF_F16, "unknown dtype %d", (int)dt);
    return PMF_OK;
}

pmf_status validate_ws(const void* ws, size_t ws_bytes, size_t need) {
    if (need == 0) return PMF_OK;
    if (ws == nullptr || ws_bytes < need)
        return set_error(PMF_EWORKSPACE, "workspace needs %zu bytes, got %zu", need, ws ? ws_bytes : (size_t)0);
    if (((uintptr_t)ws & 255u) != 0) return set_error(PMF_EWORKSPACE, "workspace must be 256-byte aligned");
    return PMF_OK;
}

}  // namespace pmf

extern "C" {

const char* pmf_version(void) { return "pmf-gb300 0.1 (sm_103a)"; }

const char* pmf_last_error(void) { return pmf::g_msg; }

const char* pmf_status_string(pmf_status s) {
    switch (s) {
        case PMF_OK: return "ok";
        case PMF_EINVAL: return "invalid argument";
        case PMF_ECUDA: return "CUDA error";
        case PMF_EWORKSPACE: return "workspace too small";
        case PMF_ETIMEOUT: return "device wait timed out";
        case PMF_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

}  // extern "C"
