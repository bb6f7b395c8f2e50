// Status strings, thread-local error messages, shared host-side validation,
// the workspace-query dispatcher, the circular-scan helper and the device
// diagnostics for the C ABI declared in include/pmf.h.
#include <math.h>
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

#ifdef PMF_DEBUG
const char* pmf_version(void) { return "pmf-gb300 0.1 (sm_103a, debug: bounds checks)"; }
#else
const char* pmf_version(void) { return "pmf-gb300 0.1 (sm_103a)"; }
#endif

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

pmf_status pmf_circular_views(int32_t P, double sad_mm, double sdd_mm, double du_mm, double dv_mm, int32_t nu,
                              int32_t nv, pmf_view* host_out) {
    PMF_REQUIRE(P >= 0 && (P == 0 || host_out != nullptr), "bad arguments");
    PMF_REQUIRE(nu > 0 && nv > 0, "detector sizes must be positive");
    PMF_REQUIRE(sad_mm > 0.0 && sdd_mm > sad_mm && isfinite(sdd_mm), "need 0 < SAD < SDD");
    PMF_REQUIRE(du_mm > 0.0 && dv_mm > 0.0 && isfinite(du_mm) && isfinite(dv_mm), "pixel pitch must be positive");
    const double two_pi = 6.283185307179586476925287;
    for (int32_t p = 0; p < P; p++) {
        const double th = two_pi * (double)p / (double)P;
        const double c = cos(th), s = sin(th);
        pmf_view& v = host_out[p];
        v.src[0] = sad_mm * c; v.src[1] = sad_mm * s; v.src[2] = 0.0;
        v.det[0] = -(sdd_mm - sad_mm) * c; v.det[1] = -(sdd_mm - sad_mm) * s; v.det[2] = 0.0;
        v.du[0] = -s * du_mm; v.du[1] = c * du_mm; v.du[2] = 0.0;
        v.dv[0] = 0.0; v.dv[1] = 0.0; v.dv[2] = dv_mm;
    }
    return PMF_OK;
}

pmf_status pmf_workspace_size(int32_t op, const pmf_ws_args* a, size_t* bytes) {
    PMF_REQUIRE(a != nullptr && bytes != nullptr, "null pointer");
    switch (op) {
        case PMF_OP_VOXELIZE: return gs_voxelize_workspace(&a->grid, a->n, a->pair_capacity, bytes);
        case PMF_OP_VOXELIZE_BACKWARD: return gs_voxelize_backward_workspace(&a->grid, a->n, a->channels, bytes);
        case PMF_OP_COMBINE_BACKWARD: return mbc_combine_backward_workspace(&a->grid, a->L, a->P, bytes);
        case PMF_OP_WARP_BACKWARD: return warp_volume_backward_workspace(&a->grid, a->P, bytes);
        case PMF_OP_WARP_COMBINE_BACKWARD: return warp_combine_backward_workspace(&a->grid, a->L, a->P, bytes);
        case PMF_OP_PROJECT_BACKWARD: return conebeam_project_backward_workspace(&a->grid, a->P, a->vol_stride, bytes);
        case PMF_OP_LOSS: return projection_loss_workspace(a->count, bytes);
    }
    return pmf::set_error(PMF_EINVAL, "unknown workspace op %d", (int)op);
}

pmf_status pmf_device_counters(uint64_t* host_out, int32_t reset) {
    PMF_REQUIRE(host_out != nullptr, "null pointer");
    unsigned long long sum[PMF_DIAG_COUNT] = {};
    pmf_status st;
    if ((st = pmf::diag_voxelize(sum, reset)) != PMF_OK) return st;
    if ((st = pmf::diag_project(sum, reset)) != PMF_OK) return st;
    if ((st = pmf::diag_warp(sum, reset)) != PMF_OK) return st;
    if ((st = pmf::diag_backproject(sum, reset)) != PMF_OK) return st;
    if ((st = pmf::diag_splat(sum, reset)) != PMF_OK) return st;
    for (int i = 0; i < PMF_DIAG_COUNT; i++) host_out[i] = (uint64_t)sum[i];
    return PMF_OK;
}

pmf_status pmf_device_status(pmf_stream stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return pmf::set_error(PMF_ECUDA, "stream: %s", cudaGetErrorString(e));
    uint64_t c[PMF_DIAG_COUNT];
    pmf_status st = pmf_device_counters(c, 0);
    if (st != PMF_OK) return st;
    if (c[PMF_DIAG_TIMEOUT] != 0)
        return pmf::set_error(PMF_ETIMEOUT, "%llu CTAs gave up waiting for a bulk copy (outputs are NaN)",
                              (unsigned long long)c[PMF_DIAG_TIMEOUT]);
    if (c[PMF_DIAG_BOUNDS] != 0)
        return pmf::set_error(PMF_EINVAL, "%llu accesses failed their bounds check and were skipped (debug build)",
                              (unsigned long long)c[PMF_DIAG_BOUNDS]);
    if (c[PMF_DIAG_NONFINITE] != 0)
        return pmf::set_error(PMF_EINVAL, "%llu launches saw a NaN or infinite input magnitude (outputs are NaN)",
                              (unsigned long long)c[PMF_DIAG_NONFINITE]);
    return PMF_OK;
}

}  // extern "C"
