// Training-step plans (pmf_plan_*) and the autotuner (pmf_autotune) of the
// projectors' launch shapes and the voxelizer's bin tiles.  A plan composes this library's entry points into one
// forward + adjoint step of Stages 2-3 (Sec. 2.3.2):
//   V = voxelize(ref) (Eq. 4-5), E_l = voxelize(mbc_l) (Sec. 2.3.1),
//   W = warp_combine(V, E, w) (Eq. 3 + Eq. 2), Y = project(W) (Eq. 6),
//   loss, dY = projection_loss(Y, M) (Eq. 10/12 or Eq. 1),
//   dW = project^T(dY), (dV, dE, dw) = warp_combine^T(dW),
//   d(ref), d(mbc_l) = voxelize^T(dV), voxelize^T(dE_l).
// The Gaussian parameters, the batch inputs and the gradient outputs are the
// caller's; the intermediate tensors and every workspace belong to the plan
// (one device allocation).  The step can be captured into a CUDA graph.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "pmf_common.cuh"

struct pmf_plan {
    pmf_batch_desc d;
    int L = 0, B = 0;
    size_t elt = 4;
    int64_t N = 0, Q = 0;
    char* mem = nullptr;
    void *V = nullptr, *E = nullptr, *W = nullptr;
    float *Y = nullptr, *dY = nullptr, *dW = nullptr, *dV = nullptr, *dE = nullptr;
    unsigned* dW_max = nullptr;  // max |dW| from the back-projector, the warp adjoint's fixed-point bound
    void* vox_ws[1 + PMF_MAX_LEVELS] = {};
    size_t vox_bytes[1 + PMF_MAX_LEVELS] = {};
    void* vb_ws[1 + PMF_MAX_LEVELS] = {};
    size_t vb_bytes[1 + PMF_MAX_LEVELS] = {};
    void* bp_ws = nullptr;
    size_t bp_bytes = 0;
    void* wc_ws = nullptr;
    size_t wc_bytes = 0;
    void* loss_ws = nullptr;
    size_t loss_bytes = 0;
    void* ssim_ws = nullptr;  // loss_kind 3 only
    size_t ssim_bytes = 0;
    void* tv_ws = nullptr;
    size_t tv_bytes = 0;
    void* norm_ws = nullptr;
    size_t norm_bytes = 0;
    pmf::MarchShape fp = pmf::default_project_shape(), bp = pmf::default_backproject_shape();  // launch shapes
    int32_t tile[1 + PMF_MAX_LEVELS][3] = {};  // voxelizer bin tile per Gaussian set (reference, then MBC levels)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // the MBC levels' voxelizer calls and adjoints run on their own streams
    cudaStream_t side[PMF_MAX_LEVELS] = {};
    cudaEvent_t fork = nullptr, join[PMF_MAX_LEVELS] = {};
};

namespace pmf {
namespace {

size_t dtype_bytes(pmf_dtype dt) { return dt == PMF_F32 ? 4 : 2; }

const pmf_gaussians& gset(const pmf_batch_desc& d, int i) { return i == 0 ? d.ref : d.mbc[i - 1]; }

pmf_status check_gaussians(const pmf_gaussians& g, int channels, const char* what) {
    PMF_REQUIRE(g.n >= 1, "%s: need at least one Gaussian", what);
    PMF_REQUIRE(g.channels == channels, "%s: channels must be %d", what, channels);
    PMF_REQUIRE(g.mean && g.scale && g.quat && g.value, "%s: null parameter pointer", what);
    PMF_REQUIRE(g.kappa > 0.0f, "%s: kappa must be positive", what);
    return PMF_OK;
}

pmf_status check_desc(const pmf_batch_desc* d) {
    PMF_REQUIRE(d != nullptr, "desc is null");
    pmf_status st = validate_grid(&d->grid);
    if (st != PMF_OK) return st;
    if ((st = validate_dtype(d->dtype)) != PMF_OK) return st;
    PMF_REQUIRE(d->w_dtype == d->dtype || d->w_dtype == PMF_F32, "w_dtype must be dtype or PMF_F32");
    PMF_REQUIRE(d->det.nu > 0 && d->det.nv > 0 && d->det.step_mm > 0.0f, "bad detector");
    PMF_REQUIRE(d->batch >= 1, "batch must be >= 1");
    PMF_REQUIRE(d->loss_kind >= 1 && d->loss_kind <= 3, "loss_kind must be 1 (L1), 2 (L2) or 3 (Eq. 14)");
    if (d->loss_kind == 3) {
        PMF_REQUIRE(isfinite(d->lambda_ssim) && isfinite(d->lambda_mbc) && isfinite(d->lambda_tv),
                    "Eq. 14 weights must be finite");
        PMF_REQUIRE(d->ssim_range > 0.0f && isfinite(d->ssim_range), "ssim_range must be positive");
        PMF_REQUIRE(d->tv_size >= 2 && d->tv_size <= d->grid.nx && d->tv_size <= d->grid.ny &&
                        d->tv_size <= d->grid.nz, "tv_size must be in [2, min(nx, ny, nz)]");
        PMF_REQUIRE(d->tv_origin != nullptr, "tv_origin is null");
    }
    PMF_REQUIRE(d->levels >= 1 && d->levels <= PMF_MAX_LEVELS, "levels must be in [1, %d]", PMF_MAX_LEVELS);
    if ((st = check_gaussians(d->ref, 1, "ref")) != PMF_OK) return st;
    for (int l = 0; l < d->levels; l++) {
        char what[16];
        snprintf(what, sizeof(what), "mbc[%d]", l);
        if ((st = check_gaussians(d->mbc[l], 3, what)) != PMF_OK) return st;
        for (int k = 0; k < 4; k++) PMF_REQUIRE(d->d_mbc[l][k] != nullptr, "d_mbc[%d][%d] is null", l, k);
    }
    for (int k = 0; k < 4; k++) PMF_REQUIRE(d->d_ref[k] != nullptr, "d_ref[%d] is null", k);
    PMF_REQUIRE(d->views && d->coeff && d->meas && d->loss && d->d_coeff, "null batch pointer");
    return PMF_OK;
}

// Key of a configuration in the tuning cache: device, SM count, the plan's
// shapes and the Gaussian counts (the launch forms do not depend on the data;
// the voxelizer's bin tile depends on the sets' sizes).
std::string tune_key(const pmf_batch_desc& d) {
    int dev = 0, sms = 0;
    cudaDeviceProp prop;
    std::string name = "unknown";
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
        name = prop.name;
        sms = prop.multiProcessorCount;
    }
    for (char& c : name)
        if (c == ' ' || c == '\t') c = '_';
    char buf[512];
    snprintf(buf, sizeof(buf), "dev=%s;sm=%d;grid=%dx%dx%d@%g,%g,%g;det=%dx%d@%g;B=%d;L=%d;dtype=%d;w=%d;n=%lld",
             name.c_str(), sms, d.grid.nx, d.grid.ny, d.grid.nz, (double)d.grid.vx, (double)d.grid.vy,
             (double)d.grid.vz, d.det.nu, d.det.nv, (double)d.det.step_mm, d.batch, d.levels, (int)d.dtype,
             (int)d.w_dtype, (long long)d.ref.n);
    std::string key = buf;
    for (int l = 0; l < d.levels; l++) key += "," + std::to_string((long long)d.mbc[l].n);
    return key;
}

std::vector<std::string> read_lines(const char* path) {
    std::vector<std::string> out;
    FILE* f = fopen(path, "r");
    if (!f) return out;
    char line[2048];
    while (fgets(line, sizeof(line), f)) {
        std::string s(line);
        while (!s.empty() && (s.back() == '\n' || s.back() == '\r')) s.pop_back();
        if (!s.empty()) out.push_back(s);
    }
    fclose(f);
    return out;
}

bool valid(const MarchShape& m, bool adjoint) { return pmf::valid_march_shape(m, adjoint); }

bool valid_tile(const int32_t* t) {
    return (t[0] == 8 || t[0] == 16) && t[1] == 8 && (t[2] == 8 || t[2] == 4);
}

// "<key> proj=<form>,<chunk>,<rays> backproj=<form>,<chunk>,<rays>[ vox=<x>x<y>x<z>,...]" (one tile per set)
bool cache_lookup(const char* path, const std::string& key, int sets, MarchShape& fp, MarchShape& bp,
                  int32_t (*tile)[3]) {
    for (const std::string& s : read_lines(path)) {
        if (s.compare(0, key.size(), key) != 0 || s.size() <= key.size() || s[key.size()] != ' ') continue;
        MarchShape a, b;
        int used = 0;
        if (sscanf(s.c_str() + key.size(), " proj=%d,%d,%d backproj=%d,%d,%d%n", &a.form, &a.chunk, &a.rays, &b.form,
                   &b.chunk, &b.rays, &used) != 6 || !valid(a, false) || !valid(b, true))
            continue;
        int32_t t[1 + PMF_MAX_LEVELS][3];
        memcpy(t, tile, sizeof(int32_t) * 3 * (size_t)sets);  // a line without vox= keeps the caller's tiles
        const char* c = s.c_str() + key.size() + used;
        const bool has = strncmp(c, " vox=", 5) == 0;
        bool ok = true;
        c += has ? 5 : 0;
        for (int i = 0; i < sets && ok && has; i++) {
            int n = 0;
            ok = sscanf(c, i == 0 ? "%dx%dx%d%n" : ",%dx%dx%d%n", &t[i][0], &t[i][1], &t[i][2], &n) == 3 &&
                 valid_tile(t[i]);
            c += n;
        }
        if (!ok) continue;
        fp = a;
        bp = b;
        memcpy(tile, t, sizeof(int32_t) * 3 * (size_t)sets);
        return true;
    }
    return false;
}

pmf_status cache_store(const char* path, const std::string& key, const MarchShape& fp, const MarchShape& bp, int sets,
                       const int32_t (*tile)[3]) {
    std::vector<std::string> lines = read_lines(path);
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return set_error(PMF_EINVAL, "cannot write %s", tmp.c_str());
    for (const std::string& s : lines)
        if (!(s.compare(0, key.size(), key) == 0 && s.size() > key.size() && s[key.size()] == ' '))
            fprintf(f, "%s\n", s.c_str());
    fprintf(f, "%s proj=%d,%d,%d backproj=%d,%d,%d vox=", key.c_str(), fp.form, fp.chunk, fp.rays, bp.form, bp.chunk,
            bp.rays);
    for (int i = 0; i < sets; i++) fprintf(f, "%s%dx%dx%d", i ? "," : "", tile[i][0], tile[i][1], tile[i][2]);
    fprintf(f, "\n");
    if (fclose(f) != 0 || rename(tmp.c_str(), path) != 0) return set_error(PMF_EINVAL, "cannot write %s", path);
    return PMF_OK;
}

#define PMF_TRY(expr)                        \
    do {                                     \
        pmf_status st_ = (expr);             \
        if (st_ != PMF_OK) return st_;       \
    } while (0)

#define PMF_TRY_CUDA(expr, what)                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (expr);                                                                   \
        if (e_ != cudaSuccess) return set_error(PMF_ECUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

pmf_status plan_project(pmf_plan* p, cudaStream_t s) {
    const pmf_batch_desc& d = p->d;
    pmf_project_item it{d.grid, d.det, p->B, d.views, p->W, p->N, p->Y};
    return project_launch(it, d.w_dtype, p->fp, s);
}

pmf_status plan_backproject(pmf_plan* p, cudaStream_t s) {
    const pmf_batch_desc& d = p->d;
    pmf_backproject_item it{d.grid, d.det, p->B, d.views, p->dY, p->dW, p->N};
    return backproject_launch(it, 0, p->bp_ws, p->bp_bytes, p->bp, s, p->dW_max);
}

pmf_status enqueue_step(pmf_plan* p, cudaStream_t s) {
    const pmf_batch_desc& d = p->d;
    const pmf_stream ps = (pmf_stream)s;
    const int64_t N = p->N;
    // fork: each MBC level voxelizes on its side stream, the reference set here
    PMF_TRY_CUDA(cudaEventRecord(p->fork, s), "cudaEventRecord");
    for (int l = 0; l < p->L; l++) {
        PMF_TRY_CUDA(cudaStreamWaitEvent(p->side[l], p->fork, 0), "cudaStreamWaitEvent");
        PMF_TRY(gs_voxelize_tiled(&d.grid, &d.mbc[l], d.dtype, p->tile[1 + l], (char*)p->E + (size_t)l * 3 * N * p->elt,
                                  p->vox_ws[1 + l], p->vox_bytes[1 + l], (pmf_stream)p->side[l]));
        PMF_TRY_CUDA(cudaEventRecord(p->join[l], p->side[l]), "cudaEventRecord");
    }
    PMF_TRY(gs_voxelize_tiled(&d.grid, &d.ref, d.dtype, p->tile[0], p->V, p->vox_ws[0], p->vox_bytes[0], ps));
    for (int l = 0; l < p->L; l++) PMF_TRY_CUDA(cudaStreamWaitEvent(s, p->join[l], 0), "cudaStreamWaitEvent");
    PMF_TRY(warp_combine_mixed(&d.grid, p->L, p->B, d.dtype, p->V, p->E, d.coeff, d.w_dtype, p->W, ps));
    PMF_TRY(plan_project(p, s));
    const bool eq14 = d.loss_kind == 3;
    PMF_TRY(projection_loss(eq14 ? 1 : d.loss_kind, p->B, p->Q, p->Y, d.meas, d.loss, p->dY, p->loss_ws,
                            p->loss_bytes, ps));
    if (eq14)
        PMF_TRY(projection_dssim(p->B, d.det.nu, d.det.nv, p->Y, d.meas, d.ssim_range, d.lambda_ssim, d.loss, p->dY, 1,
                                 p->ssim_ws, p->ssim_bytes, ps));
    PMF_TRY(plan_backproject(p, s));
    PMF_TRY(warp_combine_backward_bounded(&d.grid, p->L, p->B, d.dtype, p->V, p->E, d.coeff, p->dW, p->dW_max, p->dV,
                                          p->dE, d.d_coeff, 0, p->wc_ws, p->wc_bytes, ps));
    if (eq14) {
        PMF_TRY(tv_loss(&d.grid, d.dtype, p->V, d.tv_size, d.tv_origin, d.lambda_tv, d.loss, p->dV, 1, p->tv_ws,
                        p->tv_bytes, ps));
        PMF_TRY(mbc_normality(&d.grid, p->L, d.dtype, p->E, d.lambda_mbc, d.loss, p->dE, 1, p->norm_ws, p->norm_bytes,
                              ps));
    }
    // the same fork for the voxelizer adjoints, joined before the step ends
    PMF_TRY_CUDA(cudaEventRecord(p->fork, s), "cudaEventRecord");
    for (int l = 0; l < p->L; l++) {
        PMF_TRY_CUDA(cudaStreamWaitEvent(p->side[l], p->fork, 0), "cudaStreamWaitEvent");
        PMF_TRY(gs_voxelize_backward(&d.grid, &d.mbc[l], p->dE + (size_t)l * 3 * N, d.d_mbc[l][0], d.d_mbc[l][1],
                                     d.d_mbc[l][2], d.d_mbc[l][3], 0, p->vb_ws[1 + l], p->vb_bytes[1 + l],
                                     (pmf_stream)p->side[l]));
        PMF_TRY_CUDA(cudaEventRecord(p->join[l], p->side[l]), "cudaEventRecord");
    }
    PMF_TRY(gs_voxelize_backward(&d.grid, &d.ref, p->dV, d.d_ref[0], d.d_ref[1], d.d_ref[2], d.d_ref[3], 0,
                                 p->vb_ws[0], p->vb_bytes[0], ps));
    for (int l = 0; l < p->L; l++) PMF_TRY_CUDA(cudaStreamWaitEvent(s, p->join[l], 0), "cudaStreamWaitEvent");
    return PMF_OK;
}

// Pair-list capacity of each voxelizer: the exact (Gaussian, tile) overlap
// count of the current parameters with 25% headroom (overflow later is still
// correct, only slower; PMF_DIAG_VOXELIZE_LIST_OVERFLOW counts it).
pmf_status pair_capacities(const pmf_batch_desc& d, const int32_t (*tile)[3], int64_t* cap) {
    const int sets = 1 + d.levels;
    size_t need = 0;
    for (int i = 0; i < sets; i++) {
        size_t b;
        PMF_TRY(gs_voxelize_tiled_workspace(&d.grid, gset(d, i).n, 0, tile[i], &b));
        need = b > need ? b : need;
    }
    char* tmp = nullptr;
    PMF_TRY_CUDA(cudaMalloc(&tmp, need + 256), "cudaMalloc");
    pmf_status st = PMF_OK;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(tmp);
        return set_error(PMF_ECUDA, "cudaStreamCreate failed");
    }
    int64_t* d_pairs = (int64_t*)(tmp + need);
    for (int i = 0; i < sets && st == PMF_OK; i++) {
        st = gs_voxelize_tiled_count(&d.grid, &gset(d, i), tile[i], d_pairs, tmp, need, (pmf_stream)s);
        int64_t h = 0;
        if (st == PMF_OK && cudaMemcpyAsync(&h, d_pairs, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            st = set_error(PMF_ECUDA, "pair count copy failed");
        if (st == PMF_OK && cudaStreamSynchronize(s) != cudaSuccess) st = set_error(PMF_ECUDA, "pair count failed");
        cap[i] = h + h / 4 + 4096;
    }
    cudaStreamDestroy(s);
    cudaFree(tmp);
    return st;
}

void plan_free(pmf_plan* p);

pmf_status plan_create(const pmf_batch_desc* desc, pmf_plan** out) {
    PMF_TRY(check_desc(desc));
    pmf_plan* p = new pmf_plan();
    p->d = *desc;
    p->d.tune_cache = nullptr;  // the caller's string need not outlive the call
    p->L = desc->levels;
    p->B = desc->batch;
    p->elt = dtype_bytes(desc->dtype);
    p->N = (int64_t)desc->grid.nx * desc->grid.ny * desc->grid.nz;
    p->Q = (int64_t)desc->det.nu * desc->det.nv;
    const pmf_batch_desc& d = p->d;
    const int sets = 1 + p->L;
    for (int i = 0; i < sets; i++) {
        p->tile[i][0] = 8;
        p->tile[i][1] = 8;
        p->tile[i][2] = 8;
    }
    if (desc->tune_cache) cache_lookup(desc->tune_cache, tune_key(d), sets, p->fp, p->bp, p->tile);
    int64_t cap[1 + PMF_MAX_LEVELS];
    pmf_status st = pair_capacities(d, p->tile, cap);
    if (st != PMF_OK) {
        delete p;
        return st;
    }
    // sizes, then one allocation carved at 256-byte boundaries
    std::vector<size_t> sz;
    const size_t N = (size_t)p->N, B = (size_t)p->B, L = (size_t)p->L, Q = (size_t)p->Q;
    sz.push_back(N * p->elt);                 // V
    sz.push_back(L * 3 * N * p->elt);         // E
    sz.push_back(B * N * dtype_bytes(d.w_dtype));  // W
    sz.push_back(B * Q * 4);                  // Y
    sz.push_back(B * Q * 4);                  // dY
    sz.push_back(B * N * 4);                  // dW
    sz.push_back(N * 4);                      // dV
    sz.push_back(L * 3 * N * 4);              // dE
    sz.push_back(sizeof(unsigned));           // dW_max
    for (int i = 0; i < sets && st == PMF_OK; i++) {
        st = gs_voxelize_tiled_workspace(&d.grid, gset(d, i).n, cap[i], p->tile[i], &p->vox_bytes[i]);
        if (st == PMF_OK) st = gs_voxelize_backward_workspace(&d.grid, gset(d, i).n, gset(d, i).channels, &p->vb_bytes[i]);
    }
    if (st == PMF_OK) st = conebeam_project_backward_workspace(&d.grid, p->B, p->N, &p->bp_bytes);
    if (st == PMF_OK) st = warp_combine_backward_workspace(&d.grid, p->L, p->B, &p->wc_bytes);
    if (st == PMF_OK) st = projection_loss_workspace((int64_t)(B * Q), &p->loss_bytes);
    if (st == PMF_OK && desc->loss_kind == 3) {
        st = projection_dssim_workspace(p->B, desc->det.nu, desc->det.nv, &p->ssim_bytes);
        if (st == PMF_OK) st = tv_loss_workspace(desc->tv_size, &p->tv_bytes);
        if (st == PMF_OK) st = mbc_normality_workspace(p->L, &p->norm_bytes);
    }
    if (st != PMF_OK) {
        delete p;
        return st;
    }
    for (int i = 0; i < sets; i++) sz.push_back(p->vox_bytes[i]);
    for (int i = 0; i < sets; i++) sz.push_back(p->vb_bytes[i]);
    sz.push_back(p->bp_bytes);
    sz.push_back(p->wc_bytes);
    sz.push_back(p->loss_bytes);
    sz.push_back(p->ssim_bytes);
    sz.push_back(p->tv_bytes);
    sz.push_back(p->norm_bytes);
    size_t total = 0;
    for (size_t b : sz) total += align_up(b ? b : 1);
    if (cudaMalloc(&p->mem, total) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return set_error(PMF_ECUDA, "cudaMalloc of %zu bytes for the plan failed", total);
    }
    char* cur = p->mem;
    size_t k = 0;
    auto take = [&]() {
        char* r = cur;
        cur += align_up(sz[k] ? sz[k] : 1);
        k++;
        return (void*)r;
    };
    p->V = take();
    p->E = take();
    p->W = take();
    p->Y = (float*)take();
    p->dY = (float*)take();
    p->dW = (float*)take();
    p->dV = (float*)take();
    p->dE = (float*)take();
    p->dW_max = (unsigned*)take();
    for (int i = 0; i < sets; i++) p->vox_ws[i] = take();
    for (int i = 0; i < sets; i++) p->vb_ws[i] = take();
    p->bp_ws = take();
    p->wc_ws = take();
    p->loss_ws = take();
    p->ssim_ws = take();
    p->tv_ws = take();
    p->norm_ws = take();
    bool ok = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int l = 0; l < p->L && ok; l++)
        ok = cudaStreamCreateWithFlags(&p->side[l], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&p->join[l], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        plan_free(p);
        return set_error(PMF_ECUDA, "plan streams: %s", cudaGetErrorString(cudaGetLastError()));
    }
    *out = p;
    return PMF_OK;
}

void plan_free(pmf_plan* p) {
    if (!p) return;
    cudaDeviceSynchronize();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->mem) cudaFree(p->mem);
    for (int l = 0; l < PMF_MAX_LEVELS; l++) {
        if (p->side[l]) cudaStreamDestroy(p->side[l]);
        if (p->join[l]) cudaEventDestroy(p->join[l]);
    }
    if (p->fork) cudaEventDestroy(p->fork);
    delete p;
}

float time_ms(cudaStream_t s, int reps, pmf_status (*fn)(pmf_plan*, cudaStream_t), pmf_plan* p, pmf_status& st) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    st = fn(p, s);  // warm-up
    float best = 3.0e38f;
    for (int r = 0; r < reps && st == PMF_OK; r++) {
        cudaEventRecord(a, s);
        st = fn(p, s);
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess) st = set_error(PMF_ECUDA, "timing failed");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        best = ms < best ? ms : best;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

// Best of `reps` timed voxelizations of Gaussian set i with bin tile `tile`,
// after one warm-up; the workspace holds the tile's exact pair count (+25%)
// and the output goes to the plan's own V or E slice.
float time_voxelize(pmf_plan* p, int i, const int32_t tile[3], cudaStream_t s, int reps, pmf_status& st) {
    const pmf_batch_desc& d = p->d;
    const pmf_gaussians& gs = gset(d, i);
    void* out = i == 0 ? p->V : (char*)p->E + (size_t)(i - 1) * 3 * (size_t)p->N * p->elt;
    float best = 3.0e38f;
    size_t fixed = 0, need = 0;
    st = gs_voxelize_tiled_workspace(&d.grid, gs.n, 0, tile, &fixed);
    char* ws = nullptr;
    if (st == PMF_OK && cudaMalloc(&ws, fixed + 256) != cudaSuccess) st = set_error(PMF_ECUDA, "cudaMalloc failed");
    int64_t pairs = 0;
    if (st == PMF_OK) st = gs_voxelize_tiled_count(&d.grid, &gs, tile, (int64_t*)(ws + fixed), ws, fixed, (pmf_stream)s);
    if (st == PMF_OK && (cudaMemcpyAsync(&pairs, ws + fixed, sizeof(pairs), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                         cudaStreamSynchronize(s) != cudaSuccess))
        st = set_error(PMF_ECUDA, "pair count failed");
    if (ws) cudaFree(ws);
    ws = nullptr;
    if (st == PMF_OK) st = gs_voxelize_tiled_workspace(&d.grid, gs.n, pairs + pairs / 4 + 4096, tile, &need);
    if (st == PMF_OK && cudaMalloc(&ws, need) != cudaSuccess) st = set_error(PMF_ECUDA, "cudaMalloc failed");
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (int r = -1; r < reps && st == PMF_OK; r++) {
        cudaEventRecord(a, s);
        st = gs_voxelize_tiled(&d.grid, &gs, d.dtype, tile, out, ws, need, (pmf_stream)s);
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess) st = set_error(PMF_ECUDA, "timing failed");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (r >= 0) best = ms < best ? ms : best;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (ws) cudaFree(ws);
    return best;
}

}  // namespace
}  // namespace pmf

using namespace pmf;

extern "C" {

pmf_status pmf_plan_create(const pmf_batch_desc* desc, pmf_plan** plan) {
    PMF_REQUIRE(plan != nullptr, "plan is null");
    *plan = nullptr;
    return plan_create(desc, plan);
}

pmf_status pmf_plan_step(pmf_plan* p, pmf_stream stream) {
    PMF_REQUIRE(p != nullptr, "plan is null");
    cudaStream_t s = (cudaStream_t)stream;
    if (!p->d.use_graph) return enqueue_step(p, s);
    if (!p->exec) {
        PMF_REQUIRE(s != nullptr, "a graph-captured plan needs a created stream, not the NULL stream");
        PMF_TRY_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        pmf_status st = enqueue_step(p, s);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st != PMF_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return st != PMF_OK ? st : set_error(PMF_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&p->exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            p->exec = nullptr;
            return set_error(PMF_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        }
        p->graph = g;
    }
    PMF_TRY_CUDA(cudaGraphLaunch(p->exec, s), "cudaGraphLaunch");
    return PMF_OK;
}

pmf_status pmf_plan_tensors_get(const pmf_plan* p, pmf_plan_tensors* out) {
    PMF_REQUIRE(p != nullptr && out != nullptr, "null pointer");
    out->V = p->V;
    out->E = p->E;
    out->W = p->W;
    out->Y = p->Y;
    out->dY = p->dY;
    out->dW = p->dW;
    out->dV = p->dV;
    out->dE = p->dE;
    return PMF_OK;
}

pmf_status pmf_plan_launch_forms(const pmf_plan* p, int32_t* proj, int32_t* backproj) {
    PMF_REQUIRE(p != nullptr && proj != nullptr && backproj != nullptr, "null pointer");
    proj[0] = p->fp.form; proj[1] = p->fp.chunk; proj[2] = p->fp.rays;
    backproj[0] = p->bp.form; backproj[1] = p->bp.chunk; backproj[2] = p->bp.rays;
    return PMF_OK;
}

pmf_status pmf_plan_destroy(pmf_plan* p) {
    plan_free(p);
    return PMF_OK;
}

pmf_status pmf_autotune(const pmf_batch_desc* desc, const char* cache_path) {
    PMF_REQUIRE(cache_path != nullptr && cache_path[0] != '\0', "cache_path is empty");
    pmf_batch_desc d = *desc;
    d.use_graph = 0;
    d.tune_cache = nullptr;
    pmf_plan* p = nullptr;
    PMF_TRY(plan_create(&d, &p));
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        plan_free(p);
        return set_error(PMF_ECUDA, "cudaStreamCreate failed");
    }
    pmf_status st = enqueue_step(p, s);  // fills W and dY
    // every (form, chunk, rays): forms 0 (grid) and 2-4 persistent CTAs per
    // 1024 threads of an SM, bricks of 16, 32 or 48 samples (the adjoint also
    // 64), 128 or 256 rays
    float best_fp = 3.0e38f, best_bp = 3.0e38f;
    MarchShape fp, bp;
    for (int chunk : {32, 16, 48, 64})
        for (int rays : {256, 128})
            for (int form : {0, 1, 2, 4}) {
                if (st != PMF_OK) break;
                MarchShape m;
                m.form = form == 0 ? 0 : form * (256 / rays);
                m.chunk = chunk;
                m.rays = rays;
                float t;
                if (chunk <= 48) {
                    p->fp = m;
                    t = time_ms(s, 3, plan_project, p, st);
                    if (st == PMF_OK && t < best_fp) { best_fp = t; fp = m; }
                    if (st != PMF_OK) break;
                }
                p->bp = m;
                t = time_ms(s, 3, plan_backproject, p, st);
                if (st == PMF_OK && t < best_bp) { best_bp = t; bp = m; }
            }
    // the voxelizer's bin tile, per Gaussian set
    const int sets = 1 + d.levels;
    const int32_t cand[4][3] = {{8, 8, 8}, {16, 8, 8}, {8, 8, 4}, {16, 8, 4}};
    int32_t tile[1 + PMF_MAX_LEVELS][3];
    for (int i = 0; i < sets; i++) {
        float best = 3.0e38f;
        memcpy(tile[i], cand[0], sizeof(cand[0]));
        for (int c = 0; c < 4 && st == PMF_OK; c++) {
            const float t = time_voxelize(p, i, cand[c], s, 3, st);
            if (st == PMF_OK && t < best) {
                best = t;
                memcpy(tile[i], cand[c], sizeof(cand[c]));
            }
        }
    }
    if (st == PMF_OK && cudaStreamSynchronize(s) != cudaSuccess) st = set_error(PMF_ECUDA, "autotune failed");
    const std::string key = tune_key(d);
    cudaStreamDestroy(s);
    plan_free(p);
    if (st != PMF_OK) return st;
    return cache_store(cache_path, key, fp, bp, sets, tile);
}

pmf_status pmf_plan_voxel_tiles(const pmf_plan* p, int32_t* tiles) {
    PMF_REQUIRE(p != nullptr && tiles != nullptr, "null pointer");
    for (int i = 0; i <= p->L; i++)
        for (int k = 0; k < 3; k++) tiles[3 * i + k] = p->tile[i][k];
    return PMF_OK;
}

}  // extern "C"
