/*
 * pmf.h -- C ABI of the GB300 (sm_103a) library for the PMF-STGR forward model
 * and its adjoint (Xie, Shao & Zhang, "Time-resolved dynamic CBCT reconstruction
 * using prior-model-free spatiotemporal Gaussian representation").
 *
 * The model (Sec. 2.1-2.3): a reference volume voxelized from 3-D Gaussians
 * (Eq. 4-5), motion-basis components (MBCs) voxelized from signed Gaussians
 * (Sec. 2.3.1), per-projection DVFs d = sum_l w_l(p) x e_l (Eq. 3), the warped
 * volume I(x,p) = I_ref(x + d(x,p)) (Eq. 2), and cone-beam line integrals of it
 * (Eq. 6) compared with the measured projection under an L1 (Eq. 10/12) or L2
 * (Eq. 1) loss.
 *
 * Conventions (every call):
 *  - Pointers named d_* or marked "device" are CUDA device pointers; host
 *    structs (pmf_grid, pmf_detector, pmf_gaussians) are read on the host
 *    during the call and may be freed on return.  The caller owns every buffer;
 *    the library never allocates or frees device memory, except in
 *    pmf_plan_create / pmf_plan_destroy (a plan owns its intermediate tensors).
 *  - All device work is enqueued on `stream` (a cudaStream_t; NULL = legacy
 *    default stream) and is asynchronous: inputs must stay alive and unchanged
 *    until the stream reaches the work.  No call synchronizes.
 *  - Volumes are [nz][ny][nx], x fastest, centred on the isocentre: voxel
 *    (i,j,k) sits at ((i + 1/2 - nx/2) vx, (j + 1/2 - ny/2) vy, (k + 1/2 - nz/2) vz) mm.
 *    Trilinear interpolation reads voxels outside [0, n-1] as zero.
 *  - A DVF is SoA [P][3][N] in mm; MBC grids are [L][3][N]; temporal
 *    coefficients are float [P][L][3]; projections are float [P][nv][nu].
 *  - `dtype` is the storage type of volumes, MBC grids, DVFs and warped
 *    volumes (fp32, bf16 or fp16, round-to-nearest-even on store).  Every
 *    interpolation, ray sum and reduction runs in fp32; gradients are fp32.
 *  - Gradient outputs: accumulate = 0 overwrites, accumulate = 1 adds.
 *  - Scatter-type adjoints (back-projection, warp transpose) accumulate in
 *    64-bit fixed point with a power-of-two scale chosen per call from the
 *    largest input magnitude, so results are bit-reproducible run to run.
 *  - Errors: host-side validation happens before any launch and returns
 *    PMF_EINVAL / PMF_EWORKSPACE with nothing enqueued; a failed launch returns
 *    PMF_ECUDA.  pmf_last_error() gives a message for the calling thread.
 *  - `ws`/`ws_bytes`: caller-provided device scratch of at least the size the
 *    matching *_workspace() query returns, 256-byte aligned; its contents on
 *    entry do not matter and are clobbered.
 */
#ifndef PMF_H_
#define PMF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* pmf_stream; /* same object as cudaStream_t */

typedef enum {
    PMF_OK = 0,
    PMF_EINVAL = -1,      /* bad argument (null pointer, size, geometry) */
    PMF_ECUDA = -2,       /* a CUDA launch or call failed */
    PMF_EWORKSPACE = -3,  /* ws too small or misaligned */
    PMF_ETIMEOUT = -4,    /* a bounded device wait gave up (reported by pmf_device_status) */
    PMF_EUNSUPPORTED = -5 /* valid but not implemented (e.g. channels > 4) */
} pmf_status;

typedef enum { PMF_F32 = 0, PMF_BF16 = 1, PMF_F16 = 2 } pmf_dtype;

/* Voxel grid: sizes and voxel spacing in mm (Sec. 2.3.3: 200x200x100 at 2 mm). */
typedef struct {
    int32_t nx, ny, nz;
    float vx, vy, vz;
} pmf_grid;

/* One cone-beam view (flat detector).  src: x-ray source; det: detector
 * centre; du/dv: one-pixel step vectors (mm).  Pixel (a, b) is centred at
 * det + (a + 1/2 - nu/2) du + (b + 1/2 - nv/2) dv.  Double precision so that
 * the ray directions (source ~1 m away) keep sub-micron accuracy. */
typedef struct {
    double src[3], det[3], du[3], dv[3];
} pmf_view;

/* Detector size and the ray-march step (mm): a ray from src with unit
 * direction r is sampled at src + m * step * r for every integer m >= 0. */
typedef struct {
    int32_t nu, nv;
    float step_mm;
} pmf_detector;

/* A Gaussian set (Eq. 4): G(x) = value * exp(-q/2),
 * q = (x - mean)^T Sigma^-1 (x - mean), Sigma = R(quat/|quat|) diag(scale^2) R^T,
 * truncated to q <= kappa^2 (kappa = +INFINITY: no truncation).
 * mean [n][3] mm, scale [n][3] mm (standard deviations, > 0), quat [n][4]
 * (w,x,y,z; need not be unit length, must be non-zero), value [n][channels]
 * (channels = 1 for the reference densities, 3 for MBC vectors; signed values
 * are allowed: the negative-permitting voxelizer of Sec. 2.3.1).  All device. */
typedef struct {
    int64_t n;
    int32_t channels;
    float kappa;
    const float* mean;
    const float* scale;
    const float* quat;
    const float* value;
} pmf_gaussians;

/* ----------------------------------------------------------------- status */

const char* pmf_version(void);
/* Message for the last non-OK status returned on the calling thread. */
const char* pmf_last_error(void);
const char* pmf_status_string(pmf_status status);

/* ------------------------------------------------------ voxelizer (Eq. 4-5) */

/* Bytes of scratch gs_voxelize needs for a set of n Gaussians with room for
 * `pair_capacity` (Gaussian, 8x8x8-tile) overlaps.  Host-only. */
pmf_status gs_voxelize_workspace(const pmf_grid* grid, int64_t n, int64_t pair_capacity, size_t* bytes);

/* Exact number of (Gaussian, tile) overlaps, written to *d_pairs (device
 * int64).  ws as for gs_voxelize with pair_capacity 0. */
pmf_status gs_voxelize_count(const pmf_grid* grid, const pmf_gaussians* g, int64_t* d_pairs,
                             void* ws, size_t ws_bytes, pmf_stream stream);

/* Eq. 5 (channels = 1) and the signed MBC voxelizer (channels = 3):
 * out[c][v] = sum_i value[i][c] exp(-q_i(x_v)/2) [q_i(x_v) <= kappa^2], point
 * samples at voxel centres.  out: device [channels][N] of `dtype`.
 * Overlaps beyond the workspace's pair capacity are still handled (slower). */
pmf_status gs_voxelize(const pmf_grid* grid, const pmf_gaussians* g, pmf_dtype dtype, void* out,
                       void* ws, size_t ws_bytes, pmf_stream stream);

/* The same three calls with the bin tile chosen: tile = {x, y, z} voxels, one
 * of 8x8x8 (the default of the calls above), 16x8x8, 8x8x4 or 16x8x4 (one CTA
 * per tile, one warp per 4x4x4 sub-block).  The output does not depend on the
 * tile, bit for bit (the sums are exact integers); only the time and the
 * workspace do (fewer, larger tiles list each Gaussian in fewer tiles).
 * PMF_EUNSUPPORTED for any other tile.  pmf_autotune picks one per Gaussian
 * set for plans. */
pmf_status gs_voxelize_tiled_workspace(const pmf_grid* grid, int64_t n, int64_t pair_capacity, const int32_t tile[3],
                                      size_t* bytes);
pmf_status gs_voxelize_tiled_count(const pmf_grid* grid, const pmf_gaussians* g, const int32_t tile[3],
                                   int64_t* d_pairs, void* ws, size_t ws_bytes, pmf_stream stream);
pmf_status gs_voxelize_tiled(const pmf_grid* grid, const pmf_gaussians* g, pmf_dtype dtype, const int32_t tile[3],
                             void* out, void* ws, size_t ws_bytes, pmf_stream stream);

/* Bytes of scratch gs_voxelize_backward needs for n Gaussians of `channels`
 * channels (0 when n is large enough that no Gaussian is split).  Host-only. */
pmf_status gs_voxelize_backward_workspace(const pmf_grid* grid, int64_t n, int32_t channels, size_t* bytes);

/* Adjoint of gs_voxelize with respect to every Gaussian parameter, given
 * d_out = dL/dout (device fp32 [channels][N]).  Outputs device fp32:
 * d_mean [n][3], d_scale [n][3], d_quat [n][4] (gradient with respect to the
 * raw, unnormalised quaternion), d_value [n][channels].  The truncation
 * indicator has zero derivative.  Large Gaussians are split over several
 * warps whose partial sums are added in a fixed order (ws holds them). */
pmf_status gs_voxelize_backward(const pmf_grid* grid, const pmf_gaussians* g, const float* d_out,
                                float* d_mean, float* d_scale, float* d_quat, float* d_value,
                                int accumulate, void* ws, size_t ws_bytes, pmf_stream stream);

/* ------------------------------ Stage-1 X-ray rasterizer (Eq. 8-9) */

/* Gaussian splatting of one Gaussian set (channels = 1) into P cone-beam
 * projections, Stage 1 of Sec. 2.3.2 (Eq. 8-9):
 *   proj[p][j][i] = sum_g rho^_g exp(-1/2 (x^ - p^_g)^T Sigma^_g^-1 (x^ - p^_g))
 * over Gaussians whose 2-D Mahalanobis distance at the pixel is <= kappa (the
 * set's truncation radius; +inf: none).  Ray space of view p maps x to the
 * detector pixel coordinates (a, b) where the ray from the source through x
 * meets the detector plane, measured in pixels from the detector centre, and
 * the distance |x - src|; J is its Jacobian at the Gaussian's mean mu (Eq. 8's
 * local affine approximation, the viewing transform included),
 * Sigma~ = J Sigma J^T, Sigma^ its leading 2x2 block, p^ = (a, b)(mu),
 * rho^ = sqrt(2 pi |Sigma~| / |Sigma^|) rho (= rho sqrt(2 pi / (c^T Sigma^-1 c)),
 * c the unit ray direction through mu), and x^ the pixel centre
 * (i + 1/2 - nu/2, j + 1/2 - nv/2).  Gaussians whose mean is not in front of
 * the source contribute nothing.  views: device [P] (du, dv need not be
 * orthogonal; they must span the detector plane); proj: device [P][nv][nu]
 * fp32, overwritten.  Per-pixel sums are exact integers at a per-view scale
 * (each term < 2^21 of it), so the result does not depend on summation order.
 * The workspace (gs_rasterize_workspace) holds per-view frames, the projected
 * Gaussians and per-tile lists of at most pair_capacity (Gaussian, 16x16 tile)
 * entries; tiles whose lists do not fit scan every Gaussian of the view
 * (same result, slower, counted as PMF_DIAG_RASTER_LIST_OVERFLOW).
 * gs_rasterize_count writes the number of (Gaussian, tile) pairs the call needs
 * into *d_pairs (device int64) using the same workspace. */
pmf_status gs_rasterize_workspace(const pmf_detector* det, int32_t P, int64_t n, int64_t pair_capacity,
                                  size_t* bytes);
pmf_status gs_rasterize_count(const pmf_detector* det, int32_t P, const pmf_view* views, const pmf_gaussians* g,
                              int64_t* d_pairs, void* ws, size_t ws_bytes, pmf_stream stream);
pmf_status gs_rasterize(const pmf_detector* det, int32_t P, const pmf_view* views, const pmf_gaussians* g,
                        float* proj, void* ws, size_t ws_bytes, pmf_stream stream);

/* Adjoint of gs_rasterize: d_mean [n][3], d_scale [n][3], d_quat [n][4],
 * d_value [n] (fp32, overwritten, or added to with accumulate = 1) from
 * d_proj [P][nv][nu].  One warp per Gaussian walks its pixels in every view in
 * a fixed order, so the result is bit-reproducible; the truncation indicator
 * has zero derivative.  The workspace is gs_rasterize_workspace's (any pair
 * capacity, 0 included). */
pmf_status gs_rasterize_backward(const pmf_detector* det, int32_t P, const pmf_view* views, const pmf_gaussians* g,
                                 const float* d_proj, float* d_mean, float* d_scale, float* d_quat, float* d_value,
                                 int accumulate, void* ws, size_t ws_bytes, pmf_stream stream);

/* --------------------------------------------------- DVF combine (Eq. 3) */

/* dvf[p][k][v] = sum_l coeff[p][l][k] * mbc[l][k][v].  mbc [L][3][N], dvf
 * [P][3][N] (both `dtype`, device); coeff device fp32 [P][L][3]. */
pmf_status mbc_combine(const pmf_grid* grid, int32_t L, int32_t P, pmf_dtype dtype, const void* mbc,
                       const float* coeff, void* dvf, pmf_stream stream);

pmf_status mbc_combine_backward_workspace(const pmf_grid* grid, int32_t L, int32_t P, size_t* bytes);

/* Adjoint of mbc_combine: d_mbc[l][k][v] = sum_p d_dvf[p][k][v] coeff[p][l][k];
 * d_coeff[p][l][k] = sum_v d_dvf[p][k][v] mbc[l][k][v] (fixed-order tree
 * reduction).  d_dvf, d_mbc, d_coeff device fp32. */
pmf_status mbc_combine_backward(const pmf_grid* grid, int32_t L, int32_t P, pmf_dtype dtype, const void* mbc,
                                const float* coeff, const float* d_dvf, float* d_mbc, float* d_coeff,
                                int accumulate, void* ws, size_t ws_bytes, pmf_stream stream);

/* The same computation as mbc_combine_backward without a caller workspace, for
 * callers that cannot allocate device memory on the call path (their device
 * memory is handed out up front by their own pool, or they must avoid the
 * device-wide synchronization that allocating and freeing can cause).  The
 * paper has no counterpart: this is an interface convenience only.
 * Scratch: a fixed array of P*L*3*608 floats compiled into the library
 * (about 0.9 MB; every GPU that loads the library holds it until the process
 * exits), so P*L must be <= 128, else PMF_EWORKSPACE with nothing enqueued.
 * It allocates nothing (no cudaMalloc/cudaFree or allocating library call).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, so make that first call
 * before any stream capture; the address is looked up again when the device's
 * context has changed (after cudaDeviceReset), so make the first call after a
 * reset outside capture too.  All calls share the array and it keeps the last
 * call's contents (every slot read is rewritten first), so calls that overlap
 * on the GPU -- on different streams, or from different threads -- race;
 * serialize them. */
pmf_status mbc_combine_backward_noalloc(const pmf_grid* grid, int32_t L, int32_t P, pmf_dtype dtype,
                                        const void* mbc, const float* coeff, const float* d_dvf, float* d_mbc,
                                        float* d_coeff, int accumulate, pmf_stream stream);

/* -------------------------------------------------------- warp (Eq. 2) */

/* out[p][v] = Trilin(ref, (i,j,k) + dvf[p][:,v] / (vx,vy,vz)) (pull warp; the
 * DVF is applied in index space, so dvf = 0 returns ref exactly).
 * ref [N], dvf [P][3][N], out [P][N]: device, `dtype`. */
pmf_status warp_volume(const pmf_grid* grid, int32_t P, pmf_dtype dtype, const void* ref, const void* dvf,
                       void* out, pmf_stream stream);

pmf_status warp_volume_backward_workspace(const pmf_grid* grid, int32_t P, size_t* bytes);

/* Adjoint of warp_volume given d_out [P][N] (fp32): d_ref [N] receives the
 * trilinear-weight scatter summed over all P; d_dvf [P][3][N] (nullable) gets
 * d_out * dTrilin/du / voxel (one-sided at exact integer positions). */
pmf_status warp_volume_backward(const pmf_grid* grid, int32_t P, pmf_dtype dtype, const void* ref,
                                const void* dvf, const float* d_out, float* d_ref, float* d_dvf,
                                int accumulate, void* ws, size_t ws_bytes, pmf_stream stream);

/* Fused Eq. 3 + Eq. 2: out[p][v] = Trilin(ref, v + sum_l coeff[p][l][:] * mbc[l][:][v] / voxel).
 * The DVF is never stored; each voxel's MBC vectors are read once for all P. */
pmf_status warp_combine(const pmf_grid* grid, int32_t L, int32_t P, pmf_dtype dtype, const void* ref,
                        const void* mbc, const float* coeff, void* out, pmf_stream stream);

/* warp_combine with the warped volumes written in out_dtype, which is either
 * dtype or PMF_F32: with reference and MBC grids in bf16/fp16, the projector
 * can then read fp32 warped volumes (and stage them with bulk tensor copies). */
pmf_status warp_combine_mixed(const pmf_grid* grid, int32_t L, int32_t P, pmf_dtype dtype, const void* ref,
                              const void* mbc, const float* coeff, pmf_dtype out_dtype, void* out, pmf_stream stream);

pmf_status warp_combine_backward_workspace(const pmf_grid* grid, int32_t L, int32_t P, size_t* bytes);

/* Adjoint of warp_combine with the DVF recomputed from (mbc, coeff):
 * d_ref [N], d_mbc [L][3][N], d_coeff [P][L][3] (device fp32). */
pmf_status warp_combine_backward(const pmf_grid* grid, int32_t L, int32_t P, pmf_dtype dtype, const void* ref,
                                 const void* mbc, const float* coeff, const float* d_out, float* d_ref,
                                 float* d_mbc, float* d_coeff, int accumulate, void* ws, size_t ws_bytes,
                                 pmf_stream stream);

/* warp_combine_backward given the maximum of |d_out|: d_out_absmax_bits
 * (device, 4 bytes, read on `stream`) holds max |d_out[.]| as the bits of the
 * float with the sign cleared (0x7fffffff & bits; a NaN in d_out gives bits
 * above those of +inf), as conebeam_project_backward_absmax writes it.  That
 * maximum sets the fixed-point scale of d_ref; this call then skips its own
 * pass over d_out, and with the exact maximum its results are bit-identical to
 * warp_combine_backward's.  A larger value is a valid bound (d_ref then loses
 * low-order bits); a smaller one can overflow the accumulator.  Workspace as
 * warp_combine_backward_workspace.  PMF_EINVAL if d_out_absmax_bits is null. */
pmf_status warp_combine_backward_bounded(const pmf_grid* grid, int32_t L, int32_t P, pmf_dtype dtype,
                                         const void* ref, const void* mbc, const float* coeff,
                                         const float* d_out, const unsigned* d_out_absmax_bits, float* d_ref,
                                         float* d_mbc, float* d_coeff, int accumulate, void* ws,
                                         size_t ws_bytes, pmf_stream stream);

/* ------------------------------------------- cone-beam projector (Eq. 6) */

/* proj[p][b][a] = step * sum_{m >= 0} Trilin(vol_p, idx(src_p + m step r_pab)),
 * r_pab the unit direction from src_p to the centre of pixel (a, b), idx(x) =
 * x / voxel + n/2 - 1/2.  views: device pmf_view[P].  vol: `dtype`, device;
 * view p reads vol + p * vol_stride elements (vol_stride = 0: one volume
 * shared by all views).  proj: device fp32 [P][nv][nu]. */
pmf_status conebeam_project(const pmf_grid* grid, const pmf_detector* det, int32_t P, const pmf_view* views,
                            pmf_dtype dtype, const void* vol, int64_t vol_stride, float* proj,
                            pmf_stream stream);

pmf_status conebeam_project_backward_workspace(const pmf_grid* grid, int32_t P, int64_t vol_stride,
                                               size_t* bytes);

/* Exact adjoint of conebeam_project: d_vol (fp32, device; [P][N] with
 * vol_stride = N, or [N] with vol_stride = 0 summed over views) receives
 * step * sum over rays and samples of d_proj times the trilinear weights. */
pmf_status conebeam_project_backward(const pmf_grid* grid, const pmf_detector* det, int32_t P,
                                     const pmf_view* views, const float* d_proj, float* d_vol,
                                     int64_t vol_stride, int accumulate, void* ws, size_t ws_bytes,
                                     pmf_stream stream);

/* conebeam_project_backward that also writes max |d_vol| over every element
 * it writes (after accumulation) to d_vol_absmax_bits (device, 4 bytes, set on
 * `stream`) as the bits of the float with the sign cleared, from the kernel
 * that converts the accumulator, so a consumer that needs the bound
 * (warp_combine_backward_bounded) does not read d_vol for it.  d_vol's values
 * are those of conebeam_project_backward.  PMF_EINVAL if d_vol_absmax_bits is
 * null. */
pmf_status conebeam_project_backward_absmax(const pmf_grid* grid, const pmf_detector* det, int32_t P,
                                            const pmf_view* views, const float* d_proj, float* d_vol,
                                            int64_t vol_stride, int accumulate, void* ws, size_t ws_bytes,
                                            unsigned* d_vol_absmax_bits, pmf_stream stream);

/* ------------------------------------- batched, uneven projector launches */

/* One volume's share of a batched launch: its grid, detector and P views
 * (device pmf_view[P]), its volume(s) (`vol`, stride as for conebeam_project)
 * and its projections (device fp32 [P][nv][nu]). */
typedef struct {
    pmf_grid grid;
    pmf_detector det;
    int32_t P;
    const pmf_view* views;
    const void* vol;
    int64_t vol_stride;
    float* proj;
} pmf_project_item;

/* conebeam_project for up to 16 volumes of different sizes and view counts in
 * one launch over the concatenated (item, view, 16x16 tile) work list, one CTA
 * per work item, the items with the longest rays (volume diagonal over the
 * march step) first so that the launch does not end on a tail of slow tiles;
 * fp32 volumes whose rows are 16-byte multiples are staged by
 * bulk tensor copies (one tensor map per item).  Every item uses `dtype`.
 * Results equal per-item conebeam_project calls bit for bit.  Host-side items
 * may be freed on return. */
pmf_status conebeam_project_batched(int32_t n, const pmf_project_item* items, pmf_dtype dtype, pmf_stream stream);

/* One volume's share of a batched adjoint: d_proj (device fp32 [P][nv][nu])
 * and d_vol (device fp32, [P][N] with vol_stride = N or [N] with 0). */
typedef struct {
    pmf_grid grid;
    pmf_detector det;
    int32_t P;
    const pmf_view* views;
    const float* d_proj;
    float* d_vol;
    int64_t vol_stride;
} pmf_backproject_item;

pmf_status conebeam_project_backward_batched_workspace(int32_t n, const pmf_backproject_item* items, size_t* bytes);

/* conebeam_project_backward for up to 16 items in one launch over the work
 * list, ordered as above (plus one batched max-reduction and one batched
 * fixed-point conversion); each
 * item keeps its own fixed-point scale, so results equal per-item calls bit
 * for bit. */
pmf_status conebeam_project_backward_batched(int32_t n, const pmf_backproject_item* items, int accumulate, void* ws,
                                             size_t ws_bytes, pmf_stream stream);

/* -------------------------------------------------------- loss (Eq. 10/12) */

pmf_status projection_loss_workspace(int64_t count, size_t* bytes);

/* kind 1: L = mean |pred - meas| (Eq. 10/12); kind 2: L = mean (pred - meas)^2
 * (Eq. 1), the mean over all P * Q pixels.  loss: device fp32 scalar.
 * d_pred (nullable): sign(pred - meas)/(PQ) with sign(0) = 0, or
 * 2 (pred - meas)/(PQ).  Fixed-order reduction. */
pmf_status projection_loss(int32_t kind, int32_t P, int64_t Q, const float* pred, const float* meas,
                           float* loss, float* d_pred, void* ws, size_t ws_bytes, pmf_stream stream);

/* ------------------------------------------- Eq. 14 regularisation terms */
/* Each call sets *loss (device fp32 scalar) to weight * term, or with
 * accumulate = 1 adds weight * term to it; the gradient buffer (nullable)
 * likewise receives (or adds) weight * d term / d input.  Fixed-order
 * reductions: results are reproducible run to run. */

pmf_status projection_dssim_workspace(int32_t P, int32_t nu, int32_t nv, size_t* bytes);

/* D-SSIM of Eq. 10/12: term = (1/P) sum_p (1 - mean over pixels of
 * SSIM(pred_p, meas_p)), SSIM after Zhou et al. (2004) with the 11 x 11
 * Gaussian window of standard deviation 1.5 pixels (normalised), windowed
 * moments with zero padding outside the detector,
 * SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),
 * C1 = (0.01 data_range)^2, C2 = (0.03 data_range)^2.  pred, meas, d_pred:
 * device fp32 [P][nv][nu]; P <= 65535. */
pmf_status projection_dssim(int32_t P, int32_t nu, int32_t nv, const float* pred, const float* meas, float data_range,
                            float weight, float* loss, float* d_pred, int accumulate, void* ws, size_t ws_bytes,
                            pmf_stream stream);

pmf_status tv_loss_workspace(int32_t D, size_t* bytes);

/* Sub-volume total variation (Eq. 11/14): term = the mean over the three axes
 * of the mean |forward difference| between neighbouring voxels of the D^3
 * crop of vol (`dtype`, device [N]) whose lowest corner is voxel
 * d_origin = (x, y, z) (device int32[3], read by the kernel so a captured
 * step can take a new crop each replay; clamped so the crop lies in the
 * grid).  d_vol (device fp32 [N]) gets the subgradient (sign(0) = 0) on the
 * crop and zero elsewhere (accumulate = 0) or is left unchanged there
 * (accumulate = 1).  2 <= D <= min(nx, ny, nz). */
pmf_status tv_loss(const pmf_grid* grid, pmf_dtype dtype, const void* vol, int32_t D, const int32_t* d_origin,
                   float weight, float* loss, float* d_vol, int accumulate, void* ws, size_t ws_bytes,
                   pmf_stream stream);

pmf_status mbc_normality_workspace(int32_t L, size_t* bytes);

/* MBC normality (Eq. 13): term = (1/(3L)) sum over levels l and axes k of
 * (||e_{l,k}||^2 - 1)^2 with ||e||^2 the sum of squares over the grid (L = 3
 * gives the paper's 1/9).  mbc: `dtype`, device [L][3][N]; d_mbc: device fp32
 * [L][3][N], receives 4 (||e_{l,k}||^2 - 1) e_{l,k} / (3L) times weight. */
pmf_status mbc_normality(const pmf_grid* grid, int32_t L, pmf_dtype dtype, const void* mbc, float weight, float* loss,
                         float* d_mbc, int accumulate, void* ws, size_t ws_bytes, pmf_stream stream);

/* --------------------------------------------------------- optimiser */

/* One Adam update (Kingma & Ba 2014; the optimiser of Sec. 2.3.2) of n
 * parameters in place at step t >= 1:
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   p = p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 * param, grad, m, v: device fp32 [n]; m and v start at zero. */
pmf_status pmf_adam_step(int64_t n, float* param, const float* grad, float* m, float* v, float lr, float beta1,
                         float beta2, float eps, int32_t t, pmf_stream stream);

/* out[i][k] = mean[i][k] - offset[k] (device [n][3]; offset: device float[3]).
 * The grids are centred on the isocentre, so voxelizing the Gaussians shifted
 * by the centre c of a sub-volume on a grid of the sub-volume's size gives that
 * sub-volume (the random TV crops of Sec. 2.3.2); gradients with respect to the
 * shifted means are gradients with respect to the means.  out may equal mean. */
pmf_status pmf_shift_means(int64_t n, const float* mean, const float* offset, float* out, pmf_stream stream);

/* ------------------------------------------ adaptive density control */

/* acc[i] += |d_mean[i]| (Euclidean norm of the mean's gradient), the
 * densification statistic of Sec. 2.3.2 accumulated between controls.
 * d_mean [n][3], acc [n]: device fp32. */
pmf_status gs_grad_norm_accumulate(int64_t n, const float* d_mean, float* acc, pmf_stream stream);

/* The densification threshold of Sec. 2.3.2's control (the paper names the
 * rule, densify the Gaussians with large loss gradients, but no threshold; the
 * reading here densifies a fixed share of each set): *d_threshold (device fp32)
 * receives the (rank + 1)-th largest of stat_i = grad_acc[i] * grad_scale
 * (products rounded to fp32, as gs_density_control forms them), so exactly the
 * `rank` largest statistics lie above it when they are distinct (fewer when
 * the value at the cut is shared).  grad_acc [n]: device fp32; 0 <= rank < n,
 * 1 <= n < 2^31; one CTA, no workspace, exact (a radix select on the order of
 * the fp32 values).  PMF_EINVAL for bad arguments. */
pmf_status gs_density_threshold(int64_t n, const float* grad_acc, float grad_scale, int64_t rank, float* d_threshold,
                                pmf_stream stream);

/* Adaptive density control of Sec. 2.3.2 on one Gaussian set (any channel
 * count).  With stat_i = grad_acc[i] * grad_scale (grad_scale = 1 / steps):
 *   every channel of value_i below value_threshold in magnitude -> removed;
 *   else stat_i > grad_threshold and max(scale_i) <= scale_threshold -> cloned:
 *     two copies, each with value_i / 2;
 *   else stat_i > grad_threshold -> split: two Gaussians with means
 *     mean_i + R_i diag(scale_i) z_{i,k} (z = noise[i][k][0..2], standard normal
 *     samples the caller draws), scales scale_i / split_factor, the same
 *     quaternion and value_i / 2;
 *   else kept unchanged.
 * Outputs (device, capacity out_capacity >= 2 n) hold the controlled set in input
 * order, a densified Gaussian's two results in its place; *d_count (device int64)
 * receives the new count.  Deterministic.  Workspace: gs_density_control_workspace. */
pmf_status gs_density_control_workspace(int64_t n, size_t* bytes);
pmf_status gs_density_control(const pmf_gaussians* in, const float* grad_acc, float grad_scale, const float* noise,
                              float grad_threshold, float scale_threshold, float value_threshold, float split_factor,
                              float* out_mean, float* out_scale, float* out_quat, float* out_value,
                              int64_t out_capacity, int64_t* d_count, void* ws, size_t ws_bytes, pmf_stream stream);

/* ------------------------------------------------------------ host helpers */

/* The circular scan of Sec. 2.3.3 / Table I as pmf_view records: view p has
 * theta = 2 pi p / P, source SAD (cos theta, sin theta, 0), detector centre
 * -(SDD - SAD)(cos theta, sin theta, 0), u step du_mm (-sin theta, cos theta, 0)
 * and v step dv_mm (0, 0, 1) (flat detector opposite the source, no offset).
 * Host-only: writes P records to host_out (caller-owned host memory).
 * nu and nv are only checked (> 0): pixel positions use them at projection time. */
pmf_status pmf_circular_views(int32_t P, double sad_mm, double sdd_mm, double du_mm, double dv_mm, int32_t nu,
                              int32_t nv, pmf_view* host_out);

/* Operation codes of pmf_workspace_size, and the arguments each one reads. */
typedef enum {
    PMF_OP_VOXELIZE = 1,              /* grid, n, pair_capacity  (= gs_voxelize_workspace) */
    PMF_OP_VOXELIZE_BACKWARD = 2,     /* grid, n, channels       (= gs_voxelize_backward_workspace) */
    PMF_OP_COMBINE_BACKWARD = 3,      /* grid, L, P              (= mbc_combine_backward_workspace) */
    PMF_OP_WARP_BACKWARD = 4,         /* grid, P                 (= warp_volume_backward_workspace) */
    PMF_OP_WARP_COMBINE_BACKWARD = 5, /* grid, L, P              (= warp_combine_backward_workspace) */
    PMF_OP_PROJECT_BACKWARD = 6,      /* grid, P, vol_stride     (= conebeam_project_backward_workspace) */
    PMF_OP_LOSS = 7                   /* count                   (= projection_loss_workspace) */
} pmf_op;

typedef struct {
    pmf_grid grid;
    int64_t n;             /* Gaussians */
    int64_t pair_capacity; /* voxelizer (Gaussian, tile) list capacity */
    int64_t vol_stride;    /* projector adjoint: 0 or N */
    int64_t count;         /* loss: P * Q */
    int32_t channels, L, P;
} pmf_ws_args;

/* One entry point for every *_workspace query: *bytes = the scratch `op`
 * needs for `args`.  Host-only; PMF_EINVAL for an unknown op. */
pmf_status pmf_workspace_size(int32_t op, const pmf_ws_args* args, size_t* bytes);

/* ------------------------------------------------------ device diagnostics */

/* Counters the kernels keep on the device (per device, since the library was
 * loaded or last reset).  The slow paths give the same results, only slower;
 * PMF_DIAG_NONFINITE marks outputs that are undefined (NaN written). */
typedef enum {
    PMF_DIAG_VOXELIZE_LIST_OVERFLOW = 0,   /* voxelizer tiles whose Gaussian list overflowed the
                                              workspace's pair capacity (scanned every Gaussian instead) */
    PMF_DIAG_PROJECT_BOX_FALLBACK = 1,     /* projector chunks whose voxel box did not fit shared
                                              memory (gathered from global memory) */
    PMF_DIAG_BACKPROJECT_BOX_FALLBACK = 2, /* the same for the back-projector (global 64-bit atomics) */
    PMF_DIAG_WARP_HALO_EXIT = 3,           /* fused warp-adjoint CTAs where a displacement left the
                                              4-voxel halo (those corners use global atomics) */
    PMF_DIAG_NONFINITE = 4,                /* fixed-point scatters or voxelizations whose input
                                              magnitude was NaN or infinite (outputs set to NaN) */
    PMF_DIAG_TIMEOUT = 5,                  /* CTAs whose bounded wait for a bulk (TMA) copy ran out
                                              (about one second); their outputs are set to NaN */
    PMF_DIAG_RASTER_LIST_OVERFLOW = 6,     /* rasterizer tiles whose Gaussian list overflowed the
                                              workspace's pair capacity (scanned every Gaussian instead) */
    PMF_DIAG_BOUNDS = 7,                   /* debug builds only (PMF_DEBUG): shared-memory or list
                                              accesses whose index failed its bounds check; the access
                                              was skipped, so outputs are wrong.  Always 0 otherwise */
    PMF_DIAG_COUNT = 8
} pmf_diag;

/* Copies the current device's counters to host_out[PMF_DIAG_COUNT] and, with
 * reset != 0, zeroes them.  Synchronizes the device; not during stream capture. */
pmf_status pmf_device_counters(uint64_t* host_out, int32_t reset);

/* Synchronizes `stream` and reports what the device saw: PMF_ECUDA (with the
 * CUDA message) if the stream's work failed, PMF_ETIMEOUT if a bounded wait for
 * a bulk copy gave up, PMF_EINVAL if a non-finite input reached a fixed-point
 * scatter or (debug builds) a bounds check failed since the counters were last
 * reset, else PMF_OK.  No kernel waits on another CTA. */
pmf_status pmf_device_status(pmf_stream stream);

/* Test hook for the failure path of the bounded wait above (no counterpart in
 * the paper).  While `on` is non-zero, every later launch of the per-volume
 * bulk-copy projector (conebeam_project on fp32 volumes whose rows are 16-byte
 * multiples) arms its mbarrier for a chunk's bytes but issues no copy, so the
 * wait runs out after about 0.1 ms of clock with nothing in flight: those CTAs
 * count PMF_DIAG_TIMEOUT and write NaN to their pixels, and pmf_device_status
 * reports PMF_ETIMEOUT.  Off (0) when the library loads; set it back to 0 after
 * the test.  Synchronous (a copy to a device symbol of the current device);
 * PMF_ECUDA on failure.  Never faults or hangs the device. */
pmf_status pmf_debug_stall_bulk_copies(int32_t on);

/* ------------------------------------------------ training-step plans */

#define PMF_MAX_LEVELS 8

/* One forward + adjoint step of Stages 2-3 (Sec. 2.3.2) over a batch of B views:
 *   V = voxelize(ref), E_l = voxelize(mbc[l]), W = warp_combine(V, E, coeff),
 *   Y = project(W), loss/dY = projection_loss(Y, meas),
 *   dW = project^T(dY), (dV, dE, d_coeff) = warp_combine^T(dW),
 *   d_ref = voxelize^T(dV), d_mbc[l] = voxelize^T(dE_l).
 * Every pointer below is a caller-owned device pointer that the plan keeps:
 * it reads the inputs and writes the outputs at every pmf_plan_step, so the
 * caller refreshes their contents between steps (new views, coefficients,
 * measurements, updated Gaussian parameters) without re-creating the plan.
 * The Gaussian counts and everything else are fixed at creation. */
typedef struct {
    pmf_grid grid;
    pmf_detector det;
    pmf_dtype dtype;        /* storage of V, E, W */
    int32_t batch;          /* B >= 1 */
    int32_t loss_kind;      /* 1 = L1 (Eq. 10/12), 2 = L2 (Eq. 1), 3 = Eq. 14 (below) */
    int32_t levels;         /* L in [1, PMF_MAX_LEVELS] */
    pmf_gaussians ref;      /* channels 1 */
    pmf_gaussians mbc[PMF_MAX_LEVELS]; /* channels 3; first `levels` used */
    const pmf_view* views;  /* [B] */
    const float* coeff;     /* [B][L][3] */
    const float* meas;      /* [B][nv][nu] */
    float* loss;            /* scalar (output) */
    float* d_ref[4];        /* d_mean [n][3], d_scale [n][3], d_quat [n][4], d_value [n][1] (outputs) */
    float* d_mbc[PMF_MAX_LEVELS][4]; /* the same per level, d_value [n][3] */
    float* d_coeff;         /* [B][L][3] (output) */
    int32_t use_graph;      /* 1: the first pmf_plan_step captures the step into a CUDA graph on its
                               stream (which must not be the legacy NULL stream); later steps replay it */
    const char* tune_cache; /* nullable: file written by pmf_autotune; its entry for this
                               configuration selects the projector launch forms */
    /* loss_kind 3, the Stage 2-3 objective of Eq. 14:
     * L1 + lambda_ssim D-SSIM + lambda_mbc L_MBC + lambda_tv TV (paper: 0.25, 1, 0.05) */
    float lambda_ssim, lambda_mbc, lambda_tv;
    float ssim_range;            /* D-SSIM data range (> 0) */
    int32_t tv_size;             /* edge D of the TV crop (paper: 32) */
    const int32_t* tv_origin;    /* device int32[3]: the crop's lowest voxel (x, y, z), read at every step */
    pmf_dtype w_dtype;           /* storage of the warped volumes W: dtype or PMF_F32 (0, the default) */
} pmf_batch_desc;

typedef struct pmf_plan pmf_plan;

/* Device tensors the plan owns (valid until pmf_plan_destroy): V [N] and E [L][3][N]
 * in the plan's dtype, W [B][N] in the descriptor's w_dtype; fp32 Y, dY [B][nv][nu],
 * dW [B][N], dV [N], dE [L][3][N]. */
typedef struct {
    void* V;
    void* E;
    void* W;
    float* Y;
    float* dY;
    float* dW;
    float* dV;
    float* dE;
} pmf_plan_tensors;

/* Validates `desc`, allocates the plan's device memory (cudaMalloc: the one
 * place the library allocates), sizes each voxelizer's pair list from the
 * current Gaussians (gs_voxelize_count, synchronizing), and reads tune_cache.
 * *plan is NULL on failure. */
pmf_status pmf_plan_create(const pmf_batch_desc* desc, pmf_plan** plan);

/* Enqueues one step on `stream` (asynchronous; with use_graph, one graph launch). */
pmf_status pmf_plan_step(pmf_plan* plan, pmf_stream stream);

pmf_status pmf_plan_tensors_get(const pmf_plan* plan, pmf_plan_tensors* out);

/* Launch shapes the plan uses for the projector (proj) and its adjoint
 * (backproj), each int32[3] = {form, chunk, rays}: form 0 is one CTA per
 * (view, pixel tile) and k > 0 a persistent launch of k CTAs per SM; chunk
 * (16, 32 or 48, and for the adjoint also 64) is the number of samples per
 * staged voxel brick along the rays; rays (128 or 256) the rays per CTA.
 * Defaults {0, 48, 256} (projector) and {0, 48, 128} (adjoint), or the
 * autotuner's choice from tune_cache.  Forms give bit-identical results;
 * chunk and rays move the last bits (chunk anchors, per-CTA scales). */
pmf_status pmf_plan_launch_forms(const pmf_plan* plan, int32_t* proj, int32_t* backproj);

/* The voxelizer bin tile the plan uses for each Gaussian set (the reference
 * set, then the MBC levels): tiles[3 (1 + levels)] = {x, y, z} per set.
 * Defaults 8x8x8, or the autotuner's choice from tune_cache.  Every tile gives
 * the same bits (see gs_voxelize_tiled). */
pmf_status pmf_plan_voxel_tiles(const pmf_plan* plan, int32_t* tiles);

/* Synchronizes the device, frees the plan's memory and graph.  NULL is a no-op. */
pmf_status pmf_plan_destroy(pmf_plan* plan);

/* Times the projector and its adjoint over launch shapes (forms 0, 1, 2, 4
 * CTAs per 1024 SM threads; chunks of 16, 32 and 48 samples, for the adjoint
 * also 64; 128 and 256 rays per CTA) and each Gaussian set's voxelization over the bin tiles of
 * gs_voxelize_tiled, on desc's data (a temporary plan; CUDA events, best of 3
 * after a warm-up; the tile search allocates its own scratch), and records the
 * fastest of each in `cache_path` under a key made of the device name, SM
 * count, grid, detector, batch, levels, dtype and the sets' Gaussian counts
 * (other keys in the file are kept).  Synchronizes. */
pmf_status pmf_autotune(const pmf_batch_desc* desc, const char* cache_path);

#ifdef __cplusplus
}
#endif

#endif /* PMF_H_ */
