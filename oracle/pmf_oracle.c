/*
 * FP64 CPU oracle for the PMF-STGR forward model and its adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is read by the tests, by the smoke check
 * and by the benchmark's CPU-baseline leg; the library under test never links,
 * loads or calls it.  It shares no code, header, table or constant with the
 * CUDA path.  Every loop is the plain definition from the paper, in double
 * precision, with no tiling, fusion or reordering beyond skipping terms that are
 * exactly zero by the definition (voxels outside a Gaussian's truncation
 * ellipsoid, ray samples outside the zero-padded volume).
 *
 * Passages followed (PMF-STGR, Xie, Shao & Zhang):
 *   Eq. 4  G(x) = rho exp(-1/2 (x-p)^T Sigma^-1 (x-p))            voxelize
 *   Eq. 5  sigma(x) = sum_i G_i(x)                                 voxelize
 *   Sec. 2.3.1  negative-permitting voxelizer for signed MBC values  voxelize, C=3
 *   Eq. 3  d(x,p) = sum_i w_i(p) x e_i(x)  (per Cartesian component) combine
 *   Eq. 2  I(x,p) = I_ref(x + d(x,p))                              warp
 *   Eq. 6  I(r) = integral of sigma along the ray                   project
 *   Eq. 10/12  mean L1 over the batch; Eq. 1 squared-norm form      loss
 *   Eq. 8-9  local affine projection of each Gaussian to a 2-D Gaussian  splat (Stage 1)
 * Readings where the paper is silent:
 *   Sigma = R(q/|q|) diag(s^2) R^T with q = (w,x,y,z) and s in mm; hard
 *   truncation q_form <= kappa^2 (kappa = +inf disables it); values are sampled
 *   at voxel centres (i + 1/2 - n/2) v; interpolation is trilinear with zero
 *   padding outside [0, n-1]; the DVF is in mm and applied in index space
 *   (u = i + d/v); the line integral is the source-anchored sum
 *   step * sum_{m >= 0} Trilin(W, idx(src + m step r)) with r the unit
 *   source-to-pixel-centre direction.
 *
 * Parity: pinned by closed forms, invariants, finite differences and a NumPy
 * brute force in the oracle tests; there is no worked example in the paper to
 * match ("parity unpinned" against the paper's own numbers only).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------- geometry */

/* Voxel centre coordinate along one axis (mm): (i + 1/2 - n/2) v. */
static double centre(int64_t i, int64_t n, double v) { return ((double)i + 0.5 - 0.5 * (double)n) * v; }

/* Continuous voxel index of a coordinate: x / v + n/2 - 1/2 (inverse of centre). */
static double to_index(double x, int64_t n, double v) { return x / v + 0.5 * (double)n - 0.5; }

/* Rotation matrix of the unit quaternion q/|q|, q = (w, x, y, z); row-major R[3*i+j].
 * The columns of R are the Gaussian's principal axes: Sigma = R diag(s^2) R^T. */
static void quat_to_rot(const double q_in[4], double R[9], double qn[4], double* norm) {
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    if (qn) { qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z; }
    if (norm) *norm = n;
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

void orc_quat_to_rot(const double* q, double* R) { quat_to_rot(q, R, NULL, NULL); }

/* Index range [lo, hi] along one axis that can hold voxel centres of the
 * truncation ellipsoid: the ellipsoid {d : d^T Sigma^-1 d <= k^2} extends
 * k sqrt(Sigma_aa) from its centre along axis a.  One voxel of slack on each
 * side; the per-voxel test decides. */
static void axis_range(double mu, double half, int64_t n, double v, int64_t* lo, int64_t* hi) {
    double a = to_index(mu - half, n, v), b = to_index(mu + half, n, v);
    double l = ceil(a) - 1.0, h = floor(b) + 1.0;
    if (l < 0.0) l = 0.0;
    if (h > (double)(n - 1)) h = (double)(n - 1);
    *lo = (int64_t)l; *hi = (int64_t)h;
    if (!(a == a) || !(b == b)) { *lo = 0; *hi = n - 1; }
}

typedef struct {
    double mu[3], s[3], R[9], qn[4], qnorm;
    int64_t lo[3], hi[3];
} gauss_t;

static void prepare(gauss_t* g, const double* mean, const double* scale, const double* quat,
                    double kappa, int cull, const int64_t dims[3], const double vox[3]) {
    for (int a = 0; a < 3; a++) { g->mu[a] = mean[a]; g->s[a] = scale[a]; }
    quat_to_rot(quat, g->R, g->qn, &g->qnorm);
    for (int a = 0; a < 3; a++) {
        if (!cull || isinf(kappa)) { g->lo[a] = 0; g->hi[a] = dims[a] - 1; continue; }
        double var = 0.0;
        for (int j = 0; j < 3; j++) var += g->R[3 * a + j] * g->R[3 * a + j] * g->s[j] * g->s[j];
        axis_range(g->mu[a], kappa * sqrt(var), dims[a], vox[a], &g->lo[a], &g->hi[a]);
    }
}

/* Quadratic form q = (x-mu)^T Sigma^-1 (x-mu) = sum_j (r_j / s_j)^2, r = R^T (x-mu). */
static double qform(const gauss_t* g, const double d[3], double r[3]) {
    double q = 0.0;
    for (int j = 0; j < 3; j++) {
        r[j] = g->R[0 * 3 + j] * d[0] + g->R[1 * 3 + j] * d[1] + g->R[2 * 3 + j] * d[2];
        q += (r[j] / g->s[j]) * (r[j] / g->s[j]);
    }
    return q;
}

/* ------------------------------------------------------------ voxelization */

/* Eq. 4-5: out[c][v] = sum_g value[g][c] exp(-q_g(x_v)/2) [q_g(x_v) <= kappa^2].
 * kappa = +inf: no truncation.  cull = 0 visits every voxel for every Gaussian
 * (used to check the culled loop).  Per voxel the sum runs in Gaussian order. */
int orc_voxelize(const int64_t dims[3], const double vox[3], int64_t G, int C,
                 const double* mean, const double* scale, const double* quat, const double* value,
                 double kappa, int cull, double* out) {
    if (!(kappa > 0.0) || C < 1) return -1;
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2], N = nx * ny * nz;
    const double k2 = isinf(kappa) ? INFINITY : kappa * kappa;
    gauss_t* gs = (gauss_t*)malloc(sizeof(gauss_t) * (size_t)(G > 0 ? G : 1));
    for (int64_t g = 0; g < G; g++) prepare(&gs[g], mean + 3 * g, scale + 3 * g, quat + 4 * g, kappa, cull, dims, vox);
    memset(out, 0, sizeof(double) * (size_t)(N * C));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nz; k++) {
        for (int64_t g = 0; g < G; g++) {
            const gauss_t* ga = &gs[g];
            if (k < ga->lo[2] || k > ga->hi[2]) continue;
            for (int64_t j = ga->lo[1]; j <= ga->hi[1]; j++)
                for (int64_t i = ga->lo[0]; i <= ga->hi[0]; i++) {
                    double d[3] = {centre(i, nx, vox[0]) - ga->mu[0], centre(j, ny, vox[1]) - ga->mu[1],
                                   centre(k, nz, vox[2]) - ga->mu[2]};
                    double r[3];
                    double q = qform(ga, d, r);
                    if (!(q <= k2)) continue;
                    double e = exp(-0.5 * q);
                    int64_t v = (k * ny + j) * nx + i;
                    for (int c = 0; c < C; c++) out[c * N + v] += value[g * C + c] * e;
                }
        }
    }
    free(gs);
    return 0;
}

/* Per-voxel mass of the truncation decisions that rounding can flip:
 * amb[v] = sum_g max_c |value[g][c]| exp(-q/2) over the pairs whose q lies in
 * the band |q - kappa^2| <= eps kappa^2.  An implementation that evaluates q in
 * lower precision may keep or drop exactly these terms, so a voxel's value is
 * unique only up to amb[v].  kappa = +inf: no band, amb = 0. */
int orc_voxelize_ambiguity(const int64_t dims[3], const double vox[3], int64_t G, int C,
                           const double* mean, const double* scale, const double* quat, const double* value,
                           double kappa, double eps, double* amb) {
    if (!(kappa > 0.0) || C < 1 || !(eps >= 0.0)) return -1;
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2], N = nx * ny * nz;
    memset(amb, 0, sizeof(double) * (size_t)N);
    if (isinf(kappa)) return 0;
    const double lo2 = kappa * kappa * (1.0 - eps), hi2 = kappa * kappa * (1.0 + eps);
    gauss_t* gs = (gauss_t*)malloc(sizeof(gauss_t) * (size_t)(G > 0 ? G : 1));
    for (int64_t g = 0; g < G; g++)
        prepare(&gs[g], mean + 3 * g, scale + 3 * g, quat + 4 * g, kappa * sqrt(1.0 + eps), 1, dims, vox);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nz; k++) {
        for (int64_t g = 0; g < G; g++) {
            const gauss_t* ga = &gs[g];
            if (k < ga->lo[2] || k > ga->hi[2]) continue;
            double vmax = 0.0;
            for (int c = 0; c < C; c++) vmax = fmax(vmax, fabs(value[g * C + c]));
            for (int64_t j = ga->lo[1]; j <= ga->hi[1]; j++)
                for (int64_t i = ga->lo[0]; i <= ga->hi[0]; i++) {
                    double d[3] = {centre(i, nx, vox[0]) - ga->mu[0], centre(j, ny, vox[1]) - ga->mu[1],
                                   centre(k, nz, vox[2]) - ga->mu[2]};
                    double r[3];
                    double q = qform(ga, d, r);
                    if (q >= lo2 && q <= hi2) amb[(k * ny + j) * nx + i] += vmax * exp(-0.5 * q);
                }
        }
    }
    free(gs);
    return 0;
}

/* First-order bound on the error of q when an implementation evaluates it in
 * IEEE binary32 (unit roundoff u = 2^-24) from the inputs rounded to binary32:
 * the normalised quaternion and R (every entry within 25u absolute), 1/s_j^2
 * (2 roundings), the inverse covariance A = R diag(1/s^2) R^T (a three-term sum
 * and the doubled off-diagonal, 5 roundings), the offset d = x - mu from a
 * rounded voxel centre x (2 roundings) and the quadratic form itself (at most 6
 * sequential roundings).  With r~_j = sum_a |R_aj||d_a|, x~_j = sum_a |R_aj||x_a|
 * and |d|_1 = sum_a |d_a|, summing the first-order terms of q = sum_j (r_j/s_j)^2
 * gives
 *     |fl(q) - q| <= u sum_j (50 r~_j |d|_1 + 2 r~_j x~_j + 15 r~_j^2) / s_j^2,
 * and kappa^2 itself rounds by u kappa^2.  The tie band below uses 64 in place
 * of 50 and a caller-chosen multiple ("units") of the total. */
static double q_fp32_bound(const gauss_t* g, const double x[3], const double d[3], double k2) {
    double d1 = fabs(d[0]) + fabs(d[1]) + fabs(d[2]), b = 0.0;
    for (int j = 0; j < 3; j++) {
        double rt = 0.0, xt = 0.0;
        for (int a = 0; a < 3; a++) { rt += fabs(g->R[3 * a + j]) * fabs(d[a]); xt += fabs(g->R[3 * a + j]) * fabs(x[a]); }
        b += (64.0 * rt * d1 + 2.0 * rt * xt + 15.0 * rt * rt) / (g->s[j] * g->s[j]);
    }
    return ldexp(b + k2, -24);
}

/* The quadratic form q of one Gaussian at point x (mm) and its binary32 error
 * bound (q_fp32_bound), for the tests that pin the bound. */
void orc_qform_and_bound(const double* mean, const double* scale, const double* quat, const double x[3],
                         double kappa, double out[2]) {
    gauss_t g;
    const int64_t dims[3] = {1, 1, 1};
    const double vox[3] = {1.0, 1.0, 1.0};
    prepare(&g, mean, scale, quat, kappa, 0, dims, vox);
    double d[3] = {x[0] - g.mu[0], x[1] - g.mu[1], x[2] - g.mu[2]}, r[3];
    out[0] = qform(&g, d, r);
    out[1] = q_fp32_bound(&g, x, d, kappa * kappa);
}

/* Per-voxel mass of the truncation decisions that binary32 rounding can flip:
 * amb[v] = sum_g max_c |value[g][c]| exp(-q/2) over the pairs with
 * |q - kappa^2| <= units * q_fp32_bound (above).  offset (mm, may be NULL) is
 * added to every voxel centre for the bound only: a crop evaluated here with
 * shifted means stands for voxels whose coordinates in the full grid are
 * x + offset.  *npairs receives the number of pairs in the band.  Returns -2 if
 * a pair in the band has a band wider than the 1% margin of the bounding boxes
 * visited (pairs outside them could then reach the band too). */
int orc_voxelize_tie_band(const int64_t dims[3], const double vox[3], int64_t G, int C,
                          const double* mean, const double* scale, const double* quat, const double* value,
                          double kappa, double units, const double* offset, double* amb, int64_t* npairs) {
    if (!(kappa > 0.0) || C < 1 || !(units >= 0.0)) return -1;
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2], N = nx * ny * nz;
    memset(amb, 0, sizeof(double) * (size_t)N);
    if (npairs) *npairs = 0;
    if (isinf(kappa)) return 0;
    const double k2 = kappa * kappa, o[3] = {offset ? offset[0] : 0.0, offset ? offset[1] : 0.0,
                                             offset ? offset[2] : 0.0};
    gauss_t* gs = (gauss_t*)malloc(sizeof(gauss_t) * (size_t)(G > 0 ? G : 1));
    for (int64_t g = 0; g < G; g++)
        prepare(&gs[g], mean + 3 * g, scale + 3 * g, quat + 4 * g, kappa * sqrt(1.01), 1, dims, vox);
    int64_t count = 0;
    int wide = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : count) reduction(| : wide)
    for (int64_t k = 0; k < nz; k++) {
        for (int64_t g = 0; g < G; g++) {
            const gauss_t* ga = &gs[g];
            if (k < ga->lo[2] || k > ga->hi[2]) continue;
            double vmax = 0.0;
            for (int c = 0; c < C; c++) vmax = fmax(vmax, fabs(value[g * C + c]));
            for (int64_t j = ga->lo[1]; j <= ga->hi[1]; j++)
                for (int64_t i = ga->lo[0]; i <= ga->hi[0]; i++) {
                    double x[3] = {centre(i, nx, vox[0]), centre(j, ny, vox[1]), centre(k, nz, vox[2])};
                    double d[3] = {x[0] - ga->mu[0], x[1] - ga->mu[1], x[2] - ga->mu[2]};
                    double xf[3] = {x[0] + o[0], x[1] + o[1], x[2] + o[2]};
                    double r[3];
                    double q = qform(ga, d, r);
                    double band = units * q_fp32_bound(ga, xf, d, k2);
                    if (fabs(q - k2) <= band) {
                        if (band > 0.01 * k2) wide = 1;
                        amb[(k * ny + j) * nx + i] += vmax * exp(-0.5 * q);
                        count++;
                    }
                }
        }
    }
    free(gs);
    if (npairs) *npairs = count;
    return wide ? -2 : 0;
}

/* d R / d (w, x, y, z) for the rotation matrix written in quat_to_rot (treating
 * the normalised components as free variables); dR[comp][9]. */
static void drot_dq(const double q[4], double dR[4][9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double t[4][9] = {
        /* d/dw */ {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0},
        /* d/dx */ {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x},
        /* d/dy */ {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y},
        /* d/dz */ {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0},
    };
    memcpy(dR, t, sizeof(t));
}

/* Adjoint of orc_voxelize with respect to every Gaussian parameter (the
 * truncation indicator has zero derivative).  Gradients overwrite the outputs.
 * Chain rule per voxel: with e = exp(-q/2) and s = sum_c value_c dL/dout_c,
 *   dL/dvalue_c += dL/dout_c e,   dL/dq = -s e / 2,
 *   dq/dmu = -2 R (r / s^2),  dq/ds_j = -2 r_j^2 / s_j^3,  dq/dR_ij = 2 d_i r_j / s_j^2,
 * then dR -> d(unit quaternion) -> d(raw quaternion) through (I - qq^T)/|q|. */
int orc_voxelize_backward(const int64_t dims[3], const double vox[3], int64_t G, int C,
                          const double* mean, const double* scale, const double* quat, const double* value,
                          double kappa, const double* d_out,
                          double* d_mean, double* d_scale, double* d_quat, double* d_value) {
    if (!(kappa > 0.0) || C < 1 || C > 16) return -1;
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2], N = nx * ny * nz;
    const double k2 = isinf(kappa) ? INFINITY : kappa * kappa;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t g = 0; g < G; g++) {
        gauss_t ga;
        prepare(&ga, mean + 3 * g, scale + 3 * g, quat + 4 * g, kappa, 1, dims, vox);
        double gmu[3] = {0, 0, 0}, gs[3] = {0, 0, 0}, gR[9] = {0};
        double gval[16];
        for (int c = 0; c < C && c < 16; c++) gval[c] = 0.0;
        for (int64_t k = ga.lo[2]; k <= ga.hi[2]; k++)
            for (int64_t j = ga.lo[1]; j <= ga.hi[1]; j++)
                for (int64_t i = ga.lo[0]; i <= ga.hi[0]; i++) {
                    double d[3] = {centre(i, nx, vox[0]) - ga.mu[0], centre(j, ny, vox[1]) - ga.mu[1],
                                   centre(k, nz, vox[2]) - ga.mu[2]};
                    double r[3];
                    double q = qform(&ga, d, r);
                    if (!(q <= k2)) continue;
                    double e = exp(-0.5 * q);
                    int64_t v = (k * ny + j) * nx + i;
                    double s = 0.0;
                    for (int c = 0; c < C; c++) {
                        gval[c] += d_out[c * N + v] * e;
                        s += value[g * C + c] * d_out[c * N + v];
                    }
                    double gq = -0.5 * s * e;
                    for (int a = 0; a < 3; a++) {
                        double Ad = 0.0;
                        for (int jj = 0; jj < 3; jj++) Ad += ga.R[3 * a + jj] * r[jj] / (ga.s[jj] * ga.s[jj]);
                        gmu[a] += gq * (-2.0 * Ad);
                    }
                    for (int jj = 0; jj < 3; jj++) gs[jj] += gq * (-2.0 * r[jj] * r[jj] / (ga.s[jj] * ga.s[jj] * ga.s[jj]));
                    for (int a = 0; a < 3; a++)
                        for (int jj = 0; jj < 3; jj++) gR[3 * a + jj] += gq * (2.0 * d[a] * r[jj] / (ga.s[jj] * ga.s[jj]));
                }
        double dR[4][9], gqn[4];
        drot_dq(ga.qn, dR);
        for (int c4 = 0; c4 < 4; c4++) {
            gqn[c4] = 0.0;
            for (int t = 0; t < 9; t++) gqn[c4] += gR[t] * dR[c4][t];
        }
        double dot = gqn[0] * ga.qn[0] + gqn[1] * ga.qn[1] + gqn[2] * ga.qn[2] + gqn[3] * ga.qn[3];
        for (int c4 = 0; c4 < 4; c4++) d_quat[4 * g + c4] = (gqn[c4] - ga.qn[c4] * dot) / ga.qnorm;
        for (int a = 0; a < 3; a++) { d_mean[3 * g + a] = gmu[a]; d_scale[3 * g + a] = gs[a]; }
        for (int c = 0; c < C; c++) d_value[g * C + c] = gval[c];
    }
    return 0;
}

/* ----------------------------------------------------------------- combine */

/* Eq. 3, per Cartesian component k: D[p][k][v] = sum_l w[p][l][k] E[l][k][v]. */
void orc_combine(int64_t N, int L, int P, const double* E, const double* w, double* D) {
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < N; v++)
        for (int p = 0; p < P; p++)
            for (int k = 0; k < 3; k++) {
                double acc = 0.0;
                for (int l = 0; l < L; l++) acc += w[(p * L + l) * 3 + k] * E[((int64_t)l * 3 + k) * N + v];
                D[((int64_t)p * 3 + k) * N + v] = acc;
            }
}

/* Adjoint of orc_combine: dE[l][k][v] = sum_p dD[p][k][v] w[p][l][k];
 * dw[p][l][k] = sum_v dD[p][k][v] E[l][k][v]. */
void orc_combine_backward(int64_t N, int L, int P, const double* E, const double* w, const double* dD,
                          double* dE, double* dw) {
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < N; v++)
        for (int l = 0; l < L; l++)
            for (int k = 0; k < 3; k++) {
                double acc = 0.0;
                for (int p = 0; p < P; p++) acc += dD[((int64_t)p * 3 + k) * N + v] * w[(p * L + l) * 3 + k];
                dE[((int64_t)l * 3 + k) * N + v] = acc;
            }
    for (int p = 0; p < P; p++)
        for (int l = 0; l < L; l++)
            for (int k = 0; k < 3; k++) {
                double acc = 0.0;
                const double* a = dD + ((int64_t)p * 3 + k) * N;
                const double* b = E + ((int64_t)l * 3 + k) * N;
#pragma omp parallel for reduction(+ : acc) schedule(static)
                for (int64_t v = 0; v < N; v++) acc += a[v] * b[v];
                dw[(p * L + l) * 3 + k] = acc;
            }
}

/* ------------------------------------------------------------- trilinear */

static double vox_at(const double* V, const int64_t dims[3], int64_t i, int64_t j, int64_t k) {
    if (i < 0 || j < 0 || k < 0 || i >= dims[0] || j >= dims[1] || k >= dims[2]) return 0.0;
    return V[(k * dims[1] + j) * dims[0] + i];
}

/* Trilinear interpolation at continuous index u with zero padding: corners
 * floor(u) and floor(u)+1 per axis, weights (1-f, f), f = u - floor(u). */
static double trilin(const double* V, const int64_t dims[3], const double u[3]) {
    double fl[3], f[3];
    for (int a = 0; a < 3; a++) { fl[a] = floor(u[a]); f[a] = u[a] - fl[a]; }
    int64_t i0 = (int64_t)fl[0], j0 = (int64_t)fl[1], k0 = (int64_t)fl[2];
    double acc = 0.0;
    for (int c = 0; c < 8; c++) {
        int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
        double wgt = (di ? f[0] : 1.0 - f[0]) * (dj ? f[1] : 1.0 - f[1]) * (dk ? f[2] : 1.0 - f[2]);
        acc += wgt * vox_at(V, dims, i0 + di, j0 + dj, k0 + dk);
    }
    return acc;
}

/* Scatter g * weight to the 8 corners (adjoint of trilin with respect to V). */
static void trilin_adj(double* dV, const int64_t dims[3], const double u[3], double g) {
    double fl[3], f[3];
    for (int a = 0; a < 3; a++) { fl[a] = floor(u[a]); f[a] = u[a] - fl[a]; }
    int64_t i0 = (int64_t)fl[0], j0 = (int64_t)fl[1], k0 = (int64_t)fl[2];
    for (int c = 0; c < 8; c++) {
        int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
        int64_t i = i0 + di, j = j0 + dj, k = k0 + dk;
        if (i < 0 || j < 0 || k < 0 || i >= dims[0] || j >= dims[1] || k >= dims[2]) continue;
        double wgt = (di ? f[0] : 1.0 - f[0]) * (dj ? f[1] : 1.0 - f[1]) * (dk ? f[2] : 1.0 - f[2]);
        dV[(k * dims[1] + j) * dims[0] + i] += g * wgt;
    }
}

/* Gradient of trilin with respect to u (derivative of the weights inside the
 * floor cell; at an exact integer u this is the one-sided derivative from the
 * cell [u, u+1]). */
static void trilin_grad(const double* V, const int64_t dims[3], const double u[3], double gu[3]) {
    double fl[3], f[3];
    for (int a = 0; a < 3; a++) { fl[a] = floor(u[a]); f[a] = u[a] - fl[a]; }
    int64_t i0 = (int64_t)fl[0], j0 = (int64_t)fl[1], k0 = (int64_t)fl[2];
    gu[0] = gu[1] = gu[2] = 0.0;
    for (int c = 0; c < 8; c++) {
        int dd[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
        double val = vox_at(V, dims, i0 + dd[0], j0 + dd[1], k0 + dd[2]);
        double wv[3], dw[3];
        for (int a = 0; a < 3; a++) { wv[a] = dd[a] ? f[a] : 1.0 - f[a]; dw[a] = dd[a] ? 1.0 : -1.0; }
        gu[0] += val * dw[0] * wv[1] * wv[2];
        gu[1] += val * wv[0] * dw[1] * wv[2];
        gu[2] += val * wv[0] * wv[1] * dw[2];
    }
}

/* -------------------------------------------------------------------- warp */

/* Eq. 2 (pull warp): W[p][v] = Trilin(V, (i,j,k) + D[p][:,v] / vox). */
void orc_warp(const int64_t dims[3], const double vox[3], int P, const double* V, const double* D, double* W) {
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2], N = nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < N; v++) {
        int64_t i = v % nx, j = (v / nx) % ny, k = v / (nx * ny);
        for (int p = 0; p < P; p++) {
            const double* Dp = D + (int64_t)p * 3 * N;
            double u[3] = {(double)i + Dp[v] / vox[0], (double)j + Dp[N + v] / vox[1], (double)k + Dp[2 * N + v] / vox[2]};
            W[(int64_t)p * N + v] = trilin(V, dims, u);
        }
    }
}

/* Adjoint of orc_warp: dV = sum_p scatter of dW (overwrites dV);
 * dD[p][k][v] = dW[p][v] dTrilin/du_k / vox_k (overwrites dD). */
void orc_warp_backward(const int64_t dims[3], const double vox[3], int P, const double* V, const double* D,
                       const double* dW, double* dV, double* dD) {
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2], N = nx * ny * nz;
    memset(dV, 0, sizeof(double) * (size_t)N);
    for (int p = 0; p < P; p++) {
        const double* Dp = D + (int64_t)p * 3 * N;
#pragma omp parallel for schedule(static)
        for (int64_t v = 0; v < N; v++) {
            int64_t i = v % nx, j = (v / nx) % ny, k = v / (nx * ny);
            double u[3] = {(double)i + Dp[v] / vox[0], (double)j + Dp[N + v] / vox[1], (double)k + Dp[2 * N + v] / vox[2]};
            double gu[3];
            trilin_grad(V, dims, u, gu);
            double g = dW[(int64_t)p * N + v];
            for (int a = 0; a < 3; a++) dD[((int64_t)p * 3 + a) * N + v] = g * gu[a] / vox[a];
        }
        for (int64_t v = 0; v < N; v++) {
            int64_t i = v % nx, j = (v / nx) % ny, k = v / (nx * ny);
            double u[3] = {(double)i + Dp[v] / vox[0], (double)j + Dp[N + v] / vox[1], (double)k + Dp[2 * N + v] / vox[2]};
            trilin_adj(dV, dims, u, dW[(int64_t)p * N + v]);
        }
    }
}

/* --------------------------------------------------------------- projector */

typedef struct { double src[3], dir[3]; int64_t m_lo, m_hi; } ray_t;

/* Ray from the source through the centre of pixel (a, b) and the range of
 * sample indices m that can touch the zero-padded volume.  A sample at x
 * contributes only if |x_a| < (n_a + 1) v_a / 2 on every axis, so every such
 * sample lies inside the sphere of radius |((n+1) v / 2)| about the origin. */
static void make_ray(const double* view, int nu, int nv, int a, int b, const int64_t dims[3], const double vox[3],
                     double step, ray_t* r) {
    const double *src = view, *det = view + 3, *du = view + 6, *dv = view + 9;
    double ca = (double)a + 0.5 - 0.5 * (double)nu, cb = (double)b + 0.5 - 0.5 * (double)nv;
    double len = 0.0;
    for (int t = 0; t < 3; t++) {
        r->src[t] = src[t];
        r->dir[t] = det[t] + ca * du[t] + cb * dv[t] - src[t];
        len += r->dir[t] * r->dir[t];
    }
    len = sqrt(len);
    for (int t = 0; t < 3; t++) r->dir[t] /= len;
    double rad2 = 0.0, tc = 0.0, d2 = 0.0;
    for (int t = 0; t < 3; t++) {
        double h = 0.5 * (double)(dims[t] + 1) * vox[t];
        rad2 += h * h;
        tc -= src[t] * r->dir[t];
        d2 += src[t] * src[t];
    }
    double perp2 = d2 - tc * tc;
    if (perp2 >= rad2) { r->m_lo = 1; r->m_hi = 0; return; }
    double half = sqrt(rad2 - perp2);
    double lo = floor((tc - half) / step) - 1.0, hi = ceil((tc + half) / step) + 1.0;
    if (lo < 0.0) lo = 0.0;
    r->m_lo = (int64_t)lo; r->m_hi = (int64_t)hi;
}

/* Eq. 6, discretised: Y[p][b][a] = step * sum_{m >= 0} Trilin(vol_p, idx(src + m step r)).
 * views: [P][12] = src, detector centre, du, dv.  vol_stride = 0 shares one
 * volume between all views; otherwise view p reads vol + p * vol_stride. */
void orc_project(const int64_t dims[3], const double vox[3], int nu, int nv, double step, int P,
                 const double* views, const double* vol, int64_t vol_stride, double* Y) {
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int p = 0; p < P; p++)
        for (int b = 0; b < nv; b++) {
            const double* W = vol + (int64_t)p * vol_stride;
            for (int a = 0; a < nu; a++) {
                ray_t r;
                make_ray(views + 12 * p, nu, nv, a, b, dims, vox, step, &r);
                double acc = 0.0;
                for (int64_t m = r.m_lo; m <= r.m_hi; m++) {
                    double t = (double)m * step, u[3];
                    for (int ax = 0; ax < 3; ax++) u[ax] = to_index(r.src[ax] + t * r.dir[ax], dims[ax], vox[ax]);
                    acc += trilin(W, dims, u);
                }
                Y[((int64_t)p * nv + b) * nu + a] = step * acc;
            }
        }
}

/* Adjoint of orc_project: dvol (overwritten) = step * sum over rays and samples
 * of dY times the trilinear weights.  vol_stride = 0: one shared dvol[N];
 * otherwise dvol[P][N]. */
void orc_project_backward(const int64_t dims[3], const double vox[3], int nu, int nv, double step, int P,
                          const double* views, const double* dY, double* dvol, int64_t vol_stride) {
    const int64_t N = dims[0] * dims[1] * dims[2];
    memset(dvol, 0, sizeof(double) * (size_t)(vol_stride ? (int64_t)P * N : N));
#pragma omp parallel for schedule(dynamic, 1) if (vol_stride != 0)
    for (int p = 0; p < P; p++) {
        double* dW = dvol + (int64_t)p * vol_stride;
        for (int b = 0; b < nv; b++)
            for (int a = 0; a < nu; a++) {
                ray_t r;
                make_ray(views + 12 * p, nu, nv, a, b, dims, vox, step, &r);
                double g = step * dY[((int64_t)p * nv + b) * nu + a];
                for (int64_t m = r.m_lo; m <= r.m_hi; m++) {
                    double t = (double)m * step, u[3];
                    for (int ax = 0; ax < 3; ax++) u[ax] = to_index(r.src[ax] + t * r.dir[ax], dims[ax], vox[ax]);
                    trilin_adj(dW, dims, u, g);
                }
            }
    }
}

/* Test mode (no voxelization): step * sum_{m in [m_lo, m_hi]} sigma(src + m step r)
 * with sigma the untruncated Gaussian mixture of Eq. 5, for pinning the
 * quadrature against the closed-form line integral of Eq. 7. */
void orc_project_gaussians(int nu, int nv, double step, int P, const double* views, int64_t G,
                           const double* mean, const double* scale, const double* quat, const double* value,
                           int64_t m_lo, int64_t m_hi, double* Y) {
    gauss_t* gs = (gauss_t*)malloc(sizeof(gauss_t) * (size_t)(G > 0 ? G : 1));
    int64_t dims1[3] = {1, 1, 1};
    double vox1[3] = {1, 1, 1};
    for (int64_t g = 0; g < G; g++) prepare(&gs[g], mean + 3 * g, scale + 3 * g, quat + 4 * g, INFINITY, 0, dims1, vox1);
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int p = 0; p < P; p++)
        for (int b = 0; b < nv; b++)
            for (int a = 0; a < nu; a++) {
                const double* view = views + 12 * p;
                double ca = (double)a + 0.5 - 0.5 * (double)nu, cb = (double)b + 0.5 - 0.5 * (double)nv;
                double dir[3], len = 0.0;
                for (int t = 0; t < 3; t++) { dir[t] = view[3 + t] + ca * view[6 + t] + cb * view[9 + t] - view[t]; len += dir[t] * dir[t]; }
                len = sqrt(len);
                for (int t = 0; t < 3; t++) dir[t] /= len;
                double acc = 0.0;
                for (int64_t m = m_lo; m <= m_hi; m++) {
                    double x[3];
                    for (int t = 0; t < 3; t++) x[t] = view[t] + (double)m * step * dir[t];
                    for (int64_t g = 0; g < G; g++) {
                        double d[3] = {x[0] - gs[g].mu[0], x[1] - gs[g].mu[1], x[2] - gs[g].mu[2]}, r[3];
                        acc += value[g] * exp(-0.5 * qform(&gs[g], d, r));
                    }
                }
                Y[((int64_t)p * nv + b) * nu + a] = step * acc;
            }
    free(gs);
}

/* -------------------------------------------------------------------- loss */

/* Eq. 10/12 (L1, kind 1) and the squared form of Eq. 1 (L2, kind 2), averaged
 * over all n = B * Q pixels of the batch.  d_pred (nullable) receives
 * sign(pred - meas) / n (sign(0) = 0) or 2 (pred - meas) / n. */
double orc_loss(int kind, int64_t n, const double* pred, const double* meas, double* d_pred) {
    double acc = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double r = pred[i] - meas[i];
        if (kind == 1) {
            acc += fabs(r);
            if (d_pred) d_pred[i] = (r > 0.0 ? 1.0 : (r < 0.0 ? -1.0 : 0.0)) / (double)n;
        } else {
            acc += r * r;
            if (d_pred) d_pred[i] = 2.0 * r / (double)n;
        }
    }
    return acc / (double)n;
}

/* ------------------------------------------------ Eq. 13-14 loss terms */

/* SSIM window (Zhou et al. 2004, the customary 11 x 11 Gaussian of standard
 * deviation 1.5 pixels): w[t] for offsets t - 5, normalised so that the 2-D
 * window w[i] w[j] sums to 1. */
static void ssim_window(double w[11]) {
    double s = 0.0;
    for (int t = 0; t < 11; t++) {
        const double d = (double)(t - 5);
        w[t] = exp(-d * d / (2.0 * 1.5 * 1.5));
        s += w[t];
    }
    for (int t = 0; t < 11; t++) w[t] /= s;
}

/* Windowed sum of f(x, y) over the 11 x 11 window centred at pixel (a, b) of
 * one nv x nu image pair; pixels outside the image count as zero. */
static void window_moments(const double* X, const double* Yv, int nu, int nv, int a, int b, const double w[11],
                           double m[5]) {
    for (int k = 0; k < 5; k++) m[k] = 0.0;
    for (int j = -5; j <= 5; j++) {
        const int bb = b + j;
        if (bb < 0 || bb >= nv) continue;
        for (int i = -5; i <= 5; i++) {
            const int aa = a + i;
            if (aa < 0 || aa >= nu) continue;
            const double wt = w[j + 5] * w[i + 5];
            const double x = X[(int64_t)bb * nu + aa], y = Yv[(int64_t)bb * nu + aa];
            m[0] += wt * x;      /* mu_x */
            m[1] += wt * y;      /* mu_y */
            m[2] += wt * x * x;  /* E[x^2] */
            m[3] += wt * y * y;  /* E[y^2] */
            m[4] += wt * x * y;  /* E[xy] */
        }
    }
}

/* D-SSIM term of Eq. 10/12: the mean over the P projections of
 * 1 - mean_pixels SSIM(pred_p, meas_p), with, at every pixel,
 *   SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),
 *   s_x^2 = E[x^2] - mu_x^2, s_xy = E[xy] - mu_x mu_y (windowed, zero padding),
 *   C1 = (0.01 range)^2, C2 = (0.03 range)^2.
 * d_pred (nullable) receives d loss / d pred by the chain rule through the
 * windowed sums: pixel r enters the sums of every pixel q within its window. */
double orc_dssim(int P, int nu, int nv, const double* pred, const double* meas, double range, double* d_pred) {
    double w[11];
    ssim_window(w);
    const double C1 = (0.01 * range) * (0.01 * range), C2 = (0.03 * range) * (0.03 * range);
    const int64_t Q = (int64_t)nu * nv;
    double total = 0.0;
    double* G = (double*)malloc(sizeof(double) * 3 * (size_t)Q);  /* dS/d mu_x, dS/d E[x^2], dS/d E[xy] */
    for (int p = 0; p < P; p++) {
        const double* X = pred + (int64_t)p * Q;
        const double* Yv = meas + (int64_t)p * Q;
        double ssum = 0.0;
#pragma omp parallel for reduction(+ : ssum) schedule(static)
        for (int64_t q = 0; q < Q; q++) {
            const int a = (int)(q % nu), b = (int)(q / nu);
            double m[5];
            window_moments(X, Yv, nu, nv, a, b, w, m);
            const double mx = m[0], my = m[1];
            const double A1 = 2.0 * mx * my + C1, A2 = 2.0 * (m[4] - mx * my) + C2;
            const double B1 = mx * mx + my * my + C1, B2 = (m[2] - mx * mx) + (m[3] - my * my) + C2;
            const double S = A1 * A2 / (B1 * B2);
            ssum += S;
            G[q] = 2.0 * my * (A2 - A1) / (B1 * B2) - 2.0 * mx * S * (1.0 / B1 - 1.0 / B2);
            G[Q + q] = -S / B2;
            G[2 * Q + q] = 2.0 * A1 / (B1 * B2);
        }
        total += 1.0 - ssum / (double)Q;
        if (d_pred) {
            const double f = -1.0 / ((double)P * (double)Q);
#pragma omp parallel for schedule(static)
            for (int64_t r = 0; r < Q; r++) {
                const int a = (int)(r % nu), b = (int)(r / nu);
                double g1 = 0.0, g2 = 0.0, g3 = 0.0;
                for (int j = -5; j <= 5; j++) {
                    const int bb = b + j;
                    if (bb < 0 || bb >= nv) continue;
                    for (int i = -5; i <= 5; i++) {
                        const int aa = a + i;
                        if (aa < 0 || aa >= nu) continue;
                        const double wt = w[j + 5] * w[i + 5];
                        const int64_t q = (int64_t)bb * nu + aa;
                        g1 += wt * G[q];
                        g2 += wt * G[Q + q];
                        g3 += wt * G[2 * Q + q];
                    }
                }
                d_pred[(int64_t)p * Q + r] = f * (g1 + 2.0 * X[r] * g2 + Yv[r] * g3);
            }
        }
    }
    free(G);
    return total / (double)P;
}

/* Sub-volume total variation (the TV term of Eq. 11/14): on the D^3 crop of
 * V [nz][ny][nx] starting at voxel origin o, the mean over the three axes of
 * the mean absolute forward difference between neighbouring crop voxels
 * ((D-1) D^2 differences per axis).  dV (nullable, [N]) receives the
 * subgradient (sign(0) = 0) inside the crop and zero elsewhere. */
double orc_tv(const int64_t dims[3], const double* V, int D, const int64_t o[3], double* dV) {
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    const double per_axis = (double)(D - 1) * (double)D * (double)D;
    if (dV) memset(dV, 0, sizeof(double) * (size_t)(nx * ny * nz));
    double total = 0.0;
    for (int axis = 0; axis < 3; axis++) {
        double s = 0.0;
        for (int z = 0; z < D; z++)
            for (int y = 0; y < D; y++)
                for (int x = 0; x < D; x++) {
                    const int c[3] = {x, y, z};
                    if (c[axis] + 1 >= D) continue;
                    const int64_t v = ((o[2] + z) * ny + (o[1] + y)) * nx + (o[0] + x);
                    const int64_t step = axis == 0 ? 1 : (axis == 1 ? nx : nx * ny);
                    const double d = V[v + step] - V[v];
                    s += fabs(d);
                    if (dV) {
                        const double sg = (d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0)) / (3.0 * per_axis);
                        dV[v + step] += sg;
                        dV[v] -= sg;
                    }
                }
        total += s / per_axis;
    }
    return total / 3.0;
}

/* Eq. 13: (1 / (3 L)) sum over levels l and axes k of (||e_{l,k}||^2 - 1)^2,
 * ||e||^2 the sum of squares of the MBC volume over the grid (L = 3 gives the
 * paper's 1/9).  E is [L][3][N]; dE (nullable) receives
 * 4 (||e_{l,k}||^2 - 1) e_{l,k} / (3 L). */
double orc_mbc_normality(int L, int64_t N, const double* E, double* dE) {
    double total = 0.0;
    for (int lk = 0; lk < 3 * L; lk++) {
        const double* e = E + (int64_t)lk * N;
        double n2 = 0.0;
        for (int64_t v = 0; v < N; v++) n2 += e[v] * e[v];
        total += (n2 - 1.0) * (n2 - 1.0);
        if (dE)
            for (int64_t v = 0; v < N; v++) dE[(int64_t)lk * N + v] = 4.0 * (n2 - 1.0) * e[v] / (3.0 * L);
    }
    return total / (3.0 * L);
}

/* ------------------------------------------- Stage-1 X-ray rasterizer */
/*
 * Eq. 8-9 (Gaussian splatting of the reference Gaussians into one cone-beam
 * projection).  Ray space for view (src, det, du, dv): a point x maps to
 *   x~ = phi(x) = (a(x), b(x), |x - src|),
 * where (a, b) are the detector pixel coordinates (relative to the detector
 * centre, in pixels) at which the ray from the source through x meets the
 * detector plane, and the third coordinate is the distance along that ray, so
 * integrating over it at fixed (a, b) integrates along one X-ray.  Eq. 8 takes
 * the local affine approximation of phi at the Gaussian's mean p: with J the
 * Jacobian of the composed map (the viewing transform W is the rigid part of
 * it), Sigma~ = J Sigma J^T and p~ = phi(p).  Integrating the ray-space Gaussian
 * over its third coordinate gives Eq. 9: a 2-D Gaussian with mean p^ and
 * covariance Sigma^ (the first two rows and columns) and amplitude
 * rho^ = sqrt(2 pi |Sigma~| / |Sigma^|) rho, evaluated at pixel centres
 * x^ = (i + 1/2 - nu/2, j + 1/2 - nv/2).  Readings: a Gaussian whose mean is
 * not in front of the source (depth <= 0) contributes nothing; the 2-D Gaussian
 * is truncated to (x^ - p^)^T Sigma^-1 (x^ - p^) <= kappa^2 (kappa = +inf: none).
 */

typedef struct {
    double src[3], D[3], n[3], ut[3], vt[3], h, a0, b0;
} splat_view_t;

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Detector-plane frame of one view: unit normal n (towards the detector),
 * source-to-plane distance h, and the dual basis (ut, vt) of (du, dv) in the
 * plane, so that a point y of the plane is det + (ut.(y-det)) du + (vt.(y-det)) dv. */
static void splat_view(const double* view, splat_view_t* v) {
    const double *src = view, *det = view + 3, *du = view + 6, *dv = view + 9;
    for (int t = 0; t < 3; t++) { v->src[t] = src[t]; v->D[t] = det[t] - src[t]; }
    double n[3] = {du[1] * dv[2] - du[2] * dv[1], du[2] * dv[0] - du[0] * dv[2], du[0] * dv[1] - du[1] * dv[0]};
    double nn = sqrt(dot3(n, n));
    double sgn = dot3(n, v->D) < 0.0 ? -1.0 : 1.0;
    for (int t = 0; t < 3; t++) v->n[t] = sgn * n[t] / nn;
    v->h = dot3(v->n, v->D);
    double uu = dot3(du, du), vv = dot3(dv, dv), uv = dot3(du, dv), del = uu * vv - uv * uv;
    for (int t = 0; t < 3; t++) {
        v->ut[t] = (vv * du[t] - uv * dv[t]) / del;
        v->vt[t] = (uu * dv[t] - uv * du[t]) / del;
    }
    v->a0 = dot3(v->ut, v->D);
    v->b0 = dot3(v->vt, v->D);
}

static double det3(const double M[9]) {
    return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) + M[2] * (M[3] * M[7] - M[4] * M[6]);
}

/* The projected 2-D Gaussian of one Gaussian in one view (Eq. 8-9).
 * Out: ph[2] = p^, S[3] = (Sigma^_00, Sigma^_01, Sigma^_11), K[3] = the same
 * entries of Sigma^-1, *rho_hat, and the intermediates the adjoint needs.
 * Returns 0 when the mean is not in front of the source. */
typedef struct {
    double r[3], z, ua, vb, L, J[9], Sig[9], St[9], M[9], R[9], qn[4], qnorm, s[3];
    double ph[2], S[3], K[3], detS, detSt, rho_hat, rho;
} splat_g_t;

static int splat_project(const splat_view_t* v, const double* mean, const double* scale, const double* quat,
                         double value, splat_g_t* o) {
    for (int t = 0; t < 3; t++) o->r[t] = mean[t] - v->src[t];
    o->z = dot3(v->n, o->r);
    if (!(o->z > 0.0)) return 0;
    o->ua = dot3(v->ut, o->r);
    o->vb = dot3(v->vt, o->r);
    o->L = sqrt(dot3(o->r, o->r));
    const double h = v->h, z = o->z;
    /* phi(p): pixel coordinates of the ray through p (a0, b0: the detector centre) */
    o->ph[0] = h * o->ua / z - v->a0;
    o->ph[1] = h * o->vb / z - v->b0;
    /* J = d phi / dx at p, rows (da/dx, db/dx, d|x - src|/dx) */
    for (int t = 0; t < 3; t++) {
        o->J[t] = h / z * (v->ut[t] - o->ua / z * v->n[t]);
        o->J[3 + t] = h / z * (v->vt[t] - o->vb / z * v->n[t]);
        o->J[6 + t] = o->r[t] / o->L;
    }
    /* Sigma = R diag(s^2) R^T = M M^T with M = R diag(s) */
    quat_to_rot(quat, o->R, o->qn, &o->qnorm);
    for (int j = 0; j < 3; j++) o->s[j] = scale[j];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) o->M[3 * i + j] = o->R[3 * i + j] * scale[j];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += o->M[3 * i + k] * o->M[3 * j + k];
            o->Sig[3 * i + j] = acc;
        }
    /* Sigma~ = J Sigma J^T */
    double JS[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += o->J[3 * i + k] * o->Sig[3 * k + j];
            JS[3 * i + j] = acc;
        }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += JS[3 * i + k] * o->J[3 * j + k];
            o->St[3 * i + j] = acc;
        }
    o->S[0] = o->St[0]; o->S[1] = o->St[1]; o->S[2] = o->St[4];
    o->detS = o->S[0] * o->S[2] - o->S[1] * o->S[1];
    o->detSt = det3(o->St);
    o->K[0] = o->S[2] / o->detS; o->K[1] = -o->S[1] / o->detS; o->K[2] = o->S[0] / o->detS;
    o->rho = value;
    o->rho_hat = sqrt(2.0 * 3.14159265358979323846 * o->detSt / o->detS) * value;
    return 1;
}

/* For tests: (p^_a, p^_b, Sigma^_00, Sigma^_01, Sigma^_11, rho^, |Sigma~|, |Sigma^|) of one
 * Gaussian in one view; returns 0 (and leaves out untouched) behind the source. */
int orc_splat_params(const double* view, const double* mean, const double* scale, const double* quat, double value,
                     double* out) {
    splat_view_t v;
    splat_g_t g;
    splat_view(view, &v);
    if (!splat_project(&v, mean, scale, quat, value, &g)) return 0;
    out[0] = g.ph[0]; out[1] = g.ph[1]; out[2] = g.S[0]; out[3] = g.S[1]; out[4] = g.S[2];
    out[5] = g.rho_hat; out[6] = g.detSt; out[7] = g.detS;
    return 1;
}

/* Eq. 9: Y[p][j][i] = sum_g rho^_g exp(-1/2 (x^ - p^_g)^T Sigma^_g^-1 (x^ - p^_g)), truncated at kappa. */
void orc_splat(int nu, int nv, int P, const double* views, int64_t G, const double* mean, const double* scale,
               const double* quat, const double* value, double kappa, double* Y) {
    const double k2 = isinf(kappa) ? INFINITY : kappa * kappa;
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < P; p++) {
        splat_view_t v;
        splat_view(views + 12 * p, &v);
        double* Yp = Y + (int64_t)p * nu * nv;
        for (int64_t q = 0; q < (int64_t)nu * nv; q++) Yp[q] = 0.0;
        for (int64_t g = 0; g < G; g++) {
            splat_g_t s;
            if (!splat_project(&v, mean + 3 * g, scale + 3 * g, quat + 4 * g, value[g], &s)) continue;
            for (int j = 0; j < nv; j++)
                for (int i = 0; i < nu; i++) {
                    double da = (double)i + 0.5 - 0.5 * (double)nu - s.ph[0];
                    double db = (double)j + 0.5 - 0.5 * (double)nv - s.ph[1];
                    double q2 = s.K[0] * da * da + 2.0 * s.K[1] * da * db + s.K[2] * db * db;
                    if (!(q2 <= k2)) continue;
                    Yp[(int64_t)j * nu + i] += s.rho_hat * exp(-0.5 * q2);
                }
        }
    }
}

/* Adjoint of orc_splat with respect to every Gaussian parameter (the truncation
 * indicator has zero derivative); gradients overwrite the outputs.  Per view the
 * pixel sums give dL/drho^, dL/dp^ and dL/dSigma^-1; the chain then runs back
 * through rho^ = sqrt(2 pi |Sigma~|/|Sigma^|) rho, Sigma^-1, Sigma~ = J Sigma J^T,
 * Sigma = M M^T (M = R diag(s)), R(q/|q|), p^ = phi(p) and J(p). */
void orc_splat_backward(int nu, int nv, int P, const double* views, int64_t G, const double* mean,
                        const double* scale, const double* quat, const double* value, double kappa, const double* dY,
                        double* d_mean, double* d_scale, double* d_quat, double* d_value) {
    const double k2 = isinf(kappa) ? INFINITY : kappa * kappa;
    splat_view_t* vs = (splat_view_t*)malloc(sizeof(splat_view_t) * (size_t)(P > 0 ? P : 1));
    for (int p = 0; p < P; p++) splat_view(views + 12 * p, &vs[p]);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t g = 0; g < G; g++) {
        double gmu[3] = {0, 0, 0}, gs[3] = {0, 0, 0}, gR[9] = {0}, grho = 0.0;
        double qn[4] = {1, 0, 0, 0}, qnorm = 1.0;
        for (int p = 0; p < P; p++) {
            const splat_view_t* v = &vs[p];
            splat_g_t s;
            if (!splat_project(v, mean + 3 * g, scale + 3 * g, quat + 4 * g, value[g], &s)) continue;
            for (int c = 0; c < 4; c++) qn[c] = s.qn[c];
            qnorm = s.qnorm;
            /* pixel sums */
            double g_rh = 0.0, g_ph[2] = {0, 0}, gK[4] = {0, 0, 0, 0}; /* gK: full 2x2, row-major */
            const double* dYp = dY + (int64_t)p * nu * nv;
            for (int j = 0; j < nv; j++)
                for (int i = 0; i < nu; i++) {
                    double d[2] = {(double)i + 0.5 - 0.5 * (double)nu - s.ph[0],
                                   (double)j + 0.5 - 0.5 * (double)nv - s.ph[1]};
                    double q2 = s.K[0] * d[0] * d[0] + 2.0 * s.K[1] * d[0] * d[1] + s.K[2] * d[1] * d[1];
                    if (!(q2 <= k2)) continue;
                    double e = exp(-0.5 * q2), gy = dYp[(int64_t)j * nu + i];
                    double c = gy * s.rho_hat * e;
                    g_rh += gy * e;
                    double Kd[2] = {s.K[0] * d[0] + s.K[1] * d[1], s.K[1] * d[0] + s.K[2] * d[1]};
                    g_ph[0] += c * Kd[0];
                    g_ph[1] += c * Kd[1];
                    for (int a = 0; a < 2; a++)
                        for (int b = 0; b < 2; b++) gK[2 * a + b] += -0.5 * c * d[a] * d[b];
                }
            /* rho^ = sqrt(2 pi detSt / detS) rho */
            grho += g_rh * s.rho_hat / s.rho;
            double g_detSt = g_rh * s.rho_hat / (2.0 * s.detSt), g_detS = -g_rh * s.rho_hat / (2.0 * s.detS);
            /* K = S^-1 (full 2x2): gS = -K^T gK K^T */
            double Km[4] = {s.K[0], s.K[1], s.K[1], s.K[2]}, Sm[4] = {s.S[0], s.S[1], s.S[1], s.S[2]}, gS[4];
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++) {
                    double acc = 0.0;
                    for (int k = 0; k < 2; k++)
                        for (int l = 0; l < 2; l++) acc += Km[2 * k + a] * gK[2 * k + l] * Km[2 * b + l];
                    gS[2 * a + b] = -acc;
                }
            /* d|S|/dS = |S| S^-T */
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++) gS[2 * a + b] += g_detS * s.detS * Km[2 * b + a];
            (void)Sm;
            /* d|St|/dSt = |St| St^-T; St^-1 by cofactors */
            double C[9];
            const double* A = s.St;
            C[0] = A[4] * A[8] - A[5] * A[7]; C[1] = -(A[3] * A[8] - A[5] * A[6]); C[2] = A[3] * A[7] - A[4] * A[6];
            C[3] = -(A[1] * A[8] - A[2] * A[7]); C[4] = A[0] * A[8] - A[2] * A[6]; C[5] = -(A[0] * A[7] - A[1] * A[6]);
            C[6] = A[1] * A[5] - A[2] * A[4]; C[7] = -(A[0] * A[5] - A[2] * A[3]); C[8] = A[0] * A[4] - A[1] * A[3];
            double gSt[9];
            for (int t = 0; t < 9; t++) gSt[t] = g_detSt * C[t]; /* |St| St^-T = cofactor matrix */
            gSt[0] += gS[0]; gSt[1] += gS[1]; gSt[3] += gS[2]; gSt[4] += gS[3];
            /* St = J Sig J^T: gJ = (gSt + gSt^T) J Sig, gSig = J^T gSt J */
            double Gs[9], gJ[9], gSig[9], JSg[9];
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) Gs[3 * a + b] = gSt[3 * a + b] + gSt[3 * b + a];
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; k++) acc += s.J[3 * a + k] * s.Sig[3 * k + b];
                    JSg[3 * a + b] = acc;
                }
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; k++) acc += Gs[3 * a + k] * JSg[3 * k + b];
                    gJ[3 * a + b] = acc;
                }
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; k++)
                        for (int l = 0; l < 3; l++) acc += s.J[3 * k + a] * gSt[3 * k + l] * s.J[3 * l + b];
                    gSig[3 * a + b] = acc;
                }
            /* Sig = M M^T: gM = (gSig + gSig^T) M; M = R diag(s) */
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; k++) acc += (gSig[3 * a + k] + gSig[3 * k + a]) * s.M[3 * k + b];
                    gR[3 * a + b] += acc * s.s[b];
                    gs[b] += acc * s.R[3 * a + b];
                }
            /* p^ and J as functions of r = p - src through z, ua, vb and L */
            const double h = v->h, z = s.z;
            double g_ua = g_ph[0] * h / z, g_vb = g_ph[1] * h / z;
            double g_z = -(g_ph[0] * h * s.ua + g_ph[1] * h * s.vb) / (z * z);
            for (int t = 0; t < 3; t++) {
                g_z += gJ[t] * (-h / (z * z) * v->ut[t] + 2.0 * h * s.ua / (z * z * z) * v->n[t]);
                g_z += gJ[3 + t] * (-h / (z * z) * v->vt[t] + 2.0 * h * s.vb / (z * z * z) * v->n[t]);
                g_ua += gJ[t] * (-h / (z * z) * v->n[t]);
                g_vb += gJ[3 + t] * (-h / (z * z) * v->n[t]);
            }
            double gJt_r = (gJ[6] * s.r[0] + gJ[7] * s.r[1] + gJ[8] * s.r[2]) / s.L;
            for (int t = 0; t < 3; t++) {
                gmu[t] += (gJ[6 + t] - gJt_r * s.r[t] / s.L) / s.L;
                gmu[t] += g_ua * v->ut[t] + g_vb * v->vt[t] + g_z * v->n[t];
            }
        }
        double dR[4][9], gqn[4];
        drot_dq(qn, dR);
        for (int c4 = 0; c4 < 4; c4++) {
            gqn[c4] = 0.0;
            for (int t = 0; t < 9; t++) gqn[c4] += gR[t] * dR[c4][t];
        }
        double dotq = gqn[0] * qn[0] + gqn[1] * qn[1] + gqn[2] * qn[2] + gqn[3] * qn[3];
        for (int c4 = 0; c4 < 4; c4++) d_quat[4 * g + c4] = (gqn[c4] - qn[c4] * dotq) / qnorm;
        for (int a = 0; a < 3; a++) { d_mean[3 * g + a] = gmu[a]; d_scale[3 * g + a] = gs[a]; }
        d_value[g] = grho;
    }
    free(vs);
}
