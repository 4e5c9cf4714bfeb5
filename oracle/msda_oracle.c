/*
 * FP64 CPU oracle for Multi-Scale Deformable Aggregation (MSDA).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or helper with the CUDA library and includes nothing
 * from it.
 *
 * What is computed (the operator the paper accelerates):
 *   - Sec. 3.1: the 3D anchors of each query are projected into every camera
 *     and multi-scale deformable sampling is performed around the projected
 *     locations.
 *   - Sec. 3.2: every keypoint is projected into every camera view and the
 *     multi-scale features at the projected coordinates are extracted from
 *     the per-camera backbone maps.
 *   - Sec. 5.3: the MSDA operator fuses feature maps from several scales and
 *     cameras at dynamically predicted locations; the features are obtained
 *     by bilinear interpolation.
 *
 * The paper does not print the arithmetic, tensor layouts or coordinate
 * convention.  The readings taken here (all listed with the design notes):
 *   R1  normalised -> pixel mapping x = u*W - 0.5, y = v*H - 0.5, i.e. pixel
 *       (i, j) has its centre at ((j + 0.5)/W, (i + 0.5)/H);
 *   R2  loc[..., 0] is u (width axis), loc[..., 1] is v (height axis);
 *       spatial_shape[k, s] = (H, W);
 *   R3  per-corner zero padding; corners come from floor(); a point with
 *       x <= -1, x >= W, y <= -1 or y >= H (or a NaN coordinate) is dropped
 *       with value and gradient 0;
 *   R4  group g owns channels [g*C/G, (g+1)*C/G);
 *   R5  the weights are used as given (no renormalisation);
 *   R9  the location gradient is that of the bilinear patch selected by
 *       x0 = floor(x), y0 = floor(y);
 *   R10 the row of pixel (i, j) of camera k, scale s in batch b is
 *       b*sum_hw + start[k, s] + i*W + j.
 *
 * Layouts (all row-major, innermost last):
 *   feat   [B, sum_hw, C]            spatial_shape [Ncam, Nscale, 2] = (H, W)
 *   start  [Ncam, Nscale]            loc           [B, A, P, Ncam, 2] = (u, v)
 *   w      [B, A, P, Ncam, Nscale, G]
 *   out    [B, A, C]                 grad_out      [B, A, C]
 *
 * Forward, for every b, a and channel c in group g:
 *   out[b,a,c] = sum_p sum_k sum_s  w[b,a,p,k,s,g] * S_{b,k,s}(u, v)[c]
 *   S = (1-fx)(1-fy) F(y0,x0) + fx(1-fy) F(y0,x0+1)
 *     + (1-fx) fy  F(y0+1,x0) + fx fy   F(y0+1,x0+1)
 * with x0 = floor(x), fx = x - x0 (same for y) and F(i, j) the feature row
 * of pixel (i, j), or 0 outside [0,H) x [0,W).
 *
 * Backward, for upstream gradient go[b,a,:]:
 *   dfeat[row(i,j), c] += w * omega_ij * go[c]       (every in-bound corner)
 *   dw[b,a,p,k,s,g]     = sum_{c in g} go[c] * S[c]
 *   du += W * sum_g w_g sum_{c in g} go[c] * ((1-fy)(F01-F00) + fy(F11-F10))
 *   dv += H * sum_g w_g sum_{c in g} go[c] * ((1-fx)(F10-F00) + fx(F11-F01))
 * (summed over scales s for the same (b,a,p,k)); F01 = F(y0, x0+1) etc.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* One projected point at one scale: the four bilinear corners, their
 * interpolation weights and whether each lies inside the map (R1, R3). */
typedef struct {
    int in_range;         /* 0: the point is dropped entirely (R3)          */
    long row[4];          /* feature-row index of each corner              */
    int valid[4];         /* corner inside [0,H) x [0,W)                   */
    double omega[4];      /* bilinear weight of each corner                */
    double fx, fy;        /* fractional offsets inside the cell            */
} corners_t;

/* Corner order: 0 = (y0, x0), 1 = (y0, x0+1), 2 = (y0+1, x0), 3 = (y0+1, x0+1). */
static corners_t locate(double u, double v, int H, int W, long row0)
{
    corners_t c;
    memset(&c, 0, sizeof(c));
    double x = u * (double)W - 0.5;   /* R1 */
    double y = v * (double)H - 0.5;
    /* R3: written so that NaN fails the test and is dropped. */
    if (!(x > -1.0 && x < (double)W && y > -1.0 && y < (double)H)) return c;
    c.in_range = 1;
    double xf = floor(x), yf = floor(y);
    long x0 = (long)xf, y0 = (long)yf;
    c.fx = x - xf;
    c.fy = y - yf;
    for (int q = 0; q < 4; ++q) {
        long dy = q >> 1, dx = q & 1;
        long i = y0 + dy, j = x0 + dx;
        c.valid[q] = (i >= 0 && i < H && j >= 0 && j < W);
        c.row[q] = c.valid[q] ? row0 + i * (long)W + j : -1;
        double wx = dx ? c.fx : 1.0 - c.fx;
        double wy = dy ? c.fy : 1.0 - c.fy;
        c.omega[q] = wx * wy;
    }
    return c;
}

static int check_dims(int B, int sum_hw, int C, int Ncam, int Nscale, int A, int P, int G)
{
    if (B < 0 || sum_hw < 0 || C <= 0 || Ncam < 0 || Nscale < 0 || A < 0 || P < 0 || G <= 0) return 1;
    if (C % G != 0) return 1;
    return 0;
}

static int check_tables(const int32_t* shape, const int32_t* start, int sum_hw, int Ncam, int Nscale)
{
    for (int k = 0; k < Ncam; ++k)
        for (int s = 0; s < Nscale; ++s) {
            long H = shape[(k * Nscale + s) * 2 + 0], W = shape[(k * Nscale + s) * 2 + 1];
            long st = start[k * Nscale + s];
            if (H < 0 || W < 0 || st < 0 || st + H * W > (long)sum_hw) return 1;
        }
    return 0;
}

/* Forward of the operator (Sec. 3.1, 3.2, 5.3).  Returns 0 on success, 1 on
 * bad dimensions or tables.  nthreads > 1 splits the (b, a) loop across
 * OpenMP threads; each (b, a) owns its output row, so the result does not
 * depend on the thread count. */
int msda_oracle_forward(const double* feat, const int32_t* shape, const int32_t* start,
                        const double* loc, const double* w, double* out,
                        int B, int sum_hw, int C, int Ncam, int Nscale, int A, int P, int G,
                        int nthreads)
{
    if (check_dims(B, sum_hw, C, Ncam, Nscale, A, P, G)) return 1;
    if (check_tables(shape, start, sum_hw, Ncam, Nscale)) return 1;
    const int Cg = C / G;
    const long BA = (long)B * A;
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
#endif
    for (long ba = 0; ba < BA; ++ba) {
        const long b = ba / A;
        double* o = out + ba * C;
        for (int c = 0; c < C; ++c) o[c] = 0.0;
        for (int p = 0; p < P; ++p)
            for (int k = 0; k < Ncam; ++k) {
                const double* uv = loc + ((ba * P + p) * Ncam + k) * 2;
                for (int s = 0; s < Nscale; ++s) {
                    const int H = shape[(k * Nscale + s) * 2 + 0];
                    const int W = shape[(k * Nscale + s) * 2 + 1];
                    const long row0 = b * (long)sum_hw + start[k * Nscale + s];
                    corners_t cr = locate(uv[0], uv[1], H, W, row0);
                    if (!cr.in_range) continue;
                    const double* wg = w + (((ba * P + p) * Ncam + k) * Nscale + s) * G;
                    for (int q = 0; q < 4; ++q) {
                        if (!cr.valid[q]) continue;
                        const double* f = feat + cr.row[q] * (long)C;
                        for (int c = 0; c < C; ++c)
                            o[c] += wg[c / Cg] * cr.omega[q] * f[c];
                    }
                }
            }
    }
    return 0;
}

/* Backward of the operator (gradients of the forward above).  grad_feat is
 * overwritten (zeroed, then accumulated); grad_loc and grad_w are
 * overwritten.  Runs on one thread: the feature gradient is a scatter. */
int msda_oracle_backward(const double* feat, const int32_t* shape, const int32_t* start,
                         const double* loc, const double* w, const double* grad_out,
                         double* grad_feat, double* grad_loc, double* grad_w,
                         int B, int sum_hw, int C, int Ncam, int Nscale, int A, int P, int G)
{
    if (check_dims(B, sum_hw, C, Ncam, Nscale, A, P, G)) return 1;
    if (check_tables(shape, start, sum_hw, Ncam, Nscale)) return 1;
    const int Cg = C / G;
    const long BA = (long)B * A;
    memset(grad_feat, 0, sizeof(double) * (size_t)B * (size_t)sum_hw * (size_t)C);
    for (long ba = 0; ba < BA; ++ba) {
        const long b = ba / A;
        const double* go = grad_out + ba * C;
        for (int p = 0; p < P; ++p)
            for (int k = 0; k < Ncam; ++k) {
                const long pk = (ba * P + p) * Ncam + k;
                const double* uv = loc + pk * 2;
                double du = 0.0, dv = 0.0;
                for (int s = 0; s < Nscale; ++s) {
                    const int H = shape[(k * Nscale + s) * 2 + 0];
                    const int W = shape[(k * Nscale + s) * 2 + 1];
                    const long row0 = b * (long)sum_hw + start[k * Nscale + s];
                    const double* wg = w + (pk * Nscale + s) * G;
                    double* dwg = grad_w + (pk * Nscale + s) * G;
                    for (int g = 0; g < G; ++g) dwg[g] = 0.0;
                    corners_t cr = locate(uv[0], uv[1], H, W, row0);
                    if (!cr.in_range) continue;
                    const double fx = cr.fx, fy = cr.fy;
                    for (int c = 0; c < C; ++c) {
                        const int g = c / Cg;
                        double F[4];
                        for (int q = 0; q < 4; ++q)
                            F[q] = cr.valid[q] ? feat[cr.row[q] * (long)C + c] : 0.0;
                        double S = 0.0;
                        for (int q = 0; q < 4; ++q) S += cr.omega[q] * F[q];
                        dwg[g] += go[c] * S;
                        du += (double)W * wg[g] * go[c] * ((1.0 - fy) * (F[1] - F[0]) + fy * (F[3] - F[2]));
                        dv += (double)H * wg[g] * go[c] * ((1.0 - fx) * (F[2] - F[0]) + fx * (F[3] - F[1]));
                        for (int q = 0; q < 4; ++q)
                            if (cr.valid[q])
                                grad_feat[cr.row[q] * (long)C + c] += wg[g] * cr.omega[q] * go[c];
                    }
                }
                grad_loc[pk * 2 + 0] = du;
                grad_loc[pk * 2 + 1] = dv;
            }
    }
    return 0;
}

/* Occlusion-aware fusion (Sec. 3.2, Eq. 2): the per-camera aggregated
 * feature g_k = sum_{p,s} w[b,a,p,k,s,g] * S_{b,k,s}(loc[b,a,p,k]) is fused
 * over cameras with the visibility scores vis[b, a, k]:
 *   out[b,a,c] = sum_k vis[b,a,k] * g_k[c] / sum_k vis[b,a,k]
 * Reading: when the visibilities of an anchor sum to 0 the fused feature is
 * 0.  Computed literally: each g_k by the forward above restricted to camera
 * k, then the weighted mean.  Returns 0, or 1 on bad arguments. */
int msda_oracle_forward_oae(const double* feat, const int32_t* shape, const int32_t* start,
                            const double* loc, const double* w, const double* vis, double* out,
                            int B, int sum_hw, int C, int Ncam, int Nscale, int A, int P, int G)
{
    if (check_dims(B, sum_hw, C, Ncam, Nscale, A, P, G)) return 1;
    if (check_tables(shape, start, sum_hw, Ncam, Nscale)) return 1;
    const int Cg = C / G;
    const long BA = (long)B * A;
    double* g = (double*)malloc(sizeof(double) * (size_t)C);
    if (!g) return 1;
    for (long ba = 0; ba < BA; ++ba) {
        const long b = ba / A;
        double* o = out + ba * C;
        double vsum = 0.0;
        for (int k = 0; k < Ncam; ++k) vsum += vis[ba * Ncam + k];
        for (int c = 0; c < C; ++c) o[c] = 0.0;
        if (vsum == 0.0) continue;
        for (int k = 0; k < Ncam; ++k) {
            for (int c = 0; c < C; ++c) g[c] = 0.0;
            for (int p = 0; p < P; ++p) {
                const double* uv = loc + ((ba * P + p) * Ncam + k) * 2;
                for (int s = 0; s < Nscale; ++s) {
                    const int H = shape[(k * Nscale + s) * 2 + 0];
                    const int W = shape[(k * Nscale + s) * 2 + 1];
                    const long row0 = b * (long)sum_hw + start[k * Nscale + s];
                    corners_t cr = locate(uv[0], uv[1], H, W, row0);
                    if (!cr.in_range) continue;
                    const double* wg = w + (((ba * P + p) * Ncam + k) * Nscale + s) * G;
                    for (int q = 0; q < 4; ++q) {
                        if (!cr.valid[q]) continue;
                        const double* f = feat + cr.row[q] * (long)C;
                        for (int c = 0; c < C; ++c) g[c] += wg[c / Cg] * cr.omega[q] * f[c];
                    }
                }
            }
            const double vk = vis[ba * Ncam + k];
            for (int c = 0; c < C; ++c) o[c] += vk * g[c];
        }
        for (int c = 0; c < C; ++c) o[c] /= vsum;
    }
    free(g);
    return 0;
}

/* Keypoint prologue (Sec. 3.1, 3.2): the sampling locations of every
 * anchor keypoint in every camera.
 *   anchors [B, A, 11] = (x, y, z, w, l, h, sin yaw, cos yaw, vx, vy, vz),
 *     box centre and velocity in the world frame, sizes along the box's
 *     x (w), y (l) and z (h) axes;
 *   offsets [B, A, P, 3] keypoints in box units (fixed and learned alike);
 *   dt [B]: time from the anchor's frame to the current frame;
 *   proj [B, Ncam, 3, 4]: world -> homogeneous pixel matrix of each camera;
 *   img_wh [Ncam, 2]: image width and height in pixels.
 * Keypoint (Sec. 3.2: motion-compensated with the estimated velocity):
 *   q = R(yaw) (offset * size) + centre + velocity * dt
 * Projection: (xp, yp, zp) = proj * (q, 1); loc = (xp / zp / width,
 * yp / zp / height).  Reading: a keypoint with zp <= 1e-5 (behind or on the
 * camera plane) gets loc = (-2, -2), which the operator drops. */
int msda_oracle_keypoints(const double* anchors, const double* offsets, const double* dt,
                          const double* proj, const double* img_wh, double* loc,
                          int B, int A, int P, int Ncam)
{
    if (B < 0 || A < 0 || P < 0 || Ncam < 0) return 1;
    for (long b = 0; b < B; ++b)
        for (long a = 0; a < A; ++a) {
            const double* an = anchors + (b * A + a) * 11;
            const double sy = an[6], cy = an[7];
            for (long p = 0; p < P; ++p) {
                const double* of = offsets + ((b * A + a) * P + p) * 3;
                const double bx = of[0] * an[3], by = of[1] * an[4], bz = of[2] * an[5];
                double q[3];
                q[0] = cy * bx - sy * by + an[0] + an[8] * dt[b];
                q[1] = sy * bx + cy * by + an[1] + an[9] * dt[b];
                q[2] = bz + an[2] + an[10] * dt[b];
                for (long k = 0; k < Ncam; ++k) {
                    const double* M = proj + (b * Ncam + k) * 12;
                    double h[3];
                    for (int r = 0; r < 3; ++r)
                        h[r] = M[r * 4 + 0] * q[0] + M[r * 4 + 1] * q[1] + M[r * 4 + 2] * q[2] + M[r * 4 + 3];
                    double* o = loc + (((b * A + a) * P + p) * Ncam + k) * 2;
                    if (h[2] <= 1e-5) {
                        o[0] = -2.0;
                        o[1] = -2.0;
                    } else {
                        o[0] = h[0] / h[2] / img_wh[k * 2 + 0];
                        o[1] = h[1] / h[2] / img_wh[k * 2 + 1];
                    }
                }
            }
        }
    return 0;
}

/* Number of OpenMP threads available to the forward (1 without OpenMP). */
int msda_oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
