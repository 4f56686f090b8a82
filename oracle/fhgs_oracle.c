/*
 * FHGS oracle: a plain, slow, FP64 CPU implementation of the feature-splatting
 * hot path (arXiv 2505.19154).  TEST INFRASTRUCTURE ONLY: it is used by the
 * tests, by the smoke check and by the CPU-baseline leg of the benchmark.  The
 * product path never links, loads or calls it, and it shares no code, header
 * or constant table with the CUDA library.
 *
 * What each function follows:
 *   - orc_project / orc_project_bwd: the screen-space footprint of a 3-D
 *     Gaussian (EWA: Sigma' = J W Sigma W^T J^T + dilation I) and its inverse
 *     (the conic), which the paper takes over from the 3DGS rasterizer it
 *     builds on (Sec. 2.1, App. A); SH colour (Sec. 2.1, 3DGS background).
 *   - orc_bin_f32: the FP32 binning specification (pixel/tile rectangle and
 *     depth key, App. A "CreateTiles / DuplicateWithKeys"); a plain C float
 *     transcription, compiled with -ffp-contract=off so every operation is a
 *     single IEEE rounding in the written order.
 *   - orc_render: Eq. 4, c(x) = sum_i c_i w_i, w_i = alpha_i T_i,
 *     T_i = prod_{j<i} (1 - alpha_j), evaluated front to back (nearest first)
 *     over each 16x16 tile's depth-sorted list (App. A), and the same weights
 *     applied to the per-primitive feature f_i (the DRF path of Sec. 3.2).
 *   - orc_render_bwd: the exact derivative of Eq. 4, whose core is the
 *     App. A.2 identity dL/dalpha_k = T_k dL/dw_k - (1/(1-alpha_k))
 *     sum_{i>k} w_i dL/dw_i, plus the background term.
 *   - orc_render_brute: Eq. 4 per pixel over ALL primitives, sorted by depth,
 *     with no tiles (the brute-force definition).
 *   - orc_fuse: the compositing-weight-normalised feature fusion
 *     f_g = sum_{v,p} w_g(v,p) F_v(p) / sum_{v,p} w_g(v,p) (Sec. 3.1).
 *   - orc_splat_uv / orc_render_2dgs_brute / orc_render_2dgs_bwd_brute /
 *     orc_surfel_rect: the surfel model of Sec. 3.1 (Eq. 1-3): the pixel
 *     ray's intersection u(x) with a surfel's plane, G(u), Eq. 4 compositing
 *     per pixel over all surfels and its derivative (App. A.2 with the
 *     ray-plane solve differentiated implicitly), and the exact screen box of
 *     a surfel's footprint (dual conic); orc_bin_surfel_f32: its binary32
 *     binning rule (a padded box, integer decisions reproducible bit for bit);
 *     orc_render_2dgs / orc_render_2dgs_bwd: the tiled render and backward;
 *     orc_splat_uv_T: u(x) through the projective map T = K [a b c];
 *     orc_ndfd_2dgs / orc_ndfd_2dgs_bwd: the NDFD losses over the surfel
 *     render's weights and their derivative.
 *   - orc_point_views_f32: the paper's point-to-feature assignment
 *     (Sec. 3.1, App. A "PointsFeatureFusion"): a random visible view, the
 *     nearest pixel; binary32 projection spec (it decides integers).
 *   - orc_ndfd / orc_ndfd_bwd: the NDFD losses L_gt (Eq. 5) and L_cf
 *     (Eq. 6, App. A.1) with the activation of Sec. 3.3, over the render's
 *     weights, and their derivative through w (Sec. 3.3, App. A.2).
 *
 * Layouts (all row-major, caller-owned):
 *   camera  double[18]: width, height, fx, fy, cx, cy, then the 3x4
 *           world-to-camera matrix [R|t] row by row (OpenCV axes).
 *   params  double[12]: znear, dilation, alpha_min, alpha_max, t_eps,
 *           cutoff_sq, fov_clamp, bg_r, bg_g, bg_b, tile (16), sh_degree.
 *   means/scales double[n][3], quats double[n][4] (w,x,y,z), opac double[n],
 *   sh double[n][K][3] with K = (sh_degree+1)^2.
 *   projection record double[n][ORC_REC]: see the ORC_* indices below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_REC 24
enum {
    R_MX = 0, R_MY, R_A, R_B, R_C, R_DEPTH, R_R, R_G, R_BL, R_RAW_R, R_RAW_G,
    R_RAW_B, R_VALID, R_OP, R_SIG_A, R_SIG_B, R_SIG_C, R_EXT_X, R_EXT_Y
};

enum { P_ZNEAR = 0, P_DIL, P_AMIN, P_AMAX, P_TEPS, P_CUT, P_FOV, P_BG0, P_BG1,
       P_BG2, P_TILE, P_SHDEG };

static double cam_R(const double *cam, int i, int j) { return cam[6 + 4 * i + j]; }
static double cam_t(const double *cam, int i) { return cam[6 + 4 * i + 3]; }

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------- SH ---- */
/* Real spherical harmonics up to degree 3 in the 3DGS-family ordering and
 * sign convention.  Normalisation constants are the closed forms
 * sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the Legendre polynomial
 * prefactors, written out per basis function. */
static void sh_basis(const double d[3], double Y[16], double dY[16][3])
{
    const double x = d[0], y = d[1], z = d[2];
    const double PI = 3.14159265358979323846;
    const double c0 = 0.5 * sqrt(1.0 / PI);
    const double c1 = sqrt(3.0 / (4.0 * PI));
    const double c2a = 0.5 * sqrt(15.0 / PI);
    const double c2b = 0.25 * sqrt(5.0 / PI);
    const double c2c = 0.25 * sqrt(15.0 / PI);
    const double c3a = 0.25 * sqrt(35.0 / (2.0 * PI));
    const double c3b = 0.5 * sqrt(105.0 / PI);
    const double c3c = 0.25 * sqrt(21.0 / (2.0 * PI));
    const double c3d = 0.25 * sqrt(7.0 / PI);
    const double c3e = 0.25 * sqrt(105.0 / PI);
    double xx = x * x, yy = y * y, zz = z * z;

    Y[0] = c0;
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    Y[4] = c2a * x * y;
    Y[5] = -c2a * y * z;
    Y[6] = c2b * (2.0 * zz - xx - yy);
    Y[7] = -c2a * x * z;
    Y[8] = c2c * (xx - yy);
    Y[9] = -c3a * y * (3.0 * xx - yy);
    Y[10] = c3b * x * y * z;
    Y[11] = -c3c * y * (4.0 * zz - xx - yy);
    Y[12] = c3d * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
    Y[13] = -c3c * x * (4.0 * zz - xx - yy);
    Y[14] = c3e * z * (xx - yy);
    Y[15] = -c3a * x * (xx - 3.0 * yy);
    if (!dY) return;
    memset(dY, 0, sizeof(double) * 48);
    dY[1][1] = -c1;
    dY[2][2] = c1;
    dY[3][0] = -c1;
    dY[4][0] = c2a * y;           dY[4][1] = c2a * x;
    dY[5][1] = -c2a * z;          dY[5][2] = -c2a * y;
    dY[6][0] = -2.0 * c2b * x;    dY[6][1] = -2.0 * c2b * y;   dY[6][2] = 4.0 * c2b * z;
    dY[7][0] = -c2a * z;          dY[7][2] = -c2a * x;
    dY[8][0] = 2.0 * c2c * x;     dY[8][1] = -2.0 * c2c * y;
    dY[9][0] = -c3a * 6.0 * x * y;
    dY[9][1] = -c3a * (3.0 * xx - 3.0 * yy);
    dY[10][0] = c3b * y * z;      dY[10][1] = c3b * x * z;     dY[10][2] = c3b * x * y;
    dY[11][0] = c3c * 2.0 * x * y;
    dY[11][1] = -c3c * (4.0 * zz - xx - 3.0 * yy);
    dY[11][2] = -c3c * 8.0 * y * z;
    dY[12][0] = -c3d * 6.0 * x * z;
    dY[12][1] = -c3d * 6.0 * y * z;
    dY[12][2] = c3d * (6.0 * zz - 3.0 * xx - 3.0 * yy);
    dY[13][0] = -c3c * (4.0 * zz - 3.0 * xx - yy);
    dY[13][1] = c3c * 2.0 * x * y;
    dY[13][2] = -c3c * 8.0 * x * z;
    dY[14][0] = c3e * 2.0 * x * z;
    dY[14][1] = -c3e * 2.0 * y * z;
    dY[14][2] = c3e * (xx - yy);
    dY[15][0] = -c3a * (3.0 * xx - 3.0 * yy);
    dY[15][1] = c3a * 6.0 * x * y;
}

/* Exported for the SH pins: Y (n x 16) and dY (n x 16 x 3) at unit dirs. */
void orc_sh_basis(int64_t n, const double *dirs, double *Y, double *dY)
{
    for (int64_t i = 0; i < n; ++i)
        sh_basis(dirs + 3 * i, Y + 16 * i, dY ? (double (*)[3])(dY + 48 * i) : NULL);
}

/* ------------------------------------------------------- rotations ---- */
static void quat_to_rot(const double qn[4], double R[3][3])
{
    const double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R[0][1] = 2.0 * (x * y - w * z);
    R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z);
    R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y);
    R[2][1] = 2.0 * (y * z + w * x);
    R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

void orc_quat_to_rot(int64_t n, const double *q, double *R)
{
    for (int64_t i = 0; i < n; ++i) {
        double nq = sqrt(q[4 * i] * q[4 * i] + q[4 * i + 1] * q[4 * i + 1] +
                         q[4 * i + 2] * q[4 * i + 2] + q[4 * i + 3] * q[4 * i + 3]);
        double qn[4] = {q[4 * i] / nq, q[4 * i + 1] / nq, q[4 * i + 2] / nq, q[4 * i + 3] / nq};
        quat_to_rot(qn, (double (*)[3])(R + 9 * i));
    }
}

/* ------------------------------------------------------- projection --- */
/* Per Gaussian, FP64.  Fills the ORC_REC record; R_VALID = 0 when culled
 * (depth <= znear, non-positive determinant, or a non-finite value). */
static void project_one(const double *mu, const double *s, const double *q,
                        const double *sh, int K, const double *cam,
                        const double *prm, double *out)
{
    memset(out, 0, sizeof(double) * ORC_REC);
    const double W = cam[0], H = cam[1], fx = cam[2], fy = cam[3], cx = cam[4], cy = cam[5];
    double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(nq > 0.0) || !isfinite(nq)) return;
    double qn[4] = {q[0] / nq, q[1] / nq, q[2] / nq, q[3] / nq};
    double R[3][3];
    quat_to_rot(qn, R);
    double M[3][3], S[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] = R[i][j] * s[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            S[i][j] = M[i][0] * M[j][0] + M[i][1] * M[j][1] + M[i][2] * M[j][2];
    double t[3];
    for (int i = 0; i < 3; ++i)
        t[i] = cam_R(cam, i, 0) * mu[0] + cam_R(cam, i, 1) * mu[1] + cam_R(cam, i, 2) * mu[2] + cam_t(cam, i);
    if (!(t[2] > prm[P_ZNEAR])) return;
    double limx = prm[P_FOV] * (0.5 * W / fx), limy = prm[P_FOV] * (0.5 * H / fy);
    double ux = t[0] / t[2], uy = t[1] / t[2];
    double xh = ux > limx ? limx : (ux < -limx ? -limx : ux);
    double yh = uy > limy ? limy : (uy < -limy ? -limy : uy);
    double J[2][3] = {{fx / t[2], 0.0, -fx * xh / t[2]}, {0.0, fy / t[2], -fy * yh / t[2]}};
    double Tm[2][3];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            Tm[i][j] = J[i][0] * cam_R(cam, 0, j) + J[i][1] * cam_R(cam, 1, j) + J[i][2] * cam_R(cam, 2, j);
    double S2[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) acc += Tm[i][k] * S[k][l] * Tm[j][l];
            S2[i][j] = acc;
        }
    double a = S2[0][0] + prm[P_DIL], b = S2[0][1], c = S2[1][1] + prm[P_DIL];
    double det = a * c - b * b;
    if (!(det > 0.0)) return;
    double mx = fx * t[0] / t[2] + cx, my = fy * t[1] / t[2] + cy;
    if (!isfinite(mx) || !isfinite(my)) return;
    out[R_MX] = mx;
    out[R_MY] = my;
    out[R_A] = c / det;
    out[R_B] = -b / det;
    out[R_C] = a / det;
    out[R_DEPTH] = t[2];
    out[R_SIG_A] = a;
    out[R_SIG_B] = b;
    out[R_SIG_C] = c;
    out[R_EXT_X] = sqrt(prm[P_CUT] * a);
    out[R_EXT_Y] = sqrt(prm[P_CUT] * c);
    /* SH colour: direction from the camera centre (-R^T t) to the mean. */
    double cpos[3], v[3];
    for (int i = 0; i < 3; ++i)
        cpos[i] = -(cam_R(cam, 0, i) * cam_t(cam, 0) + cam_R(cam, 1, i) * cam_t(cam, 1) + cam_R(cam, 2, i) * cam_t(cam, 2));
    for (int i = 0; i < 3; ++i) v[i] = mu[i] - cpos[i];
    double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double d[3] = {v[0] / nv, v[1] / nv, v[2] / nv};
    double Y[16];
    sh_basis(d, Y, NULL);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc += sh[3 * k + ch] * Y[k];
        double raw = acc + 0.5;
        out[R_RAW_R + ch] = raw;
        out[R_R + ch] = raw > 0.0 ? raw : 0.0;
    }
    out[R_VALID] = 1.0;
}

void orc_project(int64_t n, const double *means, const double *scales, const double *quats,
                 const double *opac, const double *sh, int K, const double *cam,
                 const double *prm, double *rec)
{
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g) {
        project_one(means + 3 * g, scales + 3 * g, quats + 4 * g, sh + (int64_t)3 * K * g, K, cam, prm,
                    rec + (int64_t)ORC_REC * g);
        rec[(int64_t)ORC_REC * g + R_OP] = opac[g];
    }
}

/* ------------------------------------------------ FP32 binning spec --- */
/* Single-precision, contraction-free transcription of the binning rules:
 * every line is one IEEE-754 binary32 operation (or a fixed left-to-right
 * chain of them), sqrt and division correctly rounded.  Outputs per
 * Gaussian: pixel rectangle and tile rectangle (inclusive), tile count,
 * the raw bits of the view-space depth, and the FP32 footprint
 * (mean2d, conic) that the binning decisions were made from. */
static int bin_one_f32(const float *mu, const float *s, const float *q, const float *cam,
                       const float *prm, int32_t *pix, int32_t *tile, uint32_t *ntiles,
                       uint32_t *dbits, float *fp)
{
    const float W = cam[0], H = cam[1], fx = cam[2], fy = cam[3], cx = cam[4], cy = cam[5];
    const int tsz = (int)prm[P_TILE];
    float n2 = q[0] * q[0];
    n2 = n2 + q[1] * q[1];
    n2 = n2 + q[2] * q[2];
    n2 = n2 + q[3] * q[3];
    if (!(n2 > 0.0f) || !isfinite(n2)) return 0;
    float inv = 1.0f / sqrtf(n2);
    float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
    float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    float R[3][3];
    R[0][0] = 1.0f - 2.0f * (yy + zz);
    R[0][1] = 2.0f * (xy - wz);
    R[0][2] = 2.0f * (xz + wy);
    R[1][0] = 2.0f * (xy + wz);
    R[1][1] = 1.0f - 2.0f * (xx + zz);
    R[1][2] = 2.0f * (yz - wx);
    R[2][0] = 2.0f * (xz - wy);
    R[2][1] = 2.0f * (yz + wx);
    R[2][2] = 1.0f - 2.0f * (xx + yy);
    float M[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] = R[i][j] * s[j];
    float Sg[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            float acc = M[i][0] * M[j][0];
            acc = acc + M[i][1] * M[j][1];
            acc = acc + M[i][2] * M[j][2];
            Sg[i][j] = acc;
            Sg[j][i] = acc;
        }
    float t[3];
    for (int i = 0; i < 3; ++i) {
        float acc = cam[6 + 4 * i + 0] * mu[0];
        acc = acc + cam[6 + 4 * i + 1] * mu[1];
        acc = acc + cam[6 + 4 * i + 2] * mu[2];
        t[i] = acc + cam[6 + 4 * i + 3];
    }
    if (!(t[2] > prm[P_ZNEAR])) return 0;
    float limx = prm[P_FOV] * ((0.5f * W) / fx);
    float limy = prm[P_FOV] * ((0.5f * H) / fy);
    float ux = t[0] / t[2], uy = t[1] / t[2];
    float xh = fminf(limx, fmaxf(-limx, ux));
    float yh = fminf(limy, fmaxf(-limy, uy));
    float J00 = fx / t[2], J02 = -((fx * xh) / t[2]);
    float J11 = fy / t[2], J12 = -((fy * yh) / t[2]);
    float Tm[2][3];
    for (int j = 0; j < 3; ++j) {
        Tm[0][j] = J00 * cam[6 + 0 * 4 + j] + J02 * cam[6 + 2 * 4 + j];
        Tm[1][j] = J11 * cam[6 + 1 * 4 + j] + J12 * cam[6 + 2 * 4 + j];
    }
    float U[2][3];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            float acc = Tm[i][0] * Sg[0][j];
            acc = acc + Tm[i][1] * Sg[1][j];
            acc = acc + Tm[i][2] * Sg[2][j];
            U[i][j] = acc;
        }
    float a = U[0][0] * Tm[0][0];
    a = a + U[0][1] * Tm[0][1];
    a = a + U[0][2] * Tm[0][2];
    a = a + prm[P_DIL];
    float b = U[0][0] * Tm[1][0];
    b = b + U[0][1] * Tm[1][1];
    b = b + U[0][2] * Tm[1][2];
    float c = U[1][0] * Tm[1][0];
    c = c + U[1][1] * Tm[1][1];
    c = c + U[1][2] * Tm[1][2];
    c = c + prm[P_DIL];
    float ac = a * c;
    float det = ac - b * b;
    float A, B, C;
    if (det < 1e-6f * ac) {
        /* near-degenerate: determinant and inverse in binary64 */
        double dd = (double)a * (double)c - (double)b * (double)b;
        det = (float)dd;
        if (!(det > 0.0f)) return 0;
        A = (float)((double)c / dd);
        B = (float)(-(double)b / dd);
        C = (float)((double)a / dd);
    } else {
        if (!(det > 0.0f)) return 0;
        A = c / det;
        B = -(b / det);
        C = a / det;
    }
    float mx = (fx * t[0]) / t[2] + cx;
    float my = (fy * t[1]) / t[2] + cy;
    float ex = sqrtf(prm[P_CUT] * a);
    float ey = sqrtf(prm[P_CUT] * c);
    if (!isfinite(mx) || !isfinite(my) || !isfinite(ex) || !isfinite(ey)) return 0;
    float xlo = ceilf((mx - ex) - 0.5f), xhi = floorf((mx + ex) - 0.5f);
    float ylo = ceilf((my - ey) - 0.5f), yhi = floorf((my + ey) - 0.5f);
    xlo = fmaxf(xlo, 0.0f);
    ylo = fmaxf(ylo, 0.0f);
    xhi = fminf(xhi, W - 1.0f);
    yhi = fminf(yhi, H - 1.0f);
    if (xlo > xhi || ylo > yhi) return 0;
    int ix0 = (int)xlo, ix1 = (int)xhi, iy0 = (int)ylo, iy1 = (int)yhi;
    pix[0] = ix0; pix[1] = iy0; pix[2] = ix1; pix[3] = iy1;
    tile[0] = ix0 / tsz; tile[1] = iy0 / tsz; tile[2] = ix1 / tsz; tile[3] = iy1 / tsz;
    *ntiles = (uint32_t)((tile[2] - tile[0] + 1) * (tile[3] - tile[1] + 1));
    memcpy(dbits, &t[2], 4);
    fp[0] = mx; fp[1] = my; fp[2] = A; fp[3] = B; fp[4] = C; fp[5] = t[2];
    return 1;
}

void orc_bin_f32(int64_t n, const float *means, const float *scales, const float *quats,
                 const float *cam, const float *prm, int32_t *pix, int32_t *tile,
                 uint32_t *ntiles, uint32_t *dbits, float *fp)
{
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g) {
        int ok = bin_one_f32(means + 3 * g, scales + 3 * g, quats + 4 * g, cam, prm, pix + 4 * g,
                             tile + 4 * g, ntiles + g, dbits + g, fp + 6 * g);
        if (!ok) {
            for (int k = 0; k < 4; ++k) { pix[4 * g + k] = -1; tile[4 * g + k] = -1; }
            ntiles[g] = 0;
            dbits[g] = 0xFFFFFFFFu;
            for (int k = 0; k < 6; ++k) fp[6 * g + k] = 0.0f;
        }
    }
}

/* --------------------------------------------------------- render ----- */
/* One pixel, Eq. 4 front to back over an ordered candidate list.  Records
 * the contributors (index into the list, alpha, T before, weight) when
 * `rec_*` are given.  Returns the number of contributors. */
typedef struct {
    double T;
    double rgb[3];
    int32_t last;       /* (position of the last contributor in the list) + 1 */
    double margin;      /* min relative distance to its threshold of a decision
                           that decides the contributor set (cutoff, alpha_min,
                           stop); the continuous alpha_max clamp is left out */
    uint64_t sig;       /* hash of the contributor set and clamp flags */
} pix_state;

static double rel(double v, double thr) { return fabs(v - thr) / thr; }

static int composite_pixel(double px, double py, const uint32_t *list, int64_t len,
                           const double *rec, const double *feat, int D, const double *prm,
                           pix_state *st, double *F, int64_t *ci, double *calpha, double *cT,
                           double *cG, int64_t cap)
{
    const double cut = prm[P_CUT], amin = prm[P_AMIN], amax = prm[P_AMAX], teps = prm[P_TEPS];
    double T = 1.0;
    int nc = 0;
    st->rgb[0] = st->rgb[1] = st->rgb[2] = 0.0;
    st->last = 0;
    st->margin = INFINITY;
    st->sig = 1469598103934665603ull;
    if (F)
        for (int k = 0; k < D; ++k) F[k] = 0.0;
    for (int64_t k = 0; k < len; ++k) {
        const uint32_t g = list[k];
        const double *r = rec + (int64_t)ORC_REC * g;
        if (r[R_VALID] == 0.0) continue;
        double dx = px - r[R_MX], dy = py - r[R_MY];
        double q2 = r[R_A] * dx * dx + 2.0 * r[R_B] * dx * dy + r[R_C] * dy * dy;
        /* the cutoff decides membership only for a Gaussian that would pass
         * the alpha test right at the cutoff */
        double m = rel(q2, cut);
        double a_cut = r[R_OP] * exp(-0.5 * cut);
        if (a_cut > amax) a_cut = amax;
        if (a_cut >= amin * (1.0 - 1e-3) && m < st->margin) st->margin = m;
        if (q2 > cut) continue;
        double G = exp(-0.5 * q2);
        double rho = r[R_OP] * G;
        /* the alpha_max clamp is continuous in alpha: no margin */
        double alpha = rho > amax ? amax : rho;
        m = rel(alpha, amin);
        if (m < st->margin) st->margin = m;
        if (alpha < amin) continue;
        double Tn = T * (1.0 - alpha);
        m = rel(Tn, teps);
        if (m < st->margin) st->margin = m;
        if (Tn < teps) break;
        double w = alpha * T;
        st->rgb[0] += w * r[R_R];
        st->rgb[1] += w * r[R_G];
        st->rgb[2] += w * r[R_BL];
        if (F && D > 0) {
            const double *f = feat + (int64_t)D * g;
            for (int c = 0; c < D; ++c) F[c] += w * f[c];
        }
        if (ci && nc < cap) {
            ci[nc] = k;
            calpha[nc] = alpha;
            cT[nc] = T;
            cG[nc] = G;
        }
        st->sig = (st->sig ^ ((uint64_t)g * 2u + (rho > amax ? 1u : 0u))) * 1099511628211ull;
        ++nc;
        T = Tn;
        st->last = (int32_t)(k + 1);
    }
    st->T = T;
    return nc;
}


/* Tiled render of the pixels in [x0,x1) x [y0,y1) of one camera.
 * gids/ranges: the camera's depth-sorted per-tile lists (ranges[2*tile]).
 * Outputs are indexed by region pixel (row-major in the region). */
void orc_render(const double *rec, const double *feat, int D, const uint32_t *gids,
                const uint32_t *ranges, const double *cam, const double *prm, int x0, int y0,
                int x1, int y1, double *out_rgb, double *out_feat, double *out_T,
                int32_t *out_last, double *out_margin, int32_t *out_ncontrib)
{
    const int W = (int)cam[0], tsz = (int)prm[P_TILE];
    const int tiles_x = (W + tsz - 1) / tsz;
    const int rw = x1 - x0, rh = y1 - y0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t idx = 0; idx < (int64_t)rw * rh; ++idx) {
        int px = x0 + (int)(idx % rw), py = y0 + (int)(idx / rw);
        int tile = (py / tsz) * tiles_x + px / tsz;
        uint32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
        pix_state st;
        int nc = composite_pixel(px + 0.5, py + 0.5, gids + s, (int64_t)e - s, rec, feat, D, prm, &st,
                                 out_feat ? out_feat + (int64_t)D * idx : NULL, NULL, NULL, NULL, NULL, 0);
        for (int c = 0; c < 3; ++c) out_rgb[3 * idx + c] = st.rgb[c] + st.T * prm[P_BG0 + c];
        out_T[idx] = st.T;
        out_last[idx] = st.last;
        out_margin[idx] = st.margin;
        out_ncontrib[idx] = nc;
    }
}

/* Brute-force render: every pixel in the region composites ALL valid
 * Gaussians whose ellipse covers it, sorted by (depth_key, index) with no
 * tiles.  depth_key is supplied by the caller (FP32 depth bits or FP64
 * depth).  Also returns a per-pixel decision signature. */
typedef struct { double key; uint32_t g; } kd_pair;
static int kd_cmp(const void *a, const void *b)
{
    const kd_pair *x = (const kd_pair *)a, *y = (const kd_pair *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return x->g < y->g ? -1 : (x->g > y->g ? 1 : 0);
}

void orc_render_brute(int64_t n, const double *rec, const double *depth_key, const double *feat,
                      int D, const double *cam, const double *prm, int x0, int y0, int x1, int y1,
                      double *out_rgb, double *out_feat, double *out_T, double *out_margin,
                      uint64_t *out_sig)
{
    /* global depth order once, then per-pixel filtering keeps that order */
    kd_pair *order = (kd_pair *)malloc(sizeof(kd_pair) * (size_t)(n > 0 ? n : 1));
    int64_t m = 0;
    for (int64_t g = 0; g < n; ++g)
        if (rec[(int64_t)ORC_REC * g + R_VALID] != 0.0) {
            order[m].key = depth_key[g];
            order[m].g = (uint32_t)g;
            ++m;
        }
    qsort(order, (size_t)m, sizeof(kd_pair), kd_cmp);
    uint32_t *sorted = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t i = 0; i < m; ++i) sorted[i] = order[i].g;
    free(order);
    const int rw = x1 - x0, rh = y1 - y0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t idx = 0; idx < (int64_t)rw * rh; ++idx) {
        int px = x0 + (int)(idx % rw), py = y0 + (int)(idx / rw);
        pix_state st;
        composite_pixel(px + 0.5, py + 0.5, sorted, m, rec, feat, D, prm, &st,
                        out_feat ? out_feat + (int64_t)D * idx : NULL, NULL, NULL, NULL, NULL, 0);
        for (int c = 0; c < 3; ++c) out_rgb[3 * idx + c] = st.rgb[c] + st.T * prm[P_BG0 + c];
        out_T[idx] = st.T;
        out_margin[idx] = st.margin;
        out_sig[idx] = st.sig;
    }
    free(sorted);
}

/* ---------------------------------------------------- render backward -- */
/* dL/dalpha of one contributor at pixel centre (cx, cy) -> the footprint of
 * Gaussian g: alpha = min(alpha_max, op G), G = exp(-q2/2) with q2 = A dx^2 +
 * 2 B dx dy + C dy^2 and (dx, dy) = centre - mean.  The clamp passes no
 * gradient.  Accumulates (+=, atomically) into g_op, g_conic and g_mean2d. */
static void footprint_grad(const double *r, uint32_t g, double G, double dalpha, double cx, double cy,
                           double amax, double *g_mean2d, double *g_conic, double *g_op)
{
    const double rho = r[R_OP] * G;
    const double drho = rho > amax ? 0.0 : dalpha;
#pragma omp atomic
    g_op[g] += G * drho;
    const double dq2 = -0.5 * r[R_OP] * G * drho;
    const double dx = cx - r[R_MX], dy = cy - r[R_MY];
#pragma omp atomic
    g_conic[3 * g + 0] += dx * dx * dq2;
#pragma omp atomic
    g_conic[3 * g + 1] += 2.0 * dx * dy * dq2;
#pragma omp atomic
    g_conic[3 * g + 2] += dy * dy * dq2;
    const double ddx = (2.0 * r[R_A] * dx + 2.0 * r[R_B] * dy) * dq2;
    const double ddy = (2.0 * r[R_B] * dx + 2.0 * r[R_C] * dy) * dq2;
#pragma omp atomic
    g_mean2d[2 * g + 0] -= ddx;
#pragma omp atomic
    g_mean2d[2 * g + 1] -= ddy;
}

/* Gradient of L = sum_p dC_p . rgb_p + dF_p . feat_p over the region with
 * respect to each Gaussian's screen footprint and appearance.  Accumulates
 * (+=) into g_mean2d[n][2], g_conic[n][3] (A, B, C of q2 = A dx^2 +
 * 2 B dx dy + C dy^2), g_op[n], g_rgb[n][3] and, when non-NULL, g_feat[n][D].
 * The contributors are recovered by replaying the forward (exact T_i). */
#define ORC_MAXC 65536
void orc_render_bwd(const double *rec, const double *feat, int D, const uint32_t *gids,
                    const uint32_t *ranges, const double *cam, const double *prm, int x0, int y0,
                    int x1, int y1, const double *dC, const double *dF, double *g_mean2d,
                    double *g_conic, double *g_op, double *g_rgb, double *g_feat)
{
    const int W = (int)cam[0], tsz = (int)prm[P_TILE];
    const int tiles_x = (W + tsz - 1) / tsz;
    const int rw = x1 - x0, rh = y1 - y0;
    const double amax = prm[P_AMAX];
#pragma omp parallel
    {
        int64_t *ci = (int64_t *)malloc(sizeof(int64_t) * ORC_MAXC);
        double *ca = (double *)malloc(sizeof(double) * ORC_MAXC);
        double *cT = (double *)malloc(sizeof(double) * ORC_MAXC);
        double *cG = (double *)malloc(sizeof(double) * ORC_MAXC);
#pragma omp for schedule(dynamic, 16)
        for (int64_t idx = 0; idx < (int64_t)rw * rh; ++idx) {
            int px = x0 + (int)(idx % rw), py = y0 + (int)(idx / rw);
            int tile = (py / tsz) * tiles_x + px / tsz;
            uint32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
            const uint32_t *list = gids + s;
            pix_state st;
            int nc = composite_pixel(px + 0.5, py + 0.5, list, (int64_t)e - s, rec, feat, D, prm, &st,
                                     NULL, ci, ca, cT, cG, ORC_MAXC);
            if (nc > ORC_MAXC) nc = ORC_MAXC; /* never reached for the scenes used */
            const double *dc = dC + 3 * idx;
            const double *df = dF ? dF + (int64_t)D * idx : NULL;
            double S = st.T * (dc[0] * prm[P_BG0] + dc[1] * prm[P_BG1] + dc[2] * prm[P_BG2]);
            for (int j = nc - 1; j >= 0; --j) {
                const uint32_t g = list[ci[j]];
                const double *r = rec + (int64_t)ORC_REC * g;
                const double alpha = ca[j], T = cT[j], G = cG[j], w = alpha * T;
                double gw = dc[0] * r[R_R] + dc[1] * r[R_G] + dc[2] * r[R_BL];
                if (df) {
                    const double *f = feat + (int64_t)D * g;
                    for (int c = 0; c < D; ++c) gw += df[c] * f[c];
                }
                const double dalpha = T * gw - S / (1.0 - alpha);
                S += w * gw;
                for (int c = 0; c < 3; ++c) {
#pragma omp atomic
                    g_rgb[3 * g + c] += w * dc[c];
                }
                if (df && g_feat) {
                    double *gf = g_feat + (int64_t)D * g;
                    for (int c = 0; c < D; ++c) {
#pragma omp atomic
                        gf[c] += w * df[c];
                    }
                }
                footprint_grad(r, g, G, dalpha, px + 0.5, py + 0.5, amax, g_mean2d, g_conic, g_op);
            }
        }
        free(ci); free(ca); free(cT); free(cG);
    }
}

/* ------------------------------------------------ projection backward -- */
/* dL/dR (GR, 3x3) -> dL/dq (+=) through R = R(q / |q|): the derivative of
 * the rotation matrix of a unit quaternion, then the normalisation's
 * Jacobian (I - qn qn^T) / |q|. */
static void quat_grad(const double qn[4], double nq, double GR[3][3], double *gq)
{
    const double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    double gqn[4];
    gqn[0] = 2.0 * (-z * GR[0][1] + y * GR[0][2] + z * GR[1][0] - x * GR[1][2] - y * GR[2][0] + x * GR[2][1]);
    gqn[1] = 2.0 * (y * GR[0][1] + z * GR[0][2] + y * GR[1][0] - 2.0 * x * GR[1][1] - w * GR[1][2] +
                    z * GR[2][0] + w * GR[2][1] - 2.0 * x * GR[2][2]);
    gqn[2] = 2.0 * (-2.0 * y * GR[0][0] + x * GR[0][1] + w * GR[0][2] + x * GR[1][0] + z * GR[1][2] -
                    w * GR[2][0] + z * GR[2][1] - 2.0 * y * GR[2][2]);
    gqn[3] = 2.0 * (-2.0 * z * GR[0][0] - w * GR[0][1] + x * GR[0][2] + w * GR[1][0] - 2.0 * z * GR[1][1] +
                    y * GR[1][2] + x * GR[2][0] + y * GR[2][1]);
    double dot = qn[0] * gqn[0] + qn[1] * gqn[1] + qn[2] * gqn[2] + qn[3] * gqn[3];
    for (int k = 0; k < 4; ++k) gq[k] += (gqn[k] - qn[k] * dot) / nq;
}

/* Chain rule from (mean2d, conic, rgb) of one camera to the Gaussian
 * parameters; accumulates (+=) into g_means[n][3], g_scales[n][3],
 * g_quats[n][4], g_sh[n][K][3]. */
static void project_bwd_one(const double *mu, const double *s, const double *q, const double *sh,
                            int K, const double *cam, const double *prm, const double *rec,
                            const double *gm2, const double *gcon, const double *grgb,
                            double *gmu, double *gs, double *gq, double *gsh)
{
    if (rec[R_VALID] == 0.0) return;
    const double W = cam[0], H = cam[1], fx = cam[2], fy = cam[3];
    double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double qn[4] = {q[0] / nq, q[1] / nq, q[2] / nq, q[3] / nq};
    double R[3][3];
    quat_to_rot(qn, R);
    double M[3][3], S[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] = R[i][j] * s[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            S[i][j] = M[i][0] * M[j][0] + M[i][1] * M[j][1] + M[i][2] * M[j][2];
    double Rw[3][3], t[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) Rw[i][j] = cam_R(cam, i, j);
        t[i] = Rw[i][0] * mu[0] + Rw[i][1] * mu[1] + Rw[i][2] * mu[2] + cam_t(cam, i);
    }
    const double tz = t[2];
    double limx = prm[P_FOV] * (0.5 * W / fx), limy = prm[P_FOV] * (0.5 * H / fy);
    double ux = t[0] / tz, uy = t[1] / tz;
    int clx = (ux > limx) || (ux < -limx), cly = (uy > limy) || (uy < -limy);
    double xh = ux > limx ? limx : (ux < -limx ? -limx : ux);
    double yh = uy > limy ? limy : (uy < -limy ? -limy : uy);
    double J[2][3] = {{fx / tz, 0.0, -fx * xh / tz}, {0.0, fy / tz, -fy * yh / tz}};
    double Tm[2][3];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            Tm[i][j] = J[i][0] * Rw[0][j] + J[i][1] * Rw[1][j] + J[i][2] * Rw[2][j];

    /* conic = inverse of Sigma2; symmetric matrix gradient G_K */
    double Kc[2][2] = {{rec[R_A], rec[R_B]}, {rec[R_B], rec[R_C]}};
    double GK[2][2] = {{gcon[0], 0.5 * gcon[1]}, {0.5 * gcon[1], gcon[2]}};
    double tmp[2][2], G2[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) tmp[i][j] = Kc[i][0] * GK[0][j] + Kc[i][1] * GK[1][j];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) G2[i][j] = -(tmp[i][0] * Kc[0][j] + tmp[i][1] * Kc[1][j]);
    /* Sigma2 = Tm Sigma Tm^T + dil I */
    double GS[3][3], GT[2][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 2; ++k)
                for (int l = 0; l < 2; ++l) acc += Tm[k][i] * G2[k][l] * Tm[l][j];
            GS[i][j] = acc;
        }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 2; ++k)
                for (int l = 0; l < 3; ++l) acc += G2[i][k] * Tm[k][l] * S[l][j];
            GT[i][j] = 2.0 * acc;
        }
    /* Tm = J Rw */
    double GJ[2][3];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            GJ[i][j] = GT[i][0] * Rw[j][0] + GT[i][1] * Rw[j][1] + GT[i][2] * Rw[j][2];
    double gt[3] = {0.0, 0.0, 0.0};
    gt[2] += GJ[0][0] * (-fx / (tz * tz)) + GJ[1][1] * (-fy / (tz * tz));
    gt[2] += GJ[0][2] * (fx * xh / (tz * tz)) + GJ[1][2] * (fy * yh / (tz * tz));
    double gxh = GJ[0][2] * (-fx / tz), gyh = GJ[1][2] * (-fy / tz);
    if (!clx) { gt[0] += gxh / tz; gt[2] += gxh * (-t[0] / (tz * tz)); }
    if (!cly) { gt[1] += gyh / tz; gt[2] += gyh * (-t[1] / (tz * tz)); }
    /* mean2d */
    gt[0] += gm2[0] * fx / tz;
    gt[2] += gm2[0] * (-fx * t[0] / (tz * tz));
    gt[1] += gm2[1] * fy / tz;
    gt[2] += gm2[1] * (-fy * t[1] / (tz * tz));
    for (int j = 0; j < 3; ++j) gmu[j] += Rw[0][j] * gt[0] + Rw[1][j] * gt[1] + Rw[2][j] * gt[2];
    /* Sigma = M M^T, M = R diag(s) */
    double GM[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            GM[i][j] = 2.0 * (GS[i][0] * M[0][j] + GS[i][1] * M[1][j] + GS[i][2] * M[2][j]);
    double GR[3][3];
    for (int j = 0; j < 3; ++j) {
        double acc = 0.0;
        for (int i = 0; i < 3; ++i) { acc += GM[i][j] * R[i][j]; GR[i][j] = GM[i][j] * s[j]; }
        gs[j] += acc;
    }
    quat_grad(qn, nq, GR, gq);
    /* SH colour */
    double cpos[3], v[3];
    for (int i = 0; i < 3; ++i)
        cpos[i] = -(Rw[0][i] * cam_t(cam, 0) + Rw[1][i] * cam_t(cam, 1) + Rw[2][i] * cam_t(cam, 2));
    for (int i = 0; i < 3; ++i) v[i] = mu[i] - cpos[i];
    double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double d[3] = {v[0] / nv, v[1] / nv, v[2] / nv};
    double Y[16], dY[16][3];
    sh_basis(d, Y, dY);
    double graw[3];
    for (int c = 0; c < 3; ++c) graw[c] = rec[R_RAW_R + c] > 0.0 ? grgb[c] : 0.0;
    double gd[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < K; ++k) {
        double sk = 0.0;
        for (int c = 0; c < 3; ++c) {
            gsh[3 * k + c] += Y[k] * graw[c];
            sk += sh[3 * k + c] * graw[c];
        }
        for (int i = 0; i < 3; ++i) gd[i] += sk * dY[k][i];
    }
    double dd = d[0] * gd[0] + d[1] * gd[1] + d[2] * gd[2];
    for (int i = 0; i < 3; ++i) gmu[i] += (gd[i] - d[i] * dd) / nv;
}

void orc_project_bwd(int64_t n, const double *means, const double *scales, const double *quats,
                     const double *sh, int K, const double *cam, const double *prm, const double *rec,
                     const double *g_mean2d, const double *g_conic, const double *g_rgb,
                     double *g_means, double *g_scales, double *g_quats, double *g_sh)
{
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g)
        project_bwd_one(means + 3 * g, scales + 3 * g, quats + 4 * g, sh + (int64_t)3 * K * g, K, cam,
                        prm, rec + (int64_t)ORC_REC * g, g_mean2d + 2 * g, g_conic + 3 * g,
                        g_rgb + 3 * g, g_means + 3 * g, g_scales + 3 * g, g_quats + 4 * g,
                        g_sh + (int64_t)3 * K * g);
}

/* ------------------------------------------------------------ fusion -- */
/* Diagnostic for comparisons with a lower-precision renderer: adds to
 * wflip[g] a bound on how much weight Gaussian g could gain or lose at this
 * pixel if one of the pixel's threshold decisions lying within `mtol`
 * (relative) of its threshold came out the other way.  Walking the list as
 * composite_pixel does:
 *   - a position whose q^2-cutoff or alpha_min decision is near its
 *     threshold may gain or lose its own weight, at most a_thr T with a_thr
 *     the largest alpha inside the band (op e^(-cut (1 - mtol) / 2) clamped
 *     to alpha_max, or alpha_min (1 + mtol)); every later weight is then
 *     rescaled by (1 - alpha)^(+-1), i.e. moves by at most a_thr / (1 - a_thr)
 *     of itself;
 *   - a contributor whose stop decision (T (1 - alpha) vs t_eps) is near may
 *     be dropped, with every later contributor; the Gaussian that stopped
 *     the walk may be added with weight alpha T;
 *   - the alpha_max clamp is continuous and moves no weight. */
static void flip_bounds(double px, double py, const uint32_t *list, int64_t len, const double *rec,
                        const double *prm, double mtol, double *wflip)
{
    const double cut = prm[P_CUT], amin = prm[P_AMIN], amax = prm[P_AMAX], teps = prm[P_TEPS];
    double T = 1.0, ripple = 0.0;
    int dropping = 0;
    for (int64_t k = 0; k < len; ++k) {
        const uint32_t g = list[k];
        const double *r = rec + (int64_t)ORC_REC * g;
        if (r[R_VALID] == 0.0) continue;
        double dx = px - r[R_MX], dy = py - r[R_MY];
        double q2 = r[R_A] * dx * dx + 2.0 * r[R_B] * dx * dy + r[R_C] * dy * dy;
        double a_thr = 0.0;  /* largest alpha a decision within mtol of its threshold can have */
        if (rel(q2, cut) < mtol) {
            double a = r[R_OP] * exp(-0.5 * cut * (1.0 - mtol));
            a = a > amax ? amax : a;
            if (a >= amin * (1.0 - mtol)) a_thr = a;  /* else it never contributes */
        }
        double alpha = 0.0;
        if (q2 <= cut) {
            double rho = r[R_OP] * exp(-0.5 * q2);
            alpha = rho > amax ? amax : rho;
            if (rel(alpha, amin) < mtol && amin * (1.0 + mtol) > a_thr) a_thr = amin * (1.0 + mtol);
        }
        const int contributes = q2 <= cut && alpha >= amin;
        const double Tn = T * (1.0 - alpha);
        const int near_stop = contributes && rel(Tn, teps) < mtol;
        if (contributes && Tn < teps) {  /* the walk stops here */
            if (near_stop) wflip[g] += alpha * T;
            if (a_thr > 0.0) wflip[g] += a_thr * T;
            break;
        }
        const double w = contributes ? alpha * T : 0.0;
        wflip[g] += ripple * w + (dropping ? w : 0.0) + a_thr * T;
        if (near_stop) {
            wflip[g] += w;
            dropping = 1;
        }
        if (a_thr > 0.0) ripple += a_thr / (1.0 - a_thr);
        if (contributes) T = Tn;
    }
}

/* Accumulates, for one view, num[g][c] += w_g(p) F(p)[c] and
 * den[g] += w_g(p) over the region's pixels, with w the Eq. 4 weights of
 * the tiled forward.  fmap is indexed by region pixel (row-major), D wide.
 * wflip (may be NULL) accumulates, per Gaussian, the flip_bounds of the
 * pixels that have a decision within `mtol` of its threshold. */
void orc_fuse_view(const double *rec, const uint32_t *gids, const uint32_t *ranges,
                   const double *cam, const double *prm, int x0, int y0, int x1, int y1,
                   const double *fmap, int D, double *num, double *den, double *wflip, double mtol)
{
    const int W = (int)cam[0], tsz = (int)prm[P_TILE];
    const int tiles_x = (W + tsz - 1) / tsz;
    const int rw = x1 - x0, rh = y1 - y0;
#pragma omp parallel
    {
        int64_t *ci = (int64_t *)malloc(sizeof(int64_t) * ORC_MAXC);
        double *ca = (double *)malloc(sizeof(double) * ORC_MAXC);
        double *cT = (double *)malloc(sizeof(double) * ORC_MAXC);
        double *cG = (double *)malloc(sizeof(double) * ORC_MAXC);
#pragma omp for schedule(dynamic, 16)
        for (int64_t idx = 0; idx < (int64_t)rw * rh; ++idx) {
            int px = x0 + (int)(idx % rw), py = y0 + (int)(idx / rw);
            int tile = (py / tsz) * tiles_x + px / tsz;
            uint32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
            const uint32_t *list = gids + s;
            pix_state st;
            int nc = composite_pixel(px + 0.5, py + 0.5, list, (int64_t)e - s, rec, NULL, 0, prm, &st,
                                     NULL, ci, ca, cT, cG, ORC_MAXC);
            if (nc > ORC_MAXC) nc = ORC_MAXC;
            if (wflip && st.margin < mtol) {
#pragma omp critical(orc_wflip)
                flip_bounds(px + 0.5, py + 0.5, list, (int64_t)e - s, rec, prm, mtol, wflip);
            }
            const double *f = fmap + (int64_t)D * idx;
            for (int j = 0; j < nc; ++j) {
                const uint32_t g = list[ci[j]];
                const double w = ca[j] * cT[j];
#pragma omp atomic
                den[g] += w;
                for (int c = 0; c < D; ++c) {
#pragma omp atomic
                    num[(int64_t)D * g + c] += w * f[c];
                }
            }
        }
        free(ci); free(ca); free(cT); free(cG);
    }
}

/* f_g = num_g / den_g where den_g > 0, else 0 (and flag[g] = 1). */
void orc_fuse_finalize(int64_t n, int D, const double *num, const double *den, double *out,
                       int32_t *flag)
{
    for (int64_t g = 0; g < n; ++g) {
        if (den[g] > 0.0) {
            for (int c = 0; c < D; ++c) out[(int64_t)D * g + c] = num[(int64_t)D * g + c] / den[g];
            flag[g] = 0;
        } else {
            for (int c = 0; c < D; ++c) out[(int64_t)D * g + c] = 0.0;
            flag[g] = 1;
        }
    }
}

/* ------------------------------------------------------------- NDFD ---- */
/* Non-differentiable feature driving (Sec. 3.2, App. A "NDFD"): per pixel,
 * over the same tile list, weights w_i = alpha_i T_i and contributor set as
 * the render (nearest first, i = 1), with the ground-truth feature f_gt(p)
 * of that pixel:
 *   sigma_i = 1 / (1 + exp(k (phi_i - lambda))),  phi_i = cos<f_i, f_gt>
 *             (Sec. 3.3; phi_i = 0 when either vector is zero);
 *   L_gt    = sum_i w_i sigma_i                                      (Eq. 5);
 *   L_cf    = sum_i sigma_i w_i (W_{i-1} - F_{i-1} . f_i),
 *             W_n = sum_{j<=n} w_j,  F_n = sum_{j<=n} w_j f_j   (Eq. 6, App. A.1).
 * Features f_i enter L_cf through the plain dot product f_i . f_j (the paper
 * takes them unit length, where it equals the cosine). */
static double ndfd_sigma(const double *f, const double *fgt, int D, double kslope, double lam)
{
    double dot = 0.0, nf = 0.0, ng = 0.0;
    for (int c = 0; c < D; ++c) {
        dot += f[c] * fgt[c];
        nf += f[c] * f[c];
        ng += fgt[c] * fgt[c];
    }
    const double phi = (nf > 0.0 && ng > 0.0) ? dot / (sqrt(nf) * sqrt(ng)) : 0.0;
    return 1.0 / (1.0 + exp(kslope * (phi - lam)));
}

static double dotd(const double *a, const double *b, int D)
{
    double s = 0.0;
    for (int c = 0; c < D; ++c) s += a[c] * b[c];
    return s;
}

/* L_gt, L_cf and W_N of one pixel from its contributors in order (ids,
 * weights w_i), its ground-truth feature fg and the D-wide scratch F. */
static void ndfd_losses(const uint32_t *ids, const double *ws, int nc, const double *feat, int D, const double *fg,
                        double kslope, double lam, double *F, double *out_Lgt, double *out_Lcf, double *out_W)
{
    double Wc = 0.0, Lgt = 0.0, Lcf = 0.0;
    for (int c = 0; c < D; ++c) F[c] = 0.0;
    for (int j = 0; j < nc; ++j) {
        const double *f = feat + (int64_t)D * ids[j];
        const double w = ws[j];
        const double sg = ndfd_sigma(f, fg, D, kslope, lam);
        Lgt += w * sg;
        Lcf += sg * w * (Wc - dotd(F, f, D));
        Wc += w;
        for (int c = 0; c < D; ++c) F[c] += w * f[c];
    }
    *out_Lgt = Lgt;
    *out_Lcf = Lcf;
    *out_W = Wc;
}

/* fgt: region pixels x D (row-major in the region).  Outputs per region
 * pixel: L_gt, L_cf, W_N (total weight) and the contributor count. */
void orc_ndfd(const double *rec, const double *feat, int D, const uint32_t *gids, const uint32_t *ranges,
              const double *cam, const double *prm, int x0, int y0, int x1, int y1, const double *fgt,
              double kslope, double lam, double *out_Lgt, double *out_Lcf, double *out_W,
              int32_t *out_ncontrib)
{
    const int W = (int)cam[0], tsz = (int)prm[P_TILE];
    const int tiles_x = (W + tsz - 1) / tsz;
    const int rw = x1 - x0, rh = y1 - y0;
#pragma omp parallel
    {
        int64_t *ci = (int64_t *)malloc(sizeof(int64_t) * ORC_MAXC);
        double *ca = (double *)malloc(sizeof(double) * ORC_MAXC);
        double *cT = (double *)malloc(sizeof(double) * ORC_MAXC);
        double *cG = (double *)malloc(sizeof(double) * ORC_MAXC);
        uint32_t *ids = (uint32_t *)malloc(sizeof(uint32_t) * ORC_MAXC);
        double *ws = (double *)malloc(sizeof(double) * ORC_MAXC);
        double *F = (double *)malloc(sizeof(double) * (size_t)(D > 0 ? D : 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t idx = 0; idx < (int64_t)rw * rh; ++idx) {
            int px = x0 + (int)(idx % rw), py = y0 + (int)(idx / rw);
            int tile = (py / tsz) * tiles_x + px / tsz;
            uint32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
            const uint32_t *list = gids + s;
            pix_state st;
            int nc = composite_pixel(px + 0.5, py + 0.5, list, (int64_t)e - s, rec, NULL, 0, prm, &st,
                                     NULL, ci, ca, cT, cG, ORC_MAXC);
            if (nc > ORC_MAXC) nc = ORC_MAXC;
            for (int j = 0; j < nc; ++j) {
                ids[j] = list[ci[j]];
                ws[j] = ca[j] * cT[j];
            }
            double Lgt, Lcf, Wc;
            ndfd_losses(ids, ws, nc, feat, D, fgt + (int64_t)D * idx, kslope, lam, F, &Lgt, &Lcf, &Wc);
            out_Lgt[idx] = Lgt;
            out_Lcf[idx] = Lcf;
            if (out_W) out_W[idx] = Wc;
            if (out_ncontrib) out_ncontrib[idx] = nc;
        }
        free(ci); free(ca); free(cT); free(cG); free(ids); free(ws); free(F);
    }
}

/* Gradient of L = sum_p dLgt[p] L_gt(p) + dLcf[p] L_cf(p) over the region
 * with respect to each Gaussian's screen footprint (mean2d, conic) and
 * opacity; accumulates (+=) into g_mean2d[n][2], g_conic[n][3], g_op[n].
 * Features and f_gt are constants (non-differentiable).  Per contributor k:
 *   dL/dw_k = dLgt sigma_k + dLcf (sigma_k (W_{k-1} - F_{k-1} . f_k)
 *             + sum_{i>k} sigma_i w_i (1 - f_i . f_k))          (Sec. 3.3),
 * then dL/dalpha_k = T_k dL/dw_k - (1/(1 - alpha_k)) sum_{i>k} w_i dL/dw_i
 * (App. A.2), and the footprint chain of the render backward.  The suffix
 * sum over i > k is carried back to front as sum sigma_i w_i and
 * sum sigma_i w_i f_i. */
void orc_ndfd_bwd(const double *rec, const double *feat, int D, const uint32_t *gids, const uint32_t *ranges,
                  const double *cam, const double *prm, int x0, int y0, int x1, int y1, const double *fgt,
                  double kslope, double lam, const double *dLgt, const double *dLcf, double *g_mean2d,
                  double *g_conic, double *g_op)
{
    const int W = (int)cam[0], tsz = (int)prm[P_TILE];
    const int tiles_x = (W + tsz - 1) / tsz;
    const int rw = x1 - x0, rh = y1 - y0;
    const double amax = prm[P_AMAX];
#pragma omp parallel
    {
        int64_t *ci = (int64_t *)malloc(sizeof(int64_t) * ORC_MAXC);
        double *ca = (double *)malloc(sizeof(double) * ORC_MAXC);
        double *cT = (double *)malloc(sizeof(double) * ORC_MAXC);
        double *cG = (double *)malloc(sizeof(double) * ORC_MAXC);
        double *sig = (double *)malloc(sizeof(double) * ORC_MAXC);
        double *pre = (double *)malloc(sizeof(double) * ORC_MAXC);
        double *F = (double *)malloc(sizeof(double) * (size_t)(D > 0 ? D : 1));
        double *Gs = (double *)malloc(sizeof(double) * (size_t)(D > 0 ? D : 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t idx = 0; idx < (int64_t)rw * rh; ++idx) {
            int px = x0 + (int)(idx % rw), py = y0 + (int)(idx / rw);
            int tile = (py / tsz) * tiles_x + px / tsz;
            uint32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
            const uint32_t *list = gids + s;
            pix_state st;
            int nc = composite_pixel(px + 0.5, py + 0.5, list, (int64_t)e - s, rec, NULL, 0, prm, &st,
                                     NULL, ci, ca, cT, cG, ORC_MAXC);
            if (nc > ORC_MAXC) nc = ORC_MAXC;
            const double *fg = fgt + (int64_t)D * idx;
            const double cgt = dLgt[idx], ccf = dLcf[idx];
            /* front to back: sigma_k and W_{k-1} - F_{k-1} . f_k */
            double Wc = 0.0;
            for (int c = 0; c < D; ++c) F[c] = 0.0;
            for (int j = 0; j < nc; ++j) {
                const double *f = feat + (int64_t)D * list[ci[j]];
                const double w = ca[j] * cT[j];
                sig[j] = ndfd_sigma(f, fg, D, kslope, lam);
                pre[j] = Wc - dotd(F, f, D);
                Wc += w;
                for (int c = 0; c < D; ++c) F[c] += w * f[c];
            }
            /* back to front */
            double Ss = 0.0, Sw = 0.0;
            for (int c = 0; c < D; ++c) Gs[c] = 0.0;
            for (int k = nc - 1; k >= 0; --k) {
                const uint32_t g = list[ci[k]];
                const double *f = feat + (int64_t)D * g;
                const double alpha = ca[k], T = cT[k], w = alpha * T;
                const double gw = cgt * sig[k] + ccf * (sig[k] * pre[k] + Ss - dotd(Gs, f, D));
                const double dalpha = T * gw - Sw / (1.0 - alpha);
                Sw += w * gw;
                Ss += sig[k] * w;
                for (int c = 0; c < D; ++c) Gs[c] += sig[k] * w * f[c];
                footprint_grad(rec + (int64_t)ORC_REC * g, g, cG[k], dalpha, px + 0.5, py + 0.5, amax,
                               g_mean2d, g_conic, g_op);
            }
        }
        free(ci); free(ca); free(cT); free(cG); free(sig); free(pre); free(F); free(Gs);
    }
}

/* The contributors of the pixel with centre (cx, cy) over one depth-sorted
 * list, exactly as the render composites them: their positions in the list,
 * alpha_i and T_i.  Returns the count (at most cap are written). */
int orc_contributors(const double *rec, const uint32_t *list, int64_t len, const double *prm, double cx,
                     double cy, int cap, int64_t *pos, double *alpha, double *T)
{
    double *G = (double *)malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
    pix_state st;
    int nc = composite_pixel(cx, cy, list, len, rec, NULL, 0, prm, &st, NULL, pos, alpha, T, G, cap);
    free(G);
    return nc;
}

/* ------------------------------------------------- PointsFeatureFusion -- */
/* The paper's point-to-feature assignment (Sec. 3.1; App. A,
 * "PointsFeatureFusion"): a point takes the feature of the pixel it projects
 * to in one view, drawn at random among the views that see it.  Readings:
 * a view sees the point when its camera depth exceeds znear and the
 * projection (x, y) lies in [0, W) x [0, H); the pixel is (floor x, floor y)
 * (the nearest pixel centre, centres at +0.5); the draw is the k-th visible
 * view in view order with k = floor(u |M|) for a given uniform u in [0, 1)
 * (clamped to |M| - 1).  The projection decides an integer, so it is
 * specified in binary32, one rounding per operation in the written order
 * (this file is compiled with -ffp-contract=off):
 *   c = ((R_r0 X + R_r1 Y) + R_r2 Z) + t_r  for each row r,
 *   x = fx (c_x / c_z) + cx,  y = fy (c_y / c_z) + cy.
 * cams: n_views x 18 floats (width, height, fx, fy, cx, cy, [R|t] row by
 * row).  Outputs per point: the view (-1 if none sees it), the pixel index
 * y W + x in that view, and the number of views that see it. */
void orc_point_views_f32(int64_t n, const float *means, int n_views, const float *cams, float znear, const float *u,
                         int32_t *out_view, int32_t *out_pixel, int32_t *out_count)
{
    for (int64_t i = 0; i < n; ++i) {
        const float X = means[3 * i], Y = means[3 * i + 1], Z = means[3 * i + 2];
        int count = 0;
        int vis_pix[1024];
        int vis_view[1024];
        for (int v = 0; v < n_views && v < 1024; ++v) {
            const float *c = cams + 18 * v;
            const float *R = c + 6;
            const float cx_ = ((R[0] * X + R[1] * Y) + R[2] * Z) + R[3];
            const float cy_ = ((R[4] * X + R[5] * Y) + R[6] * Z) + R[7];
            const float cz_ = ((R[8] * X + R[9] * Y) + R[10] * Z) + R[11];
            if (!(cz_ > znear)) continue;
            const float qx = cx_ / cz_, qy = cy_ / cz_;
            const float x = c[2] * qx + c[4];
            const float y = c[3] * qy + c[5];
            if (!(x >= 0.0f && x < c[0] && y >= 0.0f && y < c[1])) continue;
            vis_view[count] = v;
            vis_pix[count] = (int)floorf(y) * (int)c[0] + (int)floorf(x);
            ++count;
        }
        out_count[i] = count;
        if (count == 0) {
            out_view[i] = -1;
            out_pixel[i] = -1;
            continue;
        }
        int k = (int)(u[i] * (float)count);
        if (k > count - 1) k = count - 1;
        if (k < 0) k = 0;
        out_view[i] = vis_view[k];
        out_pixel[i] = vis_pix[k];
    }
}

/* ------------------------------------------------------- 2DGS surfels -- */
/* The surfel model of Sec. 3.1 (Eq. 1-3): a primitive is the tangent plane
 * P(u, v) = p + s_u t_u u + s_v t_v v, with t_u, t_v the first two columns of
 * R (the normalised quaternion) and density G(u) = exp(-(u^2 + v^2)/2).  A
 * pixel's value is taken at u(x), the point of the plane that projects to
 * the pixel: the intersection of the pixel's camera ray with the plane,
 *   lambda d = c + u a + v b,   d = ((x - cx)/fx, (y - cy)/fy, 1),
 *   c = R_w p + t_w,  a = R_w (s_u t_u),  b = R_w (s_v t_v),
 * solved by Cramer's rule (lambda is the camera depth of the intersection).
 * A ray parallel to the plane (|det| <= 1e-12 |d| |a| |b|) misses it.
 * Returns 1 and (u, v, lambda) on a hit. */
static int splat_uv(const double *mu, const double *q, const double *s2, const double *cam, double px,
                    double py, double *u, double *v, double *lam)
{
    const double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const double qn[4] = {q[0] / nq, q[1] / nq, q[2] / nq, q[3] / nq};
    double R[3][3];
    quat_to_rot(qn, R);
    double c[3], a[3], b[3];
    for (int r = 0; r < 3; ++r) {
        c[r] = cam_t(cam, r);
        a[r] = 0.0;
        b[r] = 0.0;
        for (int k = 0; k < 3; ++k) {
            c[r] += cam_R(cam, r, k) * mu[k];
            a[r] += cam_R(cam, r, k) * R[k][0] * s2[0];
            b[r] += cam_R(cam, r, k) * R[k][1] * s2[1];
        }
    }
    const double d[3] = {(px - cam[4]) / cam[2], (py - cam[5]) / cam[3], 1.0};
    /* columns of M: d, -a, -b */
    const double m00 = d[0], m01 = -a[0], m02 = -b[0];
    const double m10 = d[1], m11 = -a[1], m12 = -b[1];
    const double m20 = d[2], m21 = -a[2], m22 = -b[2];
    const double det = m00 * (m11 * m22 - m12 * m21) - m01 * (m10 * m22 - m12 * m20) + m02 * (m10 * m21 - m11 * m20);
    const double nd = sqrt(d[0] * d[0] + d[1] * d[1] + 1.0);
    const double na = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    const double nb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    if (!(fabs(det) > 1e-12 * nd * na * nb)) return 0;
    /* Cramer: replace one column by c */
    const double dl = c[0] * (m11 * m22 - m12 * m21) - m01 * (c[1] * m22 - m12 * c[2]) + m02 * (c[1] * m21 - m11 * c[2]);
    const double du = m00 * (c[1] * m22 - m12 * c[2]) - c[0] * (m10 * m22 - m12 * m20) + m02 * (m10 * c[2] - c[1] * m20);
    const double dv = m00 * (m11 * c[2] - c[1] * m21) - m01 * (m10 * c[2] - c[1] * m20) + c[0] * (m10 * m21 - m11 * m20);
    *lam = dl / det;
    *u = du / det;
    *v = dv / det;
    return 1;
}

/* (u, v, lambda, hit) of every (pixel centre, surfel) pair given. */
void orc_splat_uv(int64_t m, const double *mu, const double *q, const double *s2, const double *cam, const double *px,
                  const double *py, double *u, double *v, double *lam, int32_t *hit)
{
    for (int64_t i = 0; i < m; ++i)
        hit[i] = splat_uv(mu + 3 * i, q + 4 * i, s2 + 2 * i, cam, px[i], py[i], u + i, v + i, lam + i);
}

/* Brute-force surfel render of the region: every pixel composites all
 * surfels whose centre lies beyond znear, in order of (depth_key, index),
 * front to back with the rules of the render (Eq. 4): alpha = min(alpha_max,
 * op G(u(x))) for u^2 + v^2 <= cutoff_sq and an intersection in front of the
 * camera (lambda > 0), skip alpha < alpha_min, stop before T (1 - alpha) <
 * t_eps; background added to RGB.  rgb: the surfels' colours [n][3]. */
void orc_render_2dgs_brute(int64_t n, const double *means, const double *quats, const double *scales2,
                           const double *opac, const double *rgb, const double *depth_key, const double *cam,
                           const double *prm, int x0, int y0, int x1, int y1, double *out_rgb, double *out_T,
                           int32_t *out_ncontrib)
{
    kd_pair *order = (kd_pair *)malloc(sizeof(kd_pair) * (size_t)(n > 0 ? n : 1));
    int64_t m = 0;
    for (int64_t g = 0; g < n; ++g) {
        double cz = cam_t(cam, 2);
        for (int k = 0; k < 3; ++k) cz += cam_R(cam, 2, k) * means[3 * g + k];
        if (cz > prm[P_ZNEAR]) {
            order[m].key = depth_key[g];
            order[m].g = (uint32_t)g;
            ++m;
        }
    }
    qsort(order, (size_t)m, sizeof(kd_pair), kd_cmp);
    const int rw = x1 - x0, rh = y1 - y0;
    const double cut = prm[P_CUT], amin = prm[P_AMIN], amax = prm[P_AMAX], teps = prm[P_TEPS];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t idx = 0; idx < (int64_t)rw * rh; ++idx) {
        const double px = x0 + (int)(idx % rw) + 0.5, py = y0 + (int)(idx / rw) + 0.5;
        double T = 1.0, acc[3] = {0.0, 0.0, 0.0};
        int nc = 0;
        for (int64_t k = 0; k < m; ++k) {
            const uint32_t g = order[k].g;
            double u, v, lam;
            if (!splat_uv(means + 3 * g, quats + 4 * g, scales2 + 2 * g, cam, px, py, &u, &v, &lam)) continue;
            if (!(lam > 0.0)) continue;
            const double r2 = u * u + v * v;
            if (r2 > cut) continue;
            const double rho = opac[g] * exp(-0.5 * r2);
            const double alpha = rho > amax ? amax : rho;
            if (alpha < amin) continue;
            const double Tn = T * (1.0 - alpha);
            if (Tn < teps) break;
            const double w = alpha * T;
            for (int ch = 0; ch < 3; ++ch) acc[ch] += w * rgb[3 * g + ch];
            T = Tn;
            ++nc;
        }
        for (int ch = 0; ch < 3; ++ch) out_rgb[3 * idx + ch] = acc[ch] + T * prm[P_BG0 + ch];
        out_T[idx] = T;
        out_ncontrib[idx] = nc;
    }
    free(order);
}

/* Screen rectangle of a surfel's footprint u^2 + v^2 <= cut (the region the
 * render can touch): the image of that ellipse of the plane is a conic, and
 * its axis-aligned bounding box follows from the dual conic
 *   C* = T diag(1, 1, -1/cut) T^T,  T = [K a, K b, K c]  (3x3, columns),
 * whose vertical tangents x = x0 solve C*00 - 2 x0 C*02 + x0^2 C*22 = 0 (and
 * likewise for y with row 1).  The ellipse must lie wholly in front of the
 * camera (its least depth c_z - sqrt(cut ((a_z)^2 + (b_z)^2)) > 0, with a, b
 * the camera-space tangent vectors scaled by s_u, s_v); otherwise its image
 * is unbounded and the rectangle is the whole image.  Output per surfel:
 * rect = (xmin, xmax, ymin, ymax) in pixel coordinates and the flag
 * bounded (1) / whole image (0). */
void orc_surfel_rect(int64_t n, const double *means, const double *quats, const double *scales2, const double *cam,
                     double cut, double *rect, int32_t *bounded)
{
    const double W = cam[0], H = cam[1], fx = cam[2], fy = cam[3], cx = cam[4], cy = cam[5];
    for (int64_t g = 0; g < n; ++g) {
        const double *q = quats + 4 * g;
        const double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        const double qn[4] = {q[0] / nq, q[1] / nq, q[2] / nq, q[3] / nq};
        double R[3][3];
        quat_to_rot(qn, R);
        double c[3], a[3], b[3];
        for (int r = 0; r < 3; ++r) {
            c[r] = cam_t(cam, r);
            a[r] = 0.0;
            b[r] = 0.0;
            for (int k = 0; k < 3; ++k) {
                c[r] += cam_R(cam, r, k) * means[3 * g + k];
                a[r] += cam_R(cam, r, k) * R[k][0] * scales2[2 * g];
                b[r] += cam_R(cam, r, k) * R[k][1] * scales2[2 * g + 1];
            }
        }
        double *out = rect + 4 * g;
        const double zmin = c[2] - sqrt(cut * (a[2] * a[2] + b[2] * b[2]));
        if (!(zmin > 0.0)) {
            out[0] = 0.0; out[1] = W; out[2] = 0.0; out[3] = H;
            bounded[g] = 0;
            continue;
        }
        /* T = K [a b c]: rows (fx a_x + cx a_z, ...), (fy a_y + cy a_z, ...), (a_z, b_z, c_z) */
        double T[3][3];
        const double *col[3] = {a, b, c};
        for (int j = 0; j < 3; ++j) {
            T[0][j] = fx * col[j][0] + cx * col[j][2];
            T[1][j] = fy * col[j][1] + cy * col[j][2];
            T[2][j] = col[j][2];
        }
        const double dq[3] = {1.0, 1.0, -1.0 / cut};
        double Cs[3][3];
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) {
                double acc = 0.0;
                for (int j = 0; j < 3; ++j) acc += T[r][j] * dq[j] * T[s][j];
                Cs[r][s] = acc;
            }
        const double dx = sqrt(fmax(0.0, Cs[0][2] * Cs[0][2] - Cs[0][0] * Cs[2][2]));
        const double dy = sqrt(fmax(0.0, Cs[1][2] * Cs[1][2] - Cs[1][1] * Cs[2][2]));
        const double x1 = (Cs[0][2] - dx) / Cs[2][2], x2 = (Cs[0][2] + dx) / Cs[2][2];
        const double y1 = (Cs[1][2] - dy) / Cs[2][2], y2 = (Cs[1][2] + dy) / Cs[2][2];
        out[0] = fmin(x1, x2); out[1] = fmax(x1, x2);
        out[2] = fmin(y1, y2); out[3] = fmax(y1, y2);
        bounded[g] = 1;
    }
}

/* dL/dalpha of contributor g at pixel centre (px, py), where the surfel
 * sits at plane coordinates (u, v) with G = exp(-(u^2 + v^2)/2), taken to
 * the surfel's opacity, mean, quaternion and (s_u, s_v); accumulates (+=).
 * alpha = min(alpha_max, op G) (the clamp passes nothing), dG/du = -u G,
 * dG/dv = -v G, and the ray-plane solve differentiated implicitly:
 * w = M^-T (0, dL/du, dL/dv), dL/dp = R_w^T w, dL/dR[:,0] = s_u u R_w^T w,
 * dL/dR[:,1] = s_v v R_w^T w, dL/ds_u = u w . (R_w R[:,0]),
 * dL/ds_v = v w . (R_w R[:,1]). */
static void surfel_alpha_chain(uint32_t g, double G, double u, double v, double dalpha, double px, double py,
                               const double *quats, const double *scales2, const double *opac, const double *cam,
                               double amax, double *g_means, double *g_quats, double *g_scales2, double *g_opac)
{
    const double rho = opac[g] * G;
    const double drho = rho > amax ? 0.0 : dalpha;
#pragma omp atomic
    g_opac[g] += G * drho;
    const double dG = opac[g] * drho;
    const double e[3] = {0.0, -u * G * dG, -v * G * dG};
    /* the surfel's frame in the camera */
    const double *q = quats + 4 * g;
    const double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const double qn[4] = {q[0] / nq, q[1] / nq, q[2] / nq, q[3] / nq};
    double R[3][3];
    quat_to_rot(qn, R);
    const double su = scales2[2 * g], sv = scales2[2 * g + 1];
    double ru[3], rv[3];   /* R_w R[:,0], R_w R[:,1] */
    for (int r = 0; r < 3; ++r) {
        ru[r] = 0.0;
        rv[r] = 0.0;
        for (int k = 0; k < 3; ++k) {
            ru[r] += cam_R(cam, r, k) * R[k][0];
            rv[r] += cam_R(cam, r, k) * R[k][1];
        }
    }
    const double d[3] = {(px - cam[4]) / cam[2], (py - cam[5]) / cam[3], 1.0};
    double M[3][3];
    for (int r = 0; r < 3; ++r) {
        M[r][0] = d[r];
        M[r][1] = -su * ru[r];
        M[r][2] = -sv * rv[r];
    }
    /* w3 = M^-T e: solve M^T w3 = e by Cramer's rule on A = M^T */
    double A[3][3];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) A[r][k] = M[k][r];
    const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                       A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                       A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    double w3[3];
    for (int col = 0; col < 3; ++col) {
        double B[3][3];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) B[r][k] = k == col ? e[r] : A[r][k];
        w3[col] = (B[0][0] * (B[1][1] * B[2][2] - B[1][2] * B[2][1]) -
                   B[0][1] * (B[1][0] * B[2][2] - B[1][2] * B[2][0]) +
                   B[0][2] * (B[1][0] * B[2][1] - B[1][1] * B[2][0])) / det;
    }
    double rt[3];   /* R_w^T w3 */
    for (int k = 0; k < 3; ++k) rt[k] = cam_R(cam, 0, k) * w3[0] + cam_R(cam, 1, k) * w3[1] + cam_R(cam, 2, k) * w3[2];
    for (int k = 0; k < 3; ++k) {
#pragma omp atomic
        g_means[3 * g + k] += rt[k];
    }
    const double gsu = u * (w3[0] * ru[0] + w3[1] * ru[1] + w3[2] * ru[2]);
    const double gsv = v * (w3[0] * rv[0] + w3[1] * rv[1] + w3[2] * rv[2]);
#pragma omp atomic
    g_scales2[2 * g] += gsu;
#pragma omp atomic
    g_scales2[2 * g + 1] += gsv;
    double GR[3][3];
    for (int k = 0; k < 3; ++k) {
        GR[k][0] = su * u * rt[k];
        GR[k][1] = sv * v * rt[k];
        GR[k][2] = 0.0;
    }
    double gq[4] = {0.0, 0.0, 0.0, 0.0};
    quat_grad(qn, nq, GR, gq);
    for (int k = 0; k < 4; ++k) {
#pragma omp atomic
        g_quats[4 * g + k] += gq[k];
    }
}

/* Gradient of L = sum_p dC[p] . rgb[p] of the surfel render with respect to
 * each surfel's mean, quaternion, (s_u, s_v), opacity and colour;
 * accumulates (+=).  dL/dalpha by the App. A.2 identity with the background
 * term, as in orc_render_bwd; then alpha = op G(u, v) (the clamp passes
 * nothing), dG/du = -u G, dG/dv = -v G, and (lambda, u, v) = M^-1 c with
 * M = [d, -a, -b] differentiated implicitly: d(lambda, u, v) =
 * M^-1 (dc + u da + v db), so with w = M^-T (0, dL/du, dL/dv):
 * dL/dp = R_w^T w, dL/dR[:,0] = s_u u R_w^T w, dL/dR[:,1] = s_v v R_w^T w,
 * dL/ds_u = u w . (R_w R[:,0]), dL/ds_v = v w . (R_w R[:,1]).
 * One pixel (centre px, py) over one depth-ordered list; cg, ca: scratch of
 * len and 5 len entries. */
static void surfel_pixel_bwd(double px, double py, const uint32_t *list, int64_t len, const double *means,
                             const double *quats, const double *scales2, const double *opac, const double *rgb,
                             const double *feat, int D, const double *dF, const double *cam, const double *prm,
                             const double *dc, uint32_t *cg, double *ca, double *g_means, double *g_quats,
                             double *g_scales2, double *g_opac, double *g_rgb, double *g_feat)
{
    const double cut = prm[P_CUT], amin = prm[P_AMIN], amax = prm[P_AMAX], teps = prm[P_TEPS];
    double T = 1.0;
    int nc = 0;
    for (int64_t k = 0; k < len; ++k) {
        const uint32_t g = list[k];
        double u, v, lam;
        if (!splat_uv(means + 3 * g, quats + 4 * g, scales2 + 2 * g, cam, px, py, &u, &v, &lam)) continue;
        if (!(lam > 0.0)) continue;
        const double r2 = u * u + v * v;
        if (r2 > cut) continue;
        const double G = exp(-0.5 * r2);
        const double rho = opac[g] * G;
        const double alpha = rho > amax ? amax : rho;
        if (alpha < amin) continue;
        const double Tn = T * (1.0 - alpha);
        if (Tn < teps) break;
        cg[nc] = g;
        ca[5 * nc + 0] = alpha;
        ca[5 * nc + 1] = T;
        ca[5 * nc + 2] = G;
        ca[5 * nc + 3] = u;
        ca[5 * nc + 4] = v;
        ++nc;
        T = Tn;
    }
    double S = T * (dc[0] * prm[P_BG0] + dc[1] * prm[P_BG1] + dc[2] * prm[P_BG2]);
    for (int j = nc - 1; j >= 0; --j) {
        const uint32_t g = cg[j];
        const double alpha = ca[5 * j], Tj = ca[5 * j + 1], G = ca[5 * j + 2], u = ca[5 * j + 3], v = ca[5 * j + 4];
        const double w = alpha * Tj;
        double gw = dc[0] * rgb[3 * g] + dc[1] * rgb[3 * g + 1] + dc[2] * rgb[3 * g + 2];
        if (feat && dF)  /* the feature term of dL/dw: dF . f_g */
            for (int k = 0; k < D; ++k) gw += dF[k] * feat[(int64_t)D * g + k];
        const double dalpha = Tj * gw - S / (1.0 - alpha);
        S += w * gw;
        for (int ch = 0; ch < 3; ++ch) {
#pragma omp atomic
            g_rgb[3 * g + ch] += w * dc[ch];
        }
        if (g_feat && dF)
            for (int k = 0; k < D; ++k) {
#pragma omp atomic
                g_feat[(int64_t)D * g + k] += w * dF[k];
            }
        surfel_alpha_chain(g, G, u, v, dalpha, px, py, quats, scales2, opac, cam, amax, g_means, g_quats, g_scales2,
                           g_opac);
    }
}

/* The backward of orc_render_2dgs_brute (every surfel with its centre
 * beyond znear, ordered by (depth_key, index), for every pixel). */
void orc_render_2dgs_bwd_brute(int64_t n, const double *means, const double *quats, const double *scales2,
                               const double *opac, const double *rgb, const double *depth_key, const double *cam,
                               const double *prm, int x0, int y0, int x1, int y1, const double *dC, double *g_means,
                               double *g_quats, double *g_scales2, double *g_opac, double *g_rgb)
{
    kd_pair *order = (kd_pair *)malloc(sizeof(kd_pair) * (size_t)(n > 0 ? n : 1));
    int64_t m = 0;
    for (int64_t g = 0; g < n; ++g) {
        double cz = cam_t(cam, 2);
        for (int k = 0; k < 3; ++k) cz += cam_R(cam, 2, k) * means[3 * g + k];
        if (cz > prm[P_ZNEAR]) {
            order[m].key = depth_key[g];
            order[m].g = (uint32_t)g;
            ++m;
        }
    }
    qsort(order, (size_t)m, sizeof(kd_pair), kd_cmp);
    uint32_t *list = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t k = 0; k < m; ++k) list[k] = order[k].g;
    free(order);
    const int rw = x1 - x0, rh = y1 - y0;
#pragma omp parallel
    {
        uint32_t *cg = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
        double *ca = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * 5);
#pragma omp for schedule(dynamic, 16)
        for (int64_t idx = 0; idx < (int64_t)rw * rh; ++idx)
            surfel_pixel_bwd(x0 + (int)(idx % rw) + 0.5, y0 + (int)(idx / rw) + 0.5, list, m, means, quats, scales2,
                             opac, rgb, NULL, 0, NULL, cam, prm, dC + 3 * idx, cg, ca, g_means, g_quats, g_scales2,
                             g_opac, g_rgb, NULL);
        free(cg); free(ca);
    }
    free(list);
}

/* The backward of orc_render_2dgs (tiled lists).  With features (feat
 * [n][D], dF [region pixels][D] and g_feat [n][D], all NULL or none),
 * dL/dw_g also takes the feature term dF . f_g and g_feat[g] += w_g dF. */
void orc_render_2dgs_bwd(int64_t n, const double *means, const double *quats, const double *scales2,
                         const double *opac, const double *rgb, const double *feat, int D, const double *dF,
                         const uint32_t *gids, const uint32_t *ranges, const double *cam, const double *prm, int x0,
                         int y0, int x1, int y1, const double *dC, double *g_means, double *g_quats,
                         double *g_scales2, double *g_opac, double *g_rgb, double *g_feat)
{
    const int W = (int)cam[0], tsz = (int)prm[P_TILE];
    const int tiles_x = (W + tsz - 1) / tsz;
    const int rw = x1 - x0, rh = y1 - y0;
    (void)n;
#pragma omp parallel
    {
        uint32_t *cg = (uint32_t *)malloc(sizeof(uint32_t) * ORC_MAXC);
        double *ca = (double *)malloc(sizeof(double) * ORC_MAXC * 5);
#pragma omp for schedule(dynamic, 16)
        for (int64_t idx = 0; idx < (int64_t)rw * rh; ++idx) {
            const int ix = x0 + (int)(idx % rw), iy = y0 + (int)(idx / rw);
            const int t = (iy / tsz) * tiles_x + ix / tsz;
            const uint32_t s0 = ranges[2 * t], e0 = ranges[2 * t + 1];
            const int64_t len = (int64_t)e0 - s0 < ORC_MAXC ? (int64_t)e0 - s0 : ORC_MAXC;
            surfel_pixel_bwd(ix + 0.5, iy + 0.5, gids + s0, len, means, quats, scales2, opac, rgb, feat, D,
                             dF ? dF + (int64_t)D * idx : NULL, cam, prm, dC + 3 * idx, cg, ca, g_means, g_quats,
                             g_scales2, g_opac, g_rgb, g_feat);
        }
        free(cg); free(ca);
    }
}

/* Binary32 binning rule for surfels (it decides integers, so it is specified
 * operation by operation; this file is compiled with -ffp-contract=off).
 *   qn = q / sqrt(((w w + x x) + y y) + z z); t_u, t_v = the first two
 *   columns of R(qn) (the formulas of quat_to_rot, each product rounded);
 *   c_r = ((W_r0 X + W_r1 Y) + W_r2 Z) + t_r;
 *   a_r = (((W_r0 R_00 + W_r1 R_10) + W_r2 R_20)) s_u, b_r likewise with
 *   column 1 and s_v;
 *   the ellipse must clear the camera: c_z - sqrt(cut ((a_z a_z) + (b_z b_z)))
 *   > znear, else the surfel is culled (no tiles);
 *   T_0j = fx k_jx + cx k_jz, T_1j = fy k_jy + cy k_jz, T_2j = k_jz for the
 *   columns k = a, b, c;
 *   C*_rs = (T_r0 T_s0 + T_r1 T_s1) - (T_r2 T_s2) / cut;
 *   the box x in [(C*_02 - e_x) / C*_22, (C*_02 + e_x) / C*_22] (ordered),
 *   e_x = sqrt(max(0, C*_02 C*_02 - C*_00 C*_22)), likewise y with row 1;
 *   widened by 1/64 of its larger side plus 1/2 px against the rounding of
 *   the above;
 *   pixels: those whose centre lies in the box, ceil(lo - 1/2) ..
 *   floor(hi - 1/2), clamped to the image; tiles: pixel / 16.
 * Outputs as orc_bin_f32: pix (x0, y0, x1, y1), tile (x0, y0, x1, y1),
 * ntiles (0 if culled or off the image) and the depth bits of c_z. */
void orc_bin_surfel_f32(int64_t n, const float *means, const float *quats, const float *scales2, const float *cam,
                        const float *prm, int32_t *pix, int32_t *tile, uint32_t *ntiles, uint32_t *dbits)
{
    const float W = cam[0], H = cam[1], fx = cam[2], fy = cam[3], cx = cam[4], cy = cam[5];
    const float *Wm = cam + 6;
    const float cut = prm[P_CUT], znear = prm[P_ZNEAR];
    const int tsz = (int)prm[P_TILE];
    for (int64_t g = 0; g < n; ++g) {
        int32_t *p4 = pix + 4 * g, *t4 = tile + 4 * g;
        ntiles[g] = 0;
        p4[0] = p4[1] = p4[2] = p4[3] = 0;
        t4[0] = t4[1] = t4[2] = t4[3] = 0;
        dbits[g] = 0xFFFFFFFFu;
        const float *q = quats + 4 * g;
        const float nq = sqrtf(((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3]);
        const float w = q[0] / nq, x = q[1] / nq, y = q[2] / nq, z = q[3] / nq;
        const float R00 = 1.0f - 2.0f * (y * y + z * z), R10 = 2.0f * (x * y + w * z), R20 = 2.0f * (x * z - w * y);
        const float R01 = 2.0f * (x * y - w * z), R11 = 1.0f - 2.0f * (x * x + z * z), R21 = 2.0f * (y * z + w * x);
        const float X = means[3 * g], Y = means[3 * g + 1], Z = means[3 * g + 2];
        float c[3], a[3], b[3];
        for (int r = 0; r < 3; ++r) {
            const float *row = Wm + 4 * r;
            c[r] = ((row[0] * X + row[1] * Y) + row[2] * Z) + row[3];
            a[r] = ((row[0] * R00 + row[1] * R10) + row[2] * R20) * scales2[2 * g];
            b[r] = ((row[0] * R01 + row[1] * R11) + row[2] * R21) * scales2[2 * g + 1];
        }
        const float zmin = c[2] - sqrtf(cut * (a[2] * a[2] + b[2] * b[2]));
        if (!(zmin > znear)) continue;
        const float *col[3] = {a, b, c};
        float T[3][3];
        for (int j = 0; j < 3; ++j) {
            T[0][j] = fx * col[j][0] + cx * col[j][2];
            T[1][j] = fy * col[j][1] + cy * col[j][2];
            T[2][j] = col[j][2];
        }
        float Cs[3][3];
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) Cs[r][s] = (T[r][0] * T[s][0] + T[r][1] * T[s][1]) - (T[r][2] * T[s][2]) / cut;
        const float ex = sqrtf(fmaxf(0.0f, Cs[0][2] * Cs[0][2] - Cs[0][0] * Cs[2][2]));
        const float ey = sqrtf(fmaxf(0.0f, Cs[1][2] * Cs[1][2] - Cs[1][1] * Cs[2][2]));
        const float xa = (Cs[0][2] - ex) / Cs[2][2], xb = (Cs[0][2] + ex) / Cs[2][2];
        const float ya = (Cs[1][2] - ey) / Cs[2][2], yb = (Cs[1][2] + ey) / Cs[2][2];
        float x0 = fminf(xa, xb), x1 = fmaxf(xa, xb), y0 = fminf(ya, yb), y1 = fmaxf(ya, yb);
        if (!isfinite(x0) || !isfinite(x1) || !isfinite(y0) || !isfinite(y1)) continue;
        const float pad = fmaxf(x1 - x0, y1 - y0) * 0.015625f + 0.5f;
        x0 = x0 - pad; x1 = x1 + pad; y0 = y0 - pad; y1 = y1 + pad;
        float xlo = ceilf(x0 - 0.5f), xhi = floorf(x1 - 0.5f);
        float ylo = ceilf(y0 - 0.5f), yhi = floorf(y1 - 0.5f);
        xlo = fmaxf(xlo, 0.0f);
        ylo = fmaxf(ylo, 0.0f);
        xhi = fminf(xhi, W - 1.0f);
        yhi = fminf(yhi, H - 1.0f);
        if (xlo > xhi || ylo > yhi) continue;
        p4[0] = (int)xlo; p4[1] = (int)ylo; p4[2] = (int)xhi; p4[3] = (int)yhi;
        t4[0] = p4[0] / tsz; t4[1] = p4[1] / tsz; t4[2] = p4[2] / tsz; t4[3] = p4[3] / tsz;
        ntiles[g] = (uint32_t)((t4[2] - t4[0] + 1) * (t4[3] - t4[1] + 1));
        memcpy(dbits + g, &c[2], 4);
    }
}

/* Tiled surfel render of the region: each pixel walks its 16x16 tile's
 * depth-sorted list (built from orc_bin_surfel_f32) with the rules of
 * orc_render_2dgs_brute.  The surfel arrays are indexed by the lists' ids.
 * feat [n][D] (NULL: none) is blended into out_feat [region pixels][D] with
 * the same weights (Eq. 4).  out_margin (NULL: none) receives, per pixel,
 * the smallest relative distance to its threshold of a decision that
 * settles the contributor set: the cutoff of a surfel that would pass the
 * alpha test there, the alpha_min test and the stop rule. */
void orc_render_2dgs(const double *means, const double *quats, const double *scales2, const double *opac,
                     const double *rgb, const double *feat, int D, const uint32_t *gids, const uint32_t *ranges,
                     const double *cam, const double *prm, int x0, int y0, int x1, int y1, double *out_rgb,
                     double *out_feat, double *out_T, int32_t *out_ncontrib, double *out_margin)
{
    const int W = (int)cam[0], tsz = (int)prm[P_TILE];
    const int tiles_x = (W + tsz - 1) / tsz;
    const int rw = x1 - x0, rh = y1 - y0;
    const double cut = prm[P_CUT], amin = prm[P_AMIN], amax = prm[P_AMAX], teps = prm[P_TEPS];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t idx = 0; idx < (int64_t)rw * rh; ++idx) {
        const int ix = x0 + (int)(idx % rw), iy = y0 + (int)(idx / rw);
        const double px = ix + 0.5, py = iy + 0.5;
        const int t = (iy / tsz) * tiles_x + ix / tsz;
        double T = 1.0, acc[3] = {0.0, 0.0, 0.0}, margin = INFINITY;
        double *F = out_feat ? out_feat + (int64_t)D * idx : NULL;
        if (F)
            for (int k = 0; k < D; ++k) F[k] = 0.0;
        int nc = 0;
        for (uint32_t k = ranges[2 * t]; k < ranges[2 * t + 1]; ++k) {
            const uint32_t g = gids[k];
            double u, v, lam;
            if (!splat_uv(means + 3 * g, quats + 4 * g, scales2 + 2 * g, cam, px, py, &u, &v, &lam)) continue;
            if (!(lam > 0.0)) continue;
            const double r2 = u * u + v * v;
            double a_cut = opac[g] * exp(-0.5 * cut);
            if (a_cut > amax) a_cut = amax;
            if (a_cut >= amin * (1.0 - 1e-3) && rel(r2, cut) < margin) margin = rel(r2, cut);
            if (r2 > cut) continue;
            const double rho = opac[g] * exp(-0.5 * r2);
            const double alpha = rho > amax ? amax : rho;
            if (rel(alpha, amin) < margin) margin = rel(alpha, amin);
            if (alpha < amin) continue;
            const double Tn = T * (1.0 - alpha);
            if (rel(Tn, teps) < margin) margin = rel(Tn, teps);
            if (Tn < teps) break;
            const double w = alpha * T;
            for (int ch = 0; ch < 3; ++ch) acc[ch] += w * rgb[3 * g + ch];
            if (F && feat)
                for (int c = 0; c < D; ++c) F[c] += w * feat[(int64_t)D * g + c];
            T = Tn;
            ++nc;
        }
        for (int ch = 0; ch < 3; ++ch) out_rgb[3 * idx + ch] = acc[ch] + T * prm[P_BG0 + ch];
        out_T[idx] = T;
        out_ncontrib[idx] = nc;
        if (out_margin) out_margin[idx] = margin;
    }
}

/* u(x) through the surfel's projective map instead of the ray solve: with
 * T = K [a b c] (a, b, c as in splat_uv) a plane point (u, v) lands on the
 * homogeneous pixel T (u, v, 1)^T, so the pixel (x, y) holds the point where
 * the two planes h_u = T_0 - x T_2 and h_v = T_1 - y T_2 (rows of T) vanish:
 *   u = (h_u1 h_v2 - h_u2 h_v1) / (h_u0 h_v1 - h_u1 h_v0),
 *   v = (h_u2 h_v0 - h_u0 h_v2) / (h_u0 h_v1 - h_u1 h_v0),
 * and the camera depth of that point is T_2 (u, v, 1)^T. */
void orc_splat_uv_T(int64_t m, const double *mu, const double *q, const double *s2, const double *cam, const double *px,
                    const double *py, double *u, double *v, double *depth)
{
    for (int64_t i = 0; i < m; ++i) {
        const double *qi = q + 4 * i;
        const double nq = sqrt(qi[0] * qi[0] + qi[1] * qi[1] + qi[2] * qi[2] + qi[3] * qi[3]);
        const double qn[4] = {qi[0] / nq, qi[1] / nq, qi[2] / nq, qi[3] / nq};
        double R[3][3];
        quat_to_rot(qn, R);
        double k3[3][3];   /* columns a, b, c in the camera */
        for (int r = 0; r < 3; ++r) {
            k3[r][2] = cam_t(cam, r);
            k3[r][0] = 0.0;
            k3[r][1] = 0.0;
            for (int k = 0; k < 3; ++k) {
                k3[r][2] += cam_R(cam, r, k) * mu[3 * i + k];
                k3[r][0] += cam_R(cam, r, k) * R[k][0] * s2[2 * i];
                k3[r][1] += cam_R(cam, r, k) * R[k][1] * s2[2 * i + 1];
            }
        }
        double T[3][3];
        for (int j = 0; j < 3; ++j) {
            T[0][j] = cam[2] * k3[0][j] + cam[4] * k3[2][j];
            T[1][j] = cam[3] * k3[1][j] + cam[5] * k3[2][j];
            T[2][j] = k3[2][j];
        }
        double hu[3], hv[3];
        for (int j = 0; j < 3; ++j) {
            hu[j] = T[0][j] - px[i] * T[2][j];
            hv[j] = T[1][j] - py[i] * T[2][j];
        }
        const double den = hu[0] * hv[1] - hu[1] * hv[0];
        u[i] = (hu[1] * hv[2] - hu[2] * hv[1]) / den;
        v[i] = (hu[2] * hv[0] - hu[0] * hv[2]) / den;
        depth[i] = T[2][0] * u[i] + T[2][1] * v[i] + T[2][2];
    }
}


/* NDFD over surfels (the paper's combination of Sec. 3.1-3.3): the
 * contributors and weights of each pixel come from the tiled surfel render
 * (orc_render_2dgs's walk), the losses from the same per-pixel arithmetic as
 * orc_ndfd. */
void orc_ndfd_2dgs(const double *means, const double *quats, const double *scales2, const double *opac,
                   const uint32_t *gids, const uint32_t *ranges, const double *cam, const double *prm, int x0, int y0,
                   int x1, int y1, const double *feat, int D, const double *fgt, double kslope, double lam,
                   double *out_Lgt, double *out_Lcf, int32_t *out_ncontrib)
{
    const int W = (int)cam[0], tsz = (int)prm[P_TILE];
    const int tiles_x = (W + tsz - 1) / tsz;
    const int rw = x1 - x0, rh = y1 - y0;
    const double cut = prm[P_CUT], amin = prm[P_AMIN], amax = prm[P_AMAX], teps = prm[P_TEPS];
#pragma omp parallel
    {
        uint32_t *ids = (uint32_t *)malloc(sizeof(uint32_t) * ORC_MAXC);
        double *ws = (double *)malloc(sizeof(double) * ORC_MAXC);
        double *F = (double *)malloc(sizeof(double) * (size_t)(D > 0 ? D : 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t idx = 0; idx < (int64_t)rw * rh; ++idx) {
            const int ix = x0 + (int)(idx % rw), iy = y0 + (int)(idx / rw);
            const double px = ix + 0.5, py = iy + 0.5;
            const int t = (iy / tsz) * tiles_x + ix / tsz;
            double T = 1.0;
            int nc = 0;
            for (uint32_t k = ranges[2 * t]; k < ranges[2 * t + 1] && nc < ORC_MAXC; ++k) {
                const uint32_t g = gids[k];
                double u, v, lamd;
                if (!splat_uv(means + 3 * g, quats + 4 * g, scales2 + 2 * g, cam, px, py, &u, &v, &lamd)) continue;
                if (!(lamd > 0.0)) continue;
                const double r2 = u * u + v * v;
                if (r2 > cut) continue;
                const double rho = opac[g] * exp(-0.5 * r2);
                const double alpha = rho > amax ? amax : rho;
                if (alpha < amin) continue;
                const double Tn = T * (1.0 - alpha);
                if (Tn < teps) break;
                ids[nc] = g;
                ws[nc] = alpha * T;
                ++nc;
                T = Tn;
            }
            double Lgt, Lcf, Wc;
            ndfd_losses(ids, ws, nc, feat, D, fgt + (int64_t)D * idx, kslope, lam, F, &Lgt, &Lcf, &Wc);
            out_Lgt[idx] = Lgt;
            out_Lcf[idx] = Lcf;
            if (out_ncontrib) out_ncontrib[idx] = nc;
        }
        free(ids); free(ws); free(F);
    }
}


/* Gradient of L = sum_p dLgt[p] L_gt(p) + dLcf[p] L_cf(p) of orc_ndfd_2dgs
 * with respect to the surfels' means, quaternions, (s_u, s_v) and
 * opacities; accumulates (+=).  dL/dw_k and dL/dalpha_k as in orc_ndfd_bwd
 * (Sec. 3.3, App. A.2), then the surfel chain of surfel_alpha_chain. */
void orc_ndfd_2dgs_bwd(const double *means, const double *quats, const double *scales2, const double *opac,
                       const uint32_t *gids, const uint32_t *ranges, const double *cam, const double *prm, int x0,
                       int y0, int x1, int y1, const double *feat, int D, const double *fgt, double kslope,
                       double lam, const double *dLgt, const double *dLcf, double *g_means, double *g_quats,
                       double *g_scales2, double *g_opac)
{
    const int W = (int)cam[0], tsz = (int)prm[P_TILE];
    const int tiles_x = (W + tsz - 1) / tsz;
    const int rw = x1 - x0, rh = y1 - y0;
    const double cut = prm[P_CUT], amin = prm[P_AMIN], amax = prm[P_AMAX], teps = prm[P_TEPS];
#pragma omp parallel
    {
        uint32_t *ids = (uint32_t *)malloc(sizeof(uint32_t) * ORC_MAXC);
        double *cs = (double *)malloc(sizeof(double) * ORC_MAXC * 7);   /* alpha, T, G, u, v, sigma, pre */
        double *F = (double *)malloc(sizeof(double) * (size_t)(D > 0 ? D : 1));
        double *Gs = (double *)malloc(sizeof(double) * (size_t)(D > 0 ? D : 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t idx = 0; idx < (int64_t)rw * rh; ++idx) {
            const int ix = x0 + (int)(idx % rw), iy = y0 + (int)(idx / rw);
            const double px = ix + 0.5, py = iy + 0.5;
            const int t = (iy / tsz) * tiles_x + ix / tsz;
            double T = 1.0;
            int nc = 0;
            for (uint32_t k = ranges[2 * t]; k < ranges[2 * t + 1] && nc < ORC_MAXC; ++k) {
                const uint32_t g = gids[k];
                double u, v, lamd;
                if (!splat_uv(means + 3 * g, quats + 4 * g, scales2 + 2 * g, cam, px, py, &u, &v, &lamd)) continue;
                if (!(lamd > 0.0)) continue;
                const double r2 = u * u + v * v;
                if (r2 > cut) continue;
                const double G = exp(-0.5 * r2);
                const double rho = opac[g] * G;
                const double alpha = rho > amax ? amax : rho;
                if (alpha < amin) continue;
                const double Tn = T * (1.0 - alpha);
                if (Tn < teps) break;
                ids[nc] = g;
                double *c = cs + 7 * nc;
                c[0] = alpha; c[1] = T; c[2] = G; c[3] = u; c[4] = v;
                ++nc;
                T = Tn;
            }
            const double *fg = fgt + (int64_t)D * idx;
            const double cgt = dLgt[idx], ccf = dLcf[idx];
            /* front to back: sigma_k and W_{k-1} - F_{k-1} . f_k */
            double Wc = 0.0;
            for (int c = 0; c < D; ++c) F[c] = 0.0;
            for (int j = 0; j < nc; ++j) {
                const double *f = feat + (int64_t)D * ids[j];
                double *c = cs + 7 * j;
                const double w = c[0] * c[1];
                c[5] = ndfd_sigma(f, fg, D, kslope, lam);
                c[6] = Wc - dotd(F, f, D);
                Wc += w;
                for (int q = 0; q < D; ++q) F[q] += w * f[q];
            }
            /* back to front */
            double Ss = 0.0, Sw = 0.0;
            for (int c = 0; c < D; ++c) Gs[c] = 0.0;
            for (int k = nc - 1; k >= 0; --k) {
                const uint32_t g = ids[k];
                const double *f = feat + (int64_t)D * g;
                const double *c = cs + 7 * k;
                const double alpha = c[0], Tk = c[1], w = alpha * Tk, sg = c[5];
                const double gw = cgt * sg + ccf * (sg * c[6] + Ss - dotd(Gs, f, D));
                const double dalpha = Tk * gw - Sw / (1.0 - alpha);
                Sw += w * gw;
                Ss += sg * w;
                for (int q = 0; q < D; ++q) Gs[q] += sg * w * f[q];
                surfel_alpha_chain(g, c[2], c[3], c[4], dalpha, px, py, quats, scales2, opac, cam, amax, g_means,
                                   g_quats, g_scales2, g_opac);
            }
        }
        free(ids); free(cs); free(F); free(Gs);
    }
}
