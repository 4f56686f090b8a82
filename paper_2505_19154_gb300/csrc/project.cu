// EWA projection + SH colour (forward) and its chain rule (backward).
//
// Forward, one thread per (camera, Gaussian): the screen footprint of a 3-D
// Gaussian (Sigma' = J W Sigma W^T J^T + dilation I, its inverse the conic,
// the rasterizer the paper takes over from 3DGS, App. A) and the SH colour
// (Sec. 2.1).  Every value that decides binning (depth, mean, covariance,
// tile rectangle) follows the FP32 binning specification: single-rounded
// binary32 operations in a fixed order (__fmul_rn & co. so that nvcc cannot
// contract them into FMAs), sqrt and division correctly rounded, binary64
// only for the determinant and inverse of near-degenerate footprints
// (det < 1e-6 a c).
#include "fhgs_internal.cuh"

namespace fhgs {
namespace {

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdv(float a, float b) { return __fdiv_rn(a, b); }

// Real SH, degree <= 3, in the 3DGS ordering and signs.  Normalisation
// constants (closed forms): 1/(2 sqrt(pi)), sqrt(3/(4 pi)), sqrt(15/pi)/2,
// sqrt(5/pi)/4, sqrt(15/pi)/4, sqrt(35/(2 pi))/4, sqrt(105/pi)/2,
// sqrt(21/(2 pi))/4, sqrt(7/pi)/4, sqrt(105/pi)/4.
constexpr float kY0 = 0.28209479177387814f;
constexpr float kY1 = 0.48860251190291992f;
constexpr float kY2a = 1.0925484305920792f;
constexpr float kY2b = 0.31539156525252005f;
constexpr float kY2c = 0.54627421529603959f;
constexpr float kY3a = 0.59004358992664352f;
constexpr float kY3b = 2.8906114426405538f;
constexpr float kY3c = 0.45704579946446572f;
constexpr float kY3d = 0.37317633259011540f;
constexpr float kY3e = 1.4453057213202769f;

__device__ __forceinline__ void sh_eval(float x, float y, float z, int K, float *Y) {
    Y[0] = kY0;
    if (K > 1) {
        Y[1] = -kY1 * y;
        Y[2] = kY1 * z;
        Y[3] = -kY1 * x;
    }
    if (K > 4) {
        float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kY2a * x * y;
        Y[5] = -kY2a * y * z;
        Y[6] = kY2b * (2.f * zz - xx - yy);
        Y[7] = -kY2a * x * z;
        Y[8] = kY2c * (xx - yy);
        if (K > 9) {
            Y[9] = -kY3a * y * (3.f * xx - yy);
            Y[10] = kY3b * x * y * z;
            Y[11] = -kY3c * y * (4.f * zz - xx - yy);
            Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -kY3c * x * (4.f * zz - xx - yy);
            Y[14] = kY3e * z * (xx - yy);
            Y[15] = -kY3a * x * (xx - 3.f * yy);
        }
    }
}

// Adds s * grad_{x,y,z} Y_k to g for every k < K (s[k] = sum_c sh[k][c] dL/draw_c).
__device__ __forceinline__ void sh_grad_accum(float x, float y, float z, int K, const float *s, float *g) {
    if (K > 1) {
        g[1] += -kY1 * s[1];
        g[2] += kY1 * s[2];
        g[0] += -kY1 * s[3];
    }
    if (K > 4) {
        float xx = x * x, yy = y * y, zz = z * z;
        g[0] += kY2a * y * s[4];
        g[1] += kY2a * x * s[4];
        g[1] += -kY2a * z * s[5];
        g[2] += -kY2a * y * s[5];
        g[0] += -2.f * kY2b * x * s[6];
        g[1] += -2.f * kY2b * y * s[6];
        g[2] += 4.f * kY2b * z * s[6];
        g[0] += -kY2a * z * s[7];
        g[2] += -kY2a * x * s[7];
        g[0] += 2.f * kY2c * x * s[8];
        g[1] += -2.f * kY2c * y * s[8];
        if (K > 9) {
            g[0] += -6.f * kY3a * x * y * s[9];
            g[1] += -kY3a * (3.f * xx - 3.f * yy) * s[9];
            g[0] += kY3b * y * z * s[10];
            g[1] += kY3b * x * z * s[10];
            g[2] += kY3b * x * y * s[10];
            g[0] += 2.f * kY3c * x * y * s[11];
            g[1] += -kY3c * (4.f * zz - xx - 3.f * yy) * s[11];
            g[2] += -8.f * kY3c * y * z * s[11];
            g[0] += -6.f * kY3d * x * z * s[12];
            g[1] += -6.f * kY3d * y * z * s[12];
            g[2] += kY3d * (6.f * zz - 3.f * xx - 3.f * yy) * s[12];
            g[0] += -kY3c * (4.f * zz - 3.f * xx - yy) * s[13];
            g[1] += 2.f * kY3c * x * y * s[13];
            g[2] += -8.f * kY3c * x * z * s[13];
            g[0] += 2.f * kY3e * x * z * s[14];
            g[1] += -2.f * kY3e * y * z * s[14];
            g[2] += kY3e * (xx - yy) * s[14];
            g[0] += -kY3a * (3.f * xx - 3.f * yy) * s[15];
            g[1] += 6.f * kY3a * x * y * s[15];
        }
    }
}

// FP32 binning specification.  Returns false if culled.
__device__ bool bin_spec(const float mu[3], const float s[3], float4 q, const DevCam &cam, const Params &p,
                         float &mx, float &my, float &cA, float &cB, float &cC, float &depth, int4 &trect,
                         uint32_t &ntiles) {
    float n2 = fm(q.x, q.x);
    n2 = fa(n2, fm(q.y, q.y));
    n2 = fa(n2, fm(q.z, q.z));
    n2 = fa(n2, fm(q.w, q.w));
    if (!(n2 > 0.f) || !isfinite(n2)) return false;
    const float inv = fdv(1.f, __fsqrt_rn(n2));
    const float w = fm(q.x, inv), x = fm(q.y, inv), y = fm(q.z, inv), z = fm(q.w, inv);
    const float xx = fm(x, x), yy = fm(y, y), zz = fm(z, z), xy = fm(x, y), xz = fm(x, z), yz = fm(y, z);
    const float wx = fm(w, x), wy = fm(w, y), wz = fm(w, z);
    float R[3][3];
    R[0][0] = fs(1.f, fm(2.f, fa(yy, zz)));
    R[0][1] = fm(2.f, fs(xy, wz));
    R[0][2] = fm(2.f, fa(xz, wy));
    R[1][0] = fm(2.f, fa(xy, wz));
    R[1][1] = fs(1.f, fm(2.f, fa(xx, zz)));
    R[1][2] = fm(2.f, fs(yz, wx));
    R[2][0] = fm(2.f, fs(xz, wy));
    R[2][1] = fm(2.f, fa(yz, wx));
    R[2][2] = fs(1.f, fm(2.f, fa(xx, yy)));
    float M[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[i][j] = fm(R[i][j], s[j]);
    float S[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            float acc = fm(M[i][0], M[j][0]);
            acc = fa(acc, fm(M[i][1], M[j][1]));
            acc = fa(acc, fm(M[i][2], M[j][2]));
            S[i][j] = acc;
            S[j][i] = acc;
        }
    float t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float acc = fm(cam.R[3 * i + 0], mu[0]);
        acc = fa(acc, fm(cam.R[3 * i + 1], mu[1]));
        acc = fa(acc, fm(cam.R[3 * i + 2], mu[2]));
        t[i] = fa(acc, cam.t[i]);
    }
    if (!(t[2] > p.znear)) return false;
    const float Wf = (float)cam.W, Hf = (float)cam.H;
    const float limx = fm(p.fov, fdv(fm(0.5f, Wf), cam.fx));
    const float limy = fm(p.fov, fdv(fm(0.5f, Hf), cam.fy));
    const float ux = fdv(t[0], t[2]), uy = fdv(t[1], t[2]);
    const float xh = fminf(limx, fmaxf(-limx, ux));
    const float yh = fminf(limy, fmaxf(-limy, uy));
    const float J00 = fdv(cam.fx, t[2]), J02 = -fdv(fm(cam.fx, xh), t[2]);
    const float J11 = fdv(cam.fy, t[2]), J12 = -fdv(fm(cam.fy, yh), t[2]);
    float T[2][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T[0][j] = fa(fm(J00, cam.R[0 * 3 + j]), fm(J02, cam.R[2 * 3 + j]));
        T[1][j] = fa(fm(J11, cam.R[1 * 3 + j]), fm(J12, cam.R[2 * 3 + j]));
    }
    float U[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float acc = fm(T[i][0], S[0][j]);
            acc = fa(acc, fm(T[i][1], S[1][j]));
            acc = fa(acc, fm(T[i][2], S[2][j]));
            U[i][j] = acc;
        }
    float a = fm(U[0][0], T[0][0]);
    a = fa(a, fm(U[0][1], T[0][1]));
    a = fa(a, fm(U[0][2], T[0][2]));
    a = fa(a, p.dil);
    float b = fm(U[0][0], T[1][0]);
    b = fa(b, fm(U[0][1], T[1][1]));
    b = fa(b, fm(U[0][2], T[1][2]));
    float c = fm(U[1][0], T[1][0]);
    c = fa(c, fm(U[1][1], T[1][1]));
    c = fa(c, fm(U[1][2], T[1][2]));
    c = fa(c, p.dil);
    const float ac = fm(a, c);
    float det = fs(ac, fm(b, b));
    if (det < fm(1e-6f, ac)) {
        const double dd = __dsub_rn(__dmul_rn((double)a, (double)c), __dmul_rn((double)b, (double)b));
        det = __double2float_rn(dd);
        if (!(det > 0.f)) return false;
        cA = __double2float_rn(__ddiv_rn((double)c, dd));
        cB = __double2float_rn(__ddiv_rn(-(double)b, dd));
        cC = __double2float_rn(__ddiv_rn((double)a, dd));
    } else {
        if (!(det > 0.f)) return false;
        cA = fdv(c, det);
        cB = -fdv(b, det);
        cC = fdv(a, det);
    }
    mx = fa(fdv(fm(cam.fx, t[0]), t[2]), cam.cx);
    my = fa(fdv(fm(cam.fy, t[1]), t[2]), cam.cy);
    const float ex = __fsqrt_rn(fm(p.cut, a));
    const float ey = __fsqrt_rn(fm(p.cut, c));
    if (!isfinite(mx) || !isfinite(my) || !isfinite(ex) || !isfinite(ey)) return false;
    float xlo = ceilf(fs(fs(mx, ex), 0.5f)), xhi = floorf(fs(fa(mx, ex), 0.5f));
    float ylo = ceilf(fs(fs(my, ey), 0.5f)), yhi = floorf(fs(fa(my, ey), 0.5f));
    xlo = fmaxf(xlo, 0.f);
    ylo = fmaxf(ylo, 0.f);
    xhi = fminf(xhi, fs(Wf, 1.f));
    yhi = fminf(yhi, fs(Hf, 1.f));
    if (xlo > xhi || ylo > yhi) return false;
    const int ix0 = (int)xlo, ix1 = (int)xhi, iy0 = (int)ylo, iy1 = (int)yhi;
    trect = make_int4(ix0 / kTile, iy0 / kTile, ix1 / kTile, iy1 / kTile);
    ntiles = (uint32_t)((trect.z - trect.x + 1) * (trect.w - trect.y + 1));
    depth = t[2];
    return true;
}

__global__ void __launch_bounds__(256) k_project(const float *__restrict__ means, const float *__restrict__ scales,
                                                 const float4 *__restrict__ quats, const float *__restrict__ opac,
                                                 const float *__restrict__ sh, long long N, CamSet cs, Params p,
                                                 ProjView pv, unsigned *status) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)cs.n * N) return;
    const int ci = (int)(e / N);
    const long long g = e - (long long)ci * N;
    const DevCam &cam = cs.c[ci];
    float mu[3] = {means[3 * g], means[3 * g + 1], means[3 * g + 2]};
    float s[3] = {scales[3 * g], scales[3 * g + 1], scales[3 * g + 2]};
    const float4 q = quats[g];
    const float op = opac[g];
    bool finite = isfinite(mu[0]) && isfinite(mu[1]) && isfinite(mu[2]) && isfinite(s[0]) && isfinite(s[1]) &&
                  isfinite(s[2]) && isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(q.w) && isfinite(op);
    const float *shg = sh + (long long)3 * p.K * g;
    float col[3] = {0.f, 0.f, 0.f};
    if (finite) {
        float Y[16];
        float v0 = mu[0] - cam.campos[0], v1 = mu[1] - cam.campos[1], v2 = mu[2] - cam.campos[2];
        float inv = rsqrtf(v0 * v0 + v1 * v1 + v2 * v2);
        sh_eval(v0 * inv, v1 * inv, v2 * inv, p.K, Y);
        for (int k = 0; k < p.K; ++k) {
            float c0 = shg[3 * k], c1 = shg[3 * k + 1], c2 = shg[3 * k + 2];
            finite = finite && isfinite(c0) && isfinite(c1) && isfinite(c2);
            col[0] += c0 * Y[k];
            col[1] += c1 * Y[k];
            col[2] += c2 * Y[k];
        }
    }
    float mx = 0.f, my = 0.f, cA = 0.f, cB = 0.f, cC = 0.f, depth = 0.f;
    int4 tr = make_int4(-1, -1, -1, -1);
    uint32_t nt = 0;
    bool ok = false;
    if (finite) {
        ok = bin_spec(mu, s, q, cam, p, mx, my, cA, cB, cC, depth, tr, nt);
    } else if (ci == 0) {
        latch(status, ST_NUMERIC);
    }
    GRec r;
    unsigned mask = 0;
    float rgb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float raw = col[c] + 0.5f;
        mask |= (raw > 0.f ? 1u : 0u) << c;
        rgb[c] = fmaxf(raw, 0.f);
    }
    r.a = make_float4(mx, my, cA, cB);
    r.b = make_float4(cC, op, rgb[0], rgb[1]);
    r.c = make_float4(rgb[2], depth, __uint_as_float(mask), 0.f);
    pv.rec[e] = r;
    pv.trect[e] = tr;
    pv.ntiles[e] = ok ? nt : 0u;
    pv.dkey[e] = ok ? __float_as_uint(depth) : 0xFFFFFFFFu;
}

// Chain rule from the per-(camera, Gaussian) render gradients
// g2d = (d mean_x, d mean_y, d A, d B, d C, d opacity, d r, d g, d b) to the
// Gaussian parameters, summed over cameras.  One thread per Gaussian.
__global__ void __launch_bounds__(128) k_project_bwd(const float *__restrict__ means, const float *__restrict__ scales,
                                                     const float4 *__restrict__ quats, const float *__restrict__ sh,
                                                     long long N, CamSet cs, Params p, ProjView pv,
                                                     const float *__restrict__ g2d, float *gmeans, float *gscales,
                                                     float *gquats, float *gopac, float *gsh) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = g < N;
    const int K = p.K;
    float gmu[3] = {0.f, 0.f, 0.f}, gs[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, gop = 0.f;
    float gshv[48];
#pragma unroll
    for (int i = 0; i < 48; ++i) gshv[i] = 0.f;
    // every gradient is linear in the footprint gradients: a Gaussian that no
    // tile composited (all of them zero) gets exact zeros, without reading
    // its parameters
    bool touched = false;
    for (int ci = 0; ci < cs.n && valid && !touched; ++ci) {
        const long long e = (long long)ci * N + g;
        if (pv.ntiles[e] == 0) continue;
        const float *gg = g2d + 12 * e;
        const float4 ga = *reinterpret_cast<const float4 *>(gg);
        const float4 gb = *reinterpret_cast<const float4 *>(gg + 4);
        touched = ga.x != 0.f || ga.y != 0.f || ga.z != 0.f || ga.w != 0.f || gb.x != 0.f || gb.y != 0.f ||
                  gb.z != 0.f || gb.w != 0.f || gg[8] != 0.f;
    }
    if (touched) {
    const float mu[3] = {means[3 * g], means[3 * g + 1], means[3 * g + 2]};
    const float s[3] = {scales[3 * g], scales[3 * g + 1], scales[3 * g + 2]};
    const float4 q4 = quats[g];
    const float *shg = sh + (long long)3 * K * g;

    // rotation from the normalised quaternion (camera independent)
    const float nq = sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float qn[4] = {q4.x / nq, q4.y / nq, q4.z / nq, q4.w / nq};
    const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    float R[3][3];
    R[0][0] = 1.f - 2.f * (y * y + z * z);
    R[0][1] = 2.f * (x * y - w * z);
    R[0][2] = 2.f * (x * z + w * y);
    R[1][0] = 2.f * (x * y + w * z);
    R[1][1] = 1.f - 2.f * (x * x + z * z);
    R[1][2] = 2.f * (y * z - w * x);
    R[2][0] = 2.f * (x * z - w * y);
    R[2][1] = 2.f * (y * z + w * x);
    R[2][2] = 1.f - 2.f * (x * x + y * y);
    float M[3][3], S[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[i][j] = R[i][j] * s[j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) S[i][j] = M[i][0] * M[j][0] + M[i][1] * M[j][1] + M[i][2] * M[j][2];
    float GS[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};

    for (int ci = 0; ci < cs.n; ++ci) {
        const long long e = (long long)ci * N + g;
        if (pv.ntiles[e] == 0) continue;
        const float *gg = g2d + 12 * e;
        const float4 ga = *reinterpret_cast<const float4 *>(gg);
        const float4 gb = *reinterpret_cast<const float4 *>(gg + 4);
        const float gbl = gg[8];
        const GRec rec = pv.rec[e];
        const DevCam &cam = cs.c[ci];
        gop += gb.y;
        // view-space mean and clamped Jacobian
        float t[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
            t[i] = cam.R[3 * i] * mu[0] + cam.R[3 * i + 1] * mu[1] + cam.R[3 * i + 2] * mu[2] + cam.t[i];
        const float tz = t[2], itz = 1.f / tz;
        const float limx = p.fov * (0.5f * cam.W / cam.fx), limy = p.fov * (0.5f * cam.H / cam.fy);
        const float ux = t[0] * itz, uy = t[1] * itz;
        const bool clx = (ux > limx) || (ux < -limx), cly = (uy > limy) || (uy < -limy);
        const float xh = fminf(limx, fmaxf(-limx, ux)), yh = fminf(limy, fmaxf(-limy, uy));
        const float J00 = cam.fx * itz, J02 = -cam.fx * xh * itz, J11 = cam.fy * itz, J12 = -cam.fy * yh * itz;
        float T[2][3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T[0][j] = J00 * cam.R[j] + J02 * cam.R[6 + j];
            T[1][j] = J11 * cam.R[3 + j] + J12 * cam.R[6 + j];
        }
        // conic K = Sigma2^-1: dL/dSigma2 = -K G_K K with G_K symmetric
        const float kA = rec.a.z, kB = rec.a.w, kC = rec.b.x;
        const float gA = ga.z, gB2 = 0.5f * ga.w, gC = gb.x;
        // tmp = K G_K
        const float t00 = kA * gA + kB * gB2, t01 = kA * gB2 + kB * gC;
        const float t10 = kB * gA + kC * gB2, t11 = kB * gB2 + kC * gC;
        const float G00 = -(t00 * kA + t01 * kB), G01 = -(t00 * kB + t01 * kC);
        const float G11 = -(t10 * kB + t11 * kC);
        const float G2[2][2] = {{G00, G01}, {G01, G11}};
        // dL/dSigma += T^T G2 T ;  dL/dT = 2 G2 T Sigma
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                GS[i][j] += T[0][i] * (G2[0][0] * T[0][j] + G2[0][1] * T[1][j]) +
                            T[1][i] * (G2[1][0] * T[0][j] + G2[1][1] * T[1][j]);
        float GT[2][3];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            float r0 = G2[i][0] * T[0][0] + G2[i][1] * T[1][0];
            float r1 = G2[i][0] * T[0][1] + G2[i][1] * T[1][1];
            float r2 = G2[i][0] * T[0][2] + G2[i][1] * T[1][2];
#pragma unroll
            for (int j = 0; j < 3; ++j) GT[i][j] = 2.f * (r0 * S[0][j] + r1 * S[1][j] + r2 * S[2][j]);
        }
        // T = J R_w  ->  dL/dJ = dL/dT R_w^T
        const float GJ00 = GT[0][0] * cam.R[0] + GT[0][1] * cam.R[1] + GT[0][2] * cam.R[2];
        const float GJ02 = GT[0][0] * cam.R[6] + GT[0][1] * cam.R[7] + GT[0][2] * cam.R[8];
        const float GJ11 = GT[1][0] * cam.R[3] + GT[1][1] * cam.R[4] + GT[1][2] * cam.R[5];
        const float GJ12 = GT[1][0] * cam.R[6] + GT[1][1] * cam.R[7] + GT[1][2] * cam.R[8];
        const float itz2 = itz * itz;
        float gt0 = 0.f, gt1 = 0.f, gt2 = 0.f;
        gt2 += -GJ00 * cam.fx * itz2 - GJ11 * cam.fy * itz2;
        gt2 += GJ02 * cam.fx * xh * itz2 + GJ12 * cam.fy * yh * itz2;
        const float gxh = -GJ02 * cam.fx * itz, gyh = -GJ12 * cam.fy * itz;
        if (!clx) {
            gt0 += gxh * itz;
            gt2 -= gxh * t[0] * itz2;
        }
        if (!cly) {
            gt1 += gyh * itz;
            gt2 -= gyh * t[1] * itz2;
        }
        // screen mean
        gt0 += ga.x * cam.fx * itz;
        gt2 -= ga.x * cam.fx * t[0] * itz2;
        gt1 += ga.y * cam.fy * itz;
        gt2 -= ga.y * cam.fy * t[1] * itz2;
#pragma unroll
        for (int j = 0; j < 3; ++j) gmu[j] += cam.R[j] * gt0 + cam.R[3 + j] * gt1 + cam.R[6 + j] * gt2;
        // SH colour
        const unsigned mask = __float_as_uint(rec.c.z);
        const float graw[3] = {(mask & 1u) ? gb.z : 0.f, (mask & 2u) ? gb.w : 0.f, (mask & 4u) ? gbl : 0.f};
        float v0 = mu[0] - cam.campos[0], v1 = mu[1] - cam.campos[1], v2 = mu[2] - cam.campos[2];
        const float inv = rsqrtf(v0 * v0 + v1 * v1 + v2 * v2);
        const float dx = v0 * inv, dy = v1 * inv, dz = v2 * inv;
        float Y[16], sk[16], gd[3] = {0.f, 0.f, 0.f};
        sh_eval(dx, dy, dz, K, Y);
        for (int k = 0; k < K; ++k) {
            sk[k] = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                gshv[3 * k + c] += Y[k] * graw[c];
                sk[k] += shg[3 * k + c] * graw[c];
            }
        }
        sh_grad_accum(dx, dy, dz, K, sk, gd);
        const float dd = dx * gd[0] + dy * gd[1] + dz * gd[2];
        gmu[0] += (gd[0] - dx * dd) * inv;
        gmu[1] += (gd[1] - dy * dd) * inv;
        gmu[2] += (gd[2] - dz * dd) * inv;
    }
    // Sigma = M M^T, M = R diag(s)
    float GM[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) GM[i][j] = 2.f * (GS[i][0] * M[0][j] + GS[i][1] * M[1][j] + GS[i][2] * M[2][j]);
    float GR[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        gs[j] = GM[0][j] * R[0][j] + GM[1][j] * R[1][j] + GM[2][j] * R[2][j];
#pragma unroll
        for (int i = 0; i < 3; ++i) GR[i][j] = GM[i][j] * s[j];
    }
    float gqn[4];
    gqn[0] = 2.f * (-z * GR[0][1] + y * GR[0][2] + z * GR[1][0] - x * GR[1][2] - y * GR[2][0] + x * GR[2][1]);
    gqn[1] = 2.f * (y * GR[0][1] + z * GR[0][2] + y * GR[1][0] - 2.f * x * GR[1][1] - w * GR[1][2] +
                    z * GR[2][0] + w * GR[2][1] - 2.f * x * GR[2][2]);
    gqn[2] = 2.f * (-2.f * y * GR[0][0] + x * GR[0][1] + w * GR[0][2] + x * GR[1][0] + z * GR[1][2] -
                    w * GR[2][0] + z * GR[2][1] - 2.f * y * GR[2][2]);
    gqn[3] = 2.f * (-2.f * z * GR[0][0] - w * GR[0][1] + x * GR[0][2] + w * GR[1][0] - 2.f * z * GR[1][1] +
                    y * GR[1][2] + x * GR[2][0] + y * GR[2][1]);
    const float dq = qn[0] * gqn[0] + qn[1] * gqn[1] + qn[2] * gqn[2] + qn[3] * gqn[3];
#pragma unroll
    for (int k = 0; k < 4; ++k) gq[k] = (gqn[k] - qn[k] * dq) / nq;

    }

    // the warp's 32 consecutive Gaussians leave through shared memory, so
    // that every store covers contiguous bytes (rows of 3 K SH floats, 3
    // mean and 3 scale floats per Gaussian)
    __shared__ float sbuf[4][32 * 49];
    const int wl = threadIdx.x >> 5, ln = threadIdx.x & 31;
    const long long g0 = g - ln;
    if (g0 >= N) return;  // warp-uniform: the whole warp lies past the end
    const int nv = (int)min(32ll, N - g0);
    float *b = sbuf[wl];
    if (valid) {
        reinterpret_cast<float4 *>(gquats)[g] = make_float4(gq[0], gq[1], gq[2], gq[3]);
        gopac[g] = gop;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) b[ln * 3 + j] = gmu[j];
    __syncwarp();
    for (int f = ln; f < 3 * nv; f += 32) gmeans[3 * g0 + f] = b[f];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 3; ++j) b[ln * 3 + j] = gs[j];
    __syncwarp();
    for (int f = ln; f < 3 * nv; f += 32) gscales[3 * g0 + f] = b[f];
    __syncwarp();
    const int F = 3 * K;
#pragma unroll
    for (int i = 0; i < 48; ++i)
        if (i < F) b[ln * 49 + i] = gshv[i];
    __syncwarp();
    float *dst = gsh + (long long)F * g0;
    for (int j = 0; j < nv; ++j)
        for (int i = ln; i < F; i += 32) dst[j * F + i] = b[j * 49 + i];
}

}  // namespace

void launch_project(const fhgs_gaussians &g, const CamSet &cs, const Params &p, ProjView pv, unsigned *status,
                    cudaStream_t st) {
    const long long total = (long long)cs.n * g.n;
    if (total == 0) return;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    note_launch(1);
    k_project<<<blocks, 256, 0, st>>>(g.means, g.scales, reinterpret_cast<const float4 *>(g.quats), g.opacities, g.sh,
                                      g.n, cs, p, pv, status);
}

void launch_project_bwd(const fhgs_gaussians &g, const CamSet &cs, const Params &p, ProjView pv, const float *g2d,
                        float *gmeans, float *gscales, float *gquats, float *gop, float *gsh, cudaStream_t st) {
    if (g.n == 0) return;
    const unsigned blocks = (unsigned)((g.n + 127) / 128);
    note_launch(1);
    k_project_bwd<<<blocks, 128, 0, st>>>(g.means, g.scales, reinterpret_cast<const float4 *>(g.quats), g.sh, g.n,
                                          cs, p, pv, g2d, gmeans, gscales, gquats, gop, gsh);
}

}  // namespace fhgs
