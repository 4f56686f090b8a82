// 2DGS surfel geometry (Sec. 3.1, Eq. 1-3): projection with the binary32
// binning rule, the per-pixel render on the CUDA cores (forward and
// backward, App. A.2) and the chain rule back to the surfel parameters.
//
// A surfel is the plane P(u, v) = p + s_u t_u u + s_v t_v v, with t_u, t_v
// the first two columns of R(q), and density G = exp(-(u^2 + v^2)/2) at the
// plane point u(x) that projects to the pixel.  In the camera, with c = W p
// + t, a = s_u W t_u, b = s_v W t_v, the map T = K [a b c] takes (u, v, 1) to
// the homogeneous pixel.  Shifting its first two rows by the projected
// centre (x_c, y_c) gives T' with T' (u, v, 1) = depth (x - x_c, y - y_c, 1),
// so per pixel
//   (u, v, 1) ~ M (dx, dy, 1),  M = T'^-1,  dx = x - x_c, dy = y - y_c,
//   u = (M00 dx + M01 dy) / w,  v = (M10 dx + M11 dy) / w,
//   w = M20 dx + M21 dy + M22  (= 1 / depth of the hit: w > 0 in front).
// T' has a zero third column above its diagonal, so M has the same shape:
// its top-left block is the inverse of A = [[fx (a_x - xi a_z), fx (b_x - xi
// b_z)], [fy (a_y - eta a_z), fy (b_y - eta b_z)]] with xi = c_x / c_z, eta
// = c_y / c_z, (M20, M21) = -(a_z, b_z) A^-1 / c_z and M22 = 1 / c_z.  The
// record holds M (in binary64, rounded once), so the per-pixel numerators
// carry no constant term and do not cancel near the centre.
//
// The binning values follow the binary32 binning rule of the surfel
// specification (the dual-conic box of the footprint u^2 + v^2 <= cutoff,
// widened against rounding), one rounding per operation in a fixed order,
// so that the tile lists are bit-exact; the rest of the path is ordinary
// FP32 (binary64 for the record).
#include "fhgs_internal.cuh"

namespace fhgs {
namespace {

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdv(float a, float b) { return __fdiv_rn(a, b); }

constexpr int kB = 64;   // surfels per shared-memory batch
constexpr int kDC = 32;  // feature channels per block

// Real SH, degree <= 3, in the 3DGS ordering and signs (the same basis as
// the EWA projection; constants from their closed forms).
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

__device__ __forceinline__ void sh_basis(float x, float y, float z, int K, float *Y) {
    Y[0] = kY0;
    if (K > 1) {
        Y[1] = -kY1 * y;
        Y[2] = kY1 * z;
        Y[3] = -kY1 * x;
    }
    if (K > 4) {
        const float xx = x * x, yy = y * y, zz = z * z;
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

// g += sum_k s[k] grad Y_k (x, y, z).
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, int K, const float *s, float *g) {
    if (K > 1) {
        g[1] += -kY1 * s[1];
        g[2] += kY1 * s[2];
        g[0] += -kY1 * s[3];
    }
    if (K > 4) {
        const float xx = x * x, yy = y * y, zz = z * z;
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

// The binary32 binning rule: tile rectangle and depth, false if culled
// (the footprint ellipse reaches znear, a non-finite box, or off the image).
__device__ bool surfel_bin_spec(const float mu[3], float su, float sv, float4 q, const DevCam &cam, const Params &p,
                                int4 &trect, uint32_t &ntiles, float &depth) {
    float n2 = fm(q.x, q.x);
    n2 = fa(n2, fm(q.y, q.y));
    n2 = fa(n2, fm(q.z, q.z));
    n2 = fa(n2, fm(q.w, q.w));
    const float nq = __fsqrt_rn(n2);
    if (!(nq > 0.f) || !isfinite(nq)) return false;
    const float w = fdv(q.x, nq), x = fdv(q.y, nq), y = fdv(q.z, nq), z = fdv(q.w, nq);
    const float R00 = fs(1.f, fm(2.f, fa(fm(y, y), fm(z, z))));
    const float R10 = fm(2.f, fa(fm(x, y), fm(w, z)));
    const float R20 = fm(2.f, fs(fm(x, z), fm(w, y)));
    const float R01 = fm(2.f, fs(fm(x, y), fm(w, z)));
    const float R11 = fs(1.f, fm(2.f, fa(fm(x, x), fm(z, z))));
    const float R21 = fm(2.f, fa(fm(y, z), fm(w, x)));
    float c[3], a[3], b[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float *row = cam.R + 3 * r;
        c[r] = fa(fa(fa(fm(row[0], mu[0]), fm(row[1], mu[1])), fm(row[2], mu[2])), cam.t[r]);
        a[r] = fm(fa(fa(fm(row[0], R00), fm(row[1], R10)), fm(row[2], R20)), su);
        b[r] = fm(fa(fa(fm(row[0], R01), fm(row[1], R11)), fm(row[2], R21)), sv);
    }
    const float zmin = fs(c[2], __fsqrt_rn(fm(p.cut, fa(fm(a[2], a[2]), fm(b[2], b[2])))));
    if (!(zmin > p.znear)) return false;
    float T[3][3];
    const float *col[3] = {a, b, c};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T[0][j] = fa(fm(cam.fx, col[j][0]), fm(cam.cx, col[j][2]));
        T[1][j] = fa(fm(cam.fy, col[j][1]), fm(cam.cy, col[j][2]));
        T[2][j] = col[j][2];
    }
    float Cs[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = 0; s < 3; ++s)
            Cs[r][s] = fs(fa(fm(T[r][0], T[s][0]), fm(T[r][1], T[s][1])), fdv(fm(T[r][2], T[s][2]), p.cut));
    const float ex = __fsqrt_rn(fmaxf(0.f, fs(fm(Cs[0][2], Cs[0][2]), fm(Cs[0][0], Cs[2][2]))));
    const float ey = __fsqrt_rn(fmaxf(0.f, fs(fm(Cs[1][2], Cs[1][2]), fm(Cs[1][1], Cs[2][2]))));
    const float xa = fdv(fs(Cs[0][2], ex), Cs[2][2]), xb = fdv(fa(Cs[0][2], ex), Cs[2][2]);
    const float ya = fdv(fs(Cs[1][2], ey), Cs[2][2]), yb = fdv(fa(Cs[1][2], ey), Cs[2][2]);
    float x0 = fminf(xa, xb), x1 = fmaxf(xa, xb), y0 = fminf(ya, yb), y1 = fmaxf(ya, yb);
    if (!isfinite(x0) || !isfinite(x1) || !isfinite(y0) || !isfinite(y1)) return false;
    const float pad = fa(fm(fmaxf(fs(x1, x0), fs(y1, y0)), 0.015625f), 0.5f);
    x0 = fs(x0, pad);
    x1 = fa(x1, pad);
    y0 = fs(y0, pad);
    y1 = fa(y1, pad);
    const float Wf = (float)cam.W, Hf = (float)cam.H;
    float xlo = ceilf(fs(x0, 0.5f)), xhi = floorf(fs(x1, 0.5f));
    float ylo = ceilf(fs(y0, 0.5f)), yhi = floorf(fs(y1, 0.5f));
    xlo = fmaxf(xlo, 0.f);
    ylo = fmaxf(ylo, 0.f);
    xhi = fminf(xhi, fs(Wf, 1.f));
    yhi = fminf(yhi, fs(Hf, 1.f));
    if (xlo > xhi || ylo > yhi) return false;
    const int ix0 = (int)xlo, ix1 = (int)xhi, iy0 = (int)ylo, iy1 = (int)yhi;
    trect = make_int4(ix0 / kTile, iy0 / kTile, ix1 / kTile, iy1 / kTile);
    ntiles = (uint32_t)((trect.z - trect.x + 1) * (trect.w - trect.y + 1));
    depth = c[2];
    return true;
}

// The surfel's camera frame in binary64: c = W p + t, a = s_u W R[:,0],
// b = s_v W R[:,1] (R from the normalised quaternion).
struct Frame64 {
    double c[3], a[3], b[3];
};

__device__ Frame64 frame64(const float mu[3], float su, float sv, float4 q, const DevCam &cam) {
    const double qw = q.x, qx = q.y, qy = q.z, qz = q.w;
    const double nq = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
    const double w = qw / nq, x = qx / nq, y = qy / nq, z = qz / nq;
    const double R00 = 1.0 - 2.0 * (y * y + z * z), R10 = 2.0 * (x * y + w * z), R20 = 2.0 * (x * z - w * y);
    const double R01 = 2.0 * (x * y - w * z), R11 = 1.0 - 2.0 * (x * x + z * z), R21 = 2.0 * (y * z + w * x);
    Frame64 f;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const double r0 = cam.R[3 * r], r1 = cam.R[3 * r + 1], r2 = cam.R[3 * r + 2];
        f.c[r] = r0 * (double)mu[0] + r1 * (double)mu[1] + r2 * (double)mu[2] + (double)cam.t[r];
        f.a[r] = (r0 * R00 + r1 * R10 + r2 * R20) * (double)su;
        f.b[r] = (r0 * R01 + r1 * R11 + r2 * R21) * (double)sv;
    }
    return f;
}

// Projection of one (camera, surfel): binning values, the render record and
// the SH colour (dir = normalise(p - camera centre), rgb = max(0, sum + 1/2)).
__global__ void __launch_bounds__(256) k_project_surfel(const float *__restrict__ means,
                                                        const float *__restrict__ scales,
                                                        const float4 *__restrict__ quats,
                                                        const float *__restrict__ opac, const float *__restrict__ sh,
                                                        long long N, CamSet cs, Params p, ProjView pv,
                                                        unsigned *status) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)cs.n * N) return;
    const int ci = (int)(e / N);
    const long long g = e - (long long)ci * N;
    const DevCam &cam = cs.c[ci];
    const float mu[3] = {means[3 * g], means[3 * g + 1], means[3 * g + 2]};
    const float su = scales[3 * g], sv = scales[3 * g + 1];
    const float4 q = quats[g];
    const float op = opac[g];
    bool finite = isfinite(mu[0]) && isfinite(mu[1]) && isfinite(mu[2]) && isfinite(su) && isfinite(sv) &&
                  isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(q.w) && isfinite(op);
    const float *shg = sh + (long long)3 * p.K * g;
    float col[3] = {0.f, 0.f, 0.f};
    if (finite) {
        float Y[16];
        const float v0 = mu[0] - cam.campos[0], v1 = mu[1] - cam.campos[1], v2 = mu[2] - cam.campos[2];
        const float inv = rsqrtf(v0 * v0 + v1 * v1 + v2 * v2);
        sh_basis(v0 * inv, v1 * inv, v2 * inv, p.K, Y);
        for (int k = 0; k < p.K; ++k) {
            const float c0 = shg[3 * k], c1 = shg[3 * k + 1], c2 = shg[3 * k + 2];
            finite = finite && isfinite(c0) && isfinite(c1) && isfinite(c2);
            col[0] += c0 * Y[k];
            col[1] += c1 * Y[k];
            col[2] += c2 * Y[k];
        }
    }
    int4 tr = make_int4(-1, -1, -1, -1);
    uint32_t nt = 0;
    float depth = 0.f;
    bool ok = false;
    if (finite) ok = surfel_bin_spec(mu, su, sv, q, cam, p, tr, nt, depth);
    else if (ci == 0) latch(status, ST_NUMERIC);
    // record: M = T'^-1 in binary64, rounded once; M22 = -1 renders nothing
    float xc = 0.f, yc = 0.f, M00 = 0.f, M01 = 0.f, M10 = 0.f, M11 = 0.f, M20 = 0.f, M21 = 0.f, M22 = -1.f;
    if (ok) {
        const Frame64 f = frame64(mu, su, sv, q, cam);
        const double cz = f.c[2], xi = f.c[0] / cz, eta = f.c[1] / cz;
        const double fx = cam.fx, fy = cam.fy;
        const double A00 = fx * (f.a[0] - xi * f.a[2]), A01 = fx * (f.b[0] - xi * f.b[2]);
        const double A10 = fy * (f.a[1] - eta * f.a[2]), A11 = fy * (f.b[1] - eta * f.b[2]);
        const double det = A00 * A11 - A01 * A10;
        if (det != 0.0 && isfinite(det)) {
            const double B00 = A11 / det, B01 = -A01 / det, B10 = -A10 / det, B11 = A00 / det;
            M00 = (float)B00;
            M01 = (float)B01;
            M10 = (float)B10;
            M11 = (float)B11;
            M20 = (float)(-(f.a[2] * B00 + f.b[2] * B10) / cz);
            M21 = (float)(-(f.a[2] * B01 + f.b[2] * B11) / cz);
            M22 = (float)(1.0 / cz);
            xc = (float)(fx * xi + (double)cam.cx);
            yc = (float)(fy * eta + (double)cam.cy);
        }
    }
    unsigned mask = 0;
    float rgb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float raw = col[c] + 0.5f;
        mask |= (raw > 0.f ? 1u : 0u) << c;
        rgb[c] = fmaxf(raw, 0.f);
    }
    SRec r;
    r.a = make_float4(xc, yc, M00, M01);
    r.b = make_float4(M10, M11, M20, M21);
    r.c = make_float4(M22, op, rgb[0], rgb[1]);
    r.d = make_float4(rgb[2], depth, __uint_as_float(mask), 0.f);
    pv.srec[e] = r;
    pv.trect[e] = tr;
    pv.ntiles[e] = ok ? nt : 0u;
    pv.dkey[e] = ok ? __float_as_uint(depth) : 0xFFFFFFFFu;
}

// ------------------------------------------------------------------ render
template <int BF16>
__device__ __forceinline__ void load8(const void *feats, int D, uint32_t g, int c, float *dst) {
    if (c >= D) {
#pragma unroll
        for (int i = 0; i < 8; ++i) dst[i] = 0.f;
        return;
    }
    if (BF16) {
        const uint4 v = *reinterpret_cast<const uint4 *>(reinterpret_cast<const __nv_bfloat16 *>(feats) +
                                                          (size_t)g * D + c);
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 f = __bfloat1622float2(h[i]);
            dst[2 * i] = f.x;
            dst[2 * i + 1] = f.y;
        }
    } else {
        const float4 *q = reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(feats) + (size_t)g * D + c);
        const float4 a = q[0], b = q[1];
        dst[0] = a.x; dst[1] = a.y; dst[2] = a.z; dst[3] = a.w;
        dst[4] = b.x; dst[5] = b.y; dst[6] = b.z; dst[7] = b.w;
    }
}

struct TileCtx {
    int ci, px, py;
    bool inside;
    long long pix;
    uint32_t s, e;
};

__device__ __forceinline__ TileCtx tile_ctx(const CamSet &cs, const uint32_t *ranges) {
    TileCtx t;
    const int tile = blockIdx.x;
    t.ci = cam_of_tile(cs, tile);
    const DevCam &cam = cs.c[t.ci];
    const int lt = tile - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    t.px = tx * kTile + (threadIdx.x & 15);
    t.py = ty * kTile + (threadIdx.x >> 4);
    t.inside = t.px < cam.W && t.py < cam.H;
    t.pix = cam.pix_off + (long long)t.py * cam.W + t.px;
    t.s = ranges[2 * tile];
    t.e = ranges[2 * tile + 1];
    return t;
}

// Forward (Eq. 4), one 256-thread block per (16x16 tile, 32-channel feature
// chunk), one pixel per thread, records and the feature chunk staged 64
// surfels at a time; the block leaves once every pixel has stopped.
template <int BF16>
__global__ void __launch_bounds__(256) k_render_fwd_surfel(long long N, CamSet cs, Params p, ProjView pv,
                                                           const uint32_t *__restrict__ gids,
                                                           const uint32_t *__restrict__ ranges, const void *feats,
                                                           int D, float *rgb, float *feat, float *Tout,
                                                           int32_t *last_out) {
    __shared__ float4 sa[kB], sb[kB], sc[kB];
    __shared__ float sbl[kB];
    __shared__ float sf[kB][kDC];
    const TileCtx tc = tile_ctx(cs, ranges);
    const int chunk = blockIdx.y, c0 = chunk * kDC;
    const bool has_feat = D > 0 && feat != nullptr;
    const SRec *rec = pv.srec + (long long)tc.ci * N;
    const float fpx = tc.px + 0.5f, fpy = tc.py + 0.5f;
    float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, acc[kDC];
#pragma unroll
    for (int c = 0; c < kDC; ++c) acc[c] = 0.f;
    int last = 0;
    bool done = !tc.inside;
    for (uint32_t base = tc.s; base < tc.e; base += kB) {
        if (__syncthreads_and(done)) break;
        const int nb = (int)min((uint32_t)kB, tc.e - base);
        if ((int)threadIdx.x < nb) {
            const SRec r = rec[gids[base + threadIdx.x]];
            sa[threadIdx.x] = r.a;
            sb[threadIdx.x] = r.b;
            sc[threadIdx.x] = r.c;
            sbl[threadIdx.x] = r.d.x;
        }
        if (has_feat) {
            const int row = threadIdx.x >> 2, part = threadIdx.x & 3;
            if (row < nb) load8<BF16>(feats, D, gids[base + row], c0 + part * 8, &sf[row][part * 8]);
        }
        __syncthreads();
        if (!done) {
            for (int j = 0; j < nb; ++j) {
                const float4 C = sc[j];
                SurfelHit h;
                if (!surfel_uv(sa[j], sb[j], C.x, fpx, fpy, p.cut, h)) continue;
                const float a = fminf(p.amax, C.y * __expf(-0.5f * h.r2));
                if (a < p.amin) continue;
                const float Tn = T * (1.f - a);
                if (Tn < p.teps) {
                    done = true;
                    break;
                }
                const float w = a * T;
                cr += w * C.z;
                cg += w * C.w;
                cb += w * sbl[j];
                if (has_feat) {
#pragma unroll
                    for (int c = 0; c < kDC; ++c) acc[c] += w * sf[j][c];
                }
                T = Tn;
                last = (int)(base - tc.s) + j + 1;
            }
        }
    }
    if (!tc.inside) return;
    if (chunk == 0) {
        rgb[3 * tc.pix + 0] = cr + T * p.bg0;
        rgb[3 * tc.pix + 1] = cg + T * p.bg1;
        rgb[3 * tc.pix + 2] = cb + T * p.bg2;
        Tout[tc.pix] = T;
        last_out[tc.pix] = last;
    }
    if (has_feat) {
        float4 *dst = reinterpret_cast<float4 *>(feat + tc.pix * D + c0);
#pragma unroll
        for (int c = 0; c < kDC; c += 4)
            if (c0 + c < D) dst[c / 4] = make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
    }
}

// Sum 32 per-lane vectors over the warp; afterwards lane l holds the total
// of component l in v[0].
__device__ __forceinline__ void warp_reduce_scatter32(float *v, int lane) {
#pragma unroll
    for (int half = 16; half >= 1; half >>= 1) {
        const bool upper = (lane & half) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? v[i] : v[i + half];
            const float keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, half);
        }
    }
}

// Sum 16 per-lane values over the warp; afterwards lanes 2k and 2k + 1 both
// hold the total of component k in v[0] (16 shuffles).
__device__ __forceinline__ void warp_reduce_scatter16(float *v, int lane) {
#pragma unroll
    for (int half = 8, off = 16; half >= 1; half >>= 1, off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? v[i] : v[i + half];
            const float keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Backward (App. A.2), back to front per pixel: T_i = T_{i+1} / (1 -
// alpha_i) from T_final, dL/dalpha_i = T_i g_i - S_i / (1 - alpha_i) with
// g_i = dC.c_i + dF.f_i (each feature chunk adds its share; the colour part
// and the background term belong to chunk 0), then through alpha = min(
// alpha_max, op G(u, v)) and u = (M00 dx + M01 dy) / w, v = (M10 dx + M11
// dy) / w, w = M20 dx + M21 dy + M22 to the 13 per-(camera, surfel) values
// d(x_c, y_c, M00, M01, M10, M11, M20, M21, M22, opacity, r, g, b), reduced
// over the warp before one atomic per value.
template <int BF16>
__global__ void __launch_bounds__(256) k_render_bwd_surfel(long long N, CamSet cs, Params p, ProjView pv,
                                                           const uint32_t *__restrict__ gids,
                                                           const uint32_t *__restrict__ ranges, const void *feats,
                                                           int D, const float *__restrict__ Tfin,
                                                           const int32_t *__restrict__ lastv,
                                                           const float *__restrict__ grgb,
                                                           const float *__restrict__ gfeat, float *g2d,
                                                           float *gfeatures) {
    __shared__ float4 sa[kB], sb[kB], sc[kB];
    __shared__ float sbl[kB];
    __shared__ uint32_t sg[kB];
    __shared__ float sf[kB][kDC];
    __shared__ int smax;
    const TileCtx tc = tile_ctx(cs, ranges);
    const int chunk = blockIdx.y, c0 = chunk * kDC;
    const int lane = threadIdx.x & 31;
    const bool has_feat = D > 0;
    const bool feat_grad = has_feat && gfeatures != nullptr;
    const SRec *rec = pv.srec + (long long)tc.ci * N;
    float *g2dc = g2d + (long long)tc.ci * N * kSurfelG2d;
    const float fpx = tc.px + 0.5f, fpy = tc.py + 0.5f;
    float T = 1.f, dC0 = 0.f, dC1 = 0.f, dC2 = 0.f, dF[kDC];
    int lastp = 0;
#pragma unroll
    for (int c = 0; c < kDC; ++c) dF[c] = 0.f;
    if (tc.inside) {
        T = Tfin[tc.pix];
        lastp = lastv[tc.pix];
        if (chunk == 0) {
            dC0 = grgb[3 * tc.pix];
            dC1 = grgb[3 * tc.pix + 1];
            dC2 = grgb[3 * tc.pix + 2];
        }
        if (has_feat && gfeat) {
            const float4 *src = reinterpret_cast<const float4 *>(gfeat + tc.pix * D + c0);
#pragma unroll
            for (int c = 0; c < kDC; c += 4)
                if (c0 + c < D) {
                    const float4 v = src[c / 4];
                    dF[c] = v.x; dF[c + 1] = v.y; dF[c + 2] = v.z; dF[c + 3] = v.w;
                }
        }
    }
    if (threadIdx.x == 0) smax = 0;
    __syncthreads();
    atomicMax(&smax, lastp);
    __syncthreads();
    const int Lmax = min(smax, (int)(tc.e - tc.s));  // a stale `last` cannot index past the list
    float S = T * (dC0 * p.bg0 + dC1 * p.bg1 + dC2 * p.bg2);
    for (int bend = Lmax; bend > 0; bend -= kB) {
        const int bstart = max(0, bend - kB), nb = bend - bstart;
        __syncthreads();
        if ((int)threadIdx.x < nb) {
            const uint32_t g = gids[tc.s + bstart + threadIdx.x];
            const SRec r = rec[g];
            sa[threadIdx.x] = r.a;
            sb[threadIdx.x] = r.b;
            sc[threadIdx.x] = r.c;
            sbl[threadIdx.x] = r.d.x;
            sg[threadIdx.x] = g;
        }
        if (has_feat) {
            const int row = threadIdx.x >> 2, part = threadIdx.x & 3;
            if (row < nb) load8<BF16>(feats, D, gids[tc.s + bstart + row], c0 + part * 8, &sf[row][part * 8]);
        }
        __syncthreads();
        for (int j = nb - 1; j >= 0; --j) {
            const float4 A = sa[j], B = sb[j], C = sc[j];
            SurfelHit h;
            bool contrib = false;
            float a = 0.f, G = 0.f, rho = 0.f;
            if (bstart + j < lastp && surfel_uv(A, B, C.x, fpx, fpy, p.cut, h)) {
                G = __expf(-0.5f * h.r2);
                rho = C.y * G;
                a = fminf(p.amax, rho);
                contrib = a >= p.amin;
            }
            if (!__any_sync(0xffffffffu, contrib)) continue;
            float v[kDC];
            float geo[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) geo[k] = 0.f;
#pragma unroll
            for (int c = 0; c < kDC; ++c) v[c] = 0.f;
            if (contrib) {
                const float oma = 1.f - a;
                T = T / oma;
                const float w = a * T;
                float gdot = dC0 * C.z + dC1 * C.w + dC2 * sbl[j];
                if (has_feat) {
#pragma unroll
                    for (int c = 0; c < kDC; ++c) gdot += dF[c] * sf[j][c];
                }
                const float dal = T * gdot - S / oma;
                S += w * gdot;
                if (feat_grad) {
#pragma unroll
                    for (int c = 0; c < kDC; ++c) v[c] = w * dF[c];
                }
                const float drho = rho > p.amax ? 0.f : dal;
                const float dr2 = -0.5f * rho * drho;            // rho = op exp(-r2 / 2)
                const float du = 2.f * h.u * dr2, dv = 2.f * h.v * dr2;
                const float dnu = du * h.iw, dnv = dv * h.iw;    // u = nu / w, v = nv / w
                const float dw = -(du * h.u + dv * h.v) * h.iw;
                const float ddx = dnu * A.z + dnv * B.x + dw * B.z;
                const float ddy = dnu * A.w + dnv * B.y + dw * B.w;
                geo[0] = -ddx;  // x_c
                geo[1] = -ddy;  // y_c
                geo[2] = dnu * h.dx;
                geo[3] = dnu * h.dy;
                geo[4] = dnv * h.dx;
                geo[5] = dnv * h.dy;
                geo[6] = dw * h.dx;
                geo[7] = dw * h.dy;
                geo[8] = dw;
                geo[9] = G * drho;
                geo[10] = w * dC0;
                geo[11] = w * dC1;
                geo[12] = w * dC2;
            }
            const uint32_t g = sg[j];
            if (feat_grad) {
                warp_reduce_scatter32(v, lane);
                if (c0 + lane < D) atomicAdd(gfeatures + (size_t)g * D + c0 + lane, v[0]);
            }
            warp_reduce_scatter16(geo, lane);
            const int k = lane >> 1;
            const int ngeo = chunk == 0 ? 13 : 10;
            if (!(lane & 1) && k < ngeo) atomicAdd(g2dc + (long long)kSurfelG2d * g + k, geo[0]);
        }
    }
}

// ---------------------------------------------------------- projection bwd
// Chain rule from the 13 per-(camera, surfel) values of the render backward
// to means, (s_u, s_v), quaternions, opacities and SH, summed over cameras.
// With B = A^-1 (the record's top-left block), (M20, M21) = -(a_z, b_z) B /
// c_z and M22 = 1 / c_z: dL/dA = -B^T dL/dB B^T, then A, x_c = fx xi + cx
// and y_c = fy eta + cy back to c, a, b, and c = W p + t, a = s_u W R[:,0],
// b = s_v W R[:,1] back to p, s and R(q).  One thread per surfel.
__global__ void __launch_bounds__(128) k_project_surfel_bwd(const float *__restrict__ means,
                                                            const float *__restrict__ scales,
                                                            const float4 *__restrict__ quats,
                                                            const float *__restrict__ sh, long long N, CamSet cs,
                                                            Params p, ProjView pv, const float *__restrict__ g2d,
                                                            float *gmeans, float *gscales, float *gquats, float *gopac,
                                                            float *gsh) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = g < N;
    const int K = p.K;
    float gmu[3] = {0.f, 0.f, 0.f}, gsu = 0.f, gsv = 0.f, gq[4] = {0.f, 0.f, 0.f, 0.f}, gop = 0.f;
    float gshv[48];
#pragma unroll
    for (int i = 0; i < 48; ++i) gshv[i] = 0.f;
    bool touched = false;
    for (int ci = 0; ci < cs.n && valid && !touched; ++ci) {
        const long long e = (long long)ci * N + g;
        if (pv.ntiles[e] == 0) continue;
        const float *gg = g2d + (long long)kSurfelG2d * e;
        for (int k = 0; k < 13 && !touched; ++k) touched = gg[k] != 0.f;
    }
    if (touched) {
        const float mu[3] = {means[3 * g], means[3 * g + 1], means[3 * g + 2]};
        const float su = scales[3 * g], sv = scales[3 * g + 1];
        const float4 q4 = quats[g];
        const float *shg = sh + (long long)3 * K * g;
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
        float GR[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        for (int ci = 0; ci < cs.n; ++ci) {
            const long long e = (long long)ci * N + g;
            if (pv.ntiles[e] == 0) continue;
            const float *gg = g2d + (long long)kSurfelG2d * e;
            float d[13];
#pragma unroll
            for (int k = 0; k < 13; ++k) d[k] = gg[k];
            const SRec rec = pv.srec[e];
            const DevCam &cam = cs.c[ci];
            gop += d[9];
            // the surfel frame in this camera
            float c[3], ru[3], rv[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const float *row = cam.R + 3 * r;
                c[r] = row[0] * mu[0] + row[1] * mu[1] + row[2] * mu[2] + cam.t[r];
                ru[r] = row[0] * R[0][0] + row[1] * R[1][0] + row[2] * R[2][0];
                rv[r] = row[0] * R[0][1] + row[1] * R[1][1] + row[2] * R[2][1];
            }
            const float az = su * ru[2], bz = sv * rv[2];
            const float cz = c[2], icz = 1.f / cz, xi = c[0] * icz, eta = c[1] * icz;
            const float B00 = rec.a.z, B01 = rec.a.w, B10 = rec.b.x, B11 = rec.b.y;
            const float m0 = rec.b.z, m1 = rec.b.w;
            float G00 = d[2], G01 = d[3], G10 = d[4], G11 = d[5];
            const float gm0 = d[6], gm1 = d[7], g22 = d[8];
            // (M20, M21) = -(a_z, b_z) B / c_z and M22 = 1 / c_z
            const float dr0 = -(B00 * gm0 + B01 * gm1) * icz;
            const float dr1 = -(B10 * gm0 + B11 * gm1) * icz;
            G00 -= az * gm0 * icz;
            G01 -= az * gm1 * icz;
            G10 -= bz * gm0 * icz;
            G11 -= bz * gm1 * icz;
            float dcz = -(m0 * gm0 + m1 * gm1) * icz - g22 * icz * icz;
            // B = A^-1: dL/dA = -B^T dL/dB B^T
            const float P00 = G00 * B00 + G01 * B01, P01 = G00 * B10 + G01 * B11;
            const float P10 = G10 * B00 + G11 * B01, P11 = G10 * B10 + G11 * B11;
            const float dA00 = -(B00 * P00 + B10 * P10), dA01 = -(B00 * P01 + B10 * P11);
            const float dA10 = -(B01 * P00 + B11 * P10), dA11 = -(B01 * P01 + B11 * P11);
            const float fx = cam.fx, fy = cam.fy;
            float da[3], db[3];
            da[0] = fx * dA00;
            db[0] = fx * dA01;
            da[1] = fy * dA10;
            db[1] = fy * dA11;
            da[2] = -fx * xi * dA00 - fy * eta * dA10 + dr0;
            db[2] = -fx * xi * dA01 - fy * eta * dA11 + dr1;
            const float dxi = -fx * (az * dA00 + bz * dA01) + fx * d[0];
            const float deta = -fy * (az * dA10 + bz * dA11) + fy * d[1];
            const float dc[3] = {dxi * icz, deta * icz, dcz - (dxi * xi + deta * eta) * icz};
            // c = W p + t, a = s_u W R[:,0], b = s_v W R[:,1]
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                gmu[k] += cam.R[k] * dc[0] + cam.R[3 + k] * dc[1] + cam.R[6 + k] * dc[2];
                const float wa = cam.R[k] * da[0] + cam.R[3 + k] * da[1] + cam.R[6 + k] * da[2];
                const float wb = cam.R[k] * db[0] + cam.R[3 + k] * db[1] + cam.R[6 + k] * db[2];
                GR[k][0] += su * wa;
                GR[k][1] += sv * wb;
            }
            gsu += ru[0] * da[0] + ru[1] * da[1] + ru[2] * da[2];
            gsv += rv[0] * db[0] + rv[1] * db[1] + rv[2] * db[2];
            // SH colour
            const unsigned mask = __float_as_uint(rec.d.z);
            const float graw[3] = {(mask & 1u) ? d[10] : 0.f, (mask & 2u) ? d[11] : 0.f, (mask & 4u) ? d[12] : 0.f};
            const float v0 = mu[0] - cam.campos[0], v1 = mu[1] - cam.campos[1], v2 = mu[2] - cam.campos[2];
            const float inv = rsqrtf(v0 * v0 + v1 * v1 + v2 * v2);
            const float ux = v0 * inv, uy = v1 * inv, uz = v2 * inv;
            float Y[16], sk[16], gd[3] = {0.f, 0.f, 0.f};
            sh_basis(ux, uy, uz, K, Y);
            for (int k = 0; k < K; ++k) {
                sk[k] = 0.f;
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    gshv[3 * k + cc] += Y[k] * graw[cc];
                    sk[k] += shg[3 * k + cc] * graw[cc];
                }
            }
            sh_basis_grad(ux, uy, uz, K, sk, gd);
            const float dd = ux * gd[0] + uy * gd[1] + uz * gd[2];
            gmu[0] += (gd[0] - ux * dd) * inv;
            gmu[1] += (gd[1] - uy * dd) * inv;
            gmu[2] += (gd[2] - uz * dd) * inv;
        }
        // R(q) from the normalised quaternion, then the normalisation
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
    if (!valid) return;
    gmeans[3 * g] = gmu[0];
    gmeans[3 * g + 1] = gmu[1];
    gmeans[3 * g + 2] = gmu[2];
    gscales[3 * g] = gsu;
    gscales[3 * g + 1] = gsv;
    gscales[3 * g + 2] = 0.f;
    reinterpret_cast<float4 *>(gquats)[g] = make_float4(gq[0], gq[1], gq[2], gq[3]);
    gopac[g] = gop;
    float *dst = gsh + (long long)3 * K * g;
    for (int i = 0; i < 3 * K; ++i) dst[i] = gshv[i];
}

}  // namespace

void launch_project_surfel(const fhgs_gaussians &g, const CamSet &cs, const Params &p, ProjView pv, unsigned *status,
                           cudaStream_t st) {
    const long long total = (long long)cs.n * g.n;
    if (total == 0) return;
    note_launch(1);
    k_project_surfel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
        g.means, g.scales, reinterpret_cast<const float4 *>(g.quats), g.opacities, g.sh, g.n, cs, p, pv, status);
}

void launch_render_fwd_surfel(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                              const void *feats, int bf16, int D, float *rgb, float *feat, float *T, int32_t *last,
                              cudaStream_t st) {
    const int nchunk = (feat && D > 0) ? (D + kDC - 1) / kDC : 1;
    dim3 grid(cs.total_tiles, nchunk);
    note_launch(1);
    if (bf16)
        k_render_fwd_surfel<1><<<grid, 256, 0, st>>>(N, cs, p, pv, bins.gids, bins.ranges, feats, D, rgb, feat, T,
                                                     last);
    else
        k_render_fwd_surfel<0><<<grid, 256, 0, st>>>(N, cs, p, pv, bins.gids, bins.ranges, feats, D, rgb, feat, T,
                                                     last);
}

void launch_render_bwd_surfel(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                              const void *feats, int bf16, int D, const float *T, const int32_t *last,
                              const float *grgb, const float *gfeat, float *g2d, float *gfeatures, cudaStream_t st) {
    const bool feats_used = D > 0 && (gfeat != nullptr || gfeatures != nullptr);
    const int nchunk = feats_used ? (D + kDC - 1) / kDC : 1;
    const int Dk = feats_used ? D : 0;
    dim3 grid(cs.total_tiles, nchunk);
    note_launch(1);
    if (bf16)
        k_render_bwd_surfel<1><<<grid, 256, 0, st>>>(N, cs, p, pv, bins.gids, bins.ranges, feats, Dk, T, last, grgb,
                                                     gfeat, g2d, gfeatures);
    else
        k_render_bwd_surfel<0><<<grid, 256, 0, st>>>(N, cs, p, pv, bins.gids, bins.ranges, feats, Dk, T, last, grgb,
                                                     gfeat, g2d, gfeatures);
}

void launch_project_surfel_bwd(const fhgs_gaussians &g, const CamSet &cs, const Params &p, ProjView pv,
                               const float *g2d, float *gmeans, float *gscales, float *gquats, float *gop,
                               float *gsh, cudaStream_t st) {
    if (g.n == 0) return;
    note_launch(1);
    k_project_surfel_bwd<<<(unsigned)((g.n + 127) / 128), 128, 0, st>>>(
        g.means, g.scales, reinterpret_cast<const float4 *>(g.quats), g.sh, g.n, cs, p, pv, g2d, gmeans, gscales,
        gquats, gop, gsh);
}

}  // namespace fhgs
