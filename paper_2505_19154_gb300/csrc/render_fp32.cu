// Plain FP32 per-pixel compositing on the CUDA cores (the baseline path) and
// the multi-view feature fusion.
//
// One 256-thread block per (16x16 tile, 32-channel feature chunk); each
// thread owns one pixel and walks the tile's depth-sorted list front to back
// (Eq. 4), keeping its 32 feature accumulators in registers.  Gaussian records
// and their feature chunk are staged in shared memory, 64 at a time; the
// block leaves the list as soon as every pixel's transmittance has hit the
// stop rule (__syncthreads_and).  The backward walks back to front (App. A.2),
// recovering T_i = T_{i+1} / (1 - alpha_i) from the stored T_final, and
// decomposes dL/dalpha over feature chunks: with g_i = dC.c_i + sum_chunks
// dF_chunk.f_i,chunk the App. A.2 expression is linear in g, so each chunk
// block adds its own share of the footprint gradients.  Per-Gaussian
// gradients are reduced over the warp with shuffles before one global atomic.
#include "fhgs_internal.cuh"

namespace fhgs {
namespace {

constexpr int kB = 64;   // Gaussians per shared-memory batch
constexpr int kDC = 32;  // feature channels per block

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
        const float4 *p = reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(feats) + (size_t)g * D + c);
        const float4 a = p[0], b = p[1];
        dst[0] = a.x; dst[1] = a.y; dst[2] = a.z; dst[3] = a.w;
        dst[4] = b.x; dst[5] = b.y; dst[6] = b.z; dst[7] = b.w;
    }
}

// Sum 32 per-lane vectors over the warp; afterwards lane l holds the total
// of component l in v[0] (31 shuffles instead of 32 x 5).
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

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
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

template <int BF16>
__global__ void __launch_bounds__(256) k_render_fwd_fp32(long long N, CamSet cs, Params p, ProjView pv,
                                                         const uint32_t *__restrict__ gids,
                                                         const uint32_t *__restrict__ ranges, const void *feats,
                                                         int D, float *rgb, float *feat, float *Tout,
                                                         int32_t *last_out) {
    __shared__ float4 sa[kB], sb[kB];
    __shared__ float sbl[kB];
    __shared__ float sf[kB][kDC];
    const TileCtx tc = tile_ctx(cs, ranges);
    const int chunk = blockIdx.y, c0 = chunk * kDC;
    const bool has_feat = D > 0 && feat != nullptr;
    const GRec *rec = pv.rec + (long long)tc.ci * N;
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
            const GRec r = rec[gids[base + threadIdx.x]];
            sa[threadIdx.x] = r.a;
            sb[threadIdx.x] = r.b;
            sbl[threadIdx.x] = r.c.x;
        }
        if (has_feat) {
            const int row = threadIdx.x >> 2, part = threadIdx.x & 3;
            if (row < nb) load8<BF16>(feats, D, gids[base + row], c0 + part * 8, &sf[row][part * 8]);
        }
        __syncthreads();
        if (!done) {
            for (int j = 0; j < nb; ++j) {
                const float4 A = sa[j], B = sb[j];
                const float dx = fpx - A.x, dy = fpy - A.y;
                const float q2 = eval_q2(dx, dy, A.z, A.w, B.x);
                if (q2 > p.cut) continue;
                const float a = fminf(p.amax, B.y * __expf(-0.5f * q2));
                if (a < p.amin) continue;
                const float Tn = T * (1.f - a);
                if (Tn < p.teps) {
                    done = true;
                    break;
                }
                const float w = a * T;
                cr += w * B.z;
                cg += w * B.w;
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

template <int BF16>
__global__ void __launch_bounds__(256) k_render_bwd_fp32(long long N, CamSet cs, Params p, ProjView pv,
                                                         const uint32_t *__restrict__ gids,
                                                         const uint32_t *__restrict__ ranges, const void *feats,
                                                         int D, const float *__restrict__ Tfin,
                                                         const int32_t *__restrict__ lastv,
                                                         const float *__restrict__ grgb,
                                                         const float *__restrict__ gfeat, float *g2d,
                                                         float *gfeatures) {
    __shared__ float4 sa[kB], sb[kB];
    __shared__ float sbl[kB];
    __shared__ uint32_t sg[kB];
    __shared__ float sf[kB][kDC];
    __shared__ int smax;
    const TileCtx tc = tile_ctx(cs, ranges);
    const int chunk = blockIdx.y, c0 = chunk * kDC;
    const int lane = threadIdx.x & 31;
    const bool has_feat = D > 0;
    const bool feat_grad = has_feat && gfeatures != nullptr;
    const GRec *rec = pv.rec + (long long)tc.ci * N;
    float *g2dc = g2d + (long long)tc.ci * N * 12;
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
            const GRec r = rec[g];
            sa[threadIdx.x] = r.a;
            sb[threadIdx.x] = r.b;
            sbl[threadIdx.x] = r.c.x;
            sg[threadIdx.x] = g;
        }
        if (has_feat) {
            const int row = threadIdx.x >> 2, part = threadIdx.x & 3;
            if (row < nb) load8<BF16>(feats, D, gids[tc.s + bstart + row], c0 + part * 8, &sf[row][part * 8]);
        }
        __syncthreads();
        for (int j = nb - 1; j >= 0; --j) {
            const float4 A = sa[j], B = sb[j];
            const float dx = fpx - A.x, dy = fpy - A.y;
            bool contrib = false;
            float a = 0.f, G = 0.f, rho = 0.f;
            if (bstart + j < lastp) {
                const float q2 = eval_q2(dx, dy, A.z, A.w, B.x);
                if (q2 <= p.cut) {
                    G = __expf(-0.5f * q2);
                    rho = B.y * G;
                    a = fminf(p.amax, rho);
                    contrib = a >= p.amin;
                }
            }
            if (!__any_sync(0xffffffffu, contrib)) continue;
            float v[kDC];
            float geo[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) geo[k] = 0.f;
#pragma unroll
            for (int c = 0; c < kDC; ++c) v[c] = 0.f;
            if (contrib) {
                const float oma = 1.f - a;
                T = T / oma;
                const float w = a * T;
                float gdot = dC0 * B.z + dC1 * B.w + dC2 * sbl[j];
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
                const float dq2 = -0.5f * rho * drho;
                geo[0] = -(2.f * A.z * dx + 2.f * A.w * dy) * dq2;
                geo[1] = -(2.f * A.w * dx + 2.f * B.x * dy) * dq2;
                geo[2] = dx * dx * dq2;
                geo[3] = 2.f * dx * dy * dq2;
                geo[4] = dy * dy * dq2;
                geo[5] = G * drho;
                geo[6] = w * dC0;
                geo[7] = w * dC1;
                geo[8] = w * dC2;
            }
            const uint32_t g = sg[j];
            if (feat_grad) {
                warp_reduce_scatter32(v, lane);
                if (c0 + lane < D) atomicAdd(gfeatures + (size_t)g * D + c0 + lane, v[0]);
            }
            const int ngeo = chunk == 0 ? 9 : 6;
#pragma unroll
            for (int k = 0; k < 9; ++k)
                if (k < ngeo) geo[k] = warp_sum(geo[k]);
            if (lane == 0) {
                float4 *dst = reinterpret_cast<float4 *>(g2dc + 12 * (long long)g);
                atomicAdd(dst, make_float4(geo[0], geo[1], geo[2], geo[3]));
                atomicAdd(dst + 1, make_float4(geo[4], geo[5], geo[6], geo[7]));
                if (chunk == 0) atomicAdd(g2dc + 12 * (long long)g + 8, geo[8]);
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_fuse_fp32(long long N, CamSet cs, Params p, ProjView pv,
                                                   const uint32_t *__restrict__ gids,
                                                   const uint32_t *__restrict__ ranges,
                                                   const FuseMaps maps, int D, float *num, float *den) {
    __shared__ float4 sa[kB], sb[kB];
    __shared__ uint32_t sg[kB];
    const TileCtx tc = tile_ctx(cs, ranges);
    const int chunk = blockIdx.y, c0 = chunk * kDC;
    const int lane = threadIdx.x & 31;
    const GRec *rec = pv.rec + (long long)tc.ci * N;
    const float fpx = tc.px + 0.5f, fpy = tc.py + 0.5f;
    float F[kDC];
#pragma unroll
    for (int c = 0; c < kDC; ++c) F[c] = 0.f;
    if (tc.inside) {
        // each camera's map is its own [H*W, D] array
        const long long mp = (long long)tc.py * cs.c[tc.ci].W + tc.px;
        const float4 *src = reinterpret_cast<const float4 *>(maps.m[tc.ci] + mp * D + c0);
#pragma unroll
        for (int c = 0; c < kDC; c += 4)
            if (c0 + c < D) {
                const float4 v = src[c / 4];
                F[c] = v.x; F[c + 1] = v.y; F[c + 2] = v.z; F[c + 3] = v.w;
            }
    }
    float T = 1.f;
    bool done = !tc.inside;
    for (uint32_t base = tc.s; base < tc.e; base += kB) {
        if (__syncthreads_and(done)) break;
        const int nb = (int)min((uint32_t)kB, tc.e - base);
        if ((int)threadIdx.x < nb) {
            const uint32_t g = gids[base + threadIdx.x];
            const GRec r = rec[g];
            sa[threadIdx.x] = r.a;
            sb[threadIdx.x] = r.b;
            sg[threadIdx.x] = g;
        }
        __syncthreads();
        for (int j = 0; j < nb; ++j) {
            float w = 0.f;
            if (!done) {
                const float4 A = sa[j], B = sb[j];
                const float dx = fpx - A.x, dy = fpy - A.y;
                const float q2 = eval_q2(dx, dy, A.z, A.w, B.x);
                if (q2 <= p.cut) {
                    const float a = fminf(p.amax, B.y * __expf(-0.5f * q2));
                    if (a >= p.amin) {
                        const float Tn = T * (1.f - a);
                        if (Tn < p.teps) {
                            done = true;
                        } else {
                            w = a * T;
                            T = Tn;
                        }
                    }
                }
            }
            if (!__any_sync(0xffffffffu, w > 0.f)) continue;
            float v[kDC];
#pragma unroll
            for (int c = 0; c < kDC; ++c) v[c] = w * F[c];
            warp_reduce_scatter32(v, lane);
            const uint32_t g = sg[j];
            if (c0 + lane < D) atomicAdd(num + (size_t)g * D + c0 + lane, v[0]);
            if (chunk == 0) {
                const float ws = warp_sum(w);
                if (lane == 0) atomicAdd(den + g, ws);
            }
        }
    }
}

__global__ void k_fuse_finalize(long long N, int D, const float *__restrict__ num, const float *__restrict__ den,
                                float *out, int normalize) {
    const long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= N) return;
    const float d = den[g];
    const float inv = d > 0.f ? 1.f / d : 0.f;
    float ss = 0.f;
    for (int c = lane; c < D; c += 32) {
        const float v = num[g * D + c] * inv;
        ss += v * v;
    }
    float scale = inv;
    if (normalize) {
        ss = warp_sum(ss);
        scale = ss > 0.f ? inv * rsqrtf(ss) : 0.f;
    }
    for (int c = lane; c < D; c += 32) out[g * D + c] = d > 0.f ? num[g * D + c] * scale : 0.f;
}

}  // namespace

void launch_render_fwd_fp32(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                            const void *feats, int bf16, int D, float *rgb, float *feat, float *T, int32_t *last,
                            cudaStream_t st) {
    const int nchunk = (feat && D > 0) ? (D + kDC - 1) / kDC : 1;
    dim3 grid(cs.total_tiles, nchunk);
    note_launch(1);
    if (bf16)
        k_render_fwd_fp32<1><<<grid, 256, 0, st>>>(N, cs, p, pv, bins.gids, bins.ranges, feats, D, rgb, feat, T, last);
    else
        k_render_fwd_fp32<0><<<grid, 256, 0, st>>>(N, cs, p, pv, bins.gids, bins.ranges, feats, D, rgb, feat, T, last);
}

void launch_render_bwd_fp32(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                            const void *feats, int bf16, int D, const float *T, const int32_t *last,
                            const float *grgb, const float *gfeat, float *g2d, float *gfeatures, cudaStream_t st) {
    // a chunk block only has work if it carries feature gradient or input
    const bool feats_used = D > 0 && (gfeat != nullptr || gfeatures != nullptr);
    const int nchunk = feats_used ? (D + kDC - 1) / kDC : 1;
    const int Dk = feats_used ? D : 0;
    dim3 grid(cs.total_tiles, nchunk);
    note_launch(1);
    if (bf16)
        k_render_bwd_fp32<1><<<grid, 256, 0, st>>>(N, cs, p, pv, bins.gids, bins.ranges, feats, Dk, T, last, grgb,
                                                  gfeat, g2d, gfeatures);
    else
        k_render_bwd_fp32<0><<<grid, 256, 0, st>>>(N, cs, p, pv, bins.gids, bins.ranges, feats, Dk, T, last, grgb,
                                                  gfeat, g2d, gfeatures);
}

void launch_fuse_fp32(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                      const FuseMaps &maps, int D, float *num, float *den, cudaStream_t st) {
    dim3 grid(cs.total_tiles, (D + kDC - 1) / kDC);
    note_launch(1);
    k_fuse_fp32<<<grid, 256, 0, st>>>(N, cs, p, pv, bins.gids, bins.ranges, maps, D, num, den);
}

void launch_fuse_finalize(long long N, int D, const float *num, const float *den, float *out, int normalize,
                          cudaStream_t st) {
    if (N == 0) return;
    const long long threads = N * 32;
    note_launch(1);
    k_fuse_finalize<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(N, D, num, den, out, normalize);
}

}  // namespace fhgs
