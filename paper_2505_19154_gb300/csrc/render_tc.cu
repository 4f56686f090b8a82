// Tensor-core (tcgen05) render kernels for sm_103a.
//
// The feature half of Eq. 4, F(p) = sum_i w_i(p) f_i, is per tile a dense
// contraction: F(P x D) += W(P x B) . Fe(B x D) with W the compositing
// weights of a batch of B depth-sorted Gaussians.  One CTA owns a half tile
// (16 x 8 = 128 pixels, one pixel per thread = one TMEM lane) and a slice of
// DN feature columns.  Per batch its threads compute the weights on the CUDA
// cores (FP32 alpha, T and RGB exactly as the FP32 path), write them as BF16
// into shared memory in the UMMA 128-byte-swizzled K-major layout, while
// cp.async stages the batch's feature rows (BF16, MN-major, swizzled); one
// thread then issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) into a
// TMEM accumulator of 128 lanes x DN columns.  Two stages overlap the next
// batch's weights and loads with the running MMAs; tcgen05.commit on an
// mbarrier frees a stage.  After the last batch the accumulator is read with
// tcgen05.ld and written once to the feature image.
//
// The backward (App. A.2) walks each half tile back to front in batches of
// 64: G(P x B) = dF(P x DN) . Fe(B x DN)^T on the tensor cores (dF split
// into BF16 hi + lo parts, two MMAs, so G carries ~16 mantissa bits), then
// the scalar pass (alpha, T, dL/dalpha, footprint gradients) on the CUDA
// cores, then dFe(B x DN) = W^T(B x P) . dF(P x DN) (hi + lo) with M padded
// to 128 by a zero block, drained from TMEM into the feature gradient with
// vector atomics.  Transmittance is recovered without a divide per Gaussian:
// per 32-Gaussian sub-batch T_start = T_end / prod(1 - alpha), then a
// forward prefix product.  dL/dalpha is linear in g_i = dC.c_i + dF.f_i, so
// each DN slice adds its own share of the footprint gradients.
//
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the kernel
// latches FHGS_ERR_TIMEOUT, waits once more (bounded) for its MMAs, frees its
// TMEM and returns.
#include "fhgs_internal.cuh"

namespace fhgs {
namespace {

constexpr uint64_t kWaitNs = 2000000000ull;

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false if it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (!mbar_try(bar, parity))
        if (globaltimer() - t0 > kWaitNs) return false;
    return true;
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor, 128-byte swizzle (atoms of 8 rows x 128 B).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;  // SWIZZLE_128B
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn, bool b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive TMEM columns of this warp's 32 lanes -> 32 floats per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(g), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Byte offset of 16-byte chunk `c` (0..7) of row `r` inside a 128B-swizzled
// atom column whose rows are 128 bytes apart (atom base 1024-aligned).
__device__ __forceinline__ uint32_t swz(uint32_t r, uint32_t c) { return r * 128u + ((c ^ (r & 7u)) << 4); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ uint8_t *align_smem_1024(uint8_t *raw) {
    return raw + ((1024u - (smem_u32(raw) & 1023u)) & 1023u);
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// ------------------------------------------------------------- forward
constexpr int kFB = 64;  // Gaussians per forward batch (MMA K)

template <int DN>
struct FwdCfg {
    static constexpr int kWBytes = 128 * 128;            // 128 px x 64 BF16 weights
    static constexpr int kFBytes = kFB * DN * 2;         // 64 rows x DN BF16 features
    static constexpr int kNSub = DN > 256 ? DN / 256 : 1;
    static constexpr int kMmaN = DN > 256 ? 256 : DN;
    static constexpr int kRecBytes = kFB * (16 + 16 + 4 + 4);
    static constexpr int kSmem = 1024 + 2 * kWBytes + 2 * kFBytes + 2 * kRecBytes + 64;
};

template <int DN>
__global__ void __launch_bounds__(128, 1)
    k_render_fwd_tc(long long N, CamSet cs, Params p, ProjView pv, const uint32_t *__restrict__ gids,
                    const uint32_t *__restrict__ ranges, const __nv_bfloat16 *__restrict__ feats, int D,
                    float *rgb, float *feat, float *Tout, int32_t *last_out, unsigned *status) {
    using C = FwdCfg<DN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align_smem_1024(smem_raw);
    uint8_t *sW = sm;                                   // [2][128 rows][128 B]
    uint8_t *sF = sm + 2 * C::kWBytes;                  // [2][DN/64 blocks][64 rows][128 B]
    float4 *sA = reinterpret_cast<float4 *>(sF + 2 * C::kFBytes);  // [2][64]
    float4 *sB = sA + 2 * kFB;                          // [2][64]
    float *sBl = reinterpret_cast<float *>(sB + 2 * kFB);          // [2][64]
    uint32_t *sGid = reinterpret_cast<uint32_t *>(sBl + 2 * kFB);  // [2][64]
    uint64_t *bar = reinterpret_cast<uint64_t *>(sGid + 2 * kFB);  // [2]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int tile = blockIdx.x >> 1, half = blockIdx.x & 1, chunk = blockIdx.y;
    const int ci = cam_of_tile(cs, tile);
    const DevCam &cam = cs.c[ci];
    const int lt = tile - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const int px = tx * kTile + (tid & 15), py = ty * kTile + half * 8 + (tid >> 4);
    const bool inside = px < cam.W && py < cam.H;
    const long long pix = cam.pix_off + (long long)py * cam.W + px;
    const uint32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
    const int d0 = chunk * DN;
    const GRec *rec = pv.rec + (long long)ci * N;

    if (warp == 0) tmem_alloc(tslot, DN);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t taddr = *tslot;
    const uint32_t sW_s = smem_u32(sW), sF_s = smem_u32(sF);
    constexpr uint32_t idesc = idesc_bf16(128, C::kMmaN, false, true);

    const float fpx = px + 0.5f, fpy = py + 0.5f;
    float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f;
    int last = 0;
    bool done = !inside;
    uint32_t phase0 = 0, phase1 = 0;
    int nbatch = 0;
    bool timeout = false;

    for (uint32_t base = s; base < e; base += kFB) {
        const int stg = nbatch & 1;
        const int nb = (int)min((uint32_t)kFB, e - base);
        if (nbatch >= 2) {  // the MMA of batch nbatch-2 must be done reading this stage
            const bool ok = mbar_wait(&bar[stg], stg ? phase1 : phase0);
            if (stg) phase1 ^= 1u; else phase0 ^= 1u;
            if (__syncthreads_or(!ok)) {
                timeout = true;
                break;
            }
        }
        if (tid < kFB) sGid[stg * kFB + tid] = tid < nb ? gids[base + tid] : 0u;
        __syncthreads();
        {   // feature rows of the batch -> sF[stg]; rows >= nb are zero-filled
            constexpr int kCPR = DN / 8;
            const uint32_t fb = sF_s + stg * C::kFBytes;
#pragma unroll 4
            for (int q = tid; q < kFB * kCPR; q += 128) {
                const int g = q / kCPR, c = q - g * kCPR;
                const bool valid = g < nb;
                const __nv_bfloat16 *src = feats + (size_t)sGid[stg * kFB + (valid ? g : 0)] * D + d0 + c * 8;
                cp_async16(fb + (c >> 3) * (kFB * 128) + swz(g, c & 7), src, valid);
            }
            cp_async_commit();
        }
        if (tid < nb) {
            const GRec r = rec[sGid[stg * kFB + tid]];
            sA[stg * kFB + tid] = r.a;
            sB[stg * kFB + tid] = r.b;
            sBl[stg * kFB + tid] = r.c.x;
        }
        __syncthreads();
        {   // compositing weights of this pixel -> row `tid` of W[stg]
            const float4 *A4 = sA + stg * kFB;
            const float4 *B4 = sB + stg * kFB;
            const float *Bl = sBl + stg * kFB;
            uint8_t *wb = sW + stg * C::kWBytes;
#pragma unroll 1
            for (int j0 = 0; j0 < kFB; j0 += 8) {
                float w8[8];
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const int j = j0 + jj;
                    float w = 0.f;
                    if (!done && j < nb) {
                        const float4 a = A4[j], b = B4[j];
                        const float dx = fpx - a.x, dy = fpy - a.y;
                        const float q2 = eval_q2(dx, dy, a.z, a.w, b.x);
                        if (q2 <= p.cut) {
                            const float al = fminf(p.amax, b.y * __expf(-0.5f * q2));
                            if (al >= p.amin) {
                                const float Tn = T * (1.f - al);
                                if (Tn < p.teps) {
                                    done = true;
                                } else {
                                    w = al * T;
                                    cr += w * b.z;
                                    cg += w * b.w;
                                    cb += w * Bl[j];
                                    T = Tn;
                                    last = (int)(base - s) + j + 1;
                                }
                            }
                        }
                    }
                    w8[jj] = w;
                }
                uint4 pk;
                pk.x = pack_bf16(w8[0], w8[1]);
                pk.y = pack_bf16(w8[2], w8[3]);
                pk.z = pack_bf16(w8[4], w8[5]);
                pk.w = pack_bf16(w8[6], w8[7]);
                *reinterpret_cast<uint4 *>(wb + swz(tid, j0 >> 3)) = pk;
            }
        }
        cp_async_wait_all();
        fence_async_smem();
        const int all_done = __syncthreads_and(done);
        if (tid == 0) {
            tc_after();
            const uint32_t wa = sW_s + stg * C::kWBytes, fb = sF_s + stg * C::kFBytes;
#pragma unroll
            for (int ks = 0; ks < kFB / 16; ++ks) {
                const uint64_t ad = sdesc(wa + ks * 32, 16, 1024);
#pragma unroll
                for (int nh = 0; nh < C::kNSub; ++nh) {
                    const uint64_t bd = sdesc(fb + nh * 4 * (kFB * 128) + ks * 2048, kFB * 128, 1024);
                    mma_bf16(taddr + nh * 256, ad, bd, idesc, (nbatch > 0 || ks > 0) ? 1u : 0u);
                }
            }
            mma_commit(&bar[stg]);
        }
        ++nbatch;
        if (all_done) break;
    }

    if (nbatch > 0 && !timeout) {  // the last commit covers every MMA issued before it
        const int stg = (nbatch - 1) & 1;
        const bool ok = mbar_wait(&bar[stg], stg ? phase1 : phase0);
        if (__syncthreads_or(!ok)) timeout = true;
    }
    if (timeout) {
        if (tid == 0) latch(status, ST_TIMEOUT);
        if (nbatch > 0) {
            const int stg = (nbatch - 1) & 1;
            mbar_wait(&bar[stg], stg ? phase1 : phase0);
        }
    } else {
        tc_after();
        float *fo = feat + pix * D + d0;
#pragma unroll 1
        for (int cc = 0; cc < DN / 32; ++cc) {
            float v[32];
            if (nbatch > 0) {
                tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + cc * 32, v);
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.f;
            }
            if (inside) {
                float4 *d4 = reinterpret_cast<float4 *>(fo + cc * 32);
#pragma unroll
                for (int i = 0; i < 8; ++i) d4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            }
        }
        if (chunk == 0 && inside) {
            rgb[3 * pix + 0] = cr + T * p.bg0;
            rgb[3 * pix + 1] = cg + T * p.bg1;
            rgb[3 * pix + 2] = cb + T * p.bg2;
            Tout[pix] = T;
            last_out[pix] = last;
        }
    }
    tc_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, DN);
}

// ------------------------------------------------------------- backward
constexpr int kBB = 64;  // Gaussians per backward batch

template <int DN>
struct BwdCfg {
    static constexpr int kNBlk = DN / 64;                 // 64-feature blocks
    static constexpr int kDBytes = kNBlk * 128 * 128;     // 128 px x DN BF16 (one of hi / lo)
    static constexpr int kFBytes = kNBlk * kBB * 128;     // 64 rows x DN BF16
    static constexpr int kWBytes = 2 * 128 * 128;         // two M blocks: weights, zeros
    static constexpr int kRecBytes = kBB * (16 + 16 + 4 + 4 + 4 + 9 * 4);
    static constexpr int kSmem = 1024 + 2 * kDBytes + kFBytes + kWBytes + kRecBytes + 64;
    static constexpr int kTmemCols = (64 + DN) <= 256 ? 256 : 512;
    static constexpr int kFCol = DN <= 128 ? 128 : 256;  // column of the dFe accumulator
};

template <int DN>
__global__ void __launch_bounds__(128, 1)
    k_render_bwd_tc(long long N, CamSet cs, Params p, ProjView pv, const uint32_t *__restrict__ gids,
                    const uint32_t *__restrict__ ranges, const __nv_bfloat16 *__restrict__ feats, int D,
                    const float *__restrict__ Tfin, const int32_t *__restrict__ lastv,
                    const float *__restrict__ grgb, const float *__restrict__ gfeat, float *g2d, float *gfeatures,
                    unsigned *status) {
    using C = BwdCfg<DN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align_smem_1024(smem_raw);
    uint8_t *sDh = sm;                                  // [DN/64][128 px][128 B]
    uint8_t *sDl = sm + C::kDBytes;
    uint8_t *sF = sm + 2 * C::kDBytes;                  // [DN/64][64 g][128 B]
    uint8_t *sW = sF + C::kFBytes;                      // [2][128 px][128 B]
    float4 *sA = reinterpret_cast<float4 *>(sW + C::kWBytes);
    float4 *sB = sA + kBB;
    float *sBl = reinterpret_cast<float *>(sB + kBB);
    uint32_t *sGid = reinterpret_cast<uint32_t *>(sBl + kBB);
    int *sFlag = reinterpret_cast<int *>(sGid + kBB);
    float *sAcc = reinterpret_cast<float *>(sFlag + kBB);  // [64][9]
    uint64_t *bar = reinterpret_cast<uint64_t *>(sAcc + kBB * 9);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2);
    int *smax = reinterpret_cast<int *>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x >> 1, half = blockIdx.x & 1, chunk = blockIdx.y;
    const int ci = cam_of_tile(cs, tile);
    const DevCam &cam = cs.c[ci];
    const int lt = tile - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const int px = tx * kTile + (tid & 15), py = ty * kTile + half * 8 + (tid >> 4);
    const bool inside = px < cam.W && py < cam.H;
    const long long pix = cam.pix_off + (long long)py * cam.W + px;
    const uint32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
    const int d0 = chunk * DN;
    const GRec *rec = pv.rec + (long long)ci * N;
    float *g2dc = g2d + (long long)ci * N * 12;
    const bool want_fg = gfeatures != nullptr;

    if (warp == 0) tmem_alloc(tslot, C::kTmemCols);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        *smax = 0;
    }
    // dF slice of this CTA's pixels -> BF16 hi / lo, K-major swizzled.  Each
    // warp copies its 32 pixel rows, 32 lanes x 16 B per 512-byte piece.
    {
        const int row0 = warp * 32;
#pragma unroll 1
        for (int r = 0; r < 32; ++r) {
            const int prow = row0 + r;
            const int qx = tx * kTile + (prow & 15), qy = ty * kTile + half * 8 + (prow >> 4);
            const bool qin = qx < cam.W && qy < cam.H && gfeat != nullptr;
            const float *src = gfeat + (cam.pix_off + (long long)qy * cam.W + qx) * D + d0;
#pragma unroll
            for (int f = lane * 4; f < DN; f += 128) {  // f: first of this lane's 4 features
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (qin) v = *reinterpret_cast<const float4 *>(src + f);
                const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
                const float2 b01 = __bfloat1622float2(h01), b23 = __bfloat1622float2(h23);
                const __nv_bfloat162 l01 = __floats2bfloat162_rn(v.x - b01.x, v.y - b01.y);
                const __nv_bfloat162 l23 = __floats2bfloat162_rn(v.z - b23.x, v.w - b23.y);
                const uint32_t off = (f >> 6) * (128 * 128) + swz(prow, (f & 63) >> 3) + ((f & 7) ? 8 : 0);
                uint2 hv, lv;
                hv.x = *reinterpret_cast<const uint32_t *>(&h01);
                hv.y = *reinterpret_cast<const uint32_t *>(&h23);
                lv.x = *reinterpret_cast<const uint32_t *>(&l01);
                lv.y = *reinterpret_cast<const uint32_t *>(&l23);
                *reinterpret_cast<uint2 *>(sDh + off) = hv;
                *reinterpret_cast<uint2 *>(sDl + off) = lv;
            }
        }
        // zero M block of the weight operand (rows 64..127 of dFe read it)
        uint4 *z = reinterpret_cast<uint4 *>(sW + 128 * 128);
        for (int i = tid; i < 128 * 128 / 16; i += 128) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    float T = 1.f, dC0 = 0.f, dC1 = 0.f, dC2 = 0.f;
    int lastp = 0;
    if (inside) {
        T = Tfin[pix];
        lastp = lastv[pix];
        if (chunk == 0) {
            dC0 = grgb[3 * pix];
            dC1 = grgb[3 * pix + 1];
            dC2 = grgb[3 * pix + 2];
        }
    }
    tc_before();
    __syncthreads();
    tc_after();
    atomicMax(smax, lastp);
    fence_async_smem();
    __syncthreads();
    const uint32_t taddr = *tslot;
    const uint32_t tG = taddr, tF = taddr + C::kFCol;
    const int Lmax = min(*smax, (int)(e - s));
    const uint32_t sDh_s = smem_u32(sDh), sDl_s = smem_u32(sDl), sF_s = smem_u32(sF), sW_s = smem_u32(sW);
    constexpr uint32_t idG = idesc_bf16(128, kBB, false, false);
    constexpr uint32_t idF = idesc_bf16(128, DN, true, true);

    const float fpx = px + 0.5f, fpy = py + 0.5f;
    float S = T * (dC0 * p.bg0 + dC1 * p.bg1 + dC2 * p.bg2);
    uint32_t phG = 0, phF = 0;
    bool timeout = false;

    for (int bend = Lmax; bend > 0 && !timeout; bend -= kBB) {
        const int bstart = max(0, bend - kBB), nb = bend - bstart;
        if (tid < kBB) {
            sGid[tid] = tid < nb ? gids[s + bstart + tid] : 0u;
            sFlag[tid] = 0;
        }
        for (int i = tid; i < kBB * 9; i += 128) sAcc[i] = 0.f;
        __syncthreads();
        {   // feature rows (K-major for G): [DN/64][64 g][128 B]
            constexpr int kCPR = DN / 8;
#pragma unroll 4
            for (int q = tid; q < kBB * kCPR; q += 128) {
                const int g = q / kCPR, c = q - g * kCPR;
                const bool valid = g < nb;
                const __nv_bfloat16 *src = feats + (size_t)sGid[valid ? g : 0] * D + d0 + c * 8;
                cp_async16(sF_s + (c >> 3) * (kBB * 128) + swz(g, c & 7), src, valid);
            }
            cp_async_commit();
        }
        if (tid < nb) {
            const GRec r = rec[sGid[tid]];
            sA[tid] = r.a;
            sB[tid] = r.b;
            sBl[tid] = r.c.x;
        }
        cp_async_wait_all();
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {  // G(px, g) = sum_d dF(px, d) Fe(g, d): hi and lo parts
            tc_after();
#pragma unroll
            for (int ks = 0; ks < DN / 16; ++ks) {
                const uint32_t koff = (ks >> 2) * (128 * 128) + (ks & 3) * 32;
                const uint64_t bd = sdesc(sF_s + (ks >> 2) * (kBB * 128) + (ks & 3) * 32, 16, 1024);
                mma_bf16(tG, sdesc(sDh_s + koff, 16, 1024), bd, idG, ks > 0 ? 1u : 0u);
                mma_bf16(tG, sdesc(sDl_s + koff, 16, 1024), bd, idG, 1u);
            }
            mma_commit(&bar[0]);
        }
        {
            const bool ok = mbar_wait(&bar[0], phG);
            phG ^= 1u;
            if (__syncthreads_or(!ok)) {
                timeout = true;
                break;
            }
        }
        tc_after();
        // back to front over two sub-batches of 32 Gaussians
#pragma unroll 1
        for (int sub = 1; sub >= 0; --sub) {
            float Gv[32];
            tmem_ld32(tG + ((uint32_t)(warp * 32) << 16) + sub * 32, Gv);
            float al[32], gx[32], Tj[32];
            float P = 1.f;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                const int j = sub * 32 + jj;
                float a = 0.f, gg = 0.f;
                if (j < nb && bstart + j < lastp) {
                    const float4 A4 = sA[j], B4 = sB[j];
                    const float dx = fpx - A4.x, dy = fpy - A4.y;
                    const float q2 = eval_q2(dx, dy, A4.z, A4.w, B4.x);
                    if (q2 <= p.cut) {
                        const float G = __expf(-0.5f * q2);
                        const float rho = B4.y * G;
                        const float aa = fminf(p.amax, rho);
                        if (aa >= p.amin) {
                            a = aa;
                            gg = rho > p.amax ? 0.f : G;
                        }
                    }
                }
                al[jj] = a;
                gx[jj] = gg;
                P *= 1.f - a;
            }
            // T before the sub-batch, then the forward prefix of transmittance
            const float Tstart = T / P;
            float t = Tstart;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                Tj[jj] = t;
                t *= 1.f - al[jj];
            }
            // App. A.2 back to front: dL/dalpha_k = T_k g_k - S_k / (1 - alpha_k)
#pragma unroll
            for (int jj = 31; jj >= 0; --jj) {
                const int j = sub * 32 + jj;
                if (al[jj] > 0.f) {
                    const float w = al[jj] * Tj[jj];
                    const float4 B4 = sB[j];
                    const float g = Gv[jj] + dC0 * B4.z + dC1 * B4.w + dC2 * sBl[j];
                    const float dal = Tj[jj] * g - S / (1.f - al[jj]);
                    S += w * g;
                    gx[jj] *= dal;  // = G dL/drho (0 where alpha is clamped)
                } else {
                    gx[jj] = 0.f;
                }
            }
            // weights (BF16) for dFe = W^T dF: Gaussians sub*32.. in row `tid`
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint4 pk;
                pk.x = pack_bf16(al[8 * q + 0] * Tj[8 * q + 0], al[8 * q + 1] * Tj[8 * q + 1]);
                pk.y = pack_bf16(al[8 * q + 2] * Tj[8 * q + 2], al[8 * q + 3] * Tj[8 * q + 3]);
                pk.z = pack_bf16(al[8 * q + 4] * Tj[8 * q + 4], al[8 * q + 5] * Tj[8 * q + 5]);
                pk.w = pack_bf16(al[8 * q + 6] * Tj[8 * q + 6], al[8 * q + 7] * Tj[8 * q + 7]);
                *reinterpret_cast<uint4 *>(sW + swz(tid, sub * 4 + q)) = pk;
            }
            // footprint gradients: reduce over the warp's pixels, then shared atomics
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                const bool c = al[jj] > 0.f;
                if (!__any_sync(0xffffffffu, c)) continue;
                const int j = sub * 32 + jj;
                const float4 A4 = sA[j], B4 = sB[j];
                const float dx = fpx - A4.x, dy = fpy - A4.y;
                const float gop = gx[jj];
                const float dq2 = -0.5f * B4.y * gop;
                const float w = al[jj] * Tj[jj];
                float v[9];
                v[0] = -(2.f * A4.z * dx + 2.f * A4.w * dy) * dq2;
                v[1] = -(2.f * A4.w * dx + 2.f * B4.x * dy) * dq2;
                v[2] = dx * dx * dq2;
                v[3] = 2.f * dx * dy * dq2;
                v[4] = dy * dy * dq2;
                v[5] = gop;
                v[6] = w * dC0;
                v[7] = w * dC1;
                v[8] = w * dC2;
                const int nv = chunk == 0 ? 9 : 6;
#pragma unroll
                for (int k = 0; k < 9; ++k)
                    if (k < nv) v[k] = warp_sum(v[k]);
                if (lane == 0) {
                    sFlag[j] = 1;
#pragma unroll
                    for (int k = 0; k < 9; ++k)
                        if (k < nv) atomicAdd(&sAcc[j * 9 + k], v[k]);
                }
            }
            T = Tstart;
        }
        fence_async_smem();
        __syncthreads();
        if (want_fg && tid == 0) {  // dFe(g, d) = sum_px W(px, g) dF(px, d): hi and lo parts
            tc_after();
#pragma unroll
            for (int ks = 0; ks < 128 / 16; ++ks) {
                const uint64_t ad = sdesc(sW_s + ks * 2048, 128 * 128, 1024);
                mma_bf16(tF, ad, sdesc(sDh_s + ks * 2048, 128 * 128, 1024), idF, ks > 0 ? 1u : 0u);
                mma_bf16(tF, ad, sdesc(sDl_s + ks * 2048, 128 * 128, 1024), idF, 1u);
            }
            mma_commit(&bar[1]);
        }
        // flush this batch's footprint gradients (one set of atomics per Gaussian)
        if (tid < nb && sFlag[tid]) {
            float4 *dst = reinterpret_cast<float4 *>(g2dc + 12 * (long long)sGid[tid]);
            const float *a = sAcc + tid * 9;
            atomicAdd(dst, make_float4(a[0], a[1], a[2], a[3]));
            atomicAdd(dst + 1, make_float4(a[4], a[5], chunk == 0 ? a[6] : 0.f, chunk == 0 ? a[7] : 0.f));
            if (chunk == 0) atomicAdd(g2dc + 12 * (long long)sGid[tid] + 8, a[8]);
        }
        if (want_fg) {
            const bool ok = mbar_wait(&bar[1], phF);
            phF ^= 1u;
            if (__syncthreads_or(!ok)) {
                timeout = true;
                break;
            }
            tc_after();
            if (warp < 2) {  // rows 0..63 of dFe live in lanes 0..63
                const bool mine = tid < nb && sFlag[tid] != 0;
                float *dst = gfeatures + (size_t)sGid[tid] * D + d0;
#pragma unroll 1
                for (int cc = 0; cc < DN / 32; ++cc) {
                    float v[32];
                    tmem_ld32(tF + ((uint32_t)(warp * 32) << 16) + cc * 32, v);
                    if (mine) {
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            atomicAdd(reinterpret_cast<float4 *>(dst + cc * 32) + i,
                                      make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]));
                    }
                }
            }
        }
        tc_before();
        __syncthreads();
        tc_after();
    }
    if (timeout) {
        if (tid == 0) latch(status, ST_TIMEOUT);
        mbar_wait(&bar[0], phG);
        if (want_fg) mbar_wait(&bar[1], phF);
    }
    tc_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, C::kTmemCols);
}

int pick_fwd_dn(int D, int d_split) {
    if (d_split == 64 || d_split == 128 || d_split == 256 || d_split == 512) return (D % d_split == 0) ? d_split : 0;
    if (D % 256 == 0) return 256;
    if (D % 128 == 0) return 128;
    if (D % 64 == 0) return 64;
    return 0;
}

int pick_bwd_dn(int D, int d_split) {
    if (d_split == 64 || d_split == 128 || d_split == 256) return (D % d_split == 0) ? d_split : 0;
    if (d_split == 512) return (D % 256 == 0) ? 256 : 0;
    if (D % 256 == 0) return 256;
    if (D % 128 == 0) return 128;
    if (D % 64 == 0) return 64;
    return 0;
}

template <typename K>
void set_smem(K kernel, int bytes) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace

int tc_supported(int D, int d_split) {
    return D > 0 && pick_fwd_dn(D, d_split) != 0 && pick_bwd_dn(D, d_split) != 0;
}

void launch_render_fwd_tc(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                          const __nv_bfloat16 *feats, int D, int d_split, float *rgb, float *feat, float *T,
                          int32_t *last, unsigned *status, cudaStream_t st) {
    const int dn = pick_fwd_dn(D, d_split);
    dim3 grid(cs.total_tiles * 2, D / dn);
    note_launch(1);
#define FHGS_FWD(DNV)                                                                                     \
    case DNV: {                                                                                           \
        set_smem(k_render_fwd_tc<DNV>, FwdCfg<DNV>::kSmem);                                              \
        k_render_fwd_tc<DNV><<<grid, 128, FwdCfg<DNV>::kSmem, st>>>(N, cs, p, pv, bins.gids, bins.ranges, feats, D, \
                                                                   rgb, feat, T, last, status);          \
        break;                                                                                            \
    }
    switch (dn) {
        FHGS_FWD(64)
        FHGS_FWD(128)
        FHGS_FWD(256)
        FHGS_FWD(512)
        default: break;
    }
#undef FHGS_FWD
}

void launch_render_bwd_tc(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                          const __nv_bfloat16 *feats, int D, int d_split, const float *T, const int32_t *last,
                          const float *grgb, const float *gfeat, float *g2d, float *gfeatures, unsigned *status,
                          cudaStream_t st) {
    const int dn = pick_bwd_dn(D, d_split);
    dim3 grid(cs.total_tiles * 2, D / dn);
    note_launch(1);
#define FHGS_BWD(DNV)                                                                                          \
    case DNV: {                                                                                                \
        set_smem(k_render_bwd_tc<DNV>, BwdCfg<DNV>::kSmem);                                                   \
        k_render_bwd_tc<DNV><<<grid, 128, BwdCfg<DNV>::kSmem, st>>>(N, cs, p, pv, bins.gids, bins.ranges, feats, D, T, \
                                                                   last, grgb, gfeat, g2d, gfeatures, status);  \
        break;                                                                                                 \
    }
    switch (dn) {
        FHGS_BWD(64)
        FHGS_BWD(128)
        FHGS_BWD(256)
        default: break;
    }
#undef FHGS_BWD
}

}  // namespace fhgs
