// Backward of the tensor-core render with dL/dF streamed through shared
// memory (App. A.2), for D a multiple of 128.
//
// One persistent CTA per SM walks the half tiles (16 x 8 = 128 pixels, one
// TMEM lane each) back to front in batches of 64 Gaussians, covering all D
// feature channels of the half tile: alpha, transmittance and the App. A.2
// recursion run once per (pixel, Gaussian), not once per feature slice.
// Per batch b, after its scalar pass, one pass over dF in chunks of 64
// channels (FP32, staged by TMA from L2, split into BF16 hi + lo in the
// 128-byte-swizzled K-major layout) issues, per chunk,
//   G_{b+1} += dF_hi . Fe_{b+1}^T and dF_lo . Fe_{b+1}^T   (128 px x 64 g),
// and, per pair of chunks, the feature gradient of batch b
//   dFe_b^T (128 channels x 64 g) = dF_hi^T . W_b,
// drained from TMEM (double-buffered) into grad_features with one coalesced
// 128-byte reduction per warp instruction while the next block runs.  The
// footprint gradients come from the pixel moments t^T X as in the sliced
// kernel (render_tc.cu), and G carries ~16 mantissa bits (hi + lo).
//
// MMA issue is spread over threads 0 (G hi), 32 (G lo), 64 (dFe) and 96
// (moments), each committing its own work; every mbarrier wait is bounded
// and a wait that runs out latches FHGS_ERR_TIMEOUT, waits once more
// (bounded) for the copies and MMAs in flight, frees TMEM and returns.
#include <cstring>

#include "fhgs_internal.cuh"
#include "tc_ptx.cuh"

namespace fhgs {
namespace {

using namespace tc;

constexpr int kSB = 64;               // Gaussians per batch (N of G, K of the moments)
constexpr int kCK = 64;               // channels per streamed chunk (one 128-byte BF16 atom row)
constexpr int kSG = 4;                // groups of four warps over the 128 pixels
constexpr int kSThreads = 128 * kSG;  // 512
constexpr int kSJ = kSB / kSG;        // Gaussians per thread and batch

// Shared memory of the CTA (byte offsets; MMA operands 1024-aligned).
struct SCfg {
    static constexpr int kStgBytes = 128 * kCK * 4;             // one FP32 chunk: 128 px x 64 ch
    static constexpr int kOffStg = 0;                           // [2] FP32 staging, [px][64] row-major
    static constexpr int kOffHi = kOffStg + 2 * kStgBytes;      // [2][128 px][64] BF16 hi (adjacent slots)
    static constexpr int kOffLo = kOffHi + 2 * 128 * 128;       // [2][128 px][64] BF16 lo
    static constexpr int kOffFe = kOffLo + 2 * 128 * 128;       // [4][64 g][64] BF16 features of the G batch
    static constexpr int kOffW = kOffFe + 4 * kSB * 128;        // [128 px][64 g] BF16 weights (MN-major B)
    static constexpr int kOffTh = kOffW + 128 * 128;            // [128 px][64 g] t hi (MN-major A)
    static constexpr int kOffTl = kOffTh + 128 * 128;           // t lo, right after t hi
    static constexpr int kOffX = kOffTl + 128 * 128;            // [2 K-blocks][16 rows][64 px] BF16 moments rows
    static constexpr int kRecBytes = kSB * 48;
    static constexpr int kOffRec = kOffX + 2 * 16 * 128;        // [2][64] records
    static constexpr int kOffGid = kOffRec + 2 * kRecBytes;     // [4][64] ids
    static constexpr int kOffRgb = kOffGid + 4 * kSB * 4;       // [2][64][3] colour sums
    static constexpr int kOffMask = kOffRgb + 2 * kSB * 3 * 4;  // [2][2] contributor masks
    static constexpr int kOffXch = kOffMask + 16;               // per pixel: P, S of groups 1..3; T, S
    static constexpr int kOffBar = kOffXch + 128 * 4 * (2 * (kSG - 1) + 2);
    static constexpr int kNBar = 13;
    static constexpr int kSmem = 1024 + kOffBar + kNBar * 8 + 8 + 16;
    static_assert(kSmem <= 232448, "streamed backward exceeds the opt-in shared memory");
    static_assert(kOffHi % 1024 == 0 && kOffFe % 1024 == 0 && kOffW % 1024 == 0 && kOffX % 1024 == 0,
                  "MMA operands must be 1024-aligned");
    // tensor memory (512 columns)
    static constexpr uint32_t kColG = 0, kColGl = 64, kColF = 128, kColM = 256, kTmemCols = 512;
};

// barrier slots
enum : int { kBarStg = 0, kBarHL = 2, kBarFe = 4, kBarDfe = 8, kBarG = 10, kBarM = 11, kBarQ = 12 };

__device__ __forceinline__ void rs_step_s(float *v, int lane, int off, int H) {
    const bool up = (lane & off) != 0;
    for (int i = 0; i < H; ++i) {
        const float send = up ? v[i] : v[i + H];
        const float keep = up ? v[i + H] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
}

__global__ void __launch_bounds__(kSThreads, 1)
    k_render_bwd_stream(long long N, CamSet cs, Params p, ProjView pv, const uint32_t *__restrict__ gids,
                        const uint32_t *__restrict__ ranges, const __nv_bfloat16 *__restrict__ feats, int D,
                        const float *__restrict__ Tfin, const int32_t *__restrict__ lastv,
                        const float *__restrict__ grgb, const __grid_constant__ CUtensorMap dfm, float *g2d,
                        float *gfeatures, unsigned *status, int n_items) {
    using C = SCfg;
    constexpr int kJ = kSJ;
    if ((int)blockIdx.x >= n_items) return;  // uniform over the CTA
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align_smem_1024(smem_raw);
    if (probe_wait_expired(p, sm, status)) return;
    uint8_t *sStg = sm + C::kOffStg;
    uint8_t *sHi = sm + C::kOffHi;
    uint8_t *sLo = sm + C::kOffLo;
    uint8_t *sFe = sm + C::kOffFe;
    uint8_t *sW = sm + C::kOffW;
    uint8_t *sTh = sm + C::kOffTh;
    uint8_t *sTl = sm + C::kOffTl;
    uint8_t *sX = sm + C::kOffX;
    auto sRgb = [&](int b) { return reinterpret_cast<float *>(sm + C::kOffRgb) + (b & 1) * kSB * 3; };
    auto sMask = [&](int b) { return reinterpret_cast<uint32_t *>(sm + C::kOffMask) + (b & 1) * 2; };
    float *xP = reinterpret_cast<float *>(sm + C::kOffXch);  // [3][128] group g's prod (1 - alpha), g >= 1
    float *xSg = xP + (kSG - 1) * 128;                         // [3][128] group g's sum w g, g >= 1
    float *xT = xSg + (kSG - 1) * 128;                         // [128] T after the batch
    float *xS = xT + 128;                                      // [128] S after the batch
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + C::kOffBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + C::kNBar);
    unsigned long long *smax = reinterpret_cast<unsigned long long *>(sm + C::kOffBar + C::kNBar * 8 + 8);
    auto srec = [&](int b) { return reinterpret_cast<GRec *>(sm + C::kOffRec + (b & 1) * C::kRecBytes); };
    auto sgid = [&](int b) { return reinterpret_cast<uint32_t *>(sm + C::kOffGid + (b & 3) * kSB * 4); };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, grp = tid >> 7, pidx = tid & 127;
    const bool want_fg = gfeatures != nullptr;
    const int nck = D / kCK;  // chunks per pass (even: D % 128 == 0)

    if (warp == 0) tmem_alloc(tslot, C::kTmemCols);
    if (tid == 0) {
        mbar_init(&bars[kBarStg + 0], 1);
        mbar_init(&bars[kBarStg + 1], 1);
        mbar_init(&bars[kBarHL + 0], 3);  // G hi, G lo and dFe issuers
        mbar_init(&bars[kBarHL + 1], 3);
        for (int f = 0; f < 4; ++f) mbar_init(&bars[kBarFe + f], 2);  // G hi and G lo issuers
        mbar_init(&bars[kBarDfe + 0], 1);
        mbar_init(&bars[kBarDfe + 1], 1);
        mbar_init(&bars[kBarG], 2);
        mbar_init(&bars[kBarM], 1);
        mbar_init(&bars[kBarQ], 4);       // quiesce on a timeout: one commit per issuing thread
        fence_mbar_init();
        smax[0] = smax[1] = 0ull;
    }
    if (tid < 2 * kSB) sRgb(0)[3 * tid] = sRgb(0)[3 * tid + 1] = sRgb(0)[3 * tid + 2] = 0.f;  // both slots
    if (tid < 4) sMask(0)[tid] = 0u;
    // pixel-moment rows of X: X[n][p] for p = i + 16 j: 1, i, j, i^2, i j, j^2
    for (int q = tid; q < 16 * 128; q += kSThreads) {
        const int n = q >> 7, pp = q & 127;
        const float i = (float)(pp & 15), jv = (float)(pp >> 4);
        const float val = n == 0 ? 1.f : n == 1 ? i : n == 2 ? jv : n == 3 ? i * i : n == 4 ? i * jv
                                                   : n == 5 ? jv * jv : 0.f;
        *reinterpret_cast<__nv_bfloat16 *>(sX + (pp >> 6) * (16 * 128) + swz(n, (pp & 63) >> 3) +
                                           2 * (pp & 7)) = __float2bfloat16_rn(val);
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t taddr = *tslot;
    const uint32_t tG = taddr + C::kColG, tGl = taddr + C::kColGl, tM = taddr + C::kColM;
    const uint32_t sW_s = smem_u32(sW), sTh_s = smem_u32(sTh), sX_s = smem_u32(sX);
    const uint32_t sHi_s = smem_u32(sHi), sLo_s = smem_u32(sLo), sFe_s = smem_u32(sFe), sStg_s = smem_u32(sStg);
    constexpr uint32_t idG = idesc_bf16(128, kSB, false, false);
    constexpr uint32_t idF = idesc_bf16(128, kSB, true, true);
    constexpr uint32_t idM = idesc_bf16(128, 16, true, false);
    const uint64_t dW0 = sdesc(sW_s, 128 * 128, 1024), dTh0 = sdesc(sTh_s, 128 * 128, 1024);
    const uint64_t dX0 = sdesc(sX_s, 16, 1024);

    // ---- bookkeeping of the barrier phases (identical in every thread) ----
    uint32_t qStg = 0;     // chunks staged and converted so far (slot q & 1)
    uint32_t qIss = 0;     // chunks whose TMA has been issued
    uint32_t nBlk = 0;     // feature-gradient blocks issued (buffer k & 1)
    uint32_t nBlkDrained = 0;
    uint32_t nG = 0, nGw = 0;  // G passes committed / waited
    uint32_t nM = 0, nMw = 0;  // moment MMAs committed / waited
    bool timeout = false;

    struct ItemGeo {
        int tile, ci, x0, y0;
    };
    auto item_geo = [&](int it) {
        ItemGeo g;
        g.tile = it >> 1;
        g.ci = cam_of_tile(cs, g.tile);
        const DevCam &cm = cs.c[g.ci];
        const int lt = g.tile - cm.tile_off;
        g.x0 = (lt % cm.tiles_x) * kTile;
        g.y0 = (lt / cm.tiles_x) * kTile + (it & 1) * 8;
        return g;
    };
    // a bounded wait by every thread; false (CTA-uniform) when it ran out
    auto wait_all = [&](uint64_t *bar, uint32_t parity) {
        const bool ok = mbar_wait(bar, parity);
        return !__syncthreads_or(!ok);
    };
    // TMA of dF chunk c (64 channels) of the half tile into staging slot
    // qIss & 1: 8 boxes of 16 pixels x 64 channels, one per image row.
    // Rows below the image read the next rows or camera (or zeros past the
    // end of the tensor); the conversion zeroes every pixel outside.
    auto issue_stage = [&](const ItemGeo &g, int c) {
        const uint32_t s = qIss & 1u;
        if (tid == 0) {
            const DevCam &cm = cs.c[g.ci];
            uint64_t *bar = &bars[kBarStg + s];
            mbar_arrive_expect_tx(bar, (uint32_t)C::kStgBytes);
#pragma unroll 1
            for (int r = 0; r < 8; ++r) {
                const long long row = cm.pix_off + (long long)(g.y0 + r) * cm.W + g.x0;
                tma_load_2d(sStg_s + s * C::kStgBytes + r * (16 * kCK * 4), &dfm, c * kCK, (int)row, bar);
            }
        }
        ++qIss;
    };

    int k = 0;
#pragma unroll 1
    for (int it = blockIdx.x; it < n_items && !timeout; it += gridDim.x, ++k) {
        const ItemGeo ig = item_geo(it);
        const DevCam &cam = cs.c[ig.ci];
        const int x0 = ig.x0, y0 = ig.y0;
        const int px = x0 + (pidx & 15), py = y0 + (pidx >> 4);
        const bool inside = px < cam.W && py < cam.H;
        const long long pix = cam.pix_off + (long long)py * cam.W + px;
        const uint32_t s0 = ranges[2 * ig.tile], e0 = ranges[2 * ig.tile + 1];
        const GRec *rec = pv.rec + (long long)ig.ci * N;
        float *g2dc = g2d + (long long)ig.ci * N * 12;
        float T = 1.f, dC0 = 0.f, dC1 = 0.f, dC2 = 0.f;
        int lastp = 0;
        if (inside) {
            T = Tfin[pix];
            lastp = lastv[pix];
            dC0 = grgb[3 * pix];
            dC1 = grgb[3 * pix + 1];
            dC2 = grgb[3 * pix + 2];
        }
        if (grp == 0) atomicMax(&smax[k & 1], ((unsigned long long)k << 32) | (uint32_t)max(lastp, 0));
        __syncthreads();
        const int Lmax = (int)min((unsigned long long)(e0 - s0), smax[k & 1] & 0xFFFFFFFFull);
        const int nbat = (Lmax + kSB - 1) / kSB;
        if (nbat == 0) continue;  // CTA-uniform: nothing to walk, no dF needed

        // Every load helper commits exactly one cp.async group in every thread.
        auto load_gid = [&](int b) {  // ids of batch b (ring slot b & 3)
            if (b < nbat && tid < kSB) {
                const int be = Lmax - b * kSB, bs = max(0, be - kSB), nb = be - bs;
                cp_async4(smem_u32(sgid(b) + tid), gids + s0 + bs + (tid < nb ? tid : 0), tid < nb);
            }
            cp_async_commit();
        };
        auto load_rec = [&](int b) {  // records of batch b (its ids have landed)
            if (b < nbat) {
                const int be = Lmax - b * kSB, bs = max(0, be - kSB), nb = be - bs;
                if (tid < nb) {
                    const uint32_t dst = smem_u32(srec(b) + tid);
                    const GRec *src = rec + sgid(b)[tid];
                    cp_async16(dst, &src->a, true);
                    cp_async16(dst + 16, &src->b, true);
                    cp_async16(dst + 32, &src->c, true);
                }
            }
            cp_async_commit();
        };
        // features of batch gb, channels [64 c, 64 c + 64), into Fe slot f
        // (one 16-byte piece per thread: 64 rows x 8 pieces); commits one
        // group, empty when !active, so that every chunk has exactly one
        auto load_fe = [&](bool active, int gb, int c, uint32_t f) {
            if (active) {
                const int be = Lmax - gb * kSB, bs = max(0, be - kSB), nb = be - bs;
                const int g = tid >> 3, cc = tid & 7;
                const uint32_t *ids = sgid(gb);
                cp_async16(sFe_s + f * (kSB * 128) + swz(g, cc),
                           feats + (size_t)ids[g < nb ? g : 0] * D + c * kCK + cc * 8, g < nb);
            }
            cp_async_commit();
        };
        // feature-gradient block kk (channels [128 kk, 128 kk + 128)) of batch
        // b, TMEM buffer nBlkDrained & 1: warp w reads lanes 32 (w % 4) + l =
        // channels and 16 Gaussian columns from 16 (w / 4); each reduction
        // instruction adds one Gaussian's 32 consecutive channels (128 B).
        auto drain_f = [&](int b, int kk) -> bool {
            const uint32_t kb = nBlkDrained;
            if (!wait_all(&bars[kBarDfe + (kb & 1u)], (kb >> 1) & 1u)) return false;
            ++nBlkDrained;
            tc_after();
            const int be = Lmax - b * kSB, bs = max(0, be - kSB), nb = be - bs;
            const int q4 = warp & 3, j0 = (warp >> 2) * 16;
            const uint64_t vmask = nb >= 64 ? ~0ull : ((1ull << nb) - 1ull);
            const uint64_t msk = ((((uint64_t)sMask(b)[1] << 32) | sMask(b)[0]) & vmask) >> j0;
            if ((msk & 0xFFFFull) != 0ull) {  // warp-uniform
                float v[16];
                tmem_ld16(taddr + C::kColF + (kb & 1u) * kSB + j0 + ((uint32_t)(q4 * 32) << 16), v);
                const uint32_t *ids = sgid(b) + j0;
                float *dst = gfeatures + kk * 128 + q4 * 32 + lane;
#pragma unroll
                for (int jj = 0; jj < 16; ++jj)
                    if ((msk >> jj) & 1ull) atomicAdd(dst + (size_t)ids[jj] * D, v[jj]);
            }
            tc_before();
            return true;
        };

        // One pass over dF: G of batch bG (if 0 <= bG < nbat) and the feature
        // gradient of batch bF (if bF >= 0 and grad_features is wanted).
        auto run_pass = [&](int bF, int bG) -> bool {
            const bool doG = bG >= 0 && bG < nbat;
            const bool doF = bF >= 0 && want_fg;
            const uint32_t q0 = qStg;  // global index of this pass's chunk 0 (even)
            // features of chunks 0 and 1, once chunks q0 - 4 and q0 - 3 have been read
            // (each thread waits for itself; a wait that ran out is made
            // uniform at the first chunk's barrier)
            bool okPre = true;
            for (int c = 0; c < 2; ++c) {
                const uint32_t qq = q0 + c, f = qq & 3u;
                if (qq >= 4) okPre = okPre && mbar_wait(&bars[kBarFe + f], ((qq >> 2) + 1) & 1u);
                load_fe(doG && okPre, bG, c, f);
            }
            issue_stage(ig, 0);
            issue_stage(ig, 1);
#pragma unroll 1
            for (int c = 0; c < nck; ++c) {
                const uint32_t q = qStg, s = q & 1u, f = q & 3u;
                // features of chunk c + 2, once chunk c - 2's G MMAs have read the slot
                bool okFe = okPre;
                okPre = true;
                if (c + 2 < nck) {
                    const uint32_t qq = q + 2, ff = qq & 3u;
                    if (qq >= 4) okFe = okFe && mbar_wait(&bars[kBarFe + ff], ((qq >> 2) + 1) & 1u);
                    load_fe(doG && okFe, bG, c + 2, ff);
                } else {
                    cp_async_commit();  // the group count stays one per chunk
                }
                // the staged chunk has landed; chunk q - 2's MMAs have read hi / lo slot s
                {
                    const bool ok = okFe && mbar_wait(&bars[kBarStg + s], (q >> 1) & 1u);
                    const bool ok2 = ok && (q < 2 || mbar_wait(&bars[kBarHL + s], ((q >> 1) + 1) & 1u));
                    if (__syncthreads_or(!ok2)) return false;
                }
                // FP32 -> BF16 hi + lo, K-major swizzled; pixels outside the camera are zero
                {
                    const int prow = tid >> 2, qq = tid & 3;
                    const int qx = x0 + (prow & 15), qy = y0 + (prow >> 4);
                    const bool qin = qx < cam.W && qy < cam.H;
                    const float4 *src = reinterpret_cast<const float4 *>(sStg + s * C::kStgBytes + prow * (kCK * 4) +
                                                                         qq * 64);
                    uint8_t *hi = sHi + s * (128 * 128), *lo = sLo + s * (128 * 128);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float4 a = qin ? src[2 * h] : make_float4(0.f, 0.f, 0.f, 0.f);
                        float4 bq = qin ? src[2 * h + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
                        const float x[8] = {a.x, a.y, a.z, a.w, bq.x, bq.y, bq.z, bq.w};
                        uint4 hv, lv;
                        uint32_t *hp = &hv.x, *lp = &lv.x;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const __nv_bfloat162 hh = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
                            const float2 hb = __bfloat1622float2(hh);
                            hp[i] = *reinterpret_cast<const uint32_t *>(&hh);
                            lp[i] = pack_bf16(x[2 * i] - hb.x, x[2 * i + 1] - hb.y);
                        }
                        const uint32_t off = swz(prow, 2 * qq + h);
                        *reinterpret_cast<uint4 *>(hi + off) = hv;
                        *reinterpret_cast<uint4 *>(lo + off) = lv;
                    }
                }
                ++qStg;
                cp_async_wait<2>();  // this chunk's features have landed (chunks c + 1, c + 2 may not)
                fence_async_smem();
                __syncthreads();
                if (c + 2 < nck) issue_stage(ig, c + 2);  // staging slot s has been read
                tc_after();
                const uint64_t aHi = sdesc(sHi_s + s * (128 * 128), 16, 1024);
                const uint64_t aLo = sdesc(sLo_s + s * (128 * 128), 16, 1024);
                const uint64_t bFe = sdesc(sFe_s + f * (kSB * 128), 16, 1024);
                if (tid == 0 || tid == 32) {
                    const bool lo = tid == 32;
                    if (doG) {
#pragma unroll
                        for (int ks = 0; ks < kCK / 16; ++ks)
                            mma_bf16(lo ? tGl : tG, (lo ? aLo : aHi) + (uint64_t)((ks * 32) >> 4),
                                     bFe + (uint64_t)((ks * 32) >> 4), idG, (c > 0 || ks > 0) ? 1u : 0u);
                    }
                    mma_commit(&bars[kBarHL + s]);
                    mma_commit(&bars[kBarFe + f]);
                    if (doG && c == nck - 1) mma_commit(&bars[kBarG]);
                }
                if (tid == 64 && (c & 1)) {
                    // channels [128 kk, 128 kk + 128): hi slots 0 and 1 as one M = 128 MN-major operand
                    if (doF) {
                        const uint32_t tF = taddr + C::kColF + (nBlk & 1u) * kSB;
                        const uint64_t aF = sdesc(sHi_s, 128 * 128, 1024);
#pragma unroll
                        for (int ks = 0; ks < 128 / 16; ++ks)
                            mma_bf16(tF, aF + (uint64_t)((ks * 2048) >> 4), dW0 + (uint64_t)((ks * 2048) >> 4), idF,
                                     ks > 0 ? 1u : 0u);
                        mma_commit(&bars[kBarDfe + (nBlk & 1u)]);
                    }
                    mma_commit(&bars[kBarHL + 0]);
                    mma_commit(&bars[kBarHL + 1]);
                }
                if ((c & 1) && doF) {
                    ++nBlk;
                    if (c >= 3 && !drain_f(bF, (c >> 1) - 1)) return false;
                }
            }
            if (doF && !drain_f(bF, nck / 2 - 1)) return false;
            if (doG) ++nG;
            return true;
        };

        // the moments of batch b into the footprint gradients, with its colour sums
        auto drain_m = [&](int b) -> bool {
            if (!wait_all(&bars[kBarM], nMw & 1u)) return false;
            ++nMw;
            tc_after();
            const int be = Lmax - b * kSB, bs = max(0, be - kSB), dnb = be - bs;
            const int q = warp & 3;
            // lanes 0..63 hold the t-hi part of Gaussian (lane) (warps 0, 1),
            // lanes 64..127 the t-lo part (warps 6, 7); both add their share,
            // the colour sums go with the hi part
            if ((grp == 0 && q < 2) || (grp == 1 && q >= 2)) {
                const bool hi = grp == 0;
                const int j = (q & 1) * 32 + lane;
                const uint32_t wmask = sMask(b)[q & 1] & (dnb >= (q & 1) * 32 + 32 ? 0xFFFFFFFFu
                                       : (dnb > (q & 1) * 32 ? (1u << (dnb - (q & 1) * 32)) - 1u : 0u));
                const bool mine = (wmask >> lane) & 1u;
                const uint32_t gid = sgid(b)[j];
                float m[16];
                tmem_ld16(tM + ((uint32_t)(q * 32) << 16), m);
                if (mine) {
                    const GRec r = srec(b)[j];
                    const float a = r.a.x - (float)x0 - 0.5f, bb = r.a.y - (float)y0 - 0.5f;
                    const float M0 = m[0], Mi = m[1], Mj = m[2], Mii = m[3], Mij = m[4], Mjj = m[5];
                    const float Sx = Mi - a * M0, Sy = Mj - bb * M0;
                    const float Sxx = Mii - 2.f * a * Mi + a * a * M0;
                    const float Sxy = Mij - a * Mj - bb * Mi + a * bb * M0;
                    const float Syy = Mjj - 2.f * bb * Mj + bb * bb * M0;
                    const float op = r.b.y, cA = r.a.z, cB = r.a.w, cC = r.b.x;
                    float4 *dst = reinterpret_cast<float4 *>(g2dc + 12 * (long long)gid);
                    atomicAdd(dst, make_float4(op * (cA * Sx + cB * Sy), op * (cB * Sx + cC * Sy),
                                               -0.5f * op * Sxx, -op * Sxy));
                    atomicAdd(dst + 1, make_float4(-0.5f * op * Syy, M0, hi ? sRgb(b)[3 * j] : 0.f,
                                                   hi ? sRgb(b)[3 * j + 1] : 0.f));
                    if (hi) atomicAdd(g2dc + 12 * (long long)gid + 8, sRgb(b)[3 * j + 2]);
                }
            }
            tc_before();
            __syncthreads();
            if (tid < kSB) sRgb(b)[3 * tid] = sRgb(b)[3 * tid + 1] = sRgb(b)[3 * tid + 2] = 0.f;
            if (tid < 2) sMask(b)[tid] = 0u;
            return true;
        };

        // ---- the item: ids of batches 0 and 1, records of batch 0, G of batch 0
        load_gid(0);
        load_gid(1);
        cp_async_wait_all();
        __syncthreads();
        load_rec(0);
        if (!run_pass(-1, 0)) {
            timeout = true;
            break;
        }
        const float fpx = px + 0.5f, fpy = py + 0.5f;
        float S = T * (dC0 * p.bg0 + dC1 * p.bg1 + dC2 * p.bg2);  // the background term of dL/dalpha
        bool fail = false;
#pragma unroll 1
        for (int b = 0; b < nbat; ++b) {
            const int be = Lmax - b * kSB, bs = max(0, be - kSB), nb = be - bs;
            cp_async_wait_all();  // records of batch b, ids of batch b + 1
            {
                const bool ok = mbar_wait(&bars[kBarG], nGw & 1u);  // G of batch b
                if (__syncthreads_or(!ok)) {
                    fail = true;
                    break;
                }
                ++nGw;
            }
            load_gid(b + 2);
            load_rec(b + 1);
            tc_after();
            const GRec *R = srec(b);
            float Gv[kJ];
            {  // G = hi part + lo part
                const uint32_t lq = ((uint32_t)((warp & 3) * 32) << 16) + grp * kJ;
                float gl[kJ];
                tmem_ld16(tG + lq, Gv);
                tmem_ld16(tGl + lq, gl);
#pragma unroll
                for (int jj = 0; jj < kJ; ++jj) Gv[jj] += gl[jj];
            }
            float al[kJ], gx[kJ], Tj[kJ];
            float P = 1.f;
            const int jlim = min(nb, lastp - bs);  // Gaussians past the batch or the pixel's last
#pragma unroll
            for (int jj = 0; jj < kJ; ++jj) {
                const int j = grp * kJ + jj;
                const float4 A4 = R[j].a, B4 = R[j].b;
                const float dx = fpx - A4.x, dy = fpy - A4.y;
                const float q2 = eval_q2(dx, dy, A4.z, A4.w, B4.x);
                const float G = gauss_q2(q2);
                const float rho = B4.y * G;
                const float aa = fminf(p.amax, rho);
                const bool ok = (j < jlim) && (q2 <= p.cut) && (aa >= p.amin);
                al[jj] = ok ? aa : 0.f;
                gx[jj] = (ok && rho <= p.amax) ? G : 0.f;
                P *= 1.f - al[jj];
            }
            if (grp >= 1) xP[(grp - 1) * 128 + pidx] = P;
            tc_before();
            __syncthreads();
            // T after this group's Gaussians (the later groups' products of
            // (1 - alpha) divided out), then T before each of them
            float Pl = 1.f;
#pragma unroll
            for (int m = 1; m < kSG; ++m)
                if (m > grp) Pl *= xP[(m - 1) * 128 + pidx];
            const float Tend = grp == kSG - 1 ? T : __fdividef(T, Pl);
            const float Tstart = __fdividef(Tend, P);
            {
                float t = Tstart;
#pragma unroll
                for (int jj = 0; jj < kJ; ++jj) {
                    Tj[jj] = t;
                    t *= 1.f - al[jj];
                }
            }
            // App. A.2 back to front: dL/dalpha_k = T_k g_k - S_k / (1 - alpha_k),
            // g_k = dC.c_k + dF.f_k; Gv becomes t_k = G dL/drho (earlier groups:
            // still without S + S_>g)
            float Sg = grp == kSG - 1 ? S : 0.f;
#pragma unroll
            for (int jj = kJ - 1; jj >= 0; --jj) {
                const int j = grp * kJ + jj;
                const bool c = al[jj] > 0.f;  // selects: records past the batch end are stale
                const float w = al[jj] * Tj[jj];
                const float4 B4 = R[j].b;
                const float gc = Gv[jj] + dC0 * B4.z + dC1 * B4.w + dC2 * R[j].c.x;
                const float g = c ? gc : 0.f;
                const float dal = Tj[jj] * g - __fdividef(Sg, 1.f - al[jj]);
                Sg = c ? Sg + w * g : Sg;
                Gv[jj] = c ? gx[jj] * dal : 0.f;
            }
            if (grp >= 1) xSg[(grp - 1) * 128 + pidx] = grp == kSG - 1 ? Sg - S : Sg;
            __syncthreads();
            if (grp < kSG - 1) {
                float Sb = S;  // suffix sum entering this group's Gaussians
#pragma unroll
                for (int m = 1; m < kSG; ++m)
                    if (m > grp) Sb += xSg[(m - 1) * 128 + pidx];
#pragma unroll
                for (int jj = 0; jj < kJ; ++jj) Gv[jj] -= __fdividef(gx[jj] * Sb, 1.f - al[jj]);
                if (grp == 0) {
                    S = Sb + Sg;
                    T = Tstart;
                    xT[pidx] = T;
                    xS[pidx] = S;
                }
            }
            // weights (B of dFe^T) and t hi / lo (A of the moments): the previous
            // batch's MMAs that read them have completed (drained and waited)
#pragma unroll
            for (int q = 0; q < kJ / 8; ++q) {
                uint4 pw, ph, pl;
                uint32_t *pwv = &pw.x, *phv = &ph.x, *plv = &pl.x;
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int j0 = 8 * q + 2 * h;
                    pwv[h] = pack_bf16(al[j0] * Tj[j0], al[j0 + 1] * Tj[j0 + 1]);
                    const __nv_bfloat162 th = __floats2bfloat162_rn(Gv[j0], Gv[j0 + 1]);
                    const float2 tb = __bfloat1622float2(th);
                    phv[h] = *reinterpret_cast<const uint32_t *>(&th);
                    plv[h] = pack_bf16(Gv[j0] - tb.x, Gv[j0 + 1] - tb.y);
                }
                const uint32_t off = swz(pidx, grp * (kJ / 8) + q);
                *reinterpret_cast<uint4 *>(sW + off) = pw;
                *reinterpret_cast<uint4 *>(sTh + off) = ph;
                *reinterpret_cast<uint4 *>(sTl + off) = pl;
            }
            // which Gaussians contribute anywhere in the half tile: one OR per warp
            uint32_t cmask = 0;
#pragma unroll
            for (int jj = 0; jj < kJ; ++jj) cmask |= (al[jj] > 0.f ? 1u : 0u) << jj;
            cmask = __reduce_or_sync(0xffffffffu, cmask);
            if (lane == 0 && cmask) atomicOr(&sMask(b)[(grp * kJ) >> 5], cmask << ((grp * kJ) & 31));
            // colour sums sum_p w dC_p per Gaussian: a reduce-scatter over the
            // warp's 32 pixels leaves lanes 2l and 2l + 1 with Gaussian kJ grp + l
            if (cmask) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float dc = c == 0 ? dC0 : (c == 1 ? dC1 : dC2);
                    float v[kJ];
#pragma unroll
                    for (int jj = 0; jj < kJ; ++jj) v[jj] = al[jj] * Tj[jj] * dc;
                    rs_step_s(v, lane, 16, kJ / 2);
                    rs_step_s(v, lane, 8, kJ / 4);
                    rs_step_s(v, lane, 4, kJ / 8);
                    rs_step_s(v, lane, 2, kJ / 16);
                    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
                    const int jl = lane >> 1;
                    if (!(lane & 1) && (cmask & (1u << jl))) atomicAdd(&sRgb(b)[3 * (grp * kJ + jl) + c], v[0]);
                }
            }
            fence_async_smem();  // weights and t (generic writes) -> the MMA operands
            __syncthreads();
            if (grp != 0) {
                T = xT[pidx];
                S = xS[pidx];
            }
            if (tid == 96) {  // moments = t^T X, t hi in rows 0..63 and t lo in rows 64..127
                tc_after();
#pragma unroll
                for (int ks = 0; ks < 128 / 16; ++ks)
                    mma_bf16(tM, dTh0 + (uint64_t)((ks * 2048) >> 4),
                             dX0 + (uint64_t)(((ks >> 2) * (16 * 128) + (ks & 3) * 32) >> 4), idM, ks > 0 ? 1u : 0u);
                mma_commit(&bars[kBarM]);
            }
            ++nM;
            if (!run_pass(b, b + 1) || !drain_m(b)) {
                fail = true;
                break;
            }
        }
        if (fail) {
            timeout = true;
            break;
        }
    }
    if (timeout) {
        // quiesce: every issuing thread commits once more, so that one wait
        // covers all its MMAs; then the staging copies in flight
        if (tid == 0) latch(status, ST_TIMEOUT);
        if (tid == 0 || tid == 32 || tid == 64 || tid == 96) mma_commit(&bars[kBarQ]);
        mbar_wait(&bars[kBarQ], 0);
        for (uint32_t q = qStg; q < qIss; ++q) mbar_wait(&bars[kBarStg + (q & 1u)], (q >> 1) & 1u);
    }
    cp_async_wait_all();
    tc_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, C::kTmemCols);
    (void)nG;
    (void)nM;
    (void)nBlk;
}

}  // namespace

bool bwd_stream_supported(int D) { return D > 0 && D % 128 == 0; }

bool launch_render_bwd_stream(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                              const __nv_bfloat16 *feats, int D, const float *T, const int32_t *last,
                              const float *grgb, const float *gfeat, float *g2d, float *gfeatures, unsigned *status,
                              cudaStream_t st) {
    CUtensorMap dfm;
    memset(&dfm, 0, sizeof(dfm));
    if (gfeat == nullptr || !bwd_stream_supported(D) || !encode_f32_rows_tmap(&dfm, gfeat, cs.total_pix, D, kCK, 16))
        return false;
    const int n_items = cs.total_tiles * 2;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const dim3 grid((unsigned)max(1, min(n_items, sms)));
    static std::atomic<unsigned long long> smem_done{0};
    allow_max_smem(smem_done, k_render_bwd_stream);
    note_launch(1);
    k_render_bwd_stream<<<grid, kSThreads, SCfg::kSmem, st>>>(N, cs, p, pv, bins.gids, bins.ranges, feats, D, T, last,
                                                              grgb, dfm, g2d, gfeatures, status, n_items);
    return true;
}

}  // namespace fhgs
