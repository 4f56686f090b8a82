// The device side of one training iteration (App. A, Alg. 1 loop body):
// the L1 photometric loss with its gradient, and an Adam update of the raw
// Gaussian parameters.
//
// Raw parameters follow the 3DGS family: means, log-scales, unnormalised
// quaternions, opacity logits and SH.  The rasterizer's backward gives the
// gradient with respect to the activated values (scales = exp(log-scales),
// opacities = sigmoid(logits)), so the update first takes them to the raw
// ones (d/dlog s = s d/ds, d/dlogit = op (1 - op) d/dop), then applies Adam
// (m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, theta -= lr m_hat /
// (sqrt(v_hat) + eps)) and writes the activated scales and opacities that
// the next forward reads.  The update is elementwise over flat arrays.
#include "fhgs_internal.cuh"

namespace fhgs {
namespace {

__global__ void __launch_bounds__(256) k_l1_loss(long long m, const float *__restrict__ a, const float *__restrict__ b,
                                                 float inv_count, float *loss, float *grad) {
    float s = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
        const float d = a[i] - b[i];
        s += fabsf(d);
        if (grad) grad[i] = d > 0.f ? inv_count : (d < 0.f ? -inv_count : 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        atomicAdd(loss, t * inv_count);
    }
}

struct AdamArgs {
    float lr[5];
    float b1, b2, eps, c1, c2;  // c1 = 1 - b1^t, c2 = 1 - b2^t
};

__device__ __forceinline__ float adam_one(float theta, float g, float &m, float &v, float lr, const AdamArgs &a) {
    m = a.b1 * m + (1.f - a.b1) * g;
    v = a.b2 * v + (1.f - a.b2) * g * g;
    return theta - lr * (m / a.c1) / (sqrtf(v / a.c2) + a.eps);
}

// Up to four gradient sets (render, NDFD, ...) that the update sums.
struct GradSets {
    const float *means[4], *scales[4], *quats[4], *opac[4], *sh[4];
    int n;
};

__device__ __forceinline__ float gsum(const float *const *g, int ns, long long j) {
    float s = g[0][j];
    for (int k = 1; k < ns; ++k) s += g[k][j];
    return s;
}

// Adam is elementwise: one flat index space over the five groups (means,
// log-scales, quaternions, opacity logits, SH), one element per thread in
// a grid-stride loop, so that every parameter, moment and gradient array is
// read and written with unit stride.  The raw-gradient factors (s for the
// log-scales, op (1 - op) for the logits) use the element's own value.
__global__ void __launch_bounds__(256) k_adam_gaussians(long long n, int K3, float *means, float *log_s, float *quats,
                                                        float *logit, float *sh, GradSets gs, float *state, AdamArgs a,
                                                        float *scales_out, float *opac_out) {
    const int ns = gs.n;
    // group boundaries in the flat index: means 3n, log-scales 3n, quats 4n, logits n, SH K3 n
    const long long e0 = 3 * n, e1 = 6 * n, e2 = 10 * n, e3 = 11 * n, e4 = (11 + (long long)K3) * n;
    // state: m and v of each group, group after group
    float *m_mu = state, *v_mu = m_mu + 3 * n;
    float *m_ls = v_mu + 3 * n, *v_ls = m_ls + 3 * n;
    float *m_q = v_ls + 3 * n, *v_q = m_q + 4 * n;
    float *m_lo = v_q + 4 * n, *v_lo = m_lo + n;
    float *m_sh = v_lo + n, *v_sh = m_sh + (long long)K3 * n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < e4; i += (long long)gridDim.x * blockDim.x) {
        if (i < e0) {
            means[i] = adam_one(means[i], gsum(gs.means, ns, i), m_mu[i], v_mu[i], a.lr[0], a);
        } else if (i < e1) {
            const long long j = i - e0;
            const float g = gsum(gs.scales, ns, j) * expf(log_s[j]);
            const float t = adam_one(log_s[j], g, m_ls[j], v_ls[j], a.lr[1], a);
            log_s[j] = t;
            if (scales_out) scales_out[j] = expf(t);
        } else if (i < e2) {
            const long long j = i - e1;
            quats[j] = adam_one(quats[j], gsum(gs.quats, ns, j), m_q[j], v_q[j], a.lr[2], a);
        } else if (i < e3) {
            const long long j = i - e2;
            const float op = 1.f / (1.f + expf(-logit[j]));
            const float g = gsum(gs.opac, ns, j) * op * (1.f - op);
            const float t = adam_one(logit[j], g, m_lo[j], v_lo[j], a.lr[3], a);
            logit[j] = t;
            if (opac_out) opac_out[j] = 1.f / (1.f + expf(-t));
        } else {
            const long long j = i - e3;
            sh[j] = adam_one(sh[j], gsum(gs.sh, ns, j), m_sh[j], v_sh[j], a.lr[4], a);
        }
    }
}

// The activated values the rasterizer reads: scales = exp(log-scales),
// opacities = sigmoid(logits), as the Adam kernel writes them after an update.
__global__ void __launch_bounds__(256) k_activate(long long n, const float *__restrict__ log_s,
                                                  const float *__restrict__ logit, float *scales, float *opac) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < 3; ++k) scales[3 * i + k] = expf(log_s[3 * i + k]);
    opac[i] = 1.f / (1.f + expf(-logit[i]));
}

// out[0] += sum x (block partial sums, one float atomic per block).
__global__ void __launch_bounds__(256) k_sum(long long m, const float *__restrict__ x, float *out) {
    float s = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
        s += x[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        atomicAdd(out, t);
    }
}

}  // namespace

void launch_l1_loss(long long m, const float *a, const float *b, float inv_count, float *loss, float *grad,
                    int sm_count, cudaStream_t st) {
    if (m == 0) return;
    note_launch(1);
    const long long want = (m + 255) / 256;
    const unsigned blocks = (unsigned)min(want, (long long)sm_count * 8);
    k_l1_loss<<<blocks, 256, 0, st>>>(m, a, b, inv_count, loss, grad);
}

void launch_adam_gaussians(long long n, int K, float *means, float *log_s, float *quats, float *logit, float *sh,
                           const fhgs_grads *grads, int n_sets, float *state, const fhgs_adam *opt, float *scales_out,
                           float *opac_out, cudaStream_t st) {
    if (n == 0) return;
    GradSets gs;
    gs.n = n_sets;
    for (int k = 0; k < 4; ++k) {
        const fhgs_grads &g = grads[k < n_sets ? k : 0];
        gs.means[k] = g.means;
        gs.scales[k] = g.scales;
        gs.quats[k] = g.quats;
        gs.opac[k] = g.opacities;
        gs.sh[k] = g.sh;
    }
    AdamArgs a;
    for (int k = 0; k < 5; ++k) a.lr[k] = opt->lr[k];
    a.b1 = opt->beta1;
    a.b2 = opt->beta2;
    a.eps = opt->eps;
    a.c1 = 1.f - powf(opt->beta1, (float)opt->step);
    a.c2 = 1.f - powf(opt->beta2, (float)opt->step);
    note_launch(1);
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long total = (11 + 3ll * K) * n;
    const unsigned blocks = (unsigned)min((total + 255) / 256, (long long)sms * 16);
    k_adam_gaussians<<<blocks, 256, 0, st>>>(n, 3 * K, means, log_s, quats, logit, sh, gs, state, a, scales_out,
                                             opac_out);
}

void launch_activate(long long n, const float *log_s, const float *logit, float *scales, float *opac,
                     cudaStream_t st) {
    if (n == 0) return;
    note_launch(1);
    k_activate<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, log_s, logit, scales, opac);
}

void launch_sum(long long m, const float *x, float *out, int sm_count, cudaStream_t st) {
    if (m == 0) return;
    note_launch(1);
    const long long want = (m + 255) / 256;
    const unsigned blocks = (unsigned)min(want, (long long)sm_count * 8);
    k_sum<<<blocks, 256, 0, st>>>(m, x, out);
}

}  // namespace fhgs
