// FP32 FMA throughput probe: the denominator of the "alu" rooflines.
//
// Every thread runs kChains independent FMA chains (enough to cover the FMA
// latency with four warps per scheduler) for `iters` rounds; a chain is
// x = x * a + b with a, b chosen so that x stays finite and non-trivial.
// The caller times the launch with CUDA events; the work is
// 2 * kChains * iters FLOP per thread.  The result is written only if it is
// impossible (never, for finite inputs), which keeps the FMAs live.
#include "fhgs_internal.cuh"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(1024) k_ffma_probe(int iters, float a, float b, float *sink) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0f && sink) sink[blockIdx.x] = s;  // never true for the probe's inputs
}

}  // namespace

extern "C" int64_t fhgs_ffma_probe(int blocks, int iters, void *stream) {
    if (blocks <= 0 || iters <= 0) return -1;
    // a = 0.5, b = 1: every chain converges to 2 and stays finite and positive
    k_ffma_probe<<<blocks, 1024, 0, (cudaStream_t)stream>>>(iters, 0.5f, 1.0f, nullptr);
    fhgs::note_launch(1);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return 2ll * kChains * 16 * (int64_t)iters * 1024 * blocks;
}
