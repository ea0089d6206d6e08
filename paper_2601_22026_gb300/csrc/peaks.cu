// Diagnostic: sustained FP32 FMA and MUFU exp2 issue rates of this GPU, the
// denominators of the compositing kernels' arithmetic roofline (which the
// measured-peaks file, a copy bandwidth and a bf16 GEMM rate, does not give).
//
// Each thread runs eight independent dependency chains for `iters`
// iterations, so every SM sub-partition has independent instructions to issue
// each cycle; the chains' results are folded into one store per thread so
// the compiler keeps them. kind 0: scalar fma.rn.f32 (2 FLOP each); kind 1:
// packed fma.rn.f32x2 (two FMAs, 4 FLOP each); kind 2: ex2.approx.f32 (one
// MUFU operation each).
#include "common.cuh"

namespace gsfit {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) alu_rate_kernel(int kind, int iters, float seed, float* __restrict__ sink) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3f * (float)(threadIdx.x + c);
    const float m = 0.999999f, b = 1e-7f;
    if (kind == 0) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = __fmaf_rn(a[c], m, b);
        }
    } else if (kind == 1) {
        float2 p[kChains / 2];
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) p[c] = make_float2(a[2 * c], a[2 * c + 1]);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains / 2; ++c) p[c] = __ffma2_rn(p[c], make_float2(m, m), make_float2(b, b));
        }
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) {
            a[2 * c] = p[c].x;
            a[2 * c + 1] = p[c].y;
        }
    } else {
        // x -> 2^(-x) stays in (0.5, 1) for x in (0, 1): a bounded chain of MUFU operations
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(a[c]) : "f"(-a[c]));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace gsfit

using namespace gsfit;

extern "C" int gsfit_selftest_alu_rate(int32_t kind, int32_t blocks, int32_t iters, float* sink, cudaStream_t stream) {
    if (kind < 0 || kind > 2 || blocks < 1 || iters < 1 || !sink) return GSFIT_ERR_INVALID_ARG;
    alu_rate_kernel<<<blocks, 256, 0, stream>>>(kind, iters, 0.5f, sink);
    GSFIT_LAUNCH_CHECK();
    return GSFIT_OK;
}
