// hr_calib.cu -- the FP32 FMA pipe's throughput on this GPU, measured.
//
// The FP64-class kernels compute with pairs of floats, so their roofline is
// the FP32 FMA pipe, not HBM.  Its nominal rate (SMs x 128 lanes x clock)
// assumes every operand of every FMA is read from the register file at full
// rate; this call measures what the pipe delivers: independent FMA chains
// whose multiplier and addend are shared (the operand-reuse best case), as
// scalar FFMA and as packed f32x2 FMA, timed with CUDA events.  Benchmarks
// state the double-float hop's FP32-pipe fraction against it.
#include "hr_host.h"

using namespace hr;

namespace {

constexpr int kChains = 16;

template <bool PAIRED>
__global__ void __launch_bounds__(256) k_fma_rate(float *sink, int iters, float b, float c)
{
    if constexpr (PAIRED) {
        float2 a[kChains / 2];
#pragma unroll
        for (int k = 0; k < kChains / 2; ++k) a[k] = make_float2(threadIdx.x * 1e-7f * k, blockIdx.x * 1e-9f * k);
        const float2 bb = make_float2(b, b), cc = make_float2(c, c);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kChains / 2; ++k) a[k] = __ffma2_rn(a[k], bb, cc);
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kChains / 2; ++k) s += a[k].x + a[k].y;
        if (s == 1234.5f) sink[0] = s; // keeps the chains alive; never true for these inputs
    } else {
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 1e-7f * k;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = __fmaf_rn(a[k], b, c);
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += a[k];
        if (s == 1234.5f) sink[0] = s;
    }
}

} // namespace

extern "C" hr_status hr_fp32_fma_rate(hr_ctx *ctx, double *scalar_lane_ops, double *paired_lane_ops,
                                      hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (!scalar_lane_ops || !paired_lane_ops) return set_error(ctx, HR_ERR_INVALID_ARG, "null result pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (ctx->sm_count > 0 ? ctx->sm_count : 152) * 8, threads = 256, iters = 4096;
    // 0.9 and a small addend keep the chains finite and away from subnormals
    const float b = 0.9f, c = 1e-3f;
    float *sink = reinterpret_cast<float *>(ctx->d_partials);
    double rate[2] = {0.0, 0.0};
    for (int paired = 0; paired < 2; ++paired) {
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) { // the first launch warms up; best of the rest
            cudaError_t e = cudaEventRecord(ctx->ev0, s);
            if (paired) k_fma_rate<true><<<blocks, threads, 0, s>>>(sink, iters, b, c);
            else k_fma_rate<false><<<blocks, threads, 0, s>>>(sink, iters, b, c);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(ctx->ev1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(ctx->ev1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return set_error(ctx, HR_ERR_CUDA, "FMA rate: %s", cudaGetErrorString(e));
            }
            if (rep > 0 && ms < best) best = ms;
        }
        rate[paired] = (double)blocks * threads * iters * kChains / (best * 1e-3);
    }
    *scalar_lane_ops = rate[0];
    *paired_lane_ops = rate[1];
    return HR_OK;
}
