// sl1m_sfu.cu -- measured issue rate of the special-function unit (MUFU).
//
// The operator kernels are bound by the SFU: per pixel-visibility pair they
// run sin and cos (and, for Gaussian pixels, exp2) on the MUFU pipe.  The
// roofline those kernels are judged against takes the MUFU rate from the
// CUDA throughput table (16 results per clock per SM); this file measures it
// on the device at hand, so that the table value is checked, not assumed.
//
// Each thread runs 8 independent dependency chains x <- f(x) of one MUFU
// function (sin.approx, cos.approx or ex2.approx, inline PTX), enough
// independent work per warp to hide the unit's latency; a persistent grid of
// several CTAs per SM keeps every SM's SFU busy.  The rate is results per
// second over the launch's CUDA-event time.
#include <cuda_runtime.h>

#include "sl1m_host.h"

namespace {

constexpr int CHAINS = 8;
constexpr int THREADS = 256;

template <int F>
__device__ __forceinline__ float mufu(float x)
{
    float y;
    if (F == 0) asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    else if (F == 1) asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    else asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));   // 2^-x keeps x in (0, 1]
    return y;
}

// F = 0: sin and cos alternating over the chains (a sincos pair per two
// results); F = 2: exp2.
template <int F>
__global__ void __launch_bounds__(THREADS) mufu_rate_kernel(float* sink, int iters)
{
    float a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = 1e-3f * (float)((threadIdx.x * 7 + k * 131) & 1023);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; k += 2) {
            a[k] = mufu<F == 0 ? 0 : 2>(a[k]);
            a[k + 1] = mufu<F == 0 ? 1 : 2>(a[k + 1]);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == 1234.5f) sink[blockIdx.x] = s;   // keeps the chains live; never true in practice
}

template <int F>
cudaError_t time_rate(int grid, int iters, cudaStream_t st, float* sink, double* per_s)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    float best = 0.0f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {     // the first is a warm-up
        cudaEventRecord(e0, st);
        mufu_rate_kernel<F><<<grid, THREADS, 0, st>>>(sink, iters);
        e = cudaGetLastError();
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess)
        *per_s = (double)grid * THREADS * CHAINS * (double)iters / (best * 1e-3);
    return e;
}

}  // namespace

extern "C" int sl1m_measure_sfu(sl1m_ctx* ctx, double* sincos_per_s, double* ex2_per_s)
{
    if (!ctx || !sincos_per_s || !ex2_per_s) return SL1M_ERR_ARG;
    if (ctx->server) return sl1m_fail(ctx, SL1M_ERR_BUSY, "a server is running on this context");
    cudaError_t e = cudaSetDevice(ctx->device);
    DBuf<float> sink;
    if (e == cudaSuccess) e = sink.alloc(4 * ctx->num_sms);
    const int grid = 4 * ctx->num_sms, iters = 4096;
    if (e == cudaSuccess) e = time_rate<0>(grid, iters, ctx->stream, sink.p, sincos_per_s);
    if (e == cudaSuccess) e = time_rate<2>(grid, iters, ctx->stream, sink.p, ex2_per_s);
    if (e != cudaSuccess) return sl1m_fail(ctx, SL1M_ERR_CUDA, "sl1m_measure_sfu: %s", cudaGetErrorString(e));
    ctx->n_launch += 8;
    return SL1M_OK;
}
