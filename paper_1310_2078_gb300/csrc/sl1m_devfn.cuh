// sl1m_devfn.cuh -- device helpers shared by the operator kernels (internal).
#pragma once
#include "sl1m_dev.h"
#include "sl1m_sincos_poly.h"

namespace sl1m {

#define TWO_PI_F 6.283185307179586f
#define INV_TWO_PI_F 0.15915494309189535f
#define LOG2E_F 1.4426950408889634f

// {u, v, -2 w, u^2 + v^2}: a streamed visibility as the adjoint's Gaussian
// terms use it (t = u l + v m + (-2 w) r^2/4, |(u,v) - w (l,m)|^2 = u^2 + v^2 + (-2 w) t).
__device__ __forceinline__ float4 vis_for_gauss(const float4 a)
{
    return make_float4(a.x, a.y, -2.0f * a.z, fmaf(a.x, a.x, a.y * a.y));
}

// {l, m, r^2/4, pi nu}: an owned Gaussian pixel as the adjoint uses it.
__device__ __forceinline__ float4 pix_for_gauss(const float4 a)
{
    return make_float4(a.x, a.y, 0.5f * a.z, 3.14159265358979f * a.w);
}

// The x, y, z of an offset in radians per turn (w unchanged).
__device__ __forceinline__ float4 to_rad(const float4 a)
{
    return make_float4(a.x * TWO_PI_F, a.y * TWO_PI_F, a.z * TWO_PI_F, a.w);
}

// x - rint(x) for |x| < 2^22, exact: adding and removing 1.5 * 2^23 rounds x
// to the nearest integer (ties to even) on the FP32 add pipe.
__device__ __forceinline__ float frac_turns(float x)
{
    const float M = 12582912.0f;
    return __fsub_rn(x, __fsub_rn(__fadd_rn(x, M), M));
}

// frac(a*b) in turns for a = ah + al, b = bh + bl: p + e == ah*bh exactly
// (TwoProduct with one fma), p - rint(p) is exact, the cross terms are small.
// The rounding is frac_turns' FP32-add trick, exact for |p| <= 2^22; the
// host refuses problems whose coordinate products could reach 2^21.
__device__ __forceinline__ float tp_frac(float ah, float al, float bh, float bl)
{
    const float p = __fmul_rn(ah, bh);
    const float e = __fmaf_rn(ah, bh, -p);
    const float f = frac_turns(p);
    const float lo = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
    return __fadd_rn(f, lo);
}

// frac(a . b) over x, y, z in turns, result in [-0.5, 0.5].
__device__ __forceinline__ float frac_dot3(const float4 ah, const float4 al,
                                           const float4 bh, const float4 bl)
{
    float s = __fadd_rn(tp_frac(ah.x, al.x, bh.x, bl.x), tp_frac(ah.y, al.y, bh.y, bl.y));
    s = __fadd_rn(s, tp_frac(ah.z, al.z, bh.z, bl.z));
    return frac_turns(s);
}

// sin and cos of ph (radians, |ph| < 2^22 turns) on the FMA pipe, for a share
// of the pairs so that the SFU is not the only pipe doing sincos: ph is reduced
// to turns f in [-1/2, 1/2]; h = sqrt(2) sin(pi f) and q = sqrt(2) cos(pi f)
// are Chebyshev interpolants in f^2 (sl1m_sincos_poly.h); then the double-angle
// formulas give sin(2 pi f) = h q and cos(2 pi f) = 1 - h^2.  Absolute error
// below 6e-7, the size of the SFU's own.  16 FMA-pipe instructions.
__device__ __forceinline__ void sincos_fma(float ph, float& s, float& c)
{
    const float f = frac_turns(ph * INV_TWO_PI_F);
    const float z = f * f;
    const float h = f * fmaf(fmaf(fmaf(fmaf(SCP4, z, SCP3), z, SCP2), z, SCP1), z, SCP0);
    const float q = fmaf(fmaf(fmaf(fmaf(SCQ4, z, SCQ3), z, SCQ2), z, SCQ1), z, SCQ0);
    s = h * q;
    c = fmaf(-h, h, 1.0f);
}

// The cosine alone by the same interpolant (the adjoint needs no sine):
// cos(2 pi f) = 1 - h^2.  11 FMA-pipe instructions.
__device__ __forceinline__ float cos_fma(float ph)
{
    const float f = frac_turns(ph * INV_TWO_PI_F);
    const float h = f * fmaf(fmaf(fmaf(fmaf(SCP4, f * f, SCP3), f * f, SCP2), f * f, SCP1), f * f, SCP0);
    return fmaf(-h, h, 1.0f);
}

// ---- bulk (TMA) copies global -> shared, completed on an mbarrier
__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// makes the barrier initialisation visible to the async (TMA) proxy
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// orders this CTA's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) writes to the same memory
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// One thread: arrive on bar (its one expected arrival) and announce `bytes`
// of copies that will complete on it.
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// src to shared dst; completes `bytes` of bar's announced transactions.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// One thread: arrive on bar expecting `bytes`, then copy them from src to dst.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar)
{
    mbar_arrive_expect(bar, bytes);
    bulk_copy(dst, src, bytes, bar);
}
// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// How long a wait for a bulk copy may take before it gives up: a copy of a
// stage (a few to 40 KB) lands in microseconds, so 20 ms is far beyond any
// wait that will still end.
constexpr unsigned long long WAIT_LIMIT_NS = 20ull * 1000 * 1000;

__device__ __forceinline__ bool mbar_try(unsigned a, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait until the phase of bar with this parity has completed, bounded by
// elapsed time: after WAIT_LIMIT_NS on the global timer it gives up and sets
// `fault`.  A thread whose `fault` is already set does not wait at all, and
// the kernels issue no further bulk copies from a thread whose `fault` is set,
// so a kernel whose copies stopped completing gives up once per thread,
// records the fault (the caller) and runs to its end; no barrier of the CTA is
// left waiting.
__device__ __forceinline__ void mbar_wait(unsigned long long* bar, unsigned parity, bool& fault)
{
    if (fault) return;
    const unsigned a = smem_u32(bar);
    for (int i = 0; i < 8; ++i)                 // the usual case: done at once or soon
        if (mbar_try(a, parity)) return;
    const unsigned long long t0 = global_ns();
    while (!mbar_try(a, parity)) {
        if (global_ns() - t0 > WAIT_LIMIT_NS) {
            fault = true;
            return;
        }
    }
}
// Dynamic shared memory of this launch, in bytes.
__device__ __forceinline__ unsigned dyn_smem_bytes()
{
    unsigned r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float dot3(const float4 a, const float4 b)
{
    return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}

// Largest p with prob_u0[p] <= u (problems with no units are skipped).
__device__ __forceinline__ int find_prob(const Plan& pl, long long u)
{
    int lo = 0, hi = pl.n_probs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pl.prob_u0[mid] <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int slot_of(const Plan& pl, int gblk)
{
    return pl.blk_poff[gblk] + ((int)blockIdx.x - pl.blk_clo[gblk]);
}

// Constants of one (visibility, Gaussian scale) pair, Eq. samlm4 in split form.
struct GaussConst {
    float beta, id, gamr, coef;  // beta = w s^2, id = 1/(1+beta^2), gamr = 2 pi beta^2 id
                                 // (radians per turn of t), coef = -pi s^2 id log2(e)
    float cphase;                // id beta s^2 (u^2+v^2)/2, turns
    float k0, k1;                // log2 of the amplitude as k0 + k1 t, t = u l + v m - w r^2/2:
                                 // |(u,v) - w (l,m)|^2 = u^2 + v^2 - 2 w t, so k0 = coef (u^2+v^2),
                                 // k1 = -2 coef w
};

__device__ __forceinline__ GaussConst gauss_const(float u, float v, float w, float sigma)
{
    GaussConst g;
    const float s2 = sigma * sigma;
    g.beta = w * s2;
    g.id = 1.0f / fmaf(g.beta, g.beta, 1.0f);
    g.gamr = g.beta * g.beta * g.id * TWO_PI_F;
    g.coef = -3.14159265358979f * s2 * g.id * LOG2E_F;
    g.cphase = 0.5f * g.id * g.beta * s2 * fmaf(u, u, v * v);
    g.k0 = g.coef * fmaf(u, u, v * v);
    g.k1 = -2.0f * g.coef * w;
    return g;
}

}  // namespace sl1m
