// sl1m_mixed.cu -- mixed-precision forward operator and adjoint of SL1M
// (Hardy 2013, Sect. 2 and 3.1) as sm_103a kernels.
//
//   forward  Vhat_k = sum_j A_kj x_j                    (Eq. sme)
//   adjoint  g_j    = sum_k Re(conj(A_kj) r_k)          (gradient, Sect. 3)
//   A_kj = g_jk P_j exp(-2 pi i (u_k l_j + v_k m_j + w_k (n_j - 1)))
//   Dirac pixels P = 1/n (Eq. deltam); Gaussian pixels (Eq. samlm4/samlm5) in
//   the real split form
//     A = (g/n) e^{Re(qc)} id (1 + i beta) exp(-2 pi i (phi_D - corr)),
//     beta = w s^2, id = 1/(1+beta^2), gam = beta^2 id,
//     Re(qc) = -pi s^2 id ((u - w l)^2 + (v - w m)^2),
//     corr = [paraxial: w nu] + gam (u l + v m - w r^2/2) - id beta s^2 (u^2+v^2)/2,
//     nu = n - 1 + r^2/2
//   (no 1/sigma^2 prefactor; wide-field residual phase w (n - 1 + r^2/2)).
//
// Phase: with X the owned element, Y the streamed one and Xc, Yc their
// granule centres,  X.Y = X.Yc + Xc.(Y - Yc) + (X - Xc).(Y - Yc) = C + B + D
// exactly.  C (per owned element and streamed granule) and B (per owned
// granule and streamed element) are reduced to fractional turns by an FP32
// TwoProduct; D is one FP32 fma chain when the tile's offset extents bound
// |D| <= D_MAX turns, else it is reduced exactly too.  On the first (common)
// path B and the owned offsets are held in radians (pre-multiplied by 2 pi),
// so B + D, at most 2 pi (1 + D_MAX) in size, goes to the SFU's sincos with
// no reduction step of its own; on the exact path the fractional turns are
// reduced exactly and then scaled.  sincos / exp2 run on the SFU in FP32;
// each granule's FP32 sum is added into FP64 accumulators.  The adjoint's
// output is real, so it takes one cosine per pair: Re(conj(A) r) =
// |A| |r| cos(arg r - arg A), with r and the gains held in polar form.
//
// Work split: a CTA owns BLK_GRAN granules of one side (one per warp, 2
// elements per lane) and streams granules of the other side through shared
// memory -- in the forward and in the gains adjoint by bulk (TMA) copies that
// complete on mbarriers, issued ahead of use; units = (owned block, streamed
// granule) are spread over a persistent grid stream-K style (Plan); partials
// are summed by the finish kernels in a fixed order.
#include <algorithm>

#include "sl1m_dev.h"
#include "sl1m_devfn.cuh"
#include "sl1m_kernels.h"

namespace sl1m {

// Gains tables in shared memory: one row of G pixels per antenna, padded to
// GP (sl1m_dev.h) so that the lanes' rows start in different banks (a row of
// antenna a starts at bank 2 a mod 32); the pixel index then enters the
// address as a constant offset.

// Set (never cleared here) by a CTA whose bounded wait for a bulk copy gave
// up; the host reads and clears it (wait_fault_read, wait_fault_clear).
__device__ unsigned int g_wait_fault;

// ----------------------------------------------------------- forward tiles

// Pair (jj, r) of every 4 streamed elements x 2 owned elements takes its
// sincos on the FMA pipe when it is one of the last NPOLY of those 8.
template <int NPOLY>
__device__ __forceinline__ constexpr bool fma_slot(int jj, int r) { return 2 * jj + r >= 8 - NPOLY; }

// UNR: groups of 4 streamed pixels per iteration of the tile's loop (the
// unrolling measured fastest: 4 in the kernel instance with Gaussian tiles,
// 8 in the Dirac-only one).
template <bool GAINS, bool EXACT, int NPOLY = 0, int UNR = 4>
__device__ __forceinline__ void fwd_dirac_tile(const float4* __restrict__ s_off,
                                               const float4* __restrict__ s_lo,
                                               const float2* __restrict__ sBa,
                                               const float2* __restrict__ s_gain,
                                               const float4 (&dx)[2], const float4 (&dxl)[2],
                                               const int2 (&ant)[2], float (&sr)[2], float (&si)[2])
{
    const float2* ga_row[2] = {s_gain + ant[0].x * GP, s_gain + ant[1].x * GP};   // GAINS only
    const float2* gb_row[2] = {s_gain + ant[0].y * GP, s_gain + ant[1].y * GP};
#pragma unroll UNR
    for (int j0 = 0; j0 < G; j0 += 4)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
        const int j = j0 + jj;
        const float4 o = s_off[j];             // {dl, dm, dn, -}
        const float2 ba = sBa[j];              // {B_j in radians, a_j = x_j / n_j}
        const float b = ba.x;
        const float4 ol = EXACT ? s_lo[j] : o;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            // with gains {|G|, arg G in turns}: a G_a conj(G_b) e^{-i ph} =
            // a |G_a| |G_b| e^{-i (ph + 2 pi (psi_b - psi_a))}
            float2 ga = make_float2(1.f, 0.f), gb = ga;
            if (GAINS) {
                ga = ga_row[r][j];
                gb = gb_row[r][j];
            }
            float ph;                          // radians
            if (EXACT) {
                ph = frac_dot3(dx[r], dxl[r], o, ol);
                if (GAINS) ph += gb.y - ga.y;
                ph = frac_turns(fmaf(b, INV_TWO_PI_F, ph)) * TWO_PI_F;
            } else {
                const float b0 = GAINS ? fmaf(gb.y - ga.y, TWO_PI_F, b) : b;
                ph = fmaf(dx[r].z, o.z, fmaf(dx[r].y, o.y, fmaf(dx[r].x, o.x, b0)));   // dx in radians
            }
            float sn, cs;
            if (!EXACT && fma_slot<NPOLY>(jj, r)) sincos_fma(ph, sn, cs);
            else __sincosf(ph, &sn, &cs);
            const float m = GAINS ? ba.y * (ga.x * gb.x) : ba.y;
            sr[r] = fmaf(m, cs, sr[r]);
            si[r] = fmaf(-m, sn, si[r]);
        }
    }
}

template <bool GAINS, bool EXACT, bool PAR>
__device__ __forceinline__ void fwd_gauss_tile(const float4* __restrict__ s_off,
                                               const float4* __restrict__ s_lo,
                                               const float4* __restrict__ s_pg,
                                               const float2* __restrict__ sBa,
                                               const float2* __restrict__ s_gain,
                                               const float4 (&xh)[2], const float4 (&dx)[2],
                                               const float4 (&dxl)[2], const GaussConst (&gc)[2],
                                               const int2 (&ant)[2], float (&sr)[2], float (&si)[2])
{
    const float2* ga_row[2] = {s_gain + ant[0].x * GP, s_gain + ant[1].x * GP};   // GAINS only
    const float2* gb_row[2] = {s_gain + ant[0].y * GP, s_gain + ant[1].y * GP};
#pragma unroll(GAINS ? 1 : 4)   // the gains variant stays within its registers
    for (int j = 0; j < G; ++j) {
        const float4 o = s_off[j];
        const float4 pg = s_pg[j];             // {l, m, r^2/2, nu}
        const float2 ba = sBa[j];
        const float b = ba.x;
        const float4 ol = EXACT ? s_lo[j] : o;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float uf = xh[r].x, vf = xh[r].y, wf = xh[r].z;
            const float t = fmaf(uf, pg.x, fmaf(vf, pg.y, -wf * pg.z));
            float2 ga = make_float2(1.f, 0.f), gb = ga;      // gains {|G|, arg G in turns}
            if (GAINS) {
                ga = ga_row[r][j];
                gb = gb_row[r][j];
            }
            float ph;                          // radians
            if (EXACT) {
                ph = fmaf(b, INV_TWO_PI_F, frac_dot3(dx[r], dxl[r], o, ol));
                if (GAINS) ph += gb.y - ga.y;
                ph = fmaf(-gc[r].gamr * INV_TWO_PI_F, t, ph);
                if (PAR) ph = fmaf(-wf, pg.w, ph);
                ph = frac_turns(ph) * TWO_PI_F;
            } else {
                const float b0 = GAINS ? fmaf(gb.y - ga.y, TWO_PI_F, b) : b;
                ph = fmaf(dx[r].z, o.z, fmaf(dx[r].y, o.y, fmaf(dx[r].x, o.x, b0)));
                ph = fmaf(-gc[r].gamr, t, ph);
                if (PAR) ph = fmaf(-wf * TWO_PI_F, pg.w, ph);
            }
            float sn, cs;
            __sincosf(ph, &sn, &cs);
            float amp = ba.y * ex2_approx(fmaf(gc[r].k1, t, gc[r].k0));   // (x/n) e^{Re(qc)}
            if (GAINS) amp *= ga.x * gb.x;
            sr[r] = fmaf(amp, cs, sr[r]);
            si[r] = fmaf(-amp, sn, si[r]);
        }
    }
}

// ---- forward with gains through the granule's pair table
// For the nb distinct antenna pairs (a_s, b_s) of the warp's visibility
// granule and BT_CH pixels j = c0 + jj of the streamed granule, the table
// holds a_j G_{j a_s} conj(G_{j b_s}) e^{-i B_j} (a_j = x_j / n_j) in polar
// form: T[s][jj] = {B_j - arg (radians, within one turn), |a_j G G|} (Dirac
// pixels) or {.., log2 |a_j G G|} (Gaussian pixels, for the amplitude's
// exponent).  A pair then starts its phase from the table entry, needs no B_j
// of its own, and accumulates with two FFMA.  Rows of BT_P, so the lanes of a
// half-warp (one pair, consecutive pixels) write distinct banks.  gtab: the
// gains in polar form {|G|, arg G in turns}.
template <bool LOG>
__device__ __forceinline__ void build_pair_table(float2* __restrict__ T, const int2* __restrict__ bl, int nb,
                                                 const float2* __restrict__ sBa,
                                                 const float2* __restrict__ gtab, int c0, int lane)
{
    for (int e = lane; e < nb * BT_CH; e += 32) {
        const int s = e / BT_CH, jj = e % BT_CH, j = c0 + jj;
        const int2 ab = bl[s];
        const float2 ga = gtab[ab.x * GP + j], gb = gtab[ab.y * GP + j];
        const float2 ba = sBa[j];                                    // {B_j (radians), a_j}
        // arg of a G_a conj(G_b) in turns: psi_a - psi_b (+ 1/2 when a_j < 0)
        const float arg = (ga.y - gb.y) + (ba.y < 0.f ? 0.5f : 0.f);
        const float ph = frac_turns(fmaf(ba.x, INV_TWO_PI_F, -arg)) * TWO_PI_F;
        const float m = fabsf(ba.y) * (ga.x * gb.x);
        T[s * BT_P + jj] = make_float2(ph, LOG ? __log2f(m) : m);   // log2(0) = -inf: amplitude 0
    }
}

template <bool EXACT>
__device__ __forceinline__ void fwd_dirac_tile_pt(const float4* __restrict__ s_off,
                                                  const float4* __restrict__ s_lo,
                                                  const float2* __restrict__ sBa,
                                                  const float2* __restrict__ gtab, float2* __restrict__ T,
                                                  const int2* __restrict__ bl, int nb, const int (&toff)[2],
                                                  const float4 (&dx)[2], const float4 (&dxl)[2], int lane,
                                                  float (&sr)[2], float (&si)[2])
{
#pragma unroll 1
    for (int c0 = 0; c0 < G; c0 += BT_CH) {
        build_pair_table<false>(T, bl, nb, sBa, gtab, c0, lane);
        __syncwarp();
#pragma unroll 8
        for (int jj = 0; jj < BT_CH; ++jj) {
            const int j = c0 + jj;
            const float4 o = s_off[j];
            const float4 ol = EXACT ? s_lo[j] : o;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const float2 t = T[toff[r] + jj];                      // {B - arg, |a g|}
                float ph;
                if (EXACT) ph = frac_turns(fmaf(t.x, INV_TWO_PI_F, frac_dot3(dx[r], dxl[r], o, ol))) * TWO_PI_F;
                else ph = fmaf(dx[r].z, o.z, fmaf(dx[r].y, o.y, fmaf(dx[r].x, o.x, t.x)));
                float sn, cs;
                __sincosf(ph, &sn, &cs);
                sr[r] = fmaf(t.y, cs, sr[r]);
                si[r] = fmaf(-t.y, sn, si[r]);
            }
        }
        __syncwarp();                                                  // table free for the next chunk
    }
}

template <bool EXACT, bool PAR>
__device__ __forceinline__ void fwd_gauss_tile_pt(const float4* __restrict__ s_off,
                                                  const float4* __restrict__ s_lo,
                                                  const float4* __restrict__ s_pg,
                                                  const float2* __restrict__ sBa,
                                                  const float2* __restrict__ gtab, float2* __restrict__ T,
                                                  const int2* __restrict__ bl, int nb, const int (&toff)[2],
                                                  const float4 (&xh)[2], const float4 (&dx)[2],
                                                  const float4 (&dxl)[2], const GaussConst (&gc)[2], int lane,
                                                  float (&sr)[2], float (&si)[2])
{
#pragma unroll 1
    for (int c0 = 0; c0 < G; c0 += BT_CH) {
        build_pair_table<true>(T, bl, nb, sBa, gtab, c0, lane);
        __syncwarp();
#pragma unroll 4
        for (int jj = 0; jj < BT_CH; ++jj) {
            const int j = c0 + jj;
            const float4 o = s_off[j];
            const float4 pg = s_pg[j];
            const float4 ol = EXACT ? s_lo[j] : o;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const float2 tv = T[toff[r] + jj];                     // {B - arg, log2 |a g|}
                const float wf = xh[r].z;
                const float t = fmaf(xh[r].x, pg.x, fmaf(xh[r].y, pg.y, -wf * pg.z));
                float ph;
                if (EXACT) {
                    ph = fmaf(tv.x, INV_TWO_PI_F, frac_dot3(dx[r], dxl[r], o, ol));
                    ph = fmaf(-gc[r].gamr * INV_TWO_PI_F, t, ph);
                    if (PAR) ph = fmaf(-wf, pg.w, ph);
                    ph = frac_turns(ph) * TWO_PI_F;
                } else {
                    ph = fmaf(dx[r].z, o.z, fmaf(dx[r].y, o.y, fmaf(dx[r].x, o.x, tv.x)));
                    ph = fmaf(-gc[r].gamr, t, ph);
                    if (PAR) ph = fmaf(-wf * TWO_PI_F, pg.w, ph);
                }
                float sn, cs;
                __sincosf(ph, &sn, &cs);
                const float amp = ex2_approx(fmaf(gc[r].k1, t, gc[r].k0 + tv.y));   // |a g| e^{Re(qc)}
                sr[r] = fmaf(amp, cs, sr[r]);
                si[r] = fmaf(-amp, sn, si[r]);
            }
        }
        __syncwarp();
    }
}

// Forward stage buffers in dynamic shared memory: two of them, each holding
// NST streamed pixel granules as they sit in HBM -- offsets {dl, dm, dn, 1/n},
// offset residuals, Gaussian data {l, m, r^2/2, nu}, x (FP64) and the granule
// headers {centre hi, centre lo, extent, {sigma, kind}} -- filled by bulk (TMA)
// copies that complete on one mbarrier per buffer.  The copies of stage s + 1
// are issued when stage s starts, so they land while stage s is computed.
template <int NST>
struct FwdStage {
    static constexpr int OFF = 0;                          // float4 [NST][G]
    static constexpr int LO = OFF + NST * G * 16;          // float4 [NST][G]
    static constexpr int PG = LO + NST * G * 16;           // float4 [NST][G]
    static constexpr int X = PG + NST * G * 16;            // double [NST][G]
    static constexpr int HDR = X + NST * G * 8;            // float4 [NST][4]
    static constexpr int BYTES = HDR + NST * 64;           // a multiple of 16
};
template <int NST>
constexpr int fwd_stage_bytes() { return 2 * FwdStage<NST>::BYTES; }

// One thread: copy the ns granules from gs of P's pixel side (the forward
// input X) into stage buffer `buf`, completing on bar.
template <int NST>
__device__ __forceinline__ void fwd_stage_load(unsigned char* buf, const DevProblem& P, const double* X, int gs,
                                               int ns, unsigned long long* bar)
{
    using S = FwdStage<NST>;
    const size_t e = (size_t)gs * G;
    const unsigned n4 = (unsigned)(ns * G * 16), n8 = (unsigned)(ns * G * 8), nh = (unsigned)(ns * 64);
    fence_proxy_async_smem();              // the buffer's last readers (generic proxy) are done
    mbar_arrive_expect(bar, 3 * n4 + n8 + nh);
    bulk_copy(buf + S::OFF, P.pix.off + e, n4, bar);
    bulk_copy(buf + S::LO, P.pix.offlo + e, n4, bar);
    bulk_copy(buf + S::PG, P.pgauss + e, n4, bar);
    bulk_copy(buf + S::X, X + e, n8, bar);
    bulk_copy(buf + S::HDR, P.pghdr + (size_t)gs * 4, nh, bar);
}

// Owned: visibilities (warp = one vis granule, lane = 2 visibilities).
// GAUSS = false: an instance for batches without Gaussian pixels, compiled
// without the Gaussian tiles (fewer live registers for the Dirac tiles).
// Streamed: pixel granules through the stage buffers, NST per stage (a tile
// shape the autotuner picks; the gains kernel stages one, since one granule's
// gains for all antennas already fill most of shared memory).  One CTA
// barrier per stage: it frees the buffer the next copies go to.
template <bool GAINS, int NST, int NPOLY = 0, bool GAUSS = true>
__global__ void __launch_bounds__(NTHREADS, GAINS ? 2 : 3)   // gains: pair-table path + gathers fit in 128
fwd_mixed_kernel(const DevProblem* __restrict__ probs, const Plan* __restrict__ plp, double2* __restrict__ partial)
{
    using S = FwdStage<NST>;
    // dynamic: [stage buffer 0][stage buffer 1][GAINS: one or two gains tables
    // [gain_rows(n_ant)][GP], each filled by a bulk copy; with two, the next
    // granule's table is copied while the current one is in use]
    extern __shared__ __align__(128) unsigned char s_dyn[];
    __shared__ float2 s_Ba[BLK_GRAN][NST][G];            // per warp: {B_j in radians, a_j = x_j / n_j}
    __shared__ __align__(8) unsigned long long s_sbar[2];   // stage buffers
    __shared__ __align__(8) unsigned long long s_gbar[2];   // GAINS: gains tables
    // GAINS: per warp, its visibility granule's pair list and pair table
    __shared__ int2 s_bl[GAINS ? BLK_GRAN : 1][GAINS ? NB_MAX : 1];
    __shared__ float2 s_pt[GAINS ? BLK_GRAN : 1][GAINS ? NB_MAX * BT_P : 1];
    float2* const s_gain = reinterpret_cast<float2*>(s_dyn + 2 * S::BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Plan pl = *plp;
    const long long c = blockIdx.x;
    long long u, u_end;
    cta_range(pl, c, u, u_end);
    int scur = 0;             // stage buffer of the current stage
    unsigned spar = 0;        // parity of the next wait on stage buffer b (bit b)
    unsigned gpar = 0;        // GAINS: parity of the next wait on gains buffer b (bit b)
    int gcur = 0;             // GAINS: gains buffer of the current stage when double-buffered
    bool fault = false;       // a bounded wait gave up
    if (threadIdx.x == 0) {
        mbar_init(&s_sbar[0], 1);
        mbar_init(&s_sbar[1], 1);
        mbar_init(&s_gbar[0], 1);
        mbar_init(&s_gbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    while (u < u_end) {
        const int p = find_prob(pl, u);
        const DevProblem& P = probs[p];
        const long long loc = u - pl.prob_u0[p];
        const double* X;
        if (!fwd_role(P, X)) {                    // problem not in this step: skip its units
            u = min(u_end, pl.prob_u0[p + 1]);
            continue;
        }
        const int upb = P.pix.n_gran;
        const int blk = (int)(loc / upb);
        const int g0 = (int)(loc % upb);
        const int g1 = (int)min((long long)upb, (long long)g0 + (u_end - u));
        const int vg = blk * BLK_GRAN + warp;
        const bool vg_ok = vg < P.vis.n_gran;
        const int e0 = (vg_ok ? vg : 0) * G + lane;     // this lane's visibilities: e0, e0 + 32
        const int gtab_n = GAINS ? gain_rows(P.n_ant) * GP : 0;                 // float2 per table
        const unsigned gbytes = (unsigned)gtab_n * (unsigned)sizeof(float2);
        const bool gdbl = GAINS && 2u * gbytes <= dyn_smem_bytes() - 2u * S::BYTES;
        // the range's first stage; its buffer's last readers finished before
        // the barrier of the previous range's last stage
        if (threadIdx.x == 0 && !fault)
            fwd_stage_load<NST>(s_dyn + scur * S::BYTES, P, X, g0, min(NST, g1 - g0), &s_sbar[scur]);

        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 xh[2] = {z4, z4}, dx[2] = {z4, z4};
        int2 ant[2] = {make_int2(0, 0), make_int2(0, 0)};
        float4 ch = z4, cl = z4, ext = z4;
        if (vg_ok) {
            ch = P.vis.cen_hi[vg];
            cl = P.vis.cen_lo[vg];
            ext = P.vis.ext[vg];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                xh[r] = P.vis.hi[e0 + 32 * r];
                dx[r] = to_rad(P.vis.off[e0 + 32 * r]);
                if (GAINS) ant[r] = P.ant[e0 + 32 * r];
            }
        }
        double tr[2] = {0.0, 0.0}, ti[2] = {0.0, 0.0};
        int nb = 0, toff[2] = {0, 0};          // GAINS: pairs in the granule's list (0: gathers)
        if (GAINS) {
            if (vg_ok) nb = P.gnb[vg];
            if (nb > 0) {
#pragma unroll
                for (int r = 0; r < 2; ++r) toff[r] = P.vslot[e0 + 32 * r] * BT_P;
                if (lane < nb) s_bl[warp][lane] = P.gbl[(size_t)vg * NB_MAX + lane];
            }
            __syncwarp();
        }

        for (int gs = g0; gs < g1; gs += NST) {
            const int ns = min(NST, g1 - gs);
            __syncthreads();                       // the previous stage is consumed
            if (threadIdx.x == 0 && !fault) {      // (a thread whose wait gave up issues no more copies)
                if (gs + NST < g1)                 // prefetch the next stage
                    fwd_stage_load<NST>(s_dyn + (scur ^ 1) * S::BYTES, P, X, gs + NST, min(NST, g1 - gs - NST),
                                        &s_sbar[scur ^ 1]);
                if (GAINS) {
                    const int b = gdbl ? gcur : 0;
                    fence_proxy_async_smem();
                    if (gs == g0 || !gdbl)
                        bulk_load(s_gain + b * gtab_n, P.gpol32 + (size_t)gs * gtab_n, gbytes, &s_gbar[b]);
                    if (gdbl && gs + 1 < g1)      // prefetch the next granule's table
                        bulk_load(s_gain + (b ^ 1) * gtab_n, P.gpol32 + (size_t)(gs + 1) * gtab_n, gbytes,
                                  &s_gbar[b ^ 1]);
                }
            }
            mbar_wait(&s_sbar[scur], (spar >> scur) & 1u, fault);
            spar ^= 1u << scur;
            const unsigned char* sb = s_dyn + scur * S::BYTES;
            const float4* s_off = reinterpret_cast<const float4*>(sb + S::OFF);
            const float4* s_lo = reinterpret_cast<const float4*>(sb + S::LO);
            const float4* s_pg = reinterpret_cast<const float4*>(sb + S::PG);
            const double* s_x = reinterpret_cast<const double*>(sb + S::X);
            const float4* s_hdr = reinterpret_cast<const float4*>(sb + S::HDR);
            scur ^= 1;
            const float2* gtab = s_gain;
            if (GAINS) {
                const int b = gdbl ? gcur : 0;
                mbar_wait(&s_gbar[b], (gpar >> b) & 1u, fault);
                gpar ^= 1u << b;
                gtab = s_gain + b * gtab_n;
                if (gdbl) gcur ^= 1;
            }
            // per warp: B_j = frac(Xc . (Y_j - Yc)) for its granule centre, and a_j = x_j / n_j
            for (int q = 0; q < ns; ++q) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = q * G + lane + 32 * h;
                    const float4 o = s_off[j];
                    s_Ba[warp][q][lane + 32 * h] = make_float2(frac_dot3(ch, cl, o, s_lo[j]) * TWO_PI_F,
                                                               __double2float_rn(s_x[j]) * o.w);
                }
            }
            __syncwarp();
            for (int q = 0; q < ns; ++q) {
                const float4 meta = s_hdr[4 * q + 3];                    // {sigma, kind, -, -}
                const int kind = (int)meta.y;
                const float4 yc_h = s_hdr[4 * q], yc_l = s_hdr[4 * q + 1];
                const bool exact = dot3(ext, s_hdr[4 * q + 2]) > D_MAX;  // warp-uniform
                const float4* q_off = s_off + q * G;
                const float4* q_lo = s_lo + q * G;
                const float4* q_pg = s_pg + q * G;
                const float2* q_Ba = s_Ba[warp][q];
                float C[2];
#pragma unroll
                for (int r = 0; r < 2; ++r) C[r] = frac_dot3(xh[r], P.vis.lo[e0 + 32 * r], yc_h, yc_l);
                float sr[2] = {0.f, 0.f}, si[2] = {0.f, 0.f};
                if (!GAUSS || kind == DIRAC) {
                    if (GAINS && nb > 0) {
                        if (exact) {
                            const float4 dxt[2] = {P.vis.off[e0], P.vis.off[e0 + 32]},
                                         dxl[2] = {P.vis.offlo[e0], P.vis.offlo[e0 + 32]};
                            fwd_dirac_tile_pt<true>(q_off, q_lo, q_Ba, gtab, s_pt[warp], s_bl[warp], nb, toff, dxt,
                                                    dxl, lane, sr, si);
                        } else {
                            fwd_dirac_tile_pt<false>(q_off, q_lo, q_Ba, gtab, s_pt[warp], s_bl[warp], nb, toff, dx,
                                                     dx, lane, sr, si);
                        }
                    } else if (exact) {
                        const float4 dxt[2] = {P.vis.off[e0], P.vis.off[e0 + 32]},
                                     dxl[2] = {P.vis.offlo[e0], P.vis.offlo[e0 + 32]};
                        fwd_dirac_tile<GAINS, true>(q_off, q_lo, q_Ba, gtab, dxt, dxl, ant, sr, si);
                    } else {
                        fwd_dirac_tile<GAINS, false, NPOLY, GAUSS ? 4 : 8>(q_off, q_lo, q_Ba, gtab, dx, dx, ant, sr, si);
                    }
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        float sn, cs;
                        __sincosf(C[r] * TWO_PI_F, &sn, &cs);          // rotate by exp(-2 pi i C)
                        tr[r] += (double)fmaf(cs, sr[r], sn * si[r]);
                        ti[r] += (double)fmaf(cs, si[r], -sn * sr[r]);
                    }
                } else {
                    const bool par = (kind == PARAXIAL);
                    GaussConst gc[2];
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        gc[r] = gauss_const(xh[r].x, xh[r].y, xh[r].z, meta.x);
                        C[r] = frac_turns(C[r] + gc[r].cphase);
                    }
                    if (GAINS && nb > 0) {
                        if (exact) {
                            const float4 dxt[2] = {P.vis.off[e0], P.vis.off[e0 + 32]},
                                         dxl[2] = {P.vis.offlo[e0], P.vis.offlo[e0 + 32]};
                            if (par) fwd_gauss_tile_pt<true, true>(q_off, q_lo, q_pg, q_Ba, gtab, s_pt[warp],
                                                                   s_bl[warp], nb, toff, xh, dxt, dxl, gc, lane, sr,
                                                                   si);
                            else fwd_gauss_tile_pt<true, false>(q_off, q_lo, q_pg, q_Ba, gtab, s_pt[warp],
                                                                s_bl[warp], nb, toff, xh, dxt, dxl, gc, lane, sr, si);
                        } else if (par) {
                            fwd_gauss_tile_pt<false, true>(q_off, q_lo, q_pg, q_Ba, gtab, s_pt[warp], s_bl[warp], nb,
                                                           toff, xh, dx, dx, gc, lane, sr, si);
                        } else {
                            fwd_gauss_tile_pt<false, false>(q_off, q_lo, q_pg, q_Ba, gtab, s_pt[warp], s_bl[warp], nb,
                                                            toff, xh, dx, dx, gc, lane, sr, si);
                        }
                    } else if (exact) {
                        const float4 dxt[2] = {P.vis.off[e0], P.vis.off[e0 + 32]},
                                     dxl[2] = {P.vis.offlo[e0], P.vis.offlo[e0 + 32]};
                        if (par) fwd_gauss_tile<GAINS, true, true>(q_off, q_lo, q_pg, q_Ba, gtab, xh, dxt, dxl, gc,
                                                                   ant, sr, si);
                        else fwd_gauss_tile<GAINS, true, false>(q_off, q_lo, q_pg, q_Ba, gtab, xh, dxt, dxl, gc, ant,
                                                                sr, si);
                    } else if (par) {
                        fwd_gauss_tile<GAINS, false, true>(q_off, q_lo, q_pg, q_Ba, gtab, xh, dx, dx, gc, ant, sr, si);
                    } else {
                        fwd_gauss_tile<GAINS, false, false>(q_off, q_lo, q_pg, q_Ba, gtab, xh, dx, dx, gc, ant, sr,
                                                            si);
                    }
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        // S id (1 + i beta), then rotate by exp(-2 pi i C)
                        const float ar = gc[r].id * fmaf(-gc[r].beta, si[r], sr[r]);
                        const float ai = gc[r].id * fmaf(gc[r].beta, sr[r], si[r]);
                        float sn, cs;
                        __sincosf(C[r] * TWO_PI_F, &sn, &cs);
                        tr[r] += (double)fmaf(cs, ar, sn * ai);
                        ti[r] += (double)fmaf(cs, ai, -sn * ar);
                    }
                }
            }
        }
        if (vg_ok) {
            const int gb = pl.prob_b0[p] + blk;
            double2* dst = partial + (size_t)slot_of(pl, gb) * BLK + warp * G + lane;
#pragma unroll
            for (int r = 0; r < 2; ++r) dst[32 * r] = make_double2(tr[r], ti[r]);
        }
        u += g1 - g0;
    }
    if (fault) atomicOr(&g_wait_fault, 1u);
}

// ----------------------------------------------------------- adjoint tiles
// The adjoint's output is real (the image is real: its gradient is Re A^H r),
// and for one pair Re(conj(A_kj) r_k) = |A_kj| |r_k| cos(theta_kj + arg r_k)
// with theta_kj = -arg A_kj: a cosine alone, not a sine and a cosine.
// r32_kernel writes r in polar form {|r|, arg r in turns}; when a stage is
// derived, arg r_k is added to the visibility's B term (so theta + arg r
// costs nothing per pair) and |r_k| rides in the same record (Gaussian
// owners: log2 |r'_k| inside the amplitude's exponent).
// With weights that are all positive, a bias of the SFU's cosine would add
// up over the N_v terms of a sum (where a sine and a cosine weighted by Re r
// and Im r of either sign cancel it), so every odd visibility k takes
// -cos(theta + pi) instead: its record carries B + arg r + 1/2 turn and the
// tile subtracts its term (odd_turn, the sign free in the FFMA).

// Half a turn for an odd streamed visibility k (see above).
__device__ __forceinline__ float odd_turn(int k) { return (k & 1) ? 0.5f : 0.f; }

// Gain of owned pixel r (0/1 of this lane) at antenna a: gains in shared
// memory, [antenna][pixel of the owned granule], rows of GP.
struct SmemGain {
    const float2* tab;
    int lane;
    __device__ float2 operator()(int a, int r) const { return tab[a * GP + lane + 32 * r]; }
};

// Dirac owners.  rec[k] = {B_k + arg r_k (radians), |r_k|, -, -}.
template <bool EXACT, int NPOLY = 0>
__device__ __forceinline__ void adj_dirac_tile(const float4* __restrict__ s_off,
                                               const float4* __restrict__ s_lo,
                                               const float4* __restrict__ s_rec,
                                               const float (&C)[2],
                                               const float4 (&dx)[2], const float4 (&dxl)[2],
                                               float (&acc)[2])
{
#pragma unroll 2
    for (int k0 = 0; k0 < G; k0 += 4)
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int k = k0 + kk;
        const float4 o = s_off[k];             // {du, dv, dw, W}
        const float2 br = *reinterpret_cast<const float2*>(s_rec + k);
        const float4 ol = EXACT ? s_lo[k] : o;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            float ph;                                  // radians; C and dx in radians unless EXACT
            if (EXACT) ph = frac_turns((C[r] + br.x * INV_TWO_PI_F) + frac_dot3(dx[r], dxl[r], o, ol)) * TWO_PI_F;
            else ph = fmaf(dx[r].z, o.z, fmaf(dx[r].y, o.y, fmaf(dx[r].x, o.x, C[r] + br.x)));
            const float cs = (!EXACT && fma_slot<NPOLY>(kk, r)) ? cos_fma(ph) : __cosf(ph);
            acc[r] = fmaf((kk & 1) ? -br.y : br.y, cs, acc[r]);   // odd k: -cos(theta + pi)
        }
    }
}

// Gaussian owners.  va[k] = {u, v, -2 w, u^2 + v^2}; rec[k] = {B_k + arg r'_k
// (radians), gamr, k1, k0 + log2 |r'_k|}: the amplitude times |r'| is
// 2^(k1 t + k0'), t = u l + v m - w r^2/2.
template <bool EXACT, bool PAR>
__device__ __forceinline__ void adj_gauss_tile(const float4* __restrict__ s_off,
                                               const float4* __restrict__ s_lo,
                                               const float4* __restrict__ s_abs,
                                               const float4* __restrict__ s_rec,
                                               const float (&C)[2],
                                               const float4 (&dx)[2], const float4 (&dxl)[2],
                                               const float4 (&pgd)[2], float (&acc)[2])
{
#pragma unroll 1
    for (int k0 = 0; k0 < G; k0 += 2)
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        const int k = k0 + kk;
        const float4 o = s_off[k];
        const float4 va = s_abs[k];
        const float4 rc = s_rec[k];
        const float4 ol = EXACT ? s_lo[k] : o;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            // pgd = {l, m, r^2/4, pi nu}: t = u l + v m - w r^2/2
            const float t = fmaf(va.x, pgd[r].x, fmaf(va.y, pgd[r].y, va.z * pgd[r].z));
            float ph;                                  // radians; C and dx in radians unless EXACT
            if (EXACT) {
                ph = (C[r] + rc.x * INV_TWO_PI_F) + frac_dot3(dx[r], dxl[r], o, ol);
                ph = fmaf(-rc.y * INV_TWO_PI_F, t, ph);
                if (PAR) ph = fmaf(va.z, pgd[r].w * INV_TWO_PI_F, ph);   // -w nu, turns
                ph = frac_turns(ph) * TWO_PI_F;
            } else {
                ph = fmaf(dx[r].z, o.z, fmaf(dx[r].y, o.y, fmaf(dx[r].x, o.x, C[r] + rc.x)));
                ph = fmaf(-rc.y, t, ph);
                if (PAR) ph = fmaf(va.z, pgd[r].w, ph);                  // -2 pi w nu
            }
            const float amp = ex2_approx(fmaf(rc.z, t, rc.w));          // |r'| e^{Re(qc)}
            acc[r] = fmaf(kk ? -amp : amp, __cosf(ph), acc[r]);           // odd k: -cos(theta + pi)
        }
    }
}

// The record of a streamed visibility for a Gaussian owner of scale sigma:
// r' = id (1 - i beta) r has |r'| = |r| / sqrt(1 + beta^2) and arg r' =
// arg r - atan(beta) (id > 0).  b: the visibility's B term in turns, with
// odd_turn's half turn for odd k; rp = {|r|, arg r in turns}; va = {u, v, -2 w,
// -}.  Returns {B + arg r' (radians), gamr, k1, k0 + log2 |r'|}.
__device__ __forceinline__ float4 adj_gauss_record(float b, float2 rp, const float4 va, float sigma)
{
    const GaussConst gc = gauss_const(va.x, va.y, -0.5f * va.z, sigma);
    b = frac_turns(b + gc.cphase);
    b = frac_turns(b + fmaf(-atanf(gc.beta), INV_TWO_PI_F, rp.y));
    const float lgr = __log2f(rp.x) - 0.5f * __log2f(fmaf(gc.beta, gc.beta, 1.0f));   // -inf when r = 0
    return make_float4(b * TWO_PI_F, gc.gamr, gc.k1, gc.k0 + lgr);
}

// Adjoint stage buffers in dynamic shared memory: two of them, each holding
// NSA streamed visibility granules as they sit in HBM -- offsets, offset
// residuals, the Gaussian form {u, v, -2 w, u^2 + v^2}, the residual r in
// polar form (written by r32_kernel just before the launch) and the granule
// centres and extents -- filled by bulk (TMA) copies on one mbarrier per
// buffer; the copies of stage s + 1 are issued when stage s starts.
template <int NSA>
struct AdjStage {
    static constexpr int OFF = 0;                      // float4 [NSA][G]
    static constexpr int LO = OFF + NSA * G * 16;      // float4 [NSA][G]
    static constexpr int GA = LO + NSA * G * 16;       // float4 [NSA][G]
    static constexpr int R = GA + NSA * G * 16;        // float2 [NSA][G] {|r|, arg r in turns}
    static constexpr int CEN = R + NSA * G * 8;        // float4 [3][NSA]: centre hi, centre lo, extent
    static constexpr int BYTES = CEN + 48 * NSA;       // a multiple of 16
};

template <int NSA>
__device__ __forceinline__ void adj_stage_load(unsigned char* buf, const DevProblem& P, int gs, int ns,
                                               unsigned long long* bar)
{
    using S = AdjStage<NSA>;
    const size_t e = (size_t)gs * G;
    const unsigned n4 = (unsigned)(ns * G * 16), n2 = (unsigned)(ns * G * 8), nc = (unsigned)(ns * 16);
    fence_proxy_async_smem();              // the buffer's last readers (generic proxy) are done
    mbar_arrive_expect(bar, 3 * n4 + n2 + 3 * nc);
    bulk_copy(buf + S::OFF, P.vis.off + e, n4, bar);
    bulk_copy(buf + S::LO, P.vis.offlo + e, n4, bar);
    bulk_copy(buf + S::GA, P.vgabs + e, n4, bar);
    bulk_copy(buf + S::R, P.r32 + e, n2, bar);
    bulk_copy(buf + S::CEN, P.vis.cen_hi + gs, nc, bar);
    bulk_copy(buf + S::CEN + 16 * NSA, P.vis.cen_lo + gs, nc, bar);
    bulk_copy(buf + S::CEN + 32 * NSA, P.vis.ext + gs, nc, bar);
}

// Owned: pixels (warp = one pixel granule, lane = 2 pixels).
// Streamed: visibility granules through the two stage buffers, NSA per stage,
// one CTA barrier per stage (it frees the buffer the next copies go to).
template <int NSA, int NPOLY = 0, bool GAUSS = true>
__global__ void __launch_bounds__(NTHREADS, 3)
adj_mixed_kernel(const DevProblem* __restrict__ probs, const Plan* __restrict__ plp, double* __restrict__ partial)
{
    using S = AdjStage<NSA>;
    extern __shared__ __align__(128) unsigned char s_dyn[];    // two stage buffers
    // per warp, the streamed visibilities' records for its owned granule:
    // Dirac {B + arg r (radians), |r|, -, -}, Gaussian adj_gauss_record's
    __shared__ float4 s_rec[BLK_GRAN][NSA][G];
    __shared__ __align__(8) unsigned long long s_sbar[2];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Plan pl = *plp;
    const long long c = blockIdx.x;
    long long u, u_end;
    cta_range(pl, c, u, u_end);
    int scur = 0;             // stage buffer of the current stage
    unsigned spar = 0;        // parity of the next wait on stage buffer b (bit b)
    bool fault = false;       // a bounded wait gave up
    if (threadIdx.x == 0) {
        mbar_init(&s_sbar[0], 1);
        mbar_init(&s_sbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    while (u < u_end) {
        const int p = find_prob(pl, u);
        const DevProblem& P = probs[p];
        const long long loc = u - pl.prob_u0[p];
        const double2* R;
        if (!adj_role(P, R)) {
            u = min(u_end, pl.prob_u0[p + 1]);
            continue;
        }
        const int upb = P.vis.n_gran;
        const int blk = (int)(loc / upb);
        const int g0 = (int)(loc % upb);
        const int g1 = (int)min((long long)upb, (long long)g0 + (u_end - u));
        // the range's first stage; its buffer's last readers finished before
        // the barrier of the previous range's last stage
        if (threadIdx.x == 0 && !fault)
            adj_stage_load<NSA>(s_dyn + scur * S::BYTES, P, g0, min(NSA, g1 - g0), &s_sbar[scur]);
        const int pgi = blk * BLK_GRAN + warp;
        const bool pg_ok = pgi < P.pix.n_gran;
        const int e0 = (pg_ok ? pgi : 0) * G + lane;     // this lane's pixels: e0, e0 + 32

        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 xh[2] = {z4, z4}, dx[2] = {z4, z4}, pgd[2] = {z4, z4};
        const int eidx[2] = {e0, e0 + 32};
        float4 ch = z4, cl = z4, ext = z4;
        int kind = DIRAC;
        float sigma = 0.f;
        if (pg_ok) {
            ch = P.pix.cen_hi[pgi];
            cl = P.pix.cen_lo[pgi];
            ext = P.pix.ext[pgi];
            kind = P.gkind[pgi];
            sigma = P.gsig[pgi];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                xh[r] = P.pix.hi[eidx[r]];
                dx[r] = to_rad(P.pix.off[eidx[r]]);
                if (GAUSS && kind != DIRAC) pgd[r] = pix_for_gauss(P.pgauss[eidx[r]]);
            }
        }
        const bool gauss = GAUSS && (kind != DIRAC);   // GAUSS = false: no Gaussian pixels in the batch
        const bool par = (kind == PARAXIAL);
        double tot[2] = {0.0, 0.0};

        for (int gs = g0; gs < g1; gs += NSA) {
            const int ns = min(NSA, g1 - gs);
            __syncthreads();                       // the previous stage is consumed
            if (threadIdx.x == 0 && !fault && gs + NSA < g1)  // prefetch the next stage
                adj_stage_load<NSA>(s_dyn + (scur ^ 1) * S::BYTES, P, gs + NSA, min(NSA, g1 - gs - NSA),
                                    &s_sbar[scur ^ 1]);
            mbar_wait(&s_sbar[scur], (spar >> scur) & 1u, fault);
            spar ^= 1u << scur;
            const unsigned char* sb = s_dyn + scur * S::BYTES;
            scur ^= 1;
            const float4* const b_off = reinterpret_cast<const float4*>(sb + S::OFF);
            const float4* const b_lo = reinterpret_cast<const float4*>(sb + S::LO);
            const float4* const b_ga = reinterpret_cast<const float4*>(sb + S::GA);
            const float2* const b_r = reinterpret_cast<const float2*>(sb + S::R);
            const float4* const b_cen = reinterpret_cast<const float4*>(sb + S::CEN);
            for (int q = 0; q < ns; ++q) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = lane + 32 * h;
                    const float b = frac_dot3(ch, cl, b_off[q * G + k], b_lo[q * G + k]) + odd_turn(k);
                    const float2 rp = b_r[q * G + k];
                    s_rec[warp][q][k] = gauss ? adj_gauss_record(b, rp, b_ga[q * G + k], sigma)
                                              : make_float4(frac_turns(b + rp.y) * TWO_PI_F, rp.x, 0.f, 0.f);
                }
            }
            __syncwarp();
            for (int q = 0; q < ns; ++q) {
                const float4 yc_h = b_cen[q], yc_l = b_cen[NSA + q];
                const bool exact = dot3(ext, b_cen[2 * NSA + q]) > D_MAX;
                float C[2];
#pragma unroll
                for (int r = 0; r < 2; ++r) C[r] = frac_dot3(xh[r], P.pix.lo[eidx[r]], yc_h, yc_l);
                const float Cr[2] = {C[0] * TWO_PI_F, C[1] * TWO_PI_F};
                float acc[2] = {0.f, 0.f};
                const float4* q_off = b_off + q * G;
                const float4* q_lo = b_lo + q * G;
                const float4* q_ga = b_ga + q * G;
                const float4* q_rec = s_rec[warp][q];
                if (!gauss) {
                    if (exact) {
                        const float4 dxt[2] = {P.pix.off[eidx[0]], P.pix.off[eidx[1]]},
                                     dxl[2] = {P.pix.offlo[eidx[0]], P.pix.offlo[eidx[1]]};
                        adj_dirac_tile<true>(q_off, q_lo, q_rec, C, dxt, dxl, acc);
                    } else {
                        adj_dirac_tile<false, NPOLY>(q_off, q_lo, q_rec, Cr, dx, dx, acc);
                    }
                } else if (exact) {
                    const float4 dxt[2] = {P.pix.off[eidx[0]], P.pix.off[eidx[1]]},
                                 dxl[2] = {P.pix.offlo[eidx[0]], P.pix.offlo[eidx[1]]};
                    if (par) adj_gauss_tile<true, true>(q_off, q_lo, q_ga, q_rec, C, dxt, dxl, pgd, acc);
                    else adj_gauss_tile<true, false>(q_off, q_lo, q_ga, q_rec, C, dxt, dxl, pgd, acc);
                } else if (par) {
                    adj_gauss_tile<false, true>(q_off, q_lo, q_ga, q_rec, Cr, dx, dx, pgd, acc);
                } else {
                    adj_gauss_tile<false, false>(q_off, q_lo, q_ga, q_rec, Cr, dx, dx, pgd, acc);
                }
#pragma unroll
                for (int r = 0; r < 2; ++r) tot[r] += (double)acc[r];
            }
        }
        if (pg_ok) {
            const int gb = pl.prob_b0[p] + blk;
            double* dst = partial + (size_t)slot_of(pl, gb) * BLK + warp * G + lane;
#pragma unroll
            for (int r = 0; r < 2; ++r) dst[32 * r] = tot[r] * P.pix.d[eidx[r]].w;
        }
        u += g1 - g0;
    }
    if (fault) atomicOr(&g_wait_fault, 1u);
}

// ---- adjoint tiles with gains
// A streamed visibility granule's members are sorted by antenna pair, so for
// an owned pixel j each pair s = (a, b) is one run of visibilities k.  With
// g_js = G_ja conj(G_jb) = M e^{2 pi i (psi_a - psi_b)} (psi = arg G in
// turns), r_k = |r_k| e^{2 pi i rho_k} and C the tile's centre term, the run
// adds
//   Re( conj(g_js) e^{2 pi i C} sum_{k in s} e^{i theta_jk} r_k )
//     = M sum_{k in s} |r_k| cos(theta_jk + 2 pi (rho_k + Phi)),
// Phi = C + psi_b - psi_a, theta = 2 pi (B + D) (+ the Gaussian terms): rho_k
// sits in the record's B term, Phi is formed once per run from the gains in
// polar form, and M multiplies the run's sum z at the run's end.
// Per record k: off = {du, dv, dw, B + rho (radians)}, kr = {pair key a << 16
// | b, |r| (Dirac owners) or k0 + log2 |r'| (Gaussian owners), k1, 0};
// Gaussian owners also read va = {u, v, -2 w, gam in radians}, the amplitude
// times |r'| being 2^(k1 t + k0') with t = u l + v m - w r^2/2.

// The run held in z, of magnitude M, into acc: acc += M z.
__device__ __forceinline__ void adjg_flush(const float (&M)[2], float (&z)[2], float (&acc)[2])
{
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        acc[r] = fmaf(M[r], z[r], acc[r]);
        z[r] = 0.f;
    }
}

// At a new pair `key` (antenna indices a = key >> 16, b = key & 0xffff, both
// valid): flush the run so far, then M = |G_ja| |G_jb| and Phi = C + psi_jb -
// psi_ja (radians; turns when EXACT) for the lane's two pixels, Ct = C in
// turns.
template <bool EXACT, class GF>
__device__ __forceinline__ void adjg_next_run(int key, int& cur, const GF& gain, const float (&Ct)[2],
                                              float (&M)[2], float (&Phi)[2], float (&z)[2], float (&acc)[2])
{
    if (key == cur) return;                       // warp-uniform: every lane has the same k
    adjg_flush(M, z, acc);
    cur = key;
    const int a = key >> 16, b = key & 0xffff;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const float2 ga = gain(a, r), gb = gain(b, r);   // {|G|, arg G in turns}
        M[r] = ga.x * gb.x;
        const float f = frac_turns(Ct[r] + (gb.y - ga.y));
        Phi[r] = EXACT ? f : f * TWO_PI_F;
    }
}

template <bool EXACT, class GF>
__device__ __forceinline__ void adjg_dirac_tile(const float4* __restrict__ s_off, const float4* __restrict__ g_lo,
                                                const float4* __restrict__ s_kr, const GF& gain,
                                                const float (&Ct)[2], const float4 (&dx)[2],
                                                const float4 (&dxl)[2], float (&acc)[2])
{
    int cur = -1;
    float M[2] = {0.f, 0.f}, Phi[2] = {0.f, 0.f}, z[2] = {0.f, 0.f};
#pragma unroll 1
    for (int k0 = 0; k0 < G; k0 += 4)
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int k = k0 + kk;
        const float4 o = s_off[k];
        const float2 kr = *reinterpret_cast<const float2*>(s_kr + k);   // {key, |r|}
        adjg_next_run<EXACT>(__float_as_int(kr.x), cur, gain, Ct, M, Phi, z, acc);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            float ph;                              // radians
            if (EXACT) ph = frac_turns((o.w * INV_TWO_PI_F + Phi[r]) + frac_dot3(dx[r], dxl[r], o, g_lo[k])) * TWO_PI_F;
            else ph = fmaf(dx[r].z, o.z, fmaf(dx[r].y, o.y, fmaf(dx[r].x, o.x, o.w + Phi[r])));
            z[r] = fmaf((kk & 1) ? -kr.y : kr.y, __cosf(ph), z[r]);   // odd k: -cos(theta + pi)
        }
    }
    adjg_flush(M, z, acc);                      // the last run
}

template <bool EXACT, bool PAR, class GF>
__device__ __forceinline__ void adjg_gauss_tile(const float4* __restrict__ s_off, const float4* __restrict__ g_lo,
                                                const float4* __restrict__ s_va, const float4* __restrict__ s_kr,
                                                const GF& gain, const float (&Ct)[2],
                                                const float4 (&dx)[2], const float4 (&dxl)[2],
                                                const float4 (&pgd)[2], float (&acc)[2])
{
    int cur = -1;
    float M[2] = {0.f, 0.f}, Phi[2] = {0.f, 0.f}, z[2] = {0.f, 0.f};
#pragma unroll 1
    for (int k0 = 0; k0 < G; k0 += 2)
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        const int k = k0 + kk;
        const float4 o = s_off[k];
        const float4 va = s_va[k];                 // {u, v, -2 w, gam (radians)}
        const float4 kr = s_kr[k];                 // {key, k0', k1, 0}
        adjg_next_run<EXACT>(__float_as_int(kr.x), cur, gain, Ct, M, Phi, z, acc);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            // pgd = {l, m, r^2/4, pi nu}: t = u l + v m - w r^2/2
            const float t = fmaf(va.x, pgd[r].x, fmaf(va.y, pgd[r].y, va.z * pgd[r].z));
            float ph;                              // radians
            if (EXACT) {
                ph = (o.w * INV_TWO_PI_F + Phi[r]) + frac_dot3(dx[r], dxl[r], o, g_lo[k]);
                ph = fmaf(-va.w * INV_TWO_PI_F, t, ph);
                if (PAR) ph = fmaf(va.z, pgd[r].w * INV_TWO_PI_F, ph);   // -w nu, turns
                ph = frac_turns(ph) * TWO_PI_F;
            } else {
                ph = fmaf(dx[r].z, o.z, fmaf(dx[r].y, o.y, fmaf(dx[r].x, o.x, o.w + Phi[r])));
                ph = fmaf(-va.w, t, ph);
                if (PAR) ph = fmaf(va.z, pgd[r].w, ph);                  // -2 pi w nu
            }
            const float amp = ex2_approx(fmaf(kr.z, t, kr.y));        // |r'| e^{Re(qc)}
            z[r] = fmaf(kk ? -amp : amp, __cosf(ph), z[r]);             // odd k: -cos(theta + pi)
        }
    }
    adjg_flush(M, z, acc);                      // the last run
}

// Adjoint with gains.  The CTA's 8 warps share one owned pixel granule at a
// time -- its gains for all antennas in shared memory as [antenna][pixel], so
// a lane's loads never conflict -- and split the streamed visibility granules
// of the run among themselves (warp w takes the w-th of every 8).  Each warp
// runs its own pipeline: lane 0 bulk-copies the raw records of the warp's
// next granule (offsets, residuals, coordinates, r, antenna pairs, centre and
// extent) into the warp's slice, which completes on the warp's mbarrier; the
// warp derives what its tiles read, then at once copies its following granule
// into the freed slice, so the copy runs under the tiles.  No CTA barrier
// inside the run.  For each owned granule the 8 warp sums are added in warp
// order (deterministic).
struct AdjRaw {                                   // one warp's slice, bytes
    static constexpr int OFF = 0, LO = 1024, HI = 2048, R = 3072, ANT = 3584, CEN = 4096;
    static constexpr int BYTES = CEN + 48;        // a multiple of 16
};

// Lane 0: copy visibility granule g of P into a warp's raw slice (r: the
// polar residual r32_kernel wrote).
__device__ __forceinline__ void adj_raw_load(unsigned char* raw, const DevProblem& P, int g, unsigned long long* bar)
{
    const size_t e = (size_t)g * G;
    fence_proxy_async_smem();                     // the slice's last readers (generic proxy) are done
    mbar_arrive_expect(bar, AdjRaw::BYTES);
    bulk_copy(raw + AdjRaw::OFF, P.vis.off + e, 1024, bar);
    bulk_copy(raw + AdjRaw::LO, P.vis.offlo + e, 1024, bar);
    bulk_copy(raw + AdjRaw::HI, P.vis.hi + e, 1024, bar);
    bulk_copy(raw + AdjRaw::R, P.r32 + e, 512, bar);
    bulk_copy(raw + AdjRaw::ANT, P.ant + e, 512, bar);
    bulk_copy(raw + AdjRaw::CEN, P.vis.cen_hi + g, 16, bar);
    bulk_copy(raw + AdjRaw::CEN + 16, P.vis.cen_lo + g, 16, bar);
    bulk_copy(raw + AdjRaw::CEN + 32, P.vis.ext + g, 16, bar);
}

__global__ void __launch_bounds__(NTHREADS, 2)
adj_mixed_gains_kernel(const DevProblem* __restrict__ probs, const Plan* __restrict__ plp,
                       double* __restrict__ partial)
{
    // per warp, what its tiles read for its current granule
    __shared__ float4 s_off[BLK_GRAN][G];       // {du, dv, dw, B + arg r (radians)}
    __shared__ float4 s_kr[BLK_GRAN][G];        // {pair key, |r| or k0 + log2 |r'|, k1, 0}
    __shared__ float4 s_va[BLK_GRAN][G];        // Gaussian owners: {u, v, -2 w, gam (radians)}
    __shared__ double s_red[BLK_GRAN][G];
    __shared__ __align__(8) unsigned long long s_wbar[BLK_GRAN];   // each warp's raw slice
    __shared__ __align__(8) unsigned long long s_gbar;             // the gains table
    // dynamic: [raw slices, BLK_GRAN x AdjRaw::BYTES][the owned granule's gains
    // in polar form [gain_rows(n_ant)][GP]], each filled by bulk (TMA) copies
    extern __shared__ __align__(128) unsigned char s_dyn[];
    float2* const s_gain = reinterpret_cast<float2*>(s_dyn + BLK_GRAN * AdjRaw::BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* const raw = s_dyn + warp * AdjRaw::BYTES;
    const float4* const raw_off = reinterpret_cast<const float4*>(raw + AdjRaw::OFF);
    const float4* const raw_lo = reinterpret_cast<const float4*>(raw + AdjRaw::LO);
    const float4* const raw_hi = reinterpret_cast<const float4*>(raw + AdjRaw::HI);
    const float2* const raw_r = reinterpret_cast<const float2*>(raw + AdjRaw::R);
    const int2* const raw_ant = reinterpret_cast<const int2*>(raw + AdjRaw::ANT);
    const float4* const raw_cen = reinterpret_cast<const float4*>(raw + AdjRaw::CEN);
    const Plan pl = *plp;
    const long long c = blockIdx.x;
    long long u, u_end;
    cta_range(pl, c, u, u_end);
    unsigned gpar = 0;          // parity of the next wait on s_gbar
    unsigned wpar = 0;          // parity of this warp's next wait on s_wbar[warp]
    bool fault = false;         // a bounded wait gave up
    if (threadIdx.x == 0) {
        mbar_init(&s_gbar, 1);
        for (int w = 0; w < BLK_GRAN; ++w) mbar_init(&s_wbar[w], 1);
        fence_mbar_init();
    }
    __syncthreads();

    while (u < u_end) {
        const int p = find_prob(pl, u);
        const DevProblem& P = probs[p];
        const long long loc = u - pl.prob_u0[p];
        const double2* R;
        if (!adj_role(P, R)) {
            u = min(u_end, pl.prob_u0[p + 1]);
            continue;
        }
        const int upb = P.vis.n_gran;
        const int blk = (int)(loc / upb);
        const int g0 = (int)(loc % upb);
        const int g1 = (int)min((long long)upb, (long long)g0 + (u_end - u));
        const int gtab_n = gain_rows(P.n_ant) * GP;      // float2 per granule table
        const int gb = pl.prob_b0[p] + blk;
        double* dst = partial + (size_t)slot_of(pl, gb) * BLK;
        for (int og = 0; og < BLK_GRAN; ++og) {
            const int pgi = blk * BLK_GRAN + og;
            if (pgi >= P.pix.n_gran) break;                  // uniform over the CTA
            __syncthreads();                                 // s_gain / s_red free again
            if (threadIdx.x == 0 && !fault) {
                fence_proxy_async_smem();                    // the table's last readers are done
                bulk_load(s_gain, P.gpol32 + (size_t)pgi * gtab_n, (unsigned)gtab_n * (unsigned)sizeof(float2),
                          &s_gbar);
            }
            if (lane == 0 && !fault && g0 + warp < g1) adj_raw_load(raw, P, g0 + warp, &s_wbar[warp]);
            const float4 ch = P.pix.cen_hi[pgi], cl = P.pix.cen_lo[pgi], ext = P.pix.ext[pgi];
            const int kind = P.gkind[pgi];
            const float sigma = P.gsig[pgi];
            const bool gauss = (kind != DIRAC), par = (kind == PARAXIAL);
            const int e0 = pgi * G + lane;
            const int eidx[2] = {e0, e0 + 32};
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            float4 xh[2], dx[2], pgd[2] = {z4, z4};
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                xh[r] = P.pix.hi[eidx[r]];
                dx[r] = to_rad(P.pix.off[eidx[r]]);
                if (gauss) pgd[r] = pix_for_gauss(P.pgauss[eidx[r]]);
            }
            const SmemGain sg{s_gain, lane};
            mbar_wait(&s_gbar, gpar, fault);
            gpar ^= 1u;
            double tot[2] = {0.0, 0.0};
            for (int g = g0 + warp; g < g1; g += BLK_GRAN) {
                mbar_wait(&s_wbar[warp], wpar, fault);
                wpar ^= 1u;
                // derive this granule's records for the tiles
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = lane + 32 * h;
                    float4 o = raw_off[k];
                    const int2 ab = raw_ant[k];
                    const float key = __int_as_float(ab.x << 16 | ab.y);   // the pair (adjg_next_run)
                    const float b = frac_dot3(ch, cl, o, raw_lo[k]) + odd_turn(k);   // turns
                    const float2 rp = raw_r[k];                             // {|r|, arg r in turns}
                    float4 kr;
                    if (gauss) {
                        const float4 va = vis_for_gauss(raw_hi[k]);
                        const float4 rec = adj_gauss_record(b, rp, va, sigma);   // {B', gamr, k1, k0'}
                        o.w = rec.x;
                        s_va[warp][k] = make_float4(va.x, va.y, va.z, rec.y);
                        kr = make_float4(key, rec.w, rec.z, 0.f);
                    } else {
                        o.w = frac_turns(b + rp.y) * TWO_PI_F;
                        kr = make_float4(key, rp.x, 0.f, 0.f);
                    }
                    s_off[warp][k] = o;
                    s_kr[warp][k] = kr;
                }
                const float4 yc_h = raw_cen[0], yc_l = raw_cen[1], yext = raw_cen[2];
                __syncwarp();                                 // the slice is read: refill it
                if (lane == 0 && !fault && g + BLK_GRAN < g1) adj_raw_load(raw, P, g + BLK_GRAN, &s_wbar[warp]);
                const bool exact = dot3(ext, yext) > D_MAX;
                float Ct[2];                          // the tile's centre term C, turns
#pragma unroll
                for (int r = 0; r < 2; ++r) Ct[r] = frac_dot3(xh[r], P.pix.lo[eidx[r]], yc_h, yc_l);
                const float4* g_lo = P.vis.offlo + (size_t)g * G;   // exact tiles only (rare)
                float acc[2] = {0.f, 0.f};
                if (!gauss) {
                    if (exact) {
                        const float4 dxt[2] = {P.pix.off[eidx[0]], P.pix.off[eidx[1]]},
                                     dxl[2] = {P.pix.offlo[eidx[0]], P.pix.offlo[eidx[1]]};
                        adjg_dirac_tile<true>(s_off[warp], g_lo, s_kr[warp], sg, Ct, dxt, dxl, acc);
                    } else {
                        adjg_dirac_tile<false>(s_off[warp], g_lo, s_kr[warp], sg, Ct, dx, dx, acc);
                    }
                } else if (exact) {
                    const float4 dxt[2] = {P.pix.off[eidx[0]], P.pix.off[eidx[1]]},
                                 dxl[2] = {P.pix.offlo[eidx[0]], P.pix.offlo[eidx[1]]};
                    if (par) adjg_gauss_tile<true, true>(s_off[warp], g_lo, s_va[warp], s_kr[warp], sg, Ct, dxt, dxl, pgd, acc);
                    else adjg_gauss_tile<true, false>(s_off[warp], g_lo, s_va[warp], s_kr[warp], sg, Ct, dxt, dxl, pgd, acc);
                } else if (par) {
                    adjg_gauss_tile<false, true>(s_off[warp], g_lo, s_va[warp], s_kr[warp], sg, Ct, dx, dx, pgd, acc);
                } else {
                    adjg_gauss_tile<false, false>(s_off[warp], g_lo, s_va[warp], s_kr[warp], sg, Ct, dx, dx, pgd, acc);
                }
#pragma unroll
                for (int r = 0; r < 2; ++r) tot[r] += (double)acc[r];
                __syncwarp();                                 // s_off ... of this warp free again
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) s_red[warp][lane + 32 * r] = tot[r];
            __syncthreads();
            if (warp == 0) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    double t = 0.0;
                    for (int w = 0; w < BLK_GRAN; ++w) t += s_red[w][lane + 32 * r];
                    dst[og * G + lane + 32 * r] = t * P.pix.d[eidx[r]].w;
                }
            }
        }
        u += g1 - g0;
    }
    if (fault) atomicOr(&g_wait_fault, 1u);
}

// ------------------------------------------------------------- launchers

// Bytes of one pixel granule's gains table in shared memory.
static int gains_table_bytes(int n_ant) { return gain_rows(n_ant) * GP * (int)sizeof(float2); }
// Dynamic shared memory of the forward: its two stage buffers and, with gains,
// one or two gains tables.  The table is double-buffered (the next granule's
// prefetched while the current one is in use) when two fit in this much; the
// kernel reads the choice back from the launch's dynamic size.  With the
// kernel's 36 KB of static shared memory the total stays within 227 KB.
constexpr int FWD_GAINS_DBL_MAX = 180 * 1024;
static int fwd_stage_bytes_of(int nst)
{
    return nst <= 1 ? fwd_stage_bytes<1>() : nst <= 2 ? fwd_stage_bytes<2>()
                                          : nst <= 4 ? fwd_stage_bytes<4>() : fwd_stage_bytes<8>();
}
int fwd_smem_bytes(int n_ant, bool gains, int nst)
{
    if (!gains) return fwd_stage_bytes_of(shape_nst(nst));
    const int t = gains_table_bytes(n_ant);
    return fwd_stage_bytes<1>() + (2 * t <= FWD_GAINS_DBL_MAX ? 2 * t : t);
}
int adj_gains_smem_bytes(int n_ant) { return BLK_GRAN * AdjRaw::BYTES + gains_table_bytes(n_ant); }
// the no-gains adjoint: two stage buffers
static int adj_stage_bytes_of(int nst)
{
    return 2 * (nst <= 2 ? AdjStage<2>::BYTES : AdjStage<4>::BYTES);
}

// r32 = the mixed adjoint's input residual in polar form, {|r|, arg r in
// turns}, for every problem of the batch that takes part in the coming adjoint
// (blockIdx.y = problem).  Modulus and argument are taken in FP64 and rounded
// once to FP32 (arg r to 3e-8 turn).
__global__ void r32_kernel(const DevProblem* __restrict__ probs)
{
    const DevProblem& P = probs[blockIdx.y];
    const double2* R;
    if (!adj_role(P, R) || !P.r32) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.vis.n_pad; i += gridDim.x * blockDim.x) {
        const double2 v = R[i];
        P.r32[i] = make_float2((float)hypot(v.x, v.y), (float)(atan2(v.y, v.x) * 0.15915494309189535));
    }
}
cudaError_t launch_r32(const DevProblem* probs, int n_probs, int max_vis_pad, cudaStream_t st)
{
    const dim3 grid((unsigned)std::max(1, std::min(1024, (max_vis_pad + 255) / 256)), (unsigned)n_probs);
    r32_kernel<<<grid, 256, 0, st>>>(probs);
    return cudaGetLastError();
}

cudaError_t wait_fault_read(unsigned* host_flag, cudaStream_t st)
{
    return cudaMemcpyFromSymbolAsync(host_flag, g_wait_fault, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, st);
}
// Self-test of the bounded wait: every thread waits on an mbarrier that
// expects one arrival which nobody makes (no copy is issued, so nothing is in
// flight).  The wait gives up after WAIT_LIMIT_NS, the CTA sets the fault flag
// as the operator kernels do, records how long thread 0 waited, and returns.
__global__ void __launch_bounds__(64) wait_selftest_kernel(unsigned long long* waited_ns)
{
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    bool fault = false;
    const unsigned long long t0 = global_ns();
    mbar_wait(&bar, 0u, fault);
    const unsigned long long t1 = global_ns();
    if (threadIdx.x == 0) {
        waited_ns[blockIdx.x] = t1 - t0;
        if (fault) atomicOr(&g_wait_fault, 1u);
    }
}
cudaError_t launch_wait_selftest(unsigned long long* waited_ns, int n_blocks, cudaStream_t st)
{
    wait_selftest_kernel<<<n_blocks, 64, 0, st>>>(waited_ns);
    return cudaGetLastError();
}
unsigned long long wait_limit_ns() { return WAIT_LIMIT_NS; }
cudaError_t wait_fault_clear(cudaStream_t st)
{
    static const unsigned zero = 0;
    return cudaMemcpyToSymbolAsync(g_wait_fault, &zero, sizeof(unsigned), 0, cudaMemcpyHostToDevice, st);
}

template <class K>
static int occ_of(K kernel, int dyn)
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, NTHREADS, dyn);
    return n < 1 ? 1 : n;
}

using FwdKernel = void (*)(const DevProblem*, const Plan*, double2*);
using AdjKernel = void (*)(const DevProblem*, const Plan*, double*);

// The no-gains kernel of a tile-shape code (nst 2 / 4 / 8, npoly 0 / 1 / 2,
// with or without the Gaussian tiles).
template <int N, bool GS>
static FwdKernel fwd_by_poly(int np)
{
    return np <= 0 ? fwd_mixed_kernel<false, N, 0, GS> : np == 1 ? fwd_mixed_kernel<false, N, 1, GS>
                                                                 : fwd_mixed_kernel<false, N, 2, GS>;
}
template <int N, bool GS>
static AdjKernel adj_by_poly(int np)
{
    return np <= 0 ? adj_mixed_kernel<N, 0, GS> : np == 1 ? adj_mixed_kernel<N, 1, GS> : adj_mixed_kernel<N, 2, GS>;
}
template <bool GS>
static FwdKernel fwd_kernel_gs(int nst, int np)
{
    return nst <= 2 ? fwd_by_poly<2, GS>(np) : nst <= 4 ? fwd_by_poly<4, GS>(np) : fwd_by_poly<8, GS>(np);
}
static FwdKernel fwd_kernel_of(int code)
{
    const int nst = shape_nst(code), np = shape_npoly(code);
    return shape_dirac_only(code) ? fwd_kernel_gs<false>(nst, np) : fwd_kernel_gs<true>(nst, np);
}
// The no-gains adjoint stages 2 or 4 granules (with 8, its stage buffers and
// per-warp records would leave room for 1 CTA per SM).
static AdjKernel adj_kernel_of(int code)
{
    const int nst = shape_nst(code), np = shape_npoly(code);
    if (shape_dirac_only(code)) return nst <= 2 ? adj_by_poly<2, false>(np) : adj_by_poly<4, false>(np);
    return nst <= 2 ? adj_by_poly<2, true>(np) : adj_by_poly<4, true>(np);
}

cudaError_t launch_forward_mixed(bool gains, int n_ant, int nst, const DevProblem* probs, const Plan* plp, int C,
                                 double2* partial, cudaStream_t st)
{
    // the dynamic shared-memory limits were raised by occupancy_mixed() when
    // the batch was built (not here: this may run under capture)
    if (gains)
        fwd_mixed_kernel<true, 1><<<C, NTHREADS, fwd_smem_bytes(n_ant, true, 1), st>>>(probs, plp, partial);
    else
        fwd_kernel_of(nst)<<<C, NTHREADS, fwd_smem_bytes(0, false, nst), st>>>(probs, plp, partial);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_mixed(bool gains, int n_ant, int nst, const DevProblem* probs, const Plan* plp, int C,
                                 double* partial, cudaStream_t st)
{
    if (gains) adj_mixed_gains_kernel<<<C, NTHREADS, adj_gains_smem_bytes(n_ant), st>>>(probs, plp, partial);
    else adj_kernel_of(nst)<<<C, NTHREADS, adj_stage_bytes_of(shape_nst(nst)), st>>>(probs, plp, partial);
    return cudaGetLastError();
}

int occupancy_mixed(int op, bool gains, int n_ant, int nst)
{
    static int fwd_smem_limit = 0, adj_smem_limit = 0;   // only ever raised
    if (op == 0) {
        if (gains) {
            const int sm = fwd_smem_bytes(n_ant, true, 1);
            if (sm > fwd_smem_limit) {
                cudaFuncSetAttribute(fwd_mixed_kernel<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
                fwd_smem_limit = sm;
            }
            return occ_of(fwd_mixed_kernel<true, 1>, sm);
        }
        const int sm = fwd_smem_bytes(0, false, nst);      // fixed per tile shape
        cudaFuncSetAttribute(fwd_kernel_of(nst), cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        return occ_of(fwd_kernel_of(nst), sm);
    }
    if (gains) {
        const int sm = adj_gains_smem_bytes(n_ant);
        if (sm > adj_smem_limit) {
            cudaFuncSetAttribute(adj_mixed_gains_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            adj_smem_limit = sm;
        }
        return occ_of(adj_mixed_gains_kernel, sm);
    }
    const int sm = adj_stage_bytes_of(shape_nst(nst));   // fixed per tile shape
    cudaFuncSetAttribute(adj_kernel_of(nst), cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    return occ_of(adj_kernel_of(nst), sm);
}

}  // namespace sl1m
