// sl1m_fp64.cu -- the "plain" FP64 forward operator and adjoint of SL1M
// (Hardy 2013, Sect. 2 and 3.1): the same stream-K decomposition of work as
// the mixed kernels, every step in FP64 (phase, sincospi, exp, accumulation).
// Gaussian pixels use the real split form of Eq. samlm4/samlm5 given in
// sl1m_mixed.cu; gains multiply by G[j][a_k] conj(G[j][b_k]).
#include "sl1m_dev.h"
#include "sl1m_devfn.cuh"
#include "sl1m_kernels.h"

namespace sl1m {

// =====================================================================
// FP64 ("plain") kernels: same decomposition of work, every step in FP64.
// =====================================================================
__device__ __forceinline__ void entry_phase64(int kind, double sigma, double u, double v, double w,
                                              const d4 pd, const d4 pg,
                                              double& amp, double& re_f, double& im_f, double& ph)
{
    // returns A/(g/n) = amp * (re_f + i im_f) * exp(-2 pi i ph)
    const double phi = fma(w, pd.z, fma(v, pd.y, u * pd.x));
    if (kind == DIRAC) {
        amp = 1.0; re_f = 1.0; im_f = 0.0; ph = phi;
        return;
    }
    const double s2 = sigma * sigma;
    const double beta = w * s2;
    const double id = 1.0 / (1.0 + beta * beta);
    const double gam = beta * beta * id;
    const double t = u * pg.x + v * pg.y - w * pg.z;
    double corr = gam * t - 0.5 * id * beta * s2 * (u * u + v * v);
    if (kind == PARAXIAL) corr += w * pg.w;
    ph = phi - corr;
    const double e1 = u - w * pg.x, e2 = v - w * pg.y;
    amp = exp(-3.141592653589793 * s2 * id * (e1 * e1 + e2 * e2)) * id;
    re_f = 1.0;
    im_f = beta;
}

__global__ void __launch_bounds__(NTHREADS)
fwd_fp64_kernel(const DevProblem* __restrict__ probs, const Plan* __restrict__ plp, double2* __restrict__ partial)
{
    __shared__ d4 s_pd[G];    // {l, m, n-1, a = x/n}
    __shared__ d4 s_pg[G];    // {l, m, r^2/2, nu}
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Plan pl = *plp;
    const long long c = blockIdx.x;
    long long u, u_end;
    cta_range(pl, c, u, u_end);
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
        d4 vd[2];
        int2 ant[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            vd[r] = make_d4(0.0, 0.0, 0.0, 0.0);
            ant[r] = make_int2(0, 0);
            if (vg_ok) {
                const int e = vg * G + lane + 32 * r;
                vd[r] = P.vis.d[e];
                if (P.gains64) ant[r] = P.ant[e];
            }
        }
        double tr[2] = {0.0, 0.0}, ti[2] = {0.0, 0.0};
        for (int g = g0; g < g1; ++g) {
            __syncthreads();
            const int kind = P.gkind[g];
            const double sigma = P.gsig64[g];
            if (threadIdx.x < G) {
                const int e = g * G + threadIdx.x;
                d4 d = P.pix.d[e];
                d.w = X[e] * d.w;
                s_pd[threadIdx.x] = d;
                if (kind != DIRAC) s_pg[threadIdx.x] = P.pgauss64[e];
            }
            __syncthreads();
            for (int j = 0; j < G; ++j) {
                const d4 pd = s_pd[j];
                const d4 pg = s_pg[j];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    double amp, fr, fi, ph;
                    entry_phase64(kind, sigma, vd[r].x, vd[r].y, vd[r].z, pd, pg, amp, fr, fi, ph);
                    ph = ph - rint(ph);
                    double sn, cs;
                    sincospi(2.0 * ph, &sn, &cs);
                    // amp (fr + i fi)(cs - i sn)
                    double er = amp * (fr * cs + fi * sn), ei = amp * (fi * cs - fr * sn);
                    if (P.gains64) {
                        const double2 ga = P.gains64[(size_t)(g * G + j) * P.n_ant + ant[r].x];
                        const double2 gb = P.gains64[(size_t)(g * G + j) * P.n_ant + ant[r].y];
                        const double gr = ga.x * gb.x + ga.y * gb.y;
                        const double gi = ga.y * gb.x - ga.x * gb.y;
                        const double t = er * gr - ei * gi;
                        ei = er * gi + ei * gr;
                        er = t;
                    }
                    tr[r] = fma(pd.w, er, tr[r]);
                    ti[r] = fma(pd.w, ei, ti[r]);
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
}

__global__ void __launch_bounds__(NTHREADS)
adj_fp64_kernel(const DevProblem* __restrict__ probs, const Plan* __restrict__ plp, double* __restrict__ partial)
{
    __shared__ d4 s_vd[G];    // {u, v, w, W}
    __shared__ double2 s_r[G];
    __shared__ int2 s_ant[G];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Plan pl = *plp;
    const long long c = blockIdx.x;
    long long u, u_end;
    cta_range(pl, c, u, u_end);
    while (u < u_end) {
        const int p = find_prob(pl, u);
        const DevProblem& P = probs[p];
        const long long loc = u - pl.prob_u0[p];
        const double2* R;
        if (!adj_role(P, R)) {                    // problem not in this step: skip its units
            u = min(u_end, pl.prob_u0[p + 1]);
            continue;
        }
        const int upb = P.vis.n_gran;
        const int blk = (int)(loc / upb);
        const int g0 = (int)(loc % upb);
        const int g1 = (int)min((long long)upb, (long long)g0 + (u_end - u));
        const int pgi = blk * BLK_GRAN + warp;
        const bool pg_ok = pgi < P.pix.n_gran;
        const int kind = pg_ok ? P.gkind[pgi] : DIRAC;
        const double sigma = pg_ok ? P.gsig64[pgi] : 0.0;
        d4 pd[2], pg[2];
        int eidx[2] = {0, 0};
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            pd[r] = pg[r] = make_d4(0.0, 0.0, 0.0, 0.0);
            if (pg_ok) {
                const int e = pgi * G + lane + 32 * r;
                eidx[r] = e;
                pd[r] = P.pix.d[e];
                if (kind != DIRAC) pg[r] = P.pgauss64[e];
            }
        }
        double tot[2] = {0.0, 0.0};
        for (int g = g0; g < g1; ++g) {
            __syncthreads();
            if (threadIdx.x < G) {
                const int e = g * G + threadIdx.x;
                s_vd[threadIdx.x] = P.vis.d[e];
                s_r[threadIdx.x] = R[e];
                if (P.gains64) s_ant[threadIdx.x] = P.ant[e];
            }
            __syncthreads();
            for (int k = 0; k < G; ++k) {
                const d4 vd = s_vd[k];
                const double2 rr = s_r[k];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    double amp, fr, fi, ph;
                    entry_phase64(kind, sigma, vd.x, vd.y, vd.z, pd[r], pg[r], amp, fr, fi, ph);
                    ph = ph - rint(ph);
                    double sn, cs;
                    sincospi(2.0 * ph, &sn, &cs);
                    double er = amp * (fr * cs + fi * sn), ei = amp * (fi * cs - fr * sn);
                    if (P.gains64) {
                        const int2 ab = s_ant[k];
                        const double2 ga = P.gains64[(size_t)eidx[r] * P.n_ant + ab.x];
                        const double2 gb = P.gains64[(size_t)eidx[r] * P.n_ant + ab.y];
                        const double gr = ga.x * gb.x + ga.y * gb.y;
                        const double gi = ga.y * gb.x - ga.x * gb.y;
                        const double t = er * gr - ei * gi;
                        ei = er * gi + ei * gr;
                        er = t;
                    }
                    // Re(conj(e) r)
                    tot[r] = fma(er, rr.x, fma(ei, rr.y, tot[r]));
                }
            }
        }
        if (pg_ok) {
            const int gb = pl.prob_b0[p] + blk;
            double* dst = partial + (size_t)slot_of(pl, gb) * BLK + warp * G + lane;
#pragma unroll
            for (int r = 0; r < 2; ++r) dst[32 * r] = tot[r] * pd[r].w;
        }
        u += g1 - g0;
    }
}

// ------------------------------------------------------------- launchers

cudaError_t launch_forward_mixed(bool gains, int n_ant, int nst, const DevProblem* probs, const Plan* plp, int C,
                                 double2* partial, cudaStream_t st);
cudaError_t launch_adjoint_mixed(bool gains, int n_ant, int nst, const DevProblem* probs, const Plan* plp, int C,
                                 double* partial, cudaStream_t st);
int occupancy_mixed(int op, bool gains, int n_ant, int nst);

cudaError_t launch_forward(int precision, bool gains, int n_ant, const DevProblem* probs,
                           const Plan* plp, int C, double2* partial, cudaStream_t st, int nst)
{
    if (precision == 0) {
        fwd_fp64_kernel<<<C, NTHREADS, 0, st>>>(probs, plp, partial);
        return cudaGetLastError();
    }
    return launch_forward_mixed(gains, n_ant, nst, probs, plp, C, partial, st);
}

cudaError_t launch_adjoint(int precision, bool gains, int n_ant, const DevProblem* probs, const Plan* plp, int C,
                           double* partial, cudaStream_t st, int nst)
{
    if (precision == 0) {
        adj_fp64_kernel<<<C, NTHREADS, 0, st>>>(probs, plp, partial);
        return cudaGetLastError();
    }
    return launch_adjoint_mixed(gains, n_ant, nst, probs, plp, C, partial, st);
}

int occupancy(int which, bool gains, int n_ant, int nst)
{
    int n = 0;
    switch (which) {
    case 0: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fwd_fp64_kernel, NTHREADS, 0); break;
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, adj_fp64_kernel, NTHREADS, 0); break;
    case 2: return occupancy_mixed(0, gains, n_ant, nst);
    case 3: return occupancy_mixed(1, gains, n_ant, nst);
    }
    return n < 1 ? 1 : n;
}

}  // namespace sl1m
