// sl1m_solver.cu -- the vector side of SL1M's FISTA (Hardy 2013, Sect. 3):
// finishing the stream-K partial sums of the operator kernels, the residual
// r = W (A y - V) and its norm, the positive soft threshold (Eq. threshp) and
// the momentum step of the algorithm box, the power iteration for L, and the
// per-problem FP64 scalars.  All reductions use a fixed order (deterministic,
// no atomics).  These kernels are bound by HBM bandwidth.
#include <math.h>

#include "sl1m_dev.h"
#include "sl1m_kernels.h"

namespace sl1m {

// ---------------------------------------------------------- permutations

__global__ void gather_real_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                   const int* __restrict__ orig, int n_pad, double scale)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x) {
        const int o = orig[i];
        dst[i] = o >= 0 ? src[o] * scale : 0.0;
    }
}

__global__ void gather_cplx_kernel(const double2* __restrict__ src, double2* __restrict__ dst,
                                   const int* __restrict__ orig, int n_pad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x) {
        const int o = orig[i];
        dst[i] = o >= 0 ? src[o] : make_double2(0.0, 0.0);
    }
}

__global__ void scatter_real_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                    const int* __restrict__ orig, int n_pad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x) {
        const int o = orig[i];
        if (o >= 0) dst[o] = src[i];
    }
}

__global__ void scatter_cplx_kernel(const double2* __restrict__ src, double2* __restrict__ dst,
                                    const int* __restrict__ orig, int n_pad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x) {
        const int o = orig[i];
        if (o >= 0) dst[o] = src[i];
    }
}

__global__ void fill_valid_kernel(double* __restrict__ dst, const int* __restrict__ orig, int n_pad,
                                  double val)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x)
        dst[i] = orig[i] >= 0 ? val : 0.0;
}

// r = W V in the library's visibility order (input of the dirty image).
__global__ void weighted_vis_kernel(const double2* __restrict__ V, const d4* __restrict__ vd,
                                    double2* __restrict__ r, int n_pad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x) {
        const double w = vd[i].w;
        r[i] = make_double2(w * V[i].x, w * V[i].y);
    }
}

static int grid_for(int n) { return n <= 0 ? 1 : (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096; }

cudaError_t launch_gather_real(const double* src, double* dst, const int* orig, int n_pad,
                               double scale, cudaStream_t st)
{
    gather_real_kernel<<<grid_for(n_pad), 256, 0, st>>>(src, dst, orig, n_pad, scale);
    return cudaGetLastError();
}
cudaError_t launch_gather_cplx(const double2* src, double2* dst, const int* orig, int n_pad,
                               cudaStream_t st)
{
    gather_cplx_kernel<<<grid_for(n_pad), 256, 0, st>>>(src, dst, orig, n_pad);
    return cudaGetLastError();
}
cudaError_t launch_scatter_real(const double* src, double* dst, const int* orig, int n_pad,
                                cudaStream_t st)
{
    scatter_real_kernel<<<grid_for(n_pad), 256, 0, st>>>(src, dst, orig, n_pad);
    return cudaGetLastError();
}
cudaError_t launch_scatter_cplx(const double2* src, double2* dst, const int* orig, int n_pad,
                                cudaStream_t st)
{
    scatter_cplx_kernel<<<grid_for(n_pad), 256, 0, st>>>(src, dst, orig, n_pad);
    return cudaGetLastError();
}
cudaError_t launch_weighted_vis(const double2* V, const d4* vd, double2* r, int n_pad, cudaStream_t st)
{
    weighted_vis_kernel<<<grid_for(n_pad), 256, 0, st>>>(V, vd, r, n_pad);
    return cudaGetLastError();
}

cudaError_t launch_fill_valid(double* dst, const int* orig, int n_pad, double val, cudaStream_t st)
{
    fill_valid_kernel<<<grid_for(n_pad), 256, 0, st>>>(dst, orig, n_pad, val);
    return cudaGetLastError();
}

// --------------------------------------------------------------- helpers

// t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2 and beta_k = (t_k - 1) / t_{k+1}
// (the momentum step of the FISTA box).
__device__ __forceinline__ void fista_beta(double t, double& t_next, double& beta)
{
    t_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    beta = (t - 1.0) / t_next;
}

__device__ __forceinline__ int find_blk_prob(const Plan& pl, int gb)
{
    int lo = 0, hi = pl.n_probs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pl.prob_b0[mid] <= gb) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Fixed-order block sum of one double per thread (256 threads).
__device__ double block_sum(double v, double* sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__device__ int block_sum_int(int v, int* sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const int r = sh[0];
    __syncthreads();
    return r;
}

// Mode of problem P in a finish kernel: FIN_OP (operator call), FIN_POWER,
// FIN_INIT, FIN_SOLVE, or -1 (P takes no part in this step).
__device__ __forceinline__ int fwd_finish_mode(const DevProblem& P)
{
    if (!P.st) return FIN_OP;
    switch (P.st->phase) {
    case PH_PINIT:
    case PH_POWER: return FIN_POWER;
    case PH_SINIT: return FIN_INIT;
    case PH_SOLVE: return FIN_SOLVE;
    default: return -1;
    }
}

__device__ __forceinline__ int adj_finish_mode(const DevProblem& P)
{
    if (!P.st) return FIN_OP;
    switch (P.st->phase) {
    case PH_POWER: return FIN_POWER;
    case PH_SOLVE: return FIN_SOLVE;
    default: return -1;
    }
}

// Sum of the ncon partial slots of element i, from slot poff on, in slot
// order.  The loads of 8 slots are issued before their additions, so they are
// in flight together (one L2 round trip per 8 slots, not per slot); the sum
// is added in the same order as one load at a time would add it.
template <class T>
__device__ __forceinline__ void add_in(T& s, const T& q);
template <>
__device__ __forceinline__ void add_in<double>(double& s, const double& q) { s += q; }
template <>
__device__ __forceinline__ void add_in<double2>(double2& s, const double2& q)
{
    s.x += q.x;
    s.y += q.y;
}
template <class T>
__device__ __forceinline__ void sum_slots(T& s, const T* __restrict__ partial, int poff, int ncon, int i)
{
    int c = 0;
    for (; c + 8 <= ncon; c += 8) {
        T q[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) q[t] = partial[(size_t)(poff + c + t) * BLK + i];
#pragma unroll
        for (int t = 0; t < 8; ++t) add_in(s, q[t]);
    }
    for (; c < ncon; ++c) add_in(s, partial[(size_t)(poff + c) * BLK + i]);
}

// ---------------------------------------------------------- forward finish
// Grid-stride over the plan's owned blocks (BLK visibilities each): sums the
// block's partial slots in CTA order, then per problem
//   FIN_OP    : fwd_out = A x
//   FIN_POWER : r = W (A x)                      (input of the next adjoint)
//   FIN_INIT  : AI_0 = A I_0, r = W (A I_0 - V), block sum W|A I_0 - V|^2
//   FIN_SOLVE : AI_k = A I_k, block sum W|A I_k - V|^2,
//               A y_{k+1} = AI_k + beta_k (AI_k - AI_{k-1})  (linearity),
//               r = W (A y_{k+1} - V)
//               (MFISTA: A z_k and its block sum only)
__global__ void __launch_bounds__(256)
fwd_finish_kernel(const DevProblem* __restrict__ probs, const Plan* __restrict__ plp,
                  const double2* __restrict__ partial)
{
    __shared__ double sh[256];
    __shared__ int shi[256];
    const Plan pl = *plp;
    for (int gb = blockIdx.x; gb < pl.n_blocks; gb += gridDim.x) {
        const int p = find_blk_prob(pl, gb);
        const DevProblem& P = probs[p];
        const int mode = fwd_finish_mode(P);
        if (mode < 0) continue;
        const int blk = gb - pl.prob_b0[p];
        const int poff = pl.blk_poff[gb], ncon = pl.blk_ncon[gb];
        double beta = 0.0;
        int par = 0, mf = 0;
        if (mode == FIN_SOLVE) {
            const SolveState& S = *P.st;
            double tn;
            fista_beta(S.t, tn, beta);
            par = (S.k + 1) & 1;
            mf = S.algo;
        }
        double bn = 0.0;
        int bad = 0;
        for (int h = 0; h < 2; ++h) {
            const int i = threadIdx.x + 256 * h;
            const int e = blk * BLK + i;
            if (e >= P.vis.n_pad) continue;
            double2 s = make_double2(0.0, 0.0);
            sum_slots(s, partial, poff, ncon, i);
            if (!isfinite(s.x) || !isfinite(s.y)) bad = 1;
            if (mode == FIN_OP) {
                P.fwd_out[e] = s;
                continue;
            }
            const SolveBufs& B = P.b;
            const double W = P.vis.d[e].w;
            if (mode == FIN_POWER) {
                B.r[e] = make_double2(W * s.x, W * s.y);
                continue;
            }
            const double2 V = P.V[e];
            const double dr = s.x - V.x, di = s.y - V.y;
            bn += W * (dr * dr + di * di);
            if (mode == FIN_INIT) {
                B.AI[0][e] = s;
                B.r[e] = make_double2(W * dr, W * di);
            } else if (mf) {
                B.AI[1][e] = s;                 // A z_k; r is formed by the mix kernel
            } else {
                const double2 old = B.AI[par ^ 1][e];
                B.AI[par][e] = s;
                const double ayr = s.x + beta * (s.x - old.x);
                const double ayi = s.y + beta * (s.y - old.y);
                B.r[e] = make_double2(W * (ayr - V.x), W * (ayi - V.y));
            }
        }
        if (mode == FIN_OP) continue;
        const int nb = block_sum_int(bad, shi);
        const double tot = block_sum(bn, sh);
        if (threadIdx.x == 0) {
            P.b.blk_badv[blk] = nb;
            if (mode != FIN_POWER) P.b.blk_r2[blk] = tot;
        }
    }
}

// ---------------------------------------------------------- adjoint finish
//   FIN_OP    : adj_out = Re A^H r
//   FIN_POWER : z = (Re A^H W A x) * inv_mu into xv (= B x_unit), block sum z^2
//   FIN_SOLVE : I_k = T^{lambda/L}(y_k - g/L)                 (Eq. threshp)
//               y_{k+1} = I_k + beta_k (I_k - I_{k-1})        (FISTA box)
//               block sums of I_k and of nnz
//               (MFISTA: z_k = T^{lambda/L}(y_k - g/L) and its sums only)
__global__ void __launch_bounds__(256)
adj_finish_kernel(const DevProblem* __restrict__ probs, const Plan* __restrict__ plp,
                  const double* __restrict__ partial)
{
    __shared__ double sh[256];
    __shared__ int shi[256];
    const Plan pl = *plp;
    for (int gb = blockIdx.x; gb < pl.n_blocks; gb += gridDim.x) {
        const int p = find_blk_prob(pl, gb);
        const DevProblem& P = probs[p];
        const int mode = adj_finish_mode(P);
        if (mode < 0) continue;
        const int blk = gb - pl.prob_b0[p];
        const int poff = pl.blk_poff[gb], ncon = pl.blk_ncon[gb];
        double inv_L = 0.0, thr = 0.0, beta = 0.0, scale = 1.0;
        int par = 0, mf = 0;
        if (mode == FIN_SOLVE) {
            const SolveState& S = *P.st;
            double tn;
            fista_beta(S.t, tn, beta);
            inv_L = 1.0 / S.L;
            thr = S.lambda / S.L;
            par = (S.k + 1) & 1;
            mf = S.algo;
        } else if (mode == FIN_POWER) {
            scale = P.st->inv_mu;
        }
        double acc = 0.0;
        int cnt = 0, bad = 0;
        for (int h = 0; h < 2; ++h) {
            const int i = threadIdx.x + 256 * h;
            const int e = blk * BLK + i;
            if (e >= P.pix.n_pad) continue;
            double s = 0.0;
            sum_slots(s, partial, poff, ncon, i);
            if (!isfinite(s)) bad = 1;
            if (mode == FIN_OP) {
                P.adj_out[e] = s;
                continue;
            }
            const SolveBufs& B = P.b;
            if (mode == FIN_POWER) {
                const double z = s * scale;
                B.xv[e] = z;
                acc += z * z;
                continue;
            }
            // FIN_SOLVE
            const double v = B.y[e] - s * inv_L;
            double In = v > thr ? v - thr : 0.0;
            if (P.pix.orig[e] < 0) In = 0.0;
            if (mf) {
                B.I[1][e] = In;                 // z_k; y is formed by the mix kernel
            } else {
                const double Io = B.I[par ^ 1][e];
                B.I[par][e] = In;
                B.y[e] = In + beta * (In - Io);
            }
            acc += In;
            cnt += In > 0.0;
        }
        if (mode == FIN_OP) continue;
        const double tot = block_sum(acc, sh);
        const int nb = block_sum_int(bad, shi);
        const int nz = block_sum_int(cnt, shi);
        if (threadIdx.x == 0) {
            const SolveBufs& B = P.b;
            if (mode == FIN_POWER) B.blk_z2[blk] = tot;
            else {
                B.blk_l1[blk] = tot;
                B.blk_nnz[blk] = nz;
            }
            B.blk_badp[blk] = nb;
        }
    }
}

// ------------------------------------------------------------------ scalars
// One warp per problem; fixed-order (lane-strided, then xor-tree) sums.
__device__ double warp_sum_fixed(const double* a, int n)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) s += a[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

__device__ long long warp_sum_fixed_i(const int* a, int n)
{
    long long s = 0;
    for (int i = threadIdx.x; i < n; i += 32) s += a[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// The phase machine of every solve in the batch (end of a tick).
__global__ void scalars_kernel(const DevProblem* __restrict__ probs, const int* __restrict__ n_probs,
                               double* __restrict__ evals)
{
    const int np = *n_probs;
    for (int p = blockIdx.x; p < np; p += gridDim.x) {
        const DevProblem& P = probs[p];
        if (!P.st) continue;
        SolveState& S = *P.st;
        const SolveBufs& B = P.b;
        const int nvb = P.vis.n_blk, npb = P.pix.n_blk;
        const int ph = S.phase;
        // pairs the operator kernels of this tick evaluated for this problem
        // (the roles of fwd_role / adj_role in the tick's phase)
        if (evals && threadIdx.x == 0) {
            const double pairs = (double)P.vis.n * (double)P.pix.n;
            if (ph == PH_PINIT || ph == PH_POWER || ph == PH_SINIT || ph == PH_SOLVE) atomicAdd(&evals[0], pairs);
            if (ph == PH_POWER || ph == PH_SOLVE) atomicAdd(&evals[1], pairs);
        }
        // the mix kernel of the previous tick has run (stream order)
        if (threadIdx.x == 0) S.mix_pending = 0;
        if (ph == PH_PINIT) {
            if (threadIdx.x == 0) S.phase = PH_POWER;
        } else if (ph == PH_POWER) {
            const double z2 = warp_sum_fixed(B.blk_z2, npb);
            const long long bad = warp_sum_fixed_i(B.blk_badv, nvb) + warp_sum_fixed_i(B.blk_badp, npb);
            if (threadIdx.x == 0) {
                const double mu = sqrt(z2);
                S.pit += 1;
                if (bad || !isfinite(mu) || mu == 0.0) {
                    S.nonfinite = (bad || !isfinite(mu)) ? 1 : 0;
                    S.mu = mu;
                    S.phase = PH_DONE;
                } else {
                    const bool conv = (S.pit > 1 && fabs(mu - S.mu_prev) <= S.ptol * mu) || S.pit >= S.pmax;
                    S.mu = mu;
                    S.mu_prev = mu;
                    S.inv_mu = 1.0 / mu;
                    if (conv) {
                        S.L = mu;
                        S.phase = S.power_only ? PH_DONE : PH_SINIT;
                    }
                }
            }
        } else if (ph == PH_SINIT) {
            const double r2 = warp_sum_fixed(B.blk_r2, nvb);
            const long long bad = warp_sum_fixed_i(B.blk_badv, nvb);
            if (threadIdx.x == 0) {
                S.resid2 = r2;
                S.E_prev = 0.5 * r2 + S.lambda * S.l1;
                S.E = S.E_prev;
                S.k = 0;
                S.t = 1.0;
                S.converged = 0;
                S.nonfinite = bad ? 1 : 0;
                S.phase = (S.max_iter <= 0 || bad) ? PH_DONE : PH_SOLVE;
            }
        } else if (ph == PH_SOLVE) {
            const double r2 = warp_sum_fixed(B.blk_r2, nvb);
            const double l1 = warp_sum_fixed(B.blk_l1, npb);
            const long long nnz = warp_sum_fixed_i(B.blk_nnz, npb);
            const long long bad = warp_sum_fixed_i(B.blk_badv, nvb) + warp_sum_fixed_i(B.blk_badp, npb);
            if (threadIdx.x == 0 && S.algo) {
                // MFISTA: keep the better of z_k and x_{k-1}; then
                // y_{k+1} = x_k + (t_k/t_{k+1})(z_k - x_k) + ((t_k-1)/t_{k+1})(x_k - x_{k-1})
                //         = x_{k-1} + c (z_k - x_{k-1}), c = 1 + (t_k-1)/t_{k+1} when z_k
                // is kept, t_k/t_{k+1} when it is not (formed by the mix kernel).
                double tn, beta;
                fista_beta(S.t, tn, beta);
                const double Fz = 0.5 * r2 + S.lambda * l1;
                const double Fx = S.E_prev;
                const int take = Fz <= Fx;
                S.take = take;
                S.cmix = take ? 1.0 + beta : S.t / tn;
                S.mix_pending = 1;
                S.k += 1;
                S.t = tn;
                S.beta = beta;
                if (take) {
                    S.resid2 = r2;
                    S.l1 = l1;
                    S.nnz = nnz;
                    S.E = Fz;
                }
                bool done = false;
                if (bad || !isfinite(Fz)) {
                    S.nonfinite = 1;
                    done = true;
                }
                if (S.tol > 0.0 && fabs(Fz - Fx) <= S.tol * Fx) {
                    S.converged = 1;
                    done = true;
                }
                if (S.k >= S.max_iter) done = true;
                S.E_prev = S.E;
                if (done) S.phase = PH_DONE;
            } else if (threadIdx.x == 0) {
                double tn, beta;
                fista_beta(S.t, tn, beta);
                const double E = 0.5 * r2 + S.lambda * l1;
                S.k += 1;
                S.t = tn;
                S.beta = beta;
                S.resid2 = r2;
                S.l1 = l1;
                S.nnz = nnz;
                S.E = E;
                bool done = false;
                if (bad || !isfinite(E)) {
                    S.nonfinite = 1;
                    done = true;
                }
                if (S.tol > 0.0 && fabs(E - S.E_prev) <= S.tol * S.E_prev) {
                    S.converged = 1;
                    done = true;
                }
                if (S.k >= S.max_iter) done = true;
                S.E_prev = E;
                if (done) S.phase = PH_DONE;
            }
        }
    }
}

// ------------------------------------------------------------ MFISTA mix
// Finishes an MFISTA step once the scalars kernel has compared F(z_k) with
// F(x_{k-1}): grid-stride over the visibility blocks of the forward plan and
// then the pixel blocks of the adjoint plan,
//   visibilities: A y_{k+1} = A x_{k-1} + c (A z_k - A x_{k-1})   (linearity)
//                 r = W (A y_{k+1} - V);  A x_k = A z_k if z_k was kept
//   pixels:       y_{k+1} = x_{k-1} + c (z_k - x_{k-1});  x_k = z_k if kept
__global__ void __launch_bounds__(256)
mfista_mix_kernel(const DevProblem* __restrict__ probs, const Plan* __restrict__ fplp,
                  const Plan* __restrict__ aplp)
{
    const Plan fp = *fplp, ap = *aplp;
    for (int gb = blockIdx.x; gb < fp.n_blocks + ap.n_blocks; gb += gridDim.x) {
        const bool vis = gb < fp.n_blocks;
        const Plan& pl = vis ? fp : ap;
        const int g = vis ? gb : gb - fp.n_blocks;
        const int p = find_blk_prob(pl, g);
        const DevProblem& P = probs[p];
        if (!P.st || !P.st->algo || !P.st->mix_pending) continue;
        const double c = P.st->cmix;
        const int take = P.st->take;
        const int blk = g - pl.prob_b0[p];
        const SolveBufs& B = P.b;
        for (int h = 0; h < 2; ++h) {
            const int e = blk * BLK + threadIdx.x + 256 * h;
            if (vis) {
                if (e >= P.vis.n_pad) continue;
                const double2 ax = B.AI[0][e], az = B.AI[1][e], V = P.V[e];
                const double W = P.vis.d[e].w;
                const double ayr = ax.x + c * (az.x - ax.x), ayi = ax.y + c * (az.y - ax.y);
                B.r[e] = make_double2(W * (ayr - V.x), W * (ayi - V.y));
                if (take) B.AI[0][e] = az;
            } else {
                if (e >= P.pix.n_pad) continue;
                const double x = B.I[0][e], z = B.I[1][e];
                B.y[e] = x + c * (z - x);
                if (take) B.I[0][e] = z;
            }
        }
    }
}

// Phase of every problem of a batch, for the host (one int per problem).
__global__ void phases_kernel(const DevProblem* __restrict__ probs, const int* __restrict__ n_probs,
                              int* __restrict__ out)
{
    const int np = *n_probs;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x)
        out[p] = probs[p].st ? probs[p].st->phase : PH_IDLE;
}

cudaError_t launch_fwd_finish(const DevProblem* probs, const Plan* plp, int grid, const double2* partial,
                              cudaStream_t st)
{
    fwd_finish_kernel<<<grid, 256, 0, st>>>(probs, plp, partial);
    return cudaGetLastError();
}

cudaError_t launch_adj_finish(const DevProblem* probs, const Plan* plp, int grid, const double* partial,
                              cudaStream_t st)
{
    adj_finish_kernel<<<grid, 256, 0, st>>>(probs, plp, partial);
    return cudaGetLastError();
}

cudaError_t launch_mfista_mix(const DevProblem* probs, const Plan* fplp, const Plan* aplp, int grid,
                              cudaStream_t st)
{
    mfista_mix_kernel<<<grid, 256, 0, st>>>(probs, fplp, aplp);
    return cudaGetLastError();
}

cudaError_t launch_scalars(const DevProblem* probs, const int* n_probs, int grid, double* evals, cudaStream_t st)
{
    scalars_kernel<<<grid, 32, 0, st>>>(probs, n_probs, evals);
    return cudaGetLastError();
}

cudaError_t launch_phases(const DevProblem* probs, const int* n_probs, int grid, int* out, cudaStream_t st)
{
    phases_kernel<<<grid, 128, 0, st>>>(probs, n_probs, out);
    return cudaGetLastError();
}

}  // namespace sl1m
