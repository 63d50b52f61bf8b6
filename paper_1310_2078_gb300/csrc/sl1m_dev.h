// sl1m_dev.h -- device-side data layout shared by the kernels and the host
// code of libsl1m.  Internal: not part of the public C ABI (include/sl1m.h).
//
// Layout in HBM (per problem, after sorting; see sl1m_host.cpp):
//   * Both sides (visibilities and pixels) are permuted into "granules" of
//     G = 64 elements by a k-d median split, so that every granule is a
//     compact box in (u,v,w) resp. (l,m).  Pixels are first grouped into
//     classes of equal (kind, sigma); each class is padded to a multiple of G
//     with inert padding (amplitude 0 / weight 0), so kind and sigma are
//     uniform per pixel granule.
//   * Per element: FP64 coordinates (x,y,z,aux) for the FP64 path, and for
//     the mixed path the FP32 hi/lo split of the absolute coordinates and of
//     the offset from the granule centre.
//   * A CTA "owns" a block of BLK_GRAN granules of one side (one granule per
//     warp, 2 elements per lane) and streams granules of the other side
//     through shared memory.  Work is split over a persistent grid by
//     "units" = (owned block, streamed granule), stream-K style; partial sums
//     land in per-(block, contributing CTA) slots that the finish kernels add
//     up in a fixed order (deterministic, no atomics).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sl1m {

// 32-byte aligned quadruple of doubles (one 256-bit access).
struct __align__(32) d4 {
    double x, y, z, w;
};
__host__ __device__ inline d4 make_d4(double x, double y, double z, double w)
{
    d4 r;
    r.x = x; r.y = y; r.z = z; r.w = w;
    return r;
}

constexpr int G = 64;                 // granule size
// Gains of one pixel granule as the mixed kernels hold them: one row of G
// pixels per antenna, padded to GP so that rows start in different shared-
// memory banks; rows are padded to an even count so that a granule's table
// (gain_rows(n_ant) x GP float2) is a multiple of 16 bytes, the unit of a
// bulk (TMA) copy.  The same layout sits in HBM, [pixel granule][row][GP].
constexpr int GP = G + 1;
__host__ __device__ inline int gain_rows(int n_ant) { return (n_ant + 1) & ~1; }
// Baselines of a visibility granule.  With gains, the members of each
// visibility granule are sorted by antenna pair (a, b); a granule of an
// interferometer's data holds few distinct pairs (the uv track of a baseline
// is compact), so the forward builds, per tile, x_j G_ja conj(G_jb) once per
// distinct pair and pixel instead of once per visibility and pixel.  Granules
// with more than NB_MAX pairs take the per-visibility gathers instead.
constexpr int NB_MAX = 28;
constexpr int BT_CH = 16;             // pixels per chunk of that table
constexpr int BT_P = BT_CH + 1;       // its padded row (rows start in different banks)
constexpr int BLK_GRAN = 8;           // owned granules per CTA (one per warp)
constexpr int BLK = G * BLK_GRAN;     // owned elements per CTA block
constexpr int NTHREADS = 256;         // 8 warps
constexpr int MAX_PROBS = 1024;       // problems per batched launch

enum Kind : int { DIRAC = 0, PARAXIAL = 1, WIDE = 2 };

// A tile (owned granule x streamed granule) whose offsets can make the FP32
// product term D = (X - Xc).(Y - Yc) exceed D_MAX turns is evaluated with
// the exact split instead (its FP32 rounding error grows like 2^-24 |D|).
constexpr float D_MAX = 6.0f;

// One side (visibilities or pixels) of a problem, sorted and padded.
struct Side {
    int n;              // real elements
    int n_pad;          // n_gran * G
    int n_gran;
    int n_blk;          // ceil(n_gran / BLK_GRAN)
    const float4* hi;     // absolute coordinates, FP32 hi part  {x,y,z,0}
    const float4* lo;     // absolute coordinates, FP32 lo part
    const float4* off;    // offset from granule centre, rounded {dx,dy,dz,aux32}
    const float4* offlo;  // offset residual: offset = off + offlo (to ~2^-48)
    const float4* cen_hi; // granule centre, hi   [n_gran]
    const float4* cen_lo; // granule centre, lo   [n_gran]
    const float4* ext;    // granule extent: max |offset| per coordinate [n_gran]
    const d4* d;     // FP64 {x, y, z, aux}
    const int* orig;      // sorted index -> caller's index, -1 for padding
};
// vis: x,y,z = u,v,w (wavelengths); aux = weight W_k (0 for padding)
// pix: x,y,z = l, m, n-1 (n-1 = -(l^2+m^2)/(1+n)); aux = 1/n (0 for padding)

// Phases of one solve, advanced on the device by the scalars kernel at the
// end of every tick (one tick = adjoint, adjoint finish, forward, forward
// finish, scalars for every problem of a batch):
//   PINIT  forward of x = 1/sqrt(n) -> r = W A x
//   POWER  power-iteration step: z = B x_unit, then r = W A z; mu = ||z||
//   SINIT  forward of I_0 -> A I_0, r = W (A I_0 - V), E_0
//   SOLVE  one FISTA step (Sect. 3 algorithm box), or one MFISTA step
//          (Beck & Teboulle 2009b), which a sixth kernel finishes (mix)
//   DONE   finished (converged, max_iter reached, or non-finite)
enum Phase : int { PH_IDLE = 0, PH_PINIT = 1, PH_POWER = 2, PH_SINIT = 3, PH_SOLVE = 4, PH_DONE = 5 };

// Solver state of one problem (device resident, FP64 scalars).
struct SolveState {
    double lambda, L, tol;
    double t;            // t_k of the momentum sequence (t_1 = 1)
    double beta;         // (t_k - 1) / t_{k+1} of the last step
    double E_prev;       // E(I_{k-1})
    double E, resid2, l1;
    long long nnz;
    int k;               // FISTA steps completed
    int max_iter;
    int phase;
    int converged;
    int nonfinite;       // 1: a non-finite value was met
    int power_only;      // 1: stop after the power iteration (L only)
    // MFISTA (algo = 1): I[0] = x_k, I[1] = z_k, AI[0] = A x_k, AI[1] = A z_k
    int algo;            // 0 FISTA, 1 MFISTA
    int take;            // last step kept z_k (F(z_k) <= F(x_{k-1}))
    int mix_pending;     // the mix kernel of this tick finishes the last step
    double cmix;         // y_{k+1} = x_{k-1} + cmix (z_k - x_{k-1})
    // power iteration
    double mu, mu_prev, inv_mu;
    int pit, pmax;
    double ptol;
};

// Per-problem solver workspace (device pointers).
struct SolveBufs {
    double* I[2];        // I_k ping-pong [pix.n_pad]
    double* y;           // y_k [pix.n_pad]
    double* xv;          // power-iteration vector [pix.n_pad]
    double2* AI[2];      // A I_k ping-pong [vis.n_pad]
    double2* r;          // W (A y - V), or W A x in the power iteration [vis.n_pad]
    double* blk_r2;      // [vis.n_blk] per-block sum W|A I - V|^2
    double* blk_l1;      // [pix.n_blk] per-block sum I
    double* blk_z2;      // [pix.n_blk] per-block sum z^2 (power)
    int* blk_nnz;        // [pix.n_blk]
    int* blk_badv;       // [vis.n_blk] non-finite flags
    int* blk_badp;       // [pix.n_blk] non-finite flags
};

struct DevProblem {
    Side vis;
    Side pix;
    const int2* ant;          // [vis.n_pad] antenna pair (a, b)
    const int* vslot;         // gains: [vis.n_pad] slot of the visibility's pair in its granule's list
    const int2* gbl;          // gains: [vis.n_gran][NB_MAX] the granule's distinct pairs, sorted
    const int* gnb;           // gains: [vis.n_gran] number of pairs, 0 if more than NB_MAX
    const double2* V;         // [vis.n_pad] measured visibilities (sorted)
    const float4* pgauss;     // [pix.n_pad] {l, m, (l^2+m^2)/2, nu = n-1+(l^2+m^2)/2}
    const d4* pgauss64;       // same in FP64
    const float* gsig;        // [pix.n_gran] sigma per pixel granule (FP32 path)
    const double* gsig64;     // [pix.n_gran] sigma per pixel granule (FP64 path)
    const int* gkind;         // [pix.n_gran] kind per pixel granule
    const float4* pghdr;      // [pix.n_gran][4] centre hi, centre lo, extent, {sigma, kind, 0, 0}
    const float4* vgabs;      // [vis.n_pad] {u, v, -2 w, u^2 + v^2} in FP32 (the adjoint's Gaussian terms)
    float2* r32;              // [vis.n_pad] the mixed adjoint's input residual in polar form,
                              // {|r|, arg r in turns} in FP32 (r32_kernel)
    const float2* gpol32;     // [pix.n_gran][gain_rows(n_ant)][GP] {|G|, arg G in turns} or null
    const double2* gains64;   // [pix.n_pad][n_ant] or null
    int n_ant;
    // operator mode (st == null): one forward x -> fwd_out or adjoint r -> adj_out
    const double* x;          // [pix.n_pad]
    const double2* r;         // [vis.n_pad]
    double2* fwd_out;         // [vis.n_pad]
    double* adj_out;          // [pix.n_pad]
    // solver mode
    SolveState* st;
    SolveBufs b;
};

// Forward input of problem P in this launch (false: P takes no part).
__device__ __forceinline__ bool fwd_role(const DevProblem& P, const double*& X)
{
    if (!P.st) { X = P.x; return true; }
    const int ph = P.st->phase;
    if (ph == PH_PINIT || ph == PH_POWER) { X = P.b.xv; return true; }
    if (ph == PH_SINIT) { X = P.b.I[0]; return true; }
    if (ph == PH_SOLVE) { X = P.b.I[P.st->algo ? 1 : (P.st->k + 1) & 1]; return true; }
    return false;
}

// Adjoint input of problem P in this launch (false: P takes no part).
__device__ __forceinline__ bool adj_role(const DevProblem& P, const double2*& R)
{
    if (!P.st) { R = P.r; return true; }
    const int ph = P.st->phase;
    if (ph == PH_POWER || ph == PH_SOLVE) { R = P.b.r; return true; }
    return false;
}

// Stream-K plan of one launch over a batch of problems (device resident).
struct Plan {
    int n_probs;
    int C;                        // CTAs of the persistent grid
    long long U;                  // total units
    const long long* prob_u0;     // [n_probs+1] first unit of each problem
    const int* prob_b0;           // [n_probs+1] first global block of each problem
    const int* blk_poff;          // [n_blocks] first partial slot of the block
    const int* blk_clo;           // [n_blocks] first CTA contributing to it
    const int* blk_ncon;          // [n_blocks] contributing CTAs
    const long long* cta_u0;      // [C+1] first unit of each CTA (cost-weighted split),
                                  // or null: CTA c takes [c U / C, (c+1) U / C)
    int n_blocks;
    int n_slots;
};

// Unit range [u, u_end) of CTA c.
__host__ __device__ inline void cta_range(const Plan& pl, long long c, long long& u, long long& u_end)
{
    if (pl.cta_u0) {
        u = pl.cta_u0[c];
        u_end = pl.cta_u0[c + 1];
    } else {
        u = (pl.U * c) / pl.C;
        u_end = (pl.U * (c + 1)) / pl.C;
    }
}

}  // namespace sl1m
