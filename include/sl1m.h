/*
 * sl1m.h -- C ABI of libsl1m, the GB300 (sm_103a) hot path of SL1M:
 * positivity-constrained L1 deconvolution of ungridded radio visibilities
 * (S. J. Hardy 2013, "Direct deconvolution of radio synthesis images using
 * L1 minimisation", A&A; arxiv 1310.2078).
 *
 * Conventions (all entry points):
 *   - Index convention: pixel j (n_pix of them), visibility k (n_vis).  The
 *     operator A is n_vis x n_pix, A_kj = the paper's M_jk (Eq. sme).
 *   - Units: u, v, w in wavelengths (Sect. 2: b = lambda (u e_u + v e_v +
 *     w e_w)); l, m direction cosines with l^2 + m^2 < 1; sigma in direction
 *     cosines; fluxes in Jy.  Complex arrays are interleaved (re, im) doubles.
 *   - Ownership: the caller owns every array it passes.  Host-pointer calls
 *     copy inputs in and results out before returning.  The *_dev calls take
 *     device pointers (CUDA global memory on the context's device), borrow
 *     them for the duration of the call and are asynchronous on the
 *     context's stream unless stated otherwise.
 *   - Every call returns an SL1M_* status.  On failure nothing that the call
 *     was to produce is valid; sl1m_last_error() gives a one-line reason.
 *   - Thread safety: a context and its problems must be used from one host
 *     thread at a time.  A running solve server (sl1m_server_start) works on
 *     a host thread of its own; the caller's sl1m_server_* calls and
 *     sl1m_last_error may run meanwhile.
 *   - Precision: SL1M_FP64 evaluates every step in FP64 ("plain" path);
 *     SL1M_MIXED evaluates sincos/exp and the multiply-accumulates in FP32
 *     after an exact FP32 reduction of the phase to fractional turns (the
 *     adjoint, whose output is real, takes r and the gains in polar form and
 *     one cosine per pair); sums over tiles, norms, step sizes and the
 *     projection stay in FP64.
 */
#ifndef SL1M_H
#define SL1M_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SL1M_OK 0
#define SL1M_ERR_ARG 1        /* null pointer, bad size, l^2+m^2 >= 1, sigma < 0,
                                 non-finite input, antenna index out of range */
#define SL1M_ERR_OOM 2        /* device or host allocation failed              */
#define SL1M_ERR_CUDA 3       /* a CUDA runtime call failed, or a kernel's
                                 bounded wait for a bulk copy into shared
                                 memory gave up (a device flag, read by every
                                 synchronous call; the *_dev calls leave it to
                                 the next synchronous call on the context)   */
#define SL1M_ERR_NONFINITE 4  /* a non-finite value appeared during a solve    */
#define SL1M_ERR_TIMEOUT 5    /* a bounded wait expired                        */
#define SL1M_ERR_BUSY 6       /* admission refused (memory budget)             */
#define SL1M_ERR_STATE 7      /* problem incomplete (no pixels/visibilities),
                                 or gains set without antenna pairs            */

#define SL1M_FP64 0
#define SL1M_MIXED 1

/* Pixel kinds.  Dirac: Eq. deltam.  Paraxial Gaussian: Eq. samlm4.
 * Wide-field Gaussian: Eq. samlm5.  (For the Gaussian kinds the factor
 * 1/sigma^2 printed in front of Eq. samlm4/5 is not applied: the pixel of
 * Eq. gaus has unit integral, so x_j is the pixel's total flux; and the
 * wide-field residual phase is w (n - 1 + (l^2+m^2)/2), the form whose
 * Taylor expansion is Eq. taylorexp.) */
#define SL1M_DIRAC 0
#define SL1M_GAUSS_PARAXIAL 1
#define SL1M_GAUSS_WIDE 2

/* Solvers (sl1m_solve_opts.algorithm). */
#define SL1M_FISTA 0          /* the algorithm box of Sect. 3                  */
#define SL1M_MFISTA 1         /* its monotone variant, Beck & Teboulle (2009b) */

typedef struct sl1m_ctx sl1m_ctx;
typedef struct sl1m_problem sl1m_problem;

/* Library version (major*10000 + minor*100 + patch). */
int sl1m_version(void);

/* Static description of a status code. */
const char* sl1m_status_string(int status);

/* Create a context on CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t to run on, or NULL for a stream the context creates and owns.
 * The context owns every device allocation made through it. */
int sl1m_create(sl1m_ctx** out, int device, void* cuda_stream);

/* Destroy a context and every problem created in it. */
int sl1m_destroy(sl1m_ctx* ctx);

/* Last error message of the context ("" if none).  The text is a copy held
 * per calling thread, valid until that thread calls this function again. */
const char* sl1m_last_error(const sl1m_ctx* ctx);

/* Create / destroy an (empty) deconvolution problem. */
int sl1m_problem_create(sl1m_ctx* ctx, sl1m_problem** out);
int sl1m_problem_destroy(sl1m_problem* prob);

/* Visibilities, Sect. 2 (Eq. samuvw): uvw [n_vis][3] in wavelengths,
 * vis [n_vis][2] the measured V_k (may be NULL: zeros), weights [n_vis] W_k
 * >= 0 or NULL (= 1; W multiplies the squared residual, W = 1 is the paper's
 * case), ant_pair [n_vis][2] antenna indices (a_k, b_k) or NULL (required
 * only with gains).  Replaces any earlier visibilities.  Copies the data. */
int sl1m_set_visibilities(sl1m_problem* prob, int64_t n_vis, const double* uvw,
                          const double* vis, const double* weights, const int32_t* ant_pair);

/* Replace only the measured visibilities V (same uvw, same order). */
int sl1m_set_vis_data(sl1m_problem* prob, const double* vis);

/* Pixels, Sect. 2.1 (pixel list (l_k, m_k), arbitrary positions):
 * lm [n_pix][2], sigma [n_pix] (NULL = 0) and kind [n_pix] (NULL = all
 * Dirac).  Gaussian kinds need sigma > 0.  Copies the data. */
int sl1m_set_pixels(sl1m_problem* prob, int64_t n_pix, const double* lm,
                    const double* sigma, const int32_t* kind);

/* Direction-dependent gains (Sect. 2: A(l,m; Z_j, chi_j); the method allows
 * a different gain for every pixel and every antenna): G [n_pix][n_ant][2],
 * per pixel and antenna; the entry for visibility k is multiplied by
 * g_jk = G[j][a_k] * conj(G[j][b_k]).  G == NULL or n_ant == 0 removes the
 * gains.  The mixed-precision kernels hold one pixel granule's gains for all
 * antennas in shared memory: n_ant <= 300 (SL1M_ERR_ARG above). */
int sl1m_set_gains(sl1m_problem* prob, int32_t n_ant, const double* G);

/* Forward operator, Eq. sme: vis_out_k = sum_j A_kj x_j.
 * x [n_pix] (host), vis_out [n_vis][2] (host).  Synchronous.
 * This and every later operator or solve call lay the problem out first and
 * return SL1M_ERR_ARG when max|u|*max|l|, max|v|*max|m| or max|w|*max|n-1|
 * reaches 2^21 turns (about 2e6 wavelengths at |l| = 1): the mixed kernels
 * split the phase exactly only below that. */
int sl1m_forward(sl1m_problem* prob, const double* x, double* vis_out, int precision);

/* Adjoint (back-projection of Sect. 3): img_out_j = sum_k Re(conj(A_kj) r_k).
 * r [n_vis][2] (host), img_out [n_pix] (host).  Synchronous. */
int sl1m_adjoint(sl1m_problem* prob, const double* r, double* img_out, int precision);

/* Device-pointer variants of the two calls above, asynchronous on the
 * context's stream (the caller synchronises before reading the output). */
int sl1m_forward_dev(sl1m_problem* prob, const double* x_dev, double* vis_out_dev, int precision);
int sl1m_adjoint_dev(sl1m_problem* prob, const double* r_dev, double* img_out_dev, int precision);

/* Forward operator for callers that cannot allocate device memory at the time
 * of the call (device memory owned by a pool or another framework, or a loop
 * that must not enter the allocator).  Same result as sl1m_forward_dev; the
 * paper has no counterpart (this is plumbing, not a step of the method).
 *   - Allocates nothing: all of its scratch (descriptor, work-split tables,
 *     input in the library's pixel order, partial sums, output before
 *     reordering) lives in one static device array of 32 MiB that every GPU
 *     loading libsl1m holds until the process exits.  Problems needing more
 *     return SL1M_ERR_ARG with the size they need.
 *   - The problem must already be laid out on the device by an earlier,
 *     allocating call of this library (e.g. sl1m_forward); otherwise
 *     SL1M_ERR_STATE.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before any
 *     stream capture.
 *   - All calls share the one array and each leaves its data there: calls
 *     whose work overlaps on the GPU (other streams, other contexts, other
 *     host threads) race and must be serialised by the caller.
 *   - x_dev [n_pix] and vis_out_dev [n_vis][2] are device pointers in the
 *     caller's order; asynchronous on the context's stream: the call enqueues
 *     its kernels (its per-call tables travel in kernel parameters, not in
 *     copies from host memory) and returns without waiting for the stream.
 *   - With gains in mixed precision, a kernel whose bounded wait for a bulk
 *     copy gives up sets the context's device fault flag; this call does not
 *     read it (that would wait for the stream).  The next synchronous call on
 *     the context reads it and returns SL1M_ERR_CUDA. */
int sl1m_forward_noalloc(sl1m_problem* prob, const double* x_dev, double* vis_out_dev, int precision);

/* Dirty image: the back-projection of the measured data, Re(A^H W V)
 * (Sect. 3: the gradient at I = 0; Sect. 4.4 proposes it as a starting
 * point).  img_out [n_pix] (host, may be NULL); lambda_max_out (may be NULL)
 * receives max_j of it, the smallest lambda for which the solution of the
 * algorithm box is exactly zero.  Synchronous. */
int sl1m_dirty_image(sl1m_problem* prob, int precision, double* img_out, double* lambda_max_out);

/* Step constant of FISTA (Sect. 3, algorithm box: L = largest eigenvalue of
 * M*M; Sect. 3.1 computes it with a routine whose method it does not give).
 * Power iteration on B = Re(A^H W A) from x = 1/sqrt(n_pix):
 * z = B x, mu = ||z||, x = z/mu, stopping when |mu_i - mu_{i-1}| <= tol*mu_i
 * or after max_iter steps; L = the last mu.  Synchronous. */
int sl1m_max_eig(sl1m_problem* prob, int max_iter, double tol, int precision,
                 double* L_out, int* iters_out);

/* Solver options.  lambda: regulariser of Eq. cme.  L: step constant, or 0 to
 * compute it with sl1m_max_eig(power_max_iter, power_tol).  rel_tol: stop
 * when |E_k - E_{k-1}| <= rel_tol * E_{k-1} (Sect. 3; 0 = run max_iter
 * steps), where E = 1/2 sum W |A I - V|^2 + lambda sum I is the objective the
 * algorithm box minimises.  x0: starting image [n_pix] (host) or NULL (zero,
 * the box's Step 0).  algorithm: SL1M_FISTA (default, zero) or SL1M_MFISTA;
 * for MFISTA, rel_tol applies to the objective change a step proposes,
 * |E(z_k) - E(x_{k-1})| <= rel_tol * E(x_{k-1}). */
typedef struct {
    double lambda;
    double L;
    double rel_tol;
    int32_t max_iter;
    int32_t precision;
    int32_t power_max_iter;   /* 0 = 50   */
    double power_tol;         /* 0 = 1e-6 */
    const double* x0;
    int32_t algorithm;        /* SL1M_FISTA (0) or SL1M_MFISTA */
} sl1m_solve_opts;

typedef struct {
    int32_t iters;        /* FISTA steps taken                                   */
    int32_t converged;    /* 1 when rel_tol was met                              */
    double E;             /* 1/2 sum W|A I - V|^2 + lambda sum I                 */
    double E_paper;       /* sum W|A I - V|^2 + lambda sum I   (Eq. cme)          */
    double resid2;        /* sum W |A I - V|^2                                   */
    double l1;            /* sum I                                               */
    int64_t nnz;          /* number of I_j > 0                                   */
    double L;             /* step constant used                                  */
    int32_t power_iters;  /* power-iteration steps (0 if L was given)            */
    double seconds;       /* wall time of the call                               */
} sl1m_solve_stats;

/* FISTA with the positive soft threshold (Sect. 3 algorithm box, Eq. threshp):
 *   I_k = T^{lambda/L}(y_k - Re A^H W (A y_k - V)/L),
 *   t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2,
 *   y_{k+1} = I_k + ((t_k - 1)/t_{k+1}) (I_k - I_{k-1}).
 * img_out [n_pix] (host) receives the last I_k; stats may be NULL.
 * With algorithm = SL1M_MFISTA, the monotone variant that Sect. 3 names
 * (Beck & Teboulle 2009b):
 *   z_k = T^{lambda/L}(y_k - Re A^H W (A y_k - V)/L),
 *   x_k = z_k if E(z_k) <= E(x_{k-1}), else x_{k-1},
 *   y_{k+1} = x_k + (t_k/t_{k+1})(z_k - x_k) + ((t_k - 1)/t_{k+1})(x_k - x_{k-1});
 * E(z_k) comes from the forward product the stopping test already needs and
 * A y_{k+1} follows by linearity, so a step costs one forward and one
 * adjoint, as a FISTA step does.  img_out receives x_k, and E never rises.
 * Synchronous.  SL1M_ERR_NONFINITE if a non-finite value appeared. */
int sl1m_solve(sl1m_problem* prob, const sl1m_solve_opts* opts, double* img_out,
               sl1m_solve_stats* stats);

/* ---- Continuous-batching solve server ---------------------------------------
 * Independent solves (the paper solves every channel and polarisation on
 * its own, Sect. 2 and 4.2) share the same forward and adjoint launches:
 * a request loop on a host thread admits queued solves as batch slots and the
 * device-memory budget allow, runs every admitted solve one FISTA step (or one
 * power-iteration step) per tick inside one captured CUDA graph, and retires
 * finished solves between rounds.  A request that arrives while others run
 * joins the next round.  While a server runs on a context, the operator and
 * solve calls of that context return SL1M_ERR_BUSY. */
#define SL1M_ADMIT_TWO_LANES 0   /* default: small and large requests in lanes  */
#define SL1M_ADMIT_ARRIVAL 1     /* one queue, strictly in arrival order         */
typedef struct {
    int64_t mem_budget_bytes;   /* 0 = 80% of the device memory free at start   */
    int32_t max_slots;          /* 0 = 64 concurrent solves                      */
    int32_t ticks_per_round;    /* 0 = 4 steps between admission/retirement     */
    int32_t precision;          /* SL1M_MIXED or SL1M_FP64 for every request     */
    int32_t admission;          /* SL1M_ADMIT_TWO_LANES or SL1M_ADMIT_ARRIVAL    */
    double max_pairs_per_tick;  /* work in flight: admit while the summed
                                   n_vis*n_pix of running solves stays below
                                   this; 0 = 4e9 (enough to fill the GPU).
                                   SL1M_ADMIT_ARRIVAL: in arrival order, one
                                   request always admitted when none runs.
                                   SL1M_ADMIT_TWO_LANES: requests of at most
                                   scale/16 pairs ("small") and the rest
                                   ("large") queue in arrival order in lanes of
                                   their own; large ones against this budget
                                   (one always admitted when no large one
                                   runs), small ones against scale/4 on top,
                                   where scale is this budget or the pairs of
                                   the largest running request if that is
                                   more; a small request never waits behind a
                                   large one that does not fit               */
} sl1m_server_opts;

/* Start the request loop (opts may be NULL for defaults). */
int sl1m_server_start(sl1m_ctx* ctx, const sl1m_server_opts* opts);

/* Queue a solve of `prob` with `opts` (opts->precision is ignored; the server's
 * applies; opts->x0 is copied).  The problem must not be changed or destroyed
 * until its result has been collected with sl1m_server_wait.  SL1M_ERR_BUSY if
 * the problem alone exceeds the memory budget. */
int sl1m_server_submit(sl1m_ctx* ctx, sl1m_problem* prob, const sl1m_solve_opts* opts, uint64_t* ticket);

/* done = 1 once the request has finished (successfully or not). */
int sl1m_server_poll(sl1m_ctx* ctx, uint64_t ticket, int* done);

/* Wait at most timeout_s seconds (< 0: no limit) for the request, then copy
 * its image (img_out [n_pix], may be NULL) and stats (stats->seconds = time
 * from submit to completion) and release the ticket.  SL1M_ERR_TIMEOUT if it
 * has not finished in time (the ticket stays valid). */
int sl1m_server_wait(sl1m_ctx* ctx, uint64_t ticket, double timeout_s, double* img_out,
                     sl1m_solve_stats* stats);

/* Finish every queued and running request, then stop the request loop.
 * Results not yet collected remain collectable with sl1m_server_wait until
 * the context is destroyed or a new server is started. */
int sl1m_server_stop(sl1m_ctx* ctx);

/* Counters of the running (or last) server. */
typedef struct {
    int64_t queued, active, finished, max_active;
    int64_t bytes_in_use, bytes_budget;
    int64_t ticks, rounds;
} sl1m_server_info_t;
int sl1m_server_info(sl1m_ctx* ctx, sl1m_server_info_t* info);

/* Autotuner of the operator kernels' tile shape: for the forward and the
 * adjoint of this problem it times, with CUDA events, every (streamed
 * granules per shared-memory stage: 2, 4 or 8; the adjoint 2 or 4) x
 * (persistent grid: 1 .. occupancy CTAs per SM) of the mixed no-gains
 * kernels, then for every stage count at its fastest grid the share npoly
 * (1 or 2 of every 8 pairs) whose sincos (adjoint: cosine) runs on the FMA
 * pipe instead of the SFU (each timed launch follows a launch of the other operator, as in a
 * solve); with gains or in FP64 only the grid is tuned.  The choice is kept in the context,
 * keyed by (precision, operator, gains, Gaussian pixels, log2 of the work
 * units); later launches of problems with the same key -- single solves and
 * server batches -- use it.  nst_out, ctas_per_sm_out and npoly_out ([2]:
 * forward, adjoint) may be NULL.  Synchronous. */
int sl1m_autotune(sl1m_problem* prob, int precision, int32_t* nst_out, int32_t* ctas_per_sm_out,
                  int32_t* npoly_out);

/* Set the tile shape the autotuner would choose, for this problem's key
 * (op 0 forward, 1 adjoint): nst 2, 4 or 8 (the adjoint 2 or 4),
 * ctas_per_sm from 1 to the kernel's occupancy, npoly 0, 1 or 2.  With gains
 * or in FP64 only ctas_per_sm may differ from the defaults (nst 4, npoly 0).
 * SL1M_ERR_ARG for a shape that does not exist or does not fit. */
int sl1m_set_tile_shape(sl1m_problem* prob, int precision, int op, int nst, int ctas_per_sm, int npoly);

/* ---- Adaptive quadtree refinement (Sect. 4.4) ---------------------------
 * The pixels set on the problem (Dirac, a regular grid of spacing delta0, no
 * gains) are solved first; then, level by level, every pixel above
 * refine_frac * (peak of the last image) is replaced by its four quadrant
 * children at half its spacing (offsets +-spacing/4), unrefined pixels are
 * kept when keep_unrefined, and the problem is solved again with `opts`
 * (L recomputed per level when opts->L == 0), starting from each parent's
 * flux shared equally among its children.  The paper splits every pixel
 * above 1% of the maximum, from 64" to 2" (5 levels).  On return the problem
 * holds the final pixel set; sl1m_get_solution gives it and the image. */
typedef struct {
    int32_t levels;          /* refinements after the first solve (0..16)      */
    double refine_frac;      /* split pixels above this fraction of the peak   */
    int32_t keep_unrefined;  /* 1: keep the pixels that are not split          */
} sl1m_refine_opts;

typedef struct {
    int32_t levels_done;         /* solves run                                   */
    int64_t n_pix[17];           /* pixels per solve                             */
    int32_t iters[17];           /* FISTA steps per solve                        */
    int32_t power_iters[17];     /* power-iteration steps per solve              */
    int64_t final_n_pix;
    double total_pair_evals;     /* pixel-visibility pairs evaluated, all solves */
    sl1m_solve_stats last;       /* stats of the last solve                      */
} sl1m_refine_stats;

int sl1m_solve_refine(sl1m_problem* prob, const sl1m_solve_opts* opts, const sl1m_refine_opts* ropts,
                      double delta0, sl1m_refine_stats* stats);

/* The problem's current pixels (lm_out [n_pix][2]) and the image of its last
 * refinement (img_out [n_pix]); any pointer may be NULL (n_pix alone sizes
 * the buffers). */
int sl1m_get_solution(const sl1m_problem* prob, int64_t* n_pix, double* lm_out, double* img_out);

/* Kernel timing with CUDA events on the context's stream (for benchmarks).
 * Kernel ids: 0 forward FP64, 1 adjoint FP64, 2 forward mixed, 3 adjoint
 * mixed, 4 forward finish, 5 adjoint finish (solver vector updates), 6 other.
 * sl1m_profile_read synchronises the stream and returns, for one kernel id,
 * the summed event time (ms), the number of launches, the pixel-visibility
 * pairs those launches evaluated and the bytes the finish kernels moved. */
int sl1m_profile_enable(sl1m_ctx* ctx, int on);
int sl1m_profile_reset(sl1m_ctx* ctx);
int sl1m_profile_read(sl1m_ctx* ctx, int kernel_id, double* ms, int64_t* launches,
                      double* pairs, double* bytes);

/* Counters since context creation or the last sl1m_counters_reset: kernel
 * launches the library issued, bytes it copied host->device (inputs and their
 * device layout, starting images) and device->host (results). */
int sl1m_counters(sl1m_ctx* ctx, int64_t* launches, int64_t* h2d_bytes, int64_t* d2h_bytes);
int sl1m_counters_reset(sl1m_ctx* ctx);

/* Host-only inspection of the work split (no GPU needed).  Work on a batch
 * of problems is cut into units (owned block of 512 elements x streamed
 * granule of 64), owned_blocks[p] * streamed_granules[p] per problem, and
 * spread over n_ctas = min(max_ctas, units) persistent CTAs.  Without
 * unit_costs, CTA c takes units [c U / C, (c+1) U / C); with unit_costs
 * [total units] (relative cost of each unit, problems in order, block-major)
 * the boundaries cut the summed cost into n_ctas equal parts, as the library
 * does for tiles of unequal cost.  Returns, per block (problems in order), the
 * first contributing CTA, their count and the first partial-sum slot, and the
 * first unit of every CTA in cta_first_unit [n_ctas+1] (may be NULL). */
int sl1m_plan_preview(int32_t n_probs, const int32_t* owned_blocks, const int32_t* streamed_granules,
                      int32_t max_ctas, const float* unit_costs, int32_t* n_ctas, int64_t* n_units,
                      int32_t* n_slots, int32_t* blk_first_cta, int32_t* blk_n_ctas, int32_t* blk_first_slot,
                      int64_t* cta_first_unit);

/* Host-only: the granule order the library uses for n points xy [n][2]:
 * order [n_pad] receives point indices, -1 for padding, so that each run of
 * 64 is a compact box (k-d median split along the wider axis at multiples of
 * 64).  n_pad = ceil(n / 64) * 64.  order may be NULL to query n_pad. */
int sl1m_granule_order(int64_t n, const double* xy, int32_t* order, int64_t* n_pad);

/* Host-only: the FP32 layout of one side that the mixed kernels read for the
 * exact phase split of Sect. 3.1's phase (X.Y = X.Yc + Xc.(Y - Yc) +
 * (X - Xc).(Y - Yc), each product from FP32 halves).  xyzw [n][4]: element
 * coordinates (x, y, z) and an auxiliary value (pixels: l, m, n - 1, 1/n;
 * visibilities: u, v, w, weight); order [n_pad]: a padded permutation of
 * 0..n-1 (-1 = padding, n_pad a multiple of 64), e.g. sl1m_granule_order's.
 * Outputs, each [n_pad][4] or [n_pad / 64][4] floats and each may be NULL:
 *   hi, lo     the element's (x, y, z) as hi = fl32(x), lo = fl32(x - hi); w 0
 *   off, offlo the same split of the offset from the granule centre; off.w =
 *              the auxiliary value (0 for padding)
 *   cen_hi, cen_lo, ext  per granule: the centre (the middle of the members'
 *              bounding box) split the same way, and the extent, an upper
 *              bound of |offset| per axis (half the box, rounded up).
 * A padding slot copies the coordinates of a member of its granule.
 * SL1M_ERR_ARG: null inputs, n_pad not a multiple of 64 or below n, an index
 * out of range or repeated.  The paper has no counterpart; it exposes, for
 * tests, what the library lays out in HBM. */
int sl1m_granule_layout(int64_t n, const double* xyzw, const int32_t* order, int64_t n_pad, float* hi,
                        float* lo, float* off, float* offlo, float* cen_hi, float* cen_lo, float* ext);

/* Device bytes the problem holds (inputs, layout and solver workspace). */
int sl1m_problem_bytes(const sl1m_problem* prob, int64_t* bytes);

/* Measured issue rate of the special-function unit (MUFU), which bounds the
 * mixed-precision operator kernels: per pixel-visibility pair they take sin
 * and cos of the phase of Eq. deltam, and exp2 of the Gaussian amplitude of
 * Eq. samlm5.  A kernel of 8 independent dependency chains per thread, over
 * 4 CTAs of 256 threads per SM, times sin.approx/cos.approx (alternating)
 * and ex2.approx with CUDA events on the context's stream (best of 3 after a
 * warm-up).  sincos_per_s_out: sin or cos results per second over the whole
 * device; ex2_per_s_out: exp2 results per second.  Synchronous. */
int sl1m_measure_sfu(sl1m_ctx* ctx, double* sincos_per_s_out, double* ex2_per_s_out);

/* Self-test of the kernels' bounded waits.  The mixed kernels wait on
 * mbarriers for their bulk copies into shared memory; each wait gives up
 * after a fixed time on the GPU's global timer (limit_ns_out), records a
 * device flag and lets its kernel run to its end, so no CTA barrier is left
 * waiting and the context stays usable; the next synchronous call reads the
 * flag and fails with SL1M_ERR_CUDA.  This call runs a kernel whose threads
 * wait on an mbarrier nobody arrives on (no copy is in flight), so the wait
 * must give up: it returns SL1M_ERR_CUDA, and waited_ns_out (may be NULL)
 * receives how long the wait lasted.  Any other status means the bounded wait
 * is broken.  Synchronous. */
int sl1m_selftest_bounded_wait(sl1m_ctx* ctx, int64_t* waited_ns_out, int64_t* limit_ns_out);

/* Share of the operator's tiles (visibility granule of 64 x pixel granule of
 * 64) that the mixed-precision kernels evaluate on the exact phase path: the
 * phase u l + v m + w (n-1) of Eq. deltam is split into granule-centre and
 * offset terms, and a tile whose granule extents could make the product of
 * the two offsets exceed 6 turns reduces that term exactly too (wide fields,
 * long baselines).  share_out in [0, 1]; n_tiles_out (may be NULL) the number
 * of tiles.  The problem must have been laid out by an operator or solve call
 * (SL1M_ERR_STATE otherwise).  Host-only, synchronous. */
int sl1m_exact_tile_share(const sl1m_problem* prob, double* share_out, int64_t* n_tiles_out);

#ifdef __cplusplus
}
#endif
#endif /* SL1M_H */
