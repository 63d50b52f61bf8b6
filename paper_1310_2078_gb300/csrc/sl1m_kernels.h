// sl1m_kernels.h -- launch wrappers of the libsl1m kernels (internal).
#pragma once
#include "sl1m_dev.h"

namespace sl1m {

enum FinishMode : int { FIN_OP = 0, FIN_POWER = 1, FIN_SOLVE = 2, FIN_INIT = 3 };

// operator kernels (sl1m_mixed.cu, sl1m_fp64.cu); precision 0 = FP64, 1 = mixed.
// plp: device-resident plan; C: its grid size (known on the host).
// nst: streamed granules per shared-memory stage of the mixed no-gains
// kernels (2, 4 or 8; the tile shape the autotuner picks).
constexpr int NST_DEFAULT = 4;
// Tile-shape code carried as `nst` below: streamed granules per stage (2, 4
// or 8) plus 16 x npoly, the pairs of every 8 whose sincos runs on the FMA
// pipe (0, 1 or 2; Dirac tiles without gains).
// Bit 8: the batch has no Gaussian pixels, so the no-gains mixed kernels may
// run an instance compiled without the Gaussian tiles.
constexpr int SHAPE_DIRAC_ONLY = 1 << 8;
constexpr int shape_code(int nst, int npoly) { return nst | (npoly << 4); }
constexpr int shape_nst(int code) { return code & 15; }
constexpr int shape_npoly(int code) { return (code >> 4) & 15; }
constexpr bool shape_dirac_only(int code) { return (code & SHAPE_DIRAC_ONLY) != 0; }
// The shape code of a launch over pixels that may (gauss) or may not hold
// Gaussian pixels.
constexpr int shape_for(int code, bool gauss) { return gauss ? (code & ~SHAPE_DIRAC_ONLY) : (code | SHAPE_DIRAC_ONLY); }
cudaError_t launch_forward(int precision, bool gains, int n_ant, const DevProblem* probs,
                           const Plan* plp, int C, double2* partial, cudaStream_t st, int nst = NST_DEFAULT);
cudaError_t launch_adjoint(int precision, bool gains, int n_ant, const DevProblem* probs, const Plan* plp, int C,
                           double* partial, cudaStream_t st, int nst = NST_DEFAULT);
// which: 0 fwd fp64, 1 adj fp64, 2 fwd mixed, 3 adj mixed
int occupancy(int which, bool gains, int n_ant, int nst = NST_DEFAULT);
int fwd_smem_bytes(int n_ant, bool gains, int nst);
// Before a mixed adjoint: each problem's input residual in polar form, {|r|,
// arg r in turns} in FP32 (r32).
cudaError_t launch_r32(const DevProblem* probs, int n_probs, int max_vis_pad, cudaStream_t st);
// The mixed gains kernels' bounded waits for their bulk copies set a device
// flag when they give up; read it into *host_flag (asynchronously on st: valid
// after the stream is synchronised) and clear it.
cudaError_t wait_fault_read(unsigned* host_flag, cudaStream_t st);
cudaError_t wait_fault_clear(cudaStream_t st);
// Self-test: n_blocks CTAs each wait on an mbarrier nobody arrives on; the
// waits give up after wait_limit_ns() and set the flag above; waited_ns
// [n_blocks] (device) receives how long each CTA's thread 0 waited.
cudaError_t launch_wait_selftest(unsigned long long* waited_ns, int n_blocks, cudaStream_t st);
unsigned long long wait_limit_ns();

// solver kernels (sl1m_solver.cu)
cudaError_t launch_gather_real(const double* src, double* dst, const int* orig, int n_pad,
                               double scale, cudaStream_t st);
cudaError_t launch_gather_cplx(const double2* src, double2* dst, const int* orig, int n_pad,
                               cudaStream_t st);
cudaError_t launch_scatter_real(const double* src, double* dst, const int* orig, int n_pad,
                                cudaStream_t st);
cudaError_t launch_scatter_cplx(const double2* src, double2* dst, const int* orig, int n_pad,
                                cudaStream_t st);
cudaError_t launch_fill_valid(double* dst, const int* orig, int n_pad, double val, cudaStream_t st);
cudaError_t launch_weighted_vis(const double2* V, const d4* vd, double2* r, int n_pad, cudaStream_t st);
cudaError_t launch_fwd_finish(const DevProblem* probs, const Plan* plp, int grid, const double2* partial,
                              cudaStream_t st);
cudaError_t launch_adj_finish(const DevProblem* probs, const Plan* plp, int grid, const double* partial,
                              cudaStream_t st);
cudaError_t launch_mfista_mix(const DevProblem* probs, const Plan* fplp, const Plan* aplp, int grid,
                              cudaStream_t st);
// evals (may be null): [0] += pairs the forward and [1] += pairs the adjoint
// evaluated in this tick, summed over the problems that took part.
cudaError_t launch_scalars(const DevProblem* probs, const int* n_probs, int grid, double* evals, cudaStream_t st);
cudaError_t launch_phases(const DevProblem* probs, const int* n_probs, int grid, int* out, cudaStream_t st);

}  // namespace sl1m
