// sl1m_host.h -- host-side structures of libsl1m (internal).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "sl1m.h"
#include "sl1m_dev.h"

// Device buffer owned by the library (cudaMalloc / cudaFree).
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    ~DBuf() { free(); }
    void free()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    cudaError_t alloc(size_t count)
    {
        free();
        if (count == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc((void**)&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        n = count;
        return cudaSuccess;
    }
    // Grow to at least `count` elements (contents are not preserved).
    cudaError_t reserve(size_t count, cudaStream_t st)
    {
        if (count <= n && p) return cudaSuccess;
        cudaStreamSynchronize(st);
        return alloc(count);
    }
    // Allocate exactly `count` and copy from host (zero-fill when `zero`);
    // returns after the copy (the host source may be a temporary).
    cudaError_t upload(const T* src, size_t count, cudaStream_t st, bool zero = false)
    {
        cudaError_t e = alloc(count);
        if (e != cudaSuccess || count == 0) return e;
        if (zero) e = cudaMemsetAsync(p, 0, count * sizeof(T), st);
        else e = cudaMemcpyAsync(p, src, count * sizeof(T), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        return cudaStreamSynchronize(st);
    }
    size_t bytes() const { return n * sizeof(T); }
};

struct HostPlan {
    std::vector<long long> u0;
    std::vector<int> b0, poff, clo, ncon;
    std::vector<long long> cta_u0;   // empty: uniform split
    long long U = 0;
    int C = 1, n_blocks = 0, n_slots = 0;
};

// Relative cost of the units of one problem in a plan: a constant per unit,
// or one value per unit (block-major, streamed granule minor).
struct UnitCost {
    double uniform = 1.0;
    std::vector<float> unit;
};

// costs == null: every unit costs the same; otherwise the CTA boundaries cut
// the summed cost into C equal parts.
void plan_host(const std::vector<int>& nb, const std::vector<int>& ns, int Cmax, HostPlan& H,
               const std::vector<const UnitCost*>* costs = nullptr);

// A plan whose tables and header live on the device (kernels take Plan*).
struct DevPlan {
    sl1m::Plan pl{};          // host copy of the header
    DBuf<long long> u0;
    DBuf<int> b0, poff, clo, ncon;
    DBuf<long long> cta;
    DBuf<sl1m::Plan> dpl;     // device header
};
cudaError_t build_plan(const std::vector<int>& nb, const std::vector<int>& ns, int Cmax, DevPlan& D,
                       cudaStream_t st, const std::vector<const UnitCost*>* costs = nullptr);

constexpr int NPROF = 7;

struct ProfRec {
    int kid;
    cudaEvent_t ev0, ev1;
    double pairs, bytes;
};

struct ProfTok {
    bool active = false;
    int kid = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

struct sl1m_problem;
struct Server;

// Device tables of a set of problems run together (one precision).
struct Batch {
    int precision = 1;
    bool solver = false;
    std::vector<sl1m_problem*> probs;
    std::vector<sl1m::DevProblem> hdesc;
    DBuf<sl1m::DevProblem> desc;
    DBuf<int> n_probs_dev;
    DBuf<int> phases_dev;
    DevPlan plan[2][2];        // [0 forward / 1 adjoint][0 no gains / 1 gains]
    bool has_class[2] = {false, false};
    int nst[2][2] = {{4, 4}, {4, 4}};   // tile shape per [op][class] (autotuned or default)
    int n_ant_max = 0;
    int fin_grid = 1, sc_grid = 1;
    double pairs_class[2] = {0, 0};
    double fin_bytes[2] = {0, 0};   // [forward finish, adjoint finish] per tick
    bool has_mfista = false;         // a tick ends with the MFISTA mix kernel
    // captured tick
    cudaGraphExec_t gexec = nullptr;
    bool graph_ok = false;
    long long tick_launches = 0;
    const void* cap_partial[2] = {nullptr, nullptr};   // the context's scratch the capture baked in
    ~Batch();
};

struct sl1m_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t upstream = nullptr;     // uploads of problems joining a running server
    bool own_stream = false;
    int num_sms = 1;
    std::string err;                     // last error message, guarded by err_mu: a running
    mutable std::mutex err_mu;           // server thread reports failures here too
    DBuf<double2> partial_f;
    DBuf<double> partial_a;
    std::vector<sl1m_problem*> problems;
    // autotuned (streamed granules per stage, CTAs per SM), keyed by
    // (precision, op, gains, Gaussian pixels, log2 of the units)
    std::map<long long, std::pair<int, int>> tune;
    Server* server = nullptr;            // running request loop
    Server* server_done = nullptr;       // stopped loop whose results are still collectable
    bool use_graphs = true;
    // profiling and counters
    bool prof = false;
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[NPROF] = {0}, prof_pairs[NPROF] = {0}, prof_bytes[NPROF] = {0};
    // pairs evaluated by the operator kernels of solver ticks, counted on the
    // device by the scalars kernel while profiling: [precision][0 fwd, 1 adj]
    DBuf<double> evals_dev;
    long long prof_n[NPROF] = {0};
    long long n_launch = 0, h2d = 0, d2h = 0;
    cudaEvent_t get_event();
    void drain_profile();
    ~sl1m_ctx();
};

void prof_begin(sl1m_ctx* ctx, int kid, ProfTok& tok);
void prof_end(sl1m_ctx* ctx, ProfTok& tok, double pairs, double bytes);
int sl1m_fail(sl1m_ctx* ctx, int code, const char* fmt, ...);

struct ProblemDev;

struct sl1m_problem {
    sl1m_ctx* ctx = nullptr;
    // caller data (host copies, caller order)
    int64_t n_vis = 0, n_pix = 0;
    int n_ant = 0;
    std::vector<double> uvw, vis, weights, lm, sigma, gains;
    std::vector<int> ant, kind;
    // device layout
    bool dirty = true;
    bool has_gauss = false;
    bool solver_ready = false;
    bool in_server = false;
    std::unique_ptr<ProblemDev> dev;
    sl1m::DevProblem hp{};          // layout part of the descriptor
    sl1m::SolveBufs hbufs{};
    std::vector<int> vis_orig, pix_orig;
    std::vector<double> last_img;             // image of the last refinement (caller's order)
    int algo = 0;                              // solver of the last init_solve (0 FISTA, 1 MFISTA)
    std::vector<float4> gext_vis, gext_pix;   // granule extents (host copies)
    std::vector<int> gkind_pix;               // pixel granule kinds
    UnitCost ucost[2][2];                      // [precision][0 forward / 1 adjoint]
    bool ucost_ok[2][2] = {{false, false}, {false, false}};
    std::unique_ptr<Batch> op_batch[2], solve_batch[2];
    const UnitCost& unit_cost(int precision, int op);

    int rebuild(cudaStream_t st);
    int ensure_solver(cudaStream_t st);
    int init_solve(const sl1m_solve_opts* o, double L, bool power_only, cudaStream_t st);
    int read_state(sl1m::SolveState& s, cudaStream_t st);
    int fetch_image(double* host_out, cudaStream_t st);
    sl1m::DevProblem solver_desc() const;
    double pairs() const;
    size_t dev_bytes() const;
    size_t estimate_bytes() const;
    ~sl1m_problem();
};

long long tune_key(int precision, int op, bool gains, bool gauss, long long units);

// batches (sl1m_host.cpp)
int batch_set(sl1m_ctx* ctx, Batch& B, const std::vector<sl1m_problem*>& probs,
              const std::vector<sl1m::DevProblem>& descs, int precision, bool solver);
int batch_op(sl1m_ctx* ctx, Batch& B, int op);
int batch_ticks(sl1m_ctx* ctx, Batch& B, int n);
int batch_phases(sl1m_ctx* ctx, Batch& B, std::vector<int>& out);

// server (sl1m_server.cpp)
void server_destroy(sl1m_ctx* ctx);
