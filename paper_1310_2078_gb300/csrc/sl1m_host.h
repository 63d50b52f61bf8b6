// sl1m_host.h -- host-side structures of libsl1m (internal).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

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
    // Allocate exactly `count` and copy from host (zero-fill when `zero`).
    cudaError_t upload(const T* src, size_t count, cudaStream_t st, bool zero = false)
    {
        cudaError_t e = alloc(count);
        if (e != cudaSuccess || count == 0) return e;
        if (zero) return cudaMemsetAsync(p, 0, count * sizeof(T), st);
        e = cudaMemcpyAsync(p, src, count * sizeof(T), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        // the host source may be a temporary: finish the copy before returning
        return cudaStreamSynchronize(st);
    }
    size_t bytes() const { return n * sizeof(T); }
};

struct HostPlan {
    std::vector<long long> u0;
    std::vector<int> b0, poff, clo, ncon;
    long long U = 0;
    int C = 1, n_blocks = 0, n_slots = 0;
};
void plan_host(const std::vector<int>& nb, const std::vector<int>& ns, int Cmax, HostPlan& H);

struct DevPlan {
    sl1m::Plan pl{};
    DBuf<long long> u0;
    DBuf<int> b0, poff, clo, ncon;
};

cudaError_t build_plan(const std::vector<int>& nb, const std::vector<int>& ns, int Cmax, DevPlan& D,
                       cudaStream_t st);

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

struct sl1m_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 1;
    std::string err;
    DBuf<double2> partial_f;
    DBuf<double> partial_a;
    std::vector<sl1m_problem*> problems;
    // profiling
    bool prof = false;
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[NPROF] = {0}, prof_pairs[NPROF] = {0}, prof_bytes[NPROF] = {0};
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
    std::unique_ptr<ProblemDev> dev;
    sl1m::DevProblem hp{};
    sl1m::DevProblem last_desc{};
    bool desc_valid = false;
    sl1m::SolveBufs hbufs{};
    std::vector<int> vis_orig, pix_orig;
    std::map<int, std::unique_ptr<DevPlan>> plans;

    int rebuild();
    int plan(int op, int precision, const sl1m::Plan** out);
    int upload_desc();
    int run_forward(int precision, int fin_mode, const sl1m::SolveBufs* bufs_dev);
    int run_adjoint(int precision, int fin_mode, const sl1m::SolveBufs* bufs_dev);
    int ensure_solver();
    void reset_operands();
    int power(int precision, int max_iter, double tol, double* L, int* iters);
    double pairs() const;
    size_t dev_bytes() const;
    ~sl1m_problem();
};
