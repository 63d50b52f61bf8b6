// sl1m_host.cpp -- host side of libsl1m: contexts, problem layout in HBM,
// stream-K launch plans, the operator calls, the power iteration for L and
// the FISTA loop (Hardy 2013, Sect. 2-3).  See include/sl1m.h for the ABI.
#include "sl1m.h"

#include <algorithm>
#include <future>
#include <thread>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "sl1m_dev.h"
#include "sl1m_host.h"
#include "sl1m_kernels.h"

using namespace sl1m;

// ====================================================================== utils

int sl1m_fail(sl1m_ctx* ctx, int code, const char* fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        std::lock_guard<std::mutex> lk(ctx->err_mu);
        ctx->err = buf;
    }
    return code;
}

#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return sl1m_fail(ctx, e_ == cudaErrorMemoryAllocation ? SL1M_ERR_OOM : SL1M_ERR_CUDA, \
                             "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define CKL(call)          \
    do {                   \
        ctx->n_launch += 1; \
        CK(call);          \
    } while (0)

#define RET(call)                     \
    do {                              \
        int s_ = (call);              \
        if (s_ != SL1M_OK) return s_; \
    } while (0)

static inline float f32hi(double x) { return (float)x; }
static inline float f32lo(double x) { return (float)(x - (double)(float)x); }

// ============================================================ k-d granules

// Order `idx[lo, hi)` so that consecutive runs of G elements are compact
// boxes: recursive split along the wider axis at a multiple of G near the
// median.  Only the last run can be shorter than G.  The two halves of a
// split are independent (disjoint ranges of idx), so down to `par_depth`
// levels the left half runs on a thread of its own: the same operations on
// the same ranges, so the same order as one thread gives.
static void kd_rec(std::vector<int>& idx, size_t lo, size_t hi, const double* x, const double* y,
                   size_t stride, int par_depth)
{
    const size_t n = hi - lo;
    if (n <= (size_t)G) return;
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    for (size_t i = lo; i < hi; ++i) {
        const double a = x[(size_t)idx[i] * stride], b = y[(size_t)idx[i] * stride];
        x0 = std::min(x0, a); x1 = std::max(x1, a);
        y0 = std::min(y0, b); y1 = std::max(y1, b);
    }
    const double* key = (x1 - x0 >= y1 - y0) ? x : y;
    const size_t ng = (n + G - 1) / G;
    const size_t left = (ng / 2) * G;
    std::nth_element(idx.begin() + lo, idx.begin() + lo + left, idx.begin() + hi,
                     [&](int a, int b) {
                         const double ka = key[(size_t)a * stride], kb = key[(size_t)b * stride];
                         return ka < kb || (ka == kb && a < b);
                     });
    if (par_depth > 0 && n >= (size_t)1 << 16) {
        std::future<void> f;
        try {
            f = std::async(std::launch::async, [&] { kd_rec(idx, lo, lo + left, x, y, stride, par_depth - 1); });
        } catch (...) {                    // no thread to be had: the left half runs here
            kd_rec(idx, lo, lo + left, x, y, stride, 0);
        }
        kd_rec(idx, lo + left, hi, x, y, stride, par_depth - 1);
        if (f.valid()) f.get();
    } else {
        kd_rec(idx, lo, lo + left, x, y, stride, 0);
        kd_rec(idx, lo + left, hi, x, y, stride, 0);
    }
}

// Levels of the k-d split that run their halves in parallel: up to the host's
// hardware threads (at most 16 leaves).
static int kd_par_depth()
{
    const unsigned t = std::max(1u, std::thread::hardware_concurrency());
    int d = 0;
    while (d < 4 && (2u << d) <= t) ++d;
    return d;
}

// Run fn(lo, hi) over [0, n) cut into contiguous chunks, one per host thread
// (at most 16), when n is large enough to pay for the threads.  For loops whose
// iterations write only their own outputs: the result is the one a single
// thread gives.
template <class F>
static void parallel_chunks(size_t n, size_t min_per_chunk, const F& fn)
{
    const size_t t = std::min<size_t>(16, std::max(1u, std::thread::hardware_concurrency()));
    const size_t nc = std::max<size_t>(1, std::min(t, n / std::max<size_t>(1, min_per_chunk)));
    if (nc <= 1) {
        fn((size_t)0, n);
        return;
    }
    std::vector<std::future<void>> fs;
    size_t done = 0;                       // chunks [0, done) run on threads
    try {
        for (size_t c = 1; c < nc; ++c) {
            fs.push_back(std::async(std::launch::async, [&fn, n, nc, c] { fn(n * c / nc, n * (c + 1) / nc); }));
            done = c;
        }
    } catch (...) {                        // no thread to be had: the rest runs here
    }
    fn(0, n / nc);
    for (size_t c = done + 1; c < nc; ++c) fn(n * c / nc, n * (c + 1) / nc);
    for (auto& f : fs) f.get();
}

// Append `members` (caller indices) in k-d order, padded with -1 to a
// multiple of G.
static void kd_append(std::vector<int>& order, std::vector<int> members, const double* x,
                      const double* y, size_t stride)
{
    kd_rec(members, 0, members.size(), x, y, stride, kd_par_depth());
    order.insert(order.end(), members.begin(), members.end());
    while (order.size() % G) order.push_back(-1);
}

// Reorder whole visibility granules (members unchanged) by the share of
// (visibility granule, pixel granule) tiles whose extents bound the phase
// product term above D_MAX turns, which the mixed kernels evaluate on the
// exact, about 3x dearer, path.  The forward's 8 warps each own one granule
// of a block and meet at every stage, so a block costs what its slowest
// granule costs: a wide granule among narrow ones leaves 7 warps idle.  A
// stable sort by that share (most granules: 0, kept in k-d order) groups the
// wide ones into the same blocks.  The share is taken against up to 1,024
// pixel granules (every ceil(n/1024)-th), with the extents as half the
// bounding box, as layout_side computes them.
static void group_by_exact_share(std::vector<int>& order, const double* uvw, const std::vector<float4>& pext)
{
    const size_t ng = order.size() / G;
    if (ng < 2 || pext.empty()) return;
    const size_t step = (pext.size() + 1023) / 1024;
    std::vector<std::pair<float, int>> key(ng);
    parallel_chunks(ng, 256, [&](size_t g0, size_t g1) {
        for (size_t g = g0; g < g1; ++g) {
            double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
            for (size_t i = g * G; i < (g + 1) * G; ++i) {
                const int o = order[i];
                if (o < 0) continue;
                for (int a = 0; a < 3; ++a) {
                    mn[a] = std::min(mn[a], uvw[3 * (size_t)o + a]);
                    mx[a] = std::max(mx[a], uvw[3 * (size_t)o + a]);
                }
            }
            const float e[3] = {(float)(0.5 * (mx[0] - mn[0])), (float)(0.5 * (mx[1] - mn[1])),
                                (float)(0.5 * (mx[2] - mn[2]))};
            int n_ex = 0, n = 0;
            for (size_t p = 0; p < pext.size(); p += step, ++n)
                n_ex += e[0] * pext[p].x + e[1] * pext[p].y + e[2] * pext[p].z > D_MAX;
            key[g] = {(float)n_ex / (float)std::max(1, n), (int)g};
        }
    });
    bool any = false;
    for (const auto& k : key) any |= k.first > 0.f;
    if (!any) return;
    std::stable_sort(key.begin(), key.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    std::vector<int> out(order.size());
    for (size_t g = 0; g < ng; ++g)
        std::copy(order.begin() + (size_t)key[g].second * G, order.begin() + ((size_t)key[g].second + 1) * G,
                  out.begin() + g * G);
    order.swap(out);
}

// With gains: sort the members of each granule (its membership is unchanged)
// by antenna pair (a, b), padding last, so that equal pairs are adjacent: the
// adjoint computes a pair's gain product once per run, and the forward lists
// the granule's distinct pairs.
static void sort_baselines(std::vector<int>& order, const std::vector<int>& ant)
{
    for (size_t g0 = 0; g0 + G <= order.size(); g0 += G)
        std::stable_sort(order.begin() + g0, order.begin() + g0 + G, [&](int x, int y) {
            if (x < 0 || y < 0) return x >= 0 && y < 0;            // padding last
            const long long kx = (long long)ant[2 * x] << 32 | (unsigned)ant[2 * x + 1];
            const long long ky = (long long)ant[2 * y] << 32 | (unsigned)ant[2 * y + 1];
            return kx < ky;
        });
}

// An allocator whose resize() leaves new elements of a trivial type
// uninitialised (every slot is written afterwards): the large host arrays of
// a layout are then first touched by the threads that fill them, not zeroed
// by one thread before.
template <class T>
struct NoInitAlloc : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = NoInitAlloc<U>;
    };
    NoInitAlloc() = default;
    template <class U>
    NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
    template <class U>
    void construct(U* p) noexcept
    {
        ::new ((void*)p) U;
    }
    template <class U, class... A>
    void construct(U* p, A&&... a)
    {
        ::new ((void*)p) U(std::forward<A>(a)...);
    }
};
template <class T>
using HostVec = std::vector<T, NoInitAlloc<T>>;

struct HostSide {
    int n = 0, n_pad = 0, n_gran = 0, n_blk = 0;
    HostVec<float4> hi, lo, off, offlo;
    std::vector<float4> cen_hi, cen_lo, ext;
    HostVec<d4> d;
    std::vector<int> orig;
};

// Fill a side from `order` (caller index per sorted slot, -1 = padding) and
// FP64 element coordinates xyz[i] = (x, y, z), aux[i].  Padding copies the
// coordinates of a real element of its granule and gets aux = 0.
static void layout_side(const std::vector<int>& order, const std::vector<d4>& xyz, int n_real,
                        HostSide& S)
{
    S.n = n_real;
    S.n_pad = (int)order.size();
    S.n_gran = S.n_pad / G;
    S.n_blk = (S.n_gran + BLK_GRAN - 1) / BLK_GRAN;
    S.orig = order;
    S.hi.resize(S.n_pad); S.lo.resize(S.n_pad); S.off.resize(S.n_pad); S.offlo.resize(S.n_pad);
    S.d.resize(S.n_pad);
    S.cen_hi.resize(S.n_gran); S.cen_lo.resize(S.n_gran); S.ext.resize(S.n_gran);
    // granules are independent: each fills only its own slots
    parallel_chunks((size_t)S.n_gran, 512, [&](size_t g0, size_t g1) {
    for (int g = (int)g0; g < (int)g1; ++g) {
        int ref = -1;
        double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
        for (int t = 0; t < G; ++t) {
            const int o = order[(size_t)g * G + t];
            if (o < 0) continue;
            ref = o;
            const double c[3] = {xyz[o].x, xyz[o].y, xyz[o].z};
            for (int a = 0; a < 3; ++a) { mn[a] = std::min(mn[a], c[a]); mx[a] = std::max(mx[a], c[a]); }
        }
        double cen[3] = {0, 0, 0};
        if (ref >= 0)
            for (int a = 0; a < 3; ++a) cen[a] = 0.5 * (mn[a] + mx[a]);
        // extent with a small margin: an upper bound of |offset| per axis
        S.ext[g] = make_float4((float)((mx[0] - mn[0]) * 0.5000001), (float)((mx[1] - mn[1]) * 0.5000001),
                               (float)((mx[2] - mn[2]) * 0.5000001), 0.f);
        if (ref < 0) S.ext[g] = make_float4(0.f, 0.f, 0.f, 0.f);
        S.cen_hi[g] = make_float4(f32hi(cen[0]), f32hi(cen[1]), f32hi(cen[2]), 0.f);
        S.cen_lo[g] = make_float4(f32lo(cen[0]), f32lo(cen[1]), f32lo(cen[2]), 0.f);
        for (int t = 0; t < G; ++t) {
            const size_t i = (size_t)g * G + t;
            const int o = order[i];
            d4 v = make_d4(cen[0], cen[1], cen[2], 0.0);
            if (o >= 0) v = xyz[o];
            else if (ref >= 0) { v = xyz[ref]; v.w = 0.0; }
            S.d[i] = v;
            const double c[3] = {v.x, v.y, v.z};
            double dd[3];
            for (int a = 0; a < 3; ++a) dd[a] = c[a] - cen[a];
            S.hi[i] = make_float4(f32hi(c[0]), f32hi(c[1]), f32hi(c[2]), 0.f);
            S.lo[i] = make_float4(f32lo(c[0]), f32lo(c[1]), f32lo(c[2]), 0.f);
            S.off[i] = make_float4(f32hi(dd[0]), f32hi(dd[1]), f32hi(dd[2]), (float)v.w);
            S.offlo[i] = make_float4(f32lo(dd[0]), f32lo(dd[1]), f32lo(dd[2]), 0.f);
        }
    }
    });
}

// ============================================================ device buffers

struct DevSide {
    DBuf<float4> hi, lo, off, offlo, cen_hi, cen_lo, ext;
    DBuf<d4> d;
    DBuf<int> orig;
};

static cudaError_t upload_side(const HostSide& H, DevSide& D, Side& S, cudaStream_t st)
{
    cudaError_t e;
#define UP(f)                                                        \
    if ((e = D.f.upload(H.f.data(), H.f.size(), st)) != cudaSuccess) return e;
    UP(hi) UP(lo) UP(off) UP(offlo) UP(cen_hi) UP(cen_lo) UP(ext) UP(d) UP(orig)
#undef UP
    S.n = H.n; S.n_pad = H.n_pad; S.n_gran = H.n_gran; S.n_blk = H.n_blk;
    S.hi = D.hi.p; S.lo = D.lo.p; S.off = D.off.p; S.offlo = D.offlo.p;
    S.cen_hi = D.cen_hi.p; S.cen_lo = D.cen_lo.p; S.ext = D.ext.p; S.d = D.d.p; S.orig = D.orig.p;
    return cudaSuccess;
}

// ================================================================= plans

// Stream-K schedule (host part): units = nb[p] * ns[p] per problem, CTA c
// takes units [c U / C, (c+1) U / C); block gb is touched by CTAs
// clo..clo+ncon-1 and owns partial slots poff..poff+ncon-1.
void plan_host(const std::vector<int>& nb, const std::vector<int>& ns, int Cmax, HostPlan& H,
               const std::vector<const UnitCost*>* costs)
{
    const int np = (int)nb.size();
    H.u0.assign(np + 1, 0);
    H.b0.assign(np + 1, 0);
    for (int p = 0; p < np; ++p) {
        H.u0[p + 1] = H.u0[p] + (long long)nb[p] * ns[p];
        H.b0[p + 1] = H.b0[p] + nb[p];
    }
    const long long U = H.u0[np];
    const int C = (int)std::max(1LL, std::min((long long)std::max(1, Cmax), U));
    H.cta_u0.clear();
    if (costs && U > 0) {
        // cumulative cost per problem; boundaries at multiples of total / C
        std::vector<double> W(np + 1, 0.0);
        for (int p = 0; p < np; ++p) {
            const UnitCost* uc = (*costs)[p];
            const long long up = H.u0[p + 1] - H.u0[p];
            double w = 0.0;
            if (uc && !uc->unit.empty() && (long long)uc->unit.size() == up) {
                for (float f : uc->unit) w += f;
            } else {
                w = (uc ? uc->uniform : 1.0) * (double)up;
            }
            W[p + 1] = W[p] + w;
        }
        const double T = W[np];
        H.cta_u0.assign(C + 1, 0);
        H.cta_u0[C] = U;
        int p = 0;
        std::vector<double> pref;
        int pref_of = -1;
        for (int c = 1; c < C; ++c) {
            const double t = T * (double)c / (double)C;
            while (p < np - 1 && W[p + 1] < t) ++p;
            const UnitCost* uc = (*costs)[p];
            const long long up = H.u0[p + 1] - H.u0[p];
            long long i;
            if (uc && !uc->unit.empty() && (long long)uc->unit.size() == up) {
                if (pref_of != p) {
                    pref.assign(up + 1, 0.0);
                    for (long long k = 0; k < up; ++k) pref[k + 1] = pref[k] + uc->unit[k];
                    pref_of = p;
                }
                i = std::lower_bound(pref.begin(), pref.end(), t - W[p]) - pref.begin();
            } else {
                const double w = (uc ? uc->uniform : 1.0);
                i = (long long)std::ceil((t - W[p]) / w - 1e-9);
            }
            i = std::max(0LL, std::min(up, i));
            H.cta_u0[c] = H.u0[p] + i;
        }
        // every CTA gets at least one unit (C <= U): a block's partial slots
        // are those of every CTA between its first and last, so none may be
        // empty in between
        for (int c = 1; c < C; ++c)
            H.cta_u0[c] = std::min(std::max(H.cta_u0[c], H.cta_u0[c - 1] + 1), U - (C - c));
    }
    auto cta_of = [&](long long x) {
        if (H.cta_u0.empty()) return (int)(((x + 1) * C + U - 1) / U - 1);
        const int c = (int)(std::upper_bound(H.cta_u0.begin(), H.cta_u0.end(), x) - H.cta_u0.begin()) - 1;
        return std::max(0, std::min(C - 1, c));
    };
    const int nblocks = H.b0[np];
    H.poff.assign(nblocks, 0);
    H.clo.assign(nblocks, 0);
    H.ncon.assign(nblocks, 0);
    int slots = 0;
    for (int p = 0; p < np; ++p) {
        for (int b = 0; b < nb[p]; ++b) {
            const int gb = H.b0[p] + b;
            H.poff[gb] = slots;
            if (ns[p] == 0 || U == 0) continue;
            const long long s0 = H.u0[p] + (long long)b * ns[p], e0 = s0 + ns[p];
            H.clo[gb] = cta_of(s0);
            H.ncon[gb] = cta_of(e0 - 1) - H.clo[gb] + 1;
            slots += H.ncon[gb];
        }
    }
    H.U = U;
    H.C = C;
    H.n_blocks = nblocks;
    H.n_slots = slots;
}

// Build a stream-K plan over problems with owned blocks nb[p] and streamed
// granules ns[p]; C CTAs at most.  Uploads the tables.
cudaError_t build_plan(const std::vector<int>& nb, const std::vector<int>& ns, int Cmax,
                       DevPlan& D, cudaStream_t st, const std::vector<const UnitCost*>* costs)
{
    HostPlan H;
    plan_host(nb, ns, Cmax, H, costs);
    cudaError_t err;
    auto up = [&](DBuf<int>& b, const std::vector<int>& v) {
        return b.upload(v.data(), std::max<size_t>(1, v.size()), st, v.empty());
    };
    if ((err = D.u0.upload(H.u0.data(), H.u0.size(), st))) return err;
    if ((err = up(D.b0, H.b0))) return err;
    if ((err = up(D.poff, H.poff))) return err;
    if ((err = up(D.clo, H.clo))) return err;
    if ((err = up(D.ncon, H.ncon))) return err;
    if (!H.cta_u0.empty()) {
        if ((err = D.cta.upload(H.cta_u0.data(), H.cta_u0.size(), st))) return err;
    } else {
        D.cta.free();
    }
    D.pl.n_probs = (int)nb.size();
    D.pl.C = H.C;
    D.pl.U = H.U;
    D.pl.prob_u0 = D.u0.p;
    D.pl.prob_b0 = D.b0.p;
    D.pl.blk_poff = D.poff.p;
    D.pl.blk_clo = D.clo.p;
    D.pl.blk_ncon = D.ncon.p;
    D.pl.cta_u0 = H.cta_u0.empty() ? nullptr : D.cta.p;
    D.pl.n_blocks = H.n_blocks;
    D.pl.n_slots = H.n_slots;
    return D.dpl.upload(&D.pl, 1, st);
}

// ================================================================ profiling

void prof_begin(sl1m_ctx* ctx, int kid, ProfTok& tok)
{
    tok.active = false;
    if (!ctx->prof) return;
    tok.active = true;
    tok.kid = kid;
    tok.ev0 = ctx->get_event();
    tok.ev1 = ctx->get_event();
    cudaEventRecord(tok.ev0, ctx->stream);
}

void prof_end(sl1m_ctx* ctx, ProfTok& tok, double pairs, double bytes)
{
    if (!tok.active) return;
    cudaEventRecord(tok.ev1, ctx->stream);
    ctx->pending.push_back({tok.kid, tok.ev0, tok.ev1, pairs, bytes});
}

cudaEvent_t sl1m_ctx::get_event()
{
    if (!ev_pool.empty()) {
        cudaEvent_t e = ev_pool.back();
        ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void sl1m_ctx::drain_profile()
{
    if (evals_dev.p) {                 // solver ticks: the pairs counted on the device
        double ev[4] = {0, 0, 0, 0};
        if (cudaMemcpyAsync(ev, evals_dev.p, sizeof ev, cudaMemcpyDeviceToHost, stream) == cudaSuccess &&
            cudaStreamSynchronize(stream) == cudaSuccess) {
            prof_pairs[0] += ev[0];    // forward FP64, adjoint FP64, forward mixed, adjoint mixed
            prof_pairs[1] += ev[1];
            prof_pairs[2] += ev[2];
            prof_pairs[3] += ev[3];
            cudaMemsetAsync(evals_dev.p, 0, sizeof ev, stream);
        }
    }
    for (auto& r : pending) {
        cudaEventSynchronize(r.ev1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.ev0, r.ev1);
        prof_ms[r.kid] += ms;
        prof_n[r.kid] += 1;
        prof_pairs[r.kid] += r.pairs;
        prof_bytes[r.kid] += r.bytes;
        ev_pool.push_back(r.ev0);
        ev_pool.push_back(r.ev1);
    }
    pending.clear();
}

sl1m_ctx::~sl1m_ctx()
{
    cudaSetDevice(device);
    drain_profile();
    for (auto e : ev_pool) cudaEventDestroy(e);
    if (upstream) cudaStreamDestroy(upstream);
    if (own_stream && stream) cudaStreamDestroy(stream);
}

// ============================================================== problem

struct ProblemDev {
    DevSide vis, pix;
    DBuf<int2> ant;
    DBuf<float4> vgabs;
    DBuf<float2> r32;
    DBuf<int> vslot, gnb;
    DBuf<int2> gbl;
    DBuf<double2> V;
    DBuf<float4> pgauss;
    DBuf<d4> pgauss64;
    DBuf<float> gsig;
    DBuf<double> gsig64;
    DBuf<int> gkind;
    DBuf<float4> pghdr;
    DBuf<float2> gpol32;
    DBuf<double2> gains64;
    // operator scratch
    DBuf<double> x_user, x_sorted, adj_sorted, img_user;
    DBuf<double2> r_user, r_sorted, fwd_sorted, vis_user;
    // solver
    DBuf<double> I0, I1, y, xv, blk_r2, blk_l1, blk_z2;
    DBuf<double2> AI0, AI1, rr;
    DBuf<int> blk_nnz, blk_badv, blk_badp;
    DBuf<SolveState> st;
};

sl1m_problem::~sl1m_problem() = default;

int sl1m_problem::rebuild(cudaStream_t st)
{
    if (!dirty) return SL1M_OK;
    if (n_vis <= 0 || n_pix <= 0)
        return sl1m_fail(ctx, SL1M_ERR_STATE, "problem needs visibilities and pixels");
    if (n_ant > 0 && ant.empty())
        return sl1m_fail(ctx, SL1M_ERR_STATE, "gains need antenna pairs in sl1m_set_visibilities");
    if (n_ant > 0) {
        for (int64_t k = 0; k < n_vis; ++k)
            if (ant[2 * k] < 0 || ant[2 * k] >= n_ant || ant[2 * k + 1] < 0 || ant[2 * k + 1] >= n_ant)
                return sl1m_fail(ctx, SL1M_ERR_ARG, "antenna index out of range at visibility %lld",
                                 (long long)k);
    }
    {
        // the mixed kernels round products of coordinates to whole turns on the
        // FP32 add pipe, exact below 2^22 turns; a centre times an offset is at
        // most twice the largest product, so each must stay below 2^21 turns
        double mu = 0, mv = 0, mw = 0, ml = 0, mm = 0, mn = 0;
        for (int64_t k = 0; k < n_vis; ++k) {
            mu = std::max(mu, std::fabs(uvw[3 * k]));
            mv = std::max(mv, std::fabs(uvw[3 * k + 1]));
            mw = std::max(mw, std::fabs(uvw[3 * k + 2]));
        }
        for (int64_t j = 0; j < n_pix; ++j) {
            const double l = lm[2 * j], m = lm[2 * j + 1], r2 = l * l + m * m;
            ml = std::max(ml, std::fabs(l));
            mm = std::max(mm, std::fabs(m));
            mn = std::max(mn, r2 / (1.0 + std::sqrt(1.0 - r2)));
        }
        const double lim = 2097152.0;
        if (mu * ml >= lim || mv * mm >= lim || mw * mn >= lim)
            return sl1m_fail(ctx, SL1M_ERR_ARG,
                             "max |u l|, |v m| or |w (n-1)| reaches 2^21 turns (%g, %g, %g): outside the "
                             "range of the exact phase split", mu * ml, mv * mm, mw * mn);
    }
    if (!dev) dev = std::make_unique<ProblemDev>();
    ProblemDev& D = *dev;
    // ---- pixels: classes of equal (kind, sigma), each in k-d order on (l, m)
    {
        std::vector<std::pair<std::pair<int, double>, int>> cls(n_pix);
        for (int64_t j = 0; j < n_pix; ++j)
            cls[j] = {{kind.empty() ? 0 : kind[j], sigma.empty() ? 0.0 : sigma[j]}, (int)j};
        // (one class, the common case: already in the order the sort gives)
        bool one_class = true;
        for (int64_t j = 1; j < n_pix && one_class; ++j) one_class = cls[j].first == cls[0].first;
        if (!one_class)
            std::stable_sort(cls.begin(), cls.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
        std::vector<int> order;
        std::vector<std::pair<int, double>> gran_cls;
        size_t i = 0;
        while (i < cls.size()) {
            size_t j = i;
            std::vector<int> members;
            while (j < cls.size() && cls[j].first == cls[i].first) members.push_back(cls[j++].second);
            const size_t before = order.size();
            kd_append(order, std::move(members), lm.data(), lm.data() + 1, 2);
            for (size_t g = before / G; g < order.size() / G; ++g)
                gran_cls.push_back({cls[i].first.first, cls[i].first.second});
            i = j;
        }
        std::vector<d4> xyz(n_pix);
        for (int64_t j = 0; j < n_pix; ++j) {
            const double l = lm[2 * j], m = lm[2 * j + 1];
            const double r2 = l * l + m * m, n = std::sqrt(1.0 - r2);
            xyz[j] = make_d4(l, m, -r2 / (1.0 + n), 1.0 / n);
        }
        HostSide H;
        layout_side(order, xyz, (int)n_pix, H);
        CK(upload_side(H, D.pix, hp.pix, st));
        gext_pix = H.ext;
        std::vector<float4> pg(H.n_pad);
        std::vector<d4> pg64(H.n_pad);
        for (int t = 0; t < H.n_pad; ++t) {
            const d4 v = H.d[t];
            const double r2h = 0.5 * (v.x * v.x + v.y * v.y);
            pg64[t] = make_d4(v.x, v.y, r2h, v.z + r2h);
            pg[t] = make_float4((float)v.x, (float)v.y, (float)r2h, (float)(v.z + r2h));
        }
        CK(D.pgauss.upload(pg.data(), pg.size(), st));
        CK(D.pgauss64.upload(pg64.data(), pg64.size(), st));
        std::vector<float> gs(H.n_gran);
        std::vector<double> gs64(H.n_gran);
        std::vector<int> gk(H.n_gran);
        has_gauss = false;
        for (int g = 0; g < H.n_gran; ++g) {
            gk[g] = gran_cls[g].first;
            gs64[g] = gran_cls[g].second;
            gs[g] = (float)gs64[g];
            has_gauss |= gk[g] != DIRAC;
        }
        CK(D.gsig.upload(gs.data(), gs.size(), st));
        CK(D.gsig64.upload(gs64.data(), gs64.size(), st));
        CK(D.gkind.upload(gk.data(), gk.size(), st));
        // per pixel granule, as the forward's bulk copies take it
        std::vector<float4> hdr((size_t)H.n_gran * 4);
        for (int g = 0; g < H.n_gran; ++g) {
            hdr[4 * (size_t)g] = H.cen_hi[g];
            hdr[4 * (size_t)g + 1] = H.cen_lo[g];
            hdr[4 * (size_t)g + 2] = H.ext[g];
            hdr[4 * (size_t)g + 3] = make_float4(gs[g], (float)gk[g], 0.f, 0.f);
        }
        CK(D.pghdr.upload(hdr.data(), hdr.size(), st));
        gkind_pix = gk;
        pix_orig = H.orig;
        if (n_ant > 0) {
            // FP32 in polar form {|G|, arg G in turns} (modulus and argument
            // taken in FP64): per pixel granule one row of GP per antenna
            // (gain_rows(n_ant) rows), the shared-memory layout, so a granule's
            // table is one bulk copy; FP64: [pixel][antenna]
            const size_t tab = (size_t)gain_rows(n_ant) * GP;
            std::vector<float2> gp32((size_t)H.n_gran * tab, make_float2(0.f, 0.f));
            std::vector<double2> g64((size_t)H.n_pad * n_ant, make_double2(0.0, 0.0));
            for (int t = 0; t < H.n_pad; ++t) {
                const int o = H.orig[t];
                if (o < 0) continue;
                const size_t row0 = (size_t)(t / G) * tab + (size_t)(t % G);
                for (int a = 0; a < n_ant; ++a) {
                    const double re = gains[((size_t)o * n_ant + a) * 2], im = gains[((size_t)o * n_ant + a) * 2 + 1];
                    gp32[row0 + (size_t)a * GP] =
                        make_float2((float)std::hypot(re, im), (float)(std::atan2(im, re) / 6.283185307179586));
                    g64[(size_t)t * n_ant + a] = make_double2(re, im);
                }
            }
            CK(D.gpol32.upload(gp32.data(), gp32.size(), st));
            CK(D.gains64.upload(g64.data(), g64.size(), st));
        } else {
            D.gpol32.free();
            D.gains64.free();
        }
    }
    // ---- visibilities: k-d order on (u, v); granules grouped by their share of
    // exact-phase tiles (after the pixels, whose extents that share needs)
    {
        std::vector<int> members(n_vis);
        for (int64_t k = 0; k < n_vis; ++k) members[k] = (int)k;
        std::vector<int> order;
        kd_append(order, std::move(members), uvw.data(), uvw.data() + 1, 3);
        group_by_exact_share(order, uvw.data(), gext_pix);
        if (n_ant > 0) sort_baselines(order, ant);
        std::vector<d4> xyz(n_vis);
        for (int64_t k = 0; k < n_vis; ++k)
            xyz[k] = make_d4(uvw[3 * k], uvw[3 * k + 1], uvw[3 * k + 2], weights.empty() ? 1.0 : weights[k]);
        HostSide H;
        layout_side(order, xyz, (int)n_vis, H);
        CK(upload_side(H, D.vis, hp.vis, st));
        gext_vis = H.ext;
        std::vector<int2> a(H.n_pad, make_int2(0, 0));
        std::vector<double2> Vs(H.n_pad, make_double2(0.0, 0.0));
        for (int i = 0; i < H.n_pad; ++i) {
            const int o = H.orig[i];
            if (o < 0) continue;
            if (!ant.empty()) a[i] = make_int2(ant[2 * o], ant[2 * o + 1]);
            Vs[i] = make_double2(vis[2 * o], vis[2 * o + 1]);
        }
        CK(D.ant.upload(a.data(), a.size(), st));
        CK(D.V.upload(Vs.data(), Vs.size(), st));
        // {u, v, -2 w, u^2 + v^2} in FP32, as the adjoint's Gaussian terms take it
        std::vector<float4> ga(H.n_pad);
        for (int i = 0; i < H.n_pad; ++i) {
            const float4 h = H.hi[i];
            ga[i] = make_float4(h.x, h.y, -2.0f * h.z, std::fmaf(h.x, h.x, h.y * h.y));
        }
        CK(D.vgabs.upload(ga.data(), ga.size(), st));
        CK(D.r32.upload(nullptr, H.n_pad, st, true));
        vis_orig = H.orig;
        if (n_ant > 0) {
            // each granule's distinct antenna pairs (adjacent after sort_baselines)
            std::vector<int> vslot(H.n_pad, 0), gnb(H.n_gran, 0);
            std::vector<int2> gbl((size_t)H.n_gran * NB_MAX, make_int2(0, 0));
            for (int g = 0; g < H.n_gran; ++g) {
                int nb = 0;
                bool over = false;
                for (int i = g * G; i < (g + 1) * G; ++i) {
                    const int2 ab = a[i];
                    if (nb == 0 || ab.x != gbl[(size_t)g * NB_MAX + nb - 1].x ||
                        ab.y != gbl[(size_t)g * NB_MAX + nb - 1].y) {
                        if (nb == NB_MAX) { over = true; break; }
                        gbl[(size_t)g * NB_MAX + nb++] = ab;
                    }
                    vslot[i] = nb - 1;
                }
                gnb[g] = over ? 0 : nb;
            }
            CK(D.vslot.upload(vslot.data(), vslot.size(), st));
            CK(D.gbl.upload(gbl.data(), gbl.size(), st));
            CK(D.gnb.upload(gnb.data(), gnb.size(), st));
        } else {
            D.vslot.free();
            D.gbl.free();
            D.gnb.free();
        }
    }
    hp.ant = D.ant.p;
    hp.vgabs = D.vgabs.p;
    hp.r32 = D.r32.p;
    hp.vslot = n_ant > 0 ? D.vslot.p : nullptr;
    hp.gbl = n_ant > 0 ? D.gbl.p : nullptr;
    hp.gnb = n_ant > 0 ? D.gnb.p : nullptr;
    hp.V = D.V.p;
    hp.pgauss = D.pgauss.p;
    hp.pgauss64 = D.pgauss64.p;
    hp.gsig = D.gsig.p;
    hp.gsig64 = D.gsig64.p;
    hp.gkind = D.gkind.p;
    hp.pghdr = D.pghdr.p;
    hp.gpol32 = n_ant > 0 ? D.gpol32.p : nullptr;
    hp.gains64 = n_ant > 0 ? D.gains64.p : nullptr;
    hp.n_ant = n_ant;
    hp.x = nullptr;
    hp.r = nullptr;
    hp.fwd_out = nullptr;
    hp.adj_out = nullptr;
    hp.st = nullptr;
    ctx->h2d += (long long)dev_bytes();
    for (auto& b : op_batch) b.reset();
    for (auto& b : solve_batch) b.reset();
    for (auto& r : ucost_ok) r[0] = r[1] = false;
    solver_ready = false;
    dirty = false;
    return SL1M_OK;
}

double sl1m_problem::pairs() const { return (double)n_vis * (double)n_pix; }

// Relative cost of the units (owned block x streamed granule) of one operator:
// a Gaussian pixel granule costs 1.34 to 1.60 times a Dirac one (measured, see
// below), a tile taking the exact phase path 3x, and gains 2x (gains problems
// run in launches of their own, so that factor only orders work across the
// two classes).  A block's 8 warps meet at each shared-memory stage, so a unit
// costs what its slowest warp costs.  Uniform problems return a constant.
const UnitCost& sl1m_problem::unit_cost(int precision, int op)
{
    UnitCost& uc = ucost[precision][op];
    if (ucost_ok[precision][op]) return uc;
    ucost_ok[precision][op] = true;
    uc.unit.clear();
    // cost of a Gaussian pair relative to a Dirac pair of the same launch,
    // measured on GB300 (4 x 128x128 pixels of one kind x 32,000 visibilities):
    // forward 1.53, adjoint 1.60 without gains; 1.34 and 1.45 with gains
    const double gfac = n_ant > 0 ? 2.0 : 1.0;
    const double gcost = n_ant > 0 ? (op == 0 ? 1.34 : 1.45) : (op == 0 ? 1.53 : 1.60);
    const auto base = [gcost](int kind) { return kind == DIRAC ? 1.0 : gcost; };
    int k0 = gkind_pix.empty() ? 0 : gkind_pix[0];
    bool one_kind = true;
    for (int k : gkind_pix) one_kind &= k == k0;
    const std::vector<float4>& own = op == 0 ? gext_vis : gext_pix;
    const std::vector<float4>& str = op == 0 ? gext_pix : gext_vis;
    float4 mo = make_float4(0.f, 0.f, 0.f, 0.f), ms = mo;
    for (const float4& e : own) { mo.x = std::max(mo.x, e.x); mo.y = std::max(mo.y, e.y); mo.z = std::max(mo.z, e.z); }
    for (const float4& e : str) { ms.x = std::max(ms.x, e.x); ms.y = std::max(ms.y, e.y); ms.z = std::max(ms.z, e.z); }
    const bool any_exact = precision == 1 && (mo.x * ms.x + mo.y * ms.y + mo.z * ms.z) > D_MAX;
    uc.uniform = base(k0) * gfac;
    if (one_kind && !any_exact) return uc;
    const int ng_own = (int)own.size(), ng_str = (int)str.size();
    const int nblk = (ng_own + BLK_GRAN - 1) / BLK_GRAN;
    uc.unit.resize((size_t)nblk * ng_str);
    for (int b = 0; b < nblk; ++b) {
        const int w1 = std::min(ng_own, (b + 1) * BLK_GRAN);
        double kb = 1.0;
        if (op == 1)
            for (int w = b * BLK_GRAN; w < w1; ++w) kb = std::max(kb, base(gkind_pix[w]));
        for (int g = 0; g < ng_str; ++g) {
            bool ex = false;
            if (any_exact) {
                const float4 s4 = str[g];
                for (int w = b * BLK_GRAN; w < w1 && !ex; ++w)
                    ex = own[w].x * s4.x + own[w].y * s4.y + own[w].z * s4.z > D_MAX;
            }
            const double kbase = op == 0 ? base(gkind_pix[g]) : kb;
            uc.unit[(size_t)b * ng_str + g] = (float)(kbase * (ex ? 3.0 : 1.0) * gfac);
        }
    }
    return uc;
}

// Device bytes a problem will hold once laid out with solver buffers
// (admission estimate; padded sizes, ~100 B per element and side).
size_t sl1m_problem::estimate_bytes() const
{
    const size_t nv = (size_t)((n_vis + G - 1) / G) * G, np = (size_t)((n_pix + G - 1) / G) * G;
    size_t b = nv * (4 * 16 + 32 + 4 + 8 + 16) + np * (4 * 16 + 32 + 4 + 16 + 32);
    if (n_ant > 0) {
        b += (size_t)gain_rows(n_ant) * GP * (np / G) * 8 + (size_t)n_ant * np * 16;   // FP32 + FP64
        b += nv * 4 + (nv / G) * (NB_MAX * 8 + 4);                                     // pair lists
    }
    b += np * 8 * 4 + nv * 16 * 3;                 // solver vectors
    b += nv * (16 + 8);                            // the adjoint's FP32 Gaussian terms and residual
    b += (nv + np) * 16 * 3;                       // operator scratch
    return b + (1 << 16);
}

int sl1m_problem::ensure_solver(cudaStream_t st)
{
    if (solver_ready) return SL1M_OK;
    ProblemDev& D = *dev;
    const size_t np = hp.pix.n_pad, nv = hp.vis.n_pad;
    CK(D.I0.alloc(np)); CK(D.I1.alloc(np)); CK(D.y.alloc(np)); CK(D.xv.alloc(np));
    CK(D.AI0.alloc(nv)); CK(D.AI1.alloc(nv)); CK(D.rr.alloc(nv));
    CK(D.blk_r2.alloc(std::max(1, hp.vis.n_blk)));
    CK(D.blk_badv.alloc(std::max(1, hp.vis.n_blk)));
    CK(D.blk_l1.alloc(std::max(1, hp.pix.n_blk)));
    CK(D.blk_z2.alloc(std::max(1, hp.pix.n_blk)));
    CK(D.blk_nnz.alloc(std::max(1, hp.pix.n_blk)));
    CK(D.blk_badp.alloc(std::max(1, hp.pix.n_blk)));
    CK(D.st.alloc(1));
    SolveBufs b;
    b.I[0] = D.I0.p; b.I[1] = D.I1.p; b.y = D.y.p; b.xv = D.xv.p;
    b.AI[0] = D.AI0.p; b.AI[1] = D.AI1.p; b.r = D.rr.p;
    b.blk_r2 = D.blk_r2.p; b.blk_l1 = D.blk_l1.p; b.blk_z2 = D.blk_z2.p;
    b.blk_nnz = D.blk_nnz.p; b.blk_badv = D.blk_badv.p; b.blk_badp = D.blk_badp.p;
    hbufs = b;
    CK(cudaMemsetAsync(D.blk_badp.p, 0, sizeof(int) * std::max(1, hp.pix.n_blk), st));
    CK(cudaMemsetAsync(D.blk_badv.p, 0, sizeof(int) * std::max(1, hp.vis.n_blk), st));
    solver_ready = true;
    return SL1M_OK;
}

DevProblem sl1m_problem::solver_desc() const
{
    DevProblem d = hp;
    d.x = nullptr;
    d.r = nullptr;
    d.fwd_out = nullptr;
    d.adj_out = nullptr;
    d.st = dev->st.p;
    d.b = hbufs;
    return d;
}

// Step 0 of the algorithm box (y_1 = I_0 = x0, t_1 = 1) and the start of the
// power iteration (x = 1/sqrt(n_pix)); phase PINIT when L is to be computed,
// SINIT when it is given.
int sl1m_problem::init_solve(const sl1m_solve_opts* o, double L, bool power_only, cudaStream_t st)
{
    RET(ensure_solver(st));
    ProblemDev& D = *dev;
    double l1_0 = 0.0;
    const size_t np = hp.pix.n_pad;
    if (o && o->x0) {
        CK(D.x_user.reserve(n_pix, st));
        CK(cudaMemcpyAsync(D.x_user.p, o->x0, sizeof(double) * n_pix, cudaMemcpyHostToDevice, st));
        CKL(launch_gather_real(D.x_user.p, D.I0.p, hp.pix.orig, hp.pix.n_pad, 1.0, st));
        for (int64_t j = 0; j < n_pix; ++j) l1_0 += o->x0[j];
        ctx->h2d += (long long)sizeof(double) * n_pix;
    } else {
        CK(cudaMemsetAsync(D.I0.p, 0, sizeof(double) * np, st));
    }
    CK(cudaMemcpyAsync(D.y.p, D.I0.p, sizeof(double) * np, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(D.I1.p, D.I0.p, sizeof(double) * np, cudaMemcpyDeviceToDevice, st));
    CKL(launch_fill_valid(D.xv.p, hp.pix.orig, hp.pix.n_pad, 1.0 / std::sqrt((double)n_pix), st));
    SolveState s0;
    memset(&s0, 0, sizeof s0);
    s0.lambda = o ? o->lambda : 0.0;
    s0.L = L;
    s0.tol = o ? o->rel_tol : 0.0;
    s0.t = 1.0;
    s0.l1 = l1_0;
    s0.max_iter = o ? o->max_iter : 0;
    s0.inv_mu = 1.0;
    s0.pmax = (o && o->power_max_iter > 0) ? o->power_max_iter : 50;
    s0.ptol = (o && o->power_tol > 0) ? o->power_tol : 1e-6;
    s0.power_only = power_only ? 1 : 0;
    s0.algo = (o && o->algorithm == SL1M_MFISTA && !power_only) ? 1 : 0;
    algo = s0.algo;
    if (o && o->x0)
        for (int64_t j = 0; j < n_pix; ++j) s0.nnz += o->x0[j] > 0.0;
    s0.phase = (L > 0.0 && !power_only) ? PH_SINIT : PH_PINIT;
    CK(cudaMemcpyAsync(D.st.p, &s0, sizeof s0, cudaMemcpyHostToDevice, st));
    // the host struct is a temporary: finish the copy before returning
    CK(cudaStreamSynchronize(st));
    return SL1M_OK;
}

int sl1m_problem::read_state(SolveState& s, cudaStream_t st)
{
    CK(cudaMemcpyAsync(&s, dev->st.p, sizeof s, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return SL1M_OK;
}

// Copy the last I_k (sorted, in I[k & 1]) to the caller's order on the host.
int sl1m_problem::fetch_image(double* host_out, cudaStream_t st)
{
    SolveState s;
    RET(read_state(s, st));
    ProblemDev& D = *dev;
    double* Ik = (!s.algo && (s.k & 1)) ? D.I1.p : D.I0.p;   // MFISTA: x_k lives in I[0]
    CK(D.img_user.reserve(n_pix, st));
    CKL(launch_scatter_real(Ik, D.img_user.p, hp.pix.orig, hp.pix.n_pad, st));
    CK(cudaMemcpyAsync(host_out, D.img_user.p, sizeof(double) * n_pix, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    ctx->d2h += (long long)sizeof(double) * n_pix;
    return SL1M_OK;
}

size_t sl1m_problem::dev_bytes() const
{
    if (!dev) return 0;
    const ProblemDev& D = *dev;
    size_t b = 0;
    auto side = [&](const DevSide& s) {
        b += s.hi.bytes() + s.lo.bytes() + s.off.bytes() + s.offlo.bytes() + s.cen_hi.bytes() +
             s.cen_lo.bytes() + s.ext.bytes() + s.d.bytes() + s.orig.bytes();
    };
    side(D.vis);
    side(D.pix);
    b += D.ant.bytes() + D.vgabs.bytes() + D.r32.bytes() + D.vslot.bytes() + D.gbl.bytes() + D.gnb.bytes() + D.V.bytes() + D.pgauss.bytes() + D.pgauss64.bytes() + D.gsig.bytes() +
         D.gsig64.bytes() + D.gkind.bytes() + D.pghdr.bytes() + D.gpol32.bytes() + D.gains64.bytes();
    b += D.x_user.bytes() + D.x_sorted.bytes() + D.adj_sorted.bytes() + D.img_user.bytes() +
         D.r_user.bytes() + D.r_sorted.bytes() + D.fwd_sorted.bytes() + D.vis_user.bytes();
    b += D.I0.bytes() + D.I1.bytes() + D.y.bytes() + D.xv.bytes() + D.blk_r2.bytes() + D.blk_l1.bytes() +
         D.blk_z2.bytes() + D.AI0.bytes() + D.AI1.bytes() + D.rr.bytes() + D.blk_nnz.bytes() +
         D.blk_badv.bytes() + D.blk_badp.bytes() + D.st.bytes();
    return b;
}

long long tune_key(int precision, int op, bool gains, bool gauss, long long units)
{
    int lg = 0;
    while (units > 1 && lg < 62) { units >>= 1; ++lg; }
    return ((long long)precision << 12) | ((long long)op << 11) | ((long long)gains << 10) |
           ((long long)gauss << 9) | lg;
}

// ================================================================ batches

Batch::~Batch()
{
    if (gexec) cudaGraphExecDestroy(gexec);
}

// Set the problems of a batch: descriptors, per (op, gains class) plans,
// partial-sum scratch.  The captured tick stays valid while every pointer it
// bakes in (tables, scratch) is unchanged.
int batch_set(sl1m_ctx* ctx, Batch& B, const std::vector<sl1m_problem*>& probs,
              const std::vector<DevProblem>& descs, int precision, bool solver)
{
    cudaStream_t st = ctx->stream;
    const int np = (int)probs.size();
    if (np == 0) return sl1m_fail(ctx, SL1M_ERR_ARG, "empty batch");
    const void* old_ptrs[6] = {B.desc.p, ctx->partial_f.p, ctx->partial_a.p, B.n_probs_dev.p,
                               B.plan[0][0].dpl.p, B.plan[1][1].dpl.p};
    const bool same_set = B.probs == probs && B.precision == precision && B.solver == solver;
    B.precision = precision;
    B.solver = solver;
    B.probs = probs;
    B.hdesc = descs;
    if (B.desc.n < (size_t)np) CK(B.desc.reserve(np, st));
    CK(cudaMemcpyAsync(B.desc.p, B.hdesc.data(), sizeof(DevProblem) * np, cudaMemcpyHostToDevice, st));
    if (!B.n_probs_dev.p) CK(B.n_probs_dev.alloc(1));
    CK(cudaMemcpyAsync(B.n_probs_dev.p, &np, sizeof(int), cudaMemcpyHostToDevice, st));
    if (B.phases_dev.n < (size_t)np) CK(B.phases_dev.reserve(np, st));
    if (!same_set) {
        B.has_class[0] = B.has_class[1] = false;
        B.n_ant_max = 0;
        B.pairs_class[0] = B.pairs_class[1] = 0;
        B.fin_bytes[0] = B.fin_bytes[1] = 0;
        for (int c = 0; c < 2; ++c) {
            std::vector<int> nbf(np), nsf(np), nba(np), nsa(np);
            for (int p = 0; p < np; ++p) {
                const bool g = probs[p]->n_ant > 0;
                const bool in = (c == 1) == g;
                const DevProblem& d = descs[p];
                nbf[p] = in ? d.vis.n_blk : 0;
                nsf[p] = in ? d.pix.n_gran : 0;
                nba[p] = in ? d.pix.n_blk : 0;
                nsa[p] = in ? d.vis.n_gran : 0;
                if (in) {
                    B.has_class[c] = true;
                    B.pairs_class[c] += probs[p]->pairs();
                    if (g) B.n_ant_max = std::max(B.n_ant_max, probs[p]->n_ant);
                }
            }
            // tile shape and grid: autotuned choice for this shape, else the default
            bool gauss = false;
            long long uf = 0, ua = 0;
            for (int p = 0; p < np; ++p) {
                gauss |= probs[p]->has_gauss && nbf[p] > 0;
                uf += (long long)nbf[p] * nsf[p];
                ua += (long long)nba[p] * nsa[p];
            }
            int kf = 0, ka = 0;
            B.nst[0][c] = B.nst[1][c] = NST_DEFAULT;
            const auto tf = ctx->tune.find(tune_key(precision, 0, c == 1, gauss, uf));
            const auto ta = ctx->tune.find(tune_key(precision, 1, c == 1, gauss, ua));
            if (tf != ctx->tune.end()) { B.nst[0][c] = tf->second.first; kf = tf->second.second; }
            if (ta != ctx->tune.end()) { B.nst[1][c] = ta->second.first; ka = ta->second.second; }
            if (precision != 0 && c == 0) {         // no Gaussian pixels: the Dirac-only instances
                B.nst[0][c] = shape_for(B.nst[0][c], gauss);
                B.nst[1][c] = shape_for(B.nst[1][c], gauss);
            }
            const int occf = occupancy(precision == 0 ? 0 : 2, c == 1, std::max(1, B.n_ant_max), B.nst[0][c]);
            const int occa = occupancy(precision == 0 ? 1 : 3, c == 1, std::max(1, B.n_ant_max), B.nst[1][c]);
            kf = kf > 0 ? std::min(kf, occf) : occf;
            ka = ka > 0 ? std::min(ka, occa) : occa;
            std::vector<const UnitCost*> cf(np), ca(np);
            for (int p = 0; p < np; ++p) {
                cf[p] = &probs[p]->unit_cost(precision == 0 ? 0 : 1, 0);
                ca[p] = &probs[p]->unit_cost(precision == 0 ? 0 : 1, 1);
            }
            CK(build_plan(nbf, nsf, ctx->num_sms * kf, B.plan[0][c], st, &cf));
            CK(build_plan(nba, nsa, ctx->num_sms * ka, B.plan[1][c], st, &ca));
            CK(ctx->partial_f.reserve((size_t)std::max(1, B.plan[0][c].pl.n_slots) * BLK, st));
            CK(ctx->partial_a.reserve((size_t)std::max(1, B.plan[1][c].pl.n_slots) * BLK, st));
            B.fin_bytes[0] += (double)B.plan[0][c].pl.n_slots * BLK * 16.0;
            B.fin_bytes[1] += (double)B.plan[1][c].pl.n_slots * BLK * 8.0;
        }
        int nblk = 0;
        for (int p = 0; p < np; ++p) {
            nblk = std::max({nblk, descs[p].vis.n_blk, descs[p].pix.n_blk});
            B.fin_bytes[0] += descs[p].vis.n_pad * (solver ? 16.0 * 5 + 32 : 48.0);
            B.fin_bytes[1] += descs[p].pix.n_pad * (solver ? 8.0 * 5 + 4 : 8.0);
        }
        B.fin_grid = std::max(1, std::min(4 * ctx->num_sms, nblk * np));
        B.sc_grid = std::max(1, std::min(ctx->num_sms * 4, np));
    }
    const void* new_ptrs[6] = {B.desc.p, ctx->partial_f.p, ctx->partial_a.p, B.n_probs_dev.p,
                               B.plan[0][0].dpl.p, B.plan[1][1].dpl.p};
    if (!same_set || memcmp(old_ptrs, new_ptrs, sizeof old_ptrs) != 0) B.graph_ok = false;
    return SL1M_OK;
}

static int launch_op_class(sl1m_ctx* ctx, Batch& B, int op, int c)
{
    if (!B.has_class[c]) return SL1M_OK;
    cudaStream_t st = ctx->stream;
    const DevPlan& P = B.plan[op][c];
    ProfTok tk;
    if (op == 0) {
        prof_begin(ctx, B.precision == 0 ? 0 : 2, tk);
        CKL(launch_forward(B.precision, c == 1, B.n_ant_max, B.desc.p, P.dpl.p, P.pl.C, ctx->partial_f.p, st,
                           B.nst[0][c]));
        prof_end(ctx, tk, B.solver ? 0.0 : B.pairs_class[c], 0.0);   // solver ticks: counted on the device
        prof_begin(ctx, 4, tk);
        CKL(launch_fwd_finish(B.desc.p, P.dpl.p, std::min(B.fin_grid, std::max(1, P.pl.n_blocks)),
                              ctx->partial_f.p, st));
        prof_end(ctx, tk, 0.0, B.fin_bytes[0]);
    } else {
        // the mixed adjoints read r in polar form, written once for the whole
        // batch before its first class
        if (B.precision != 0 && (c == 0 || !B.has_class[0])) {
            int vmax = 1;
            for (const DevProblem& d : B.hdesc) vmax = std::max(vmax, d.vis.n_pad);
            CKL(launch_r32(B.desc.p, (int)B.hdesc.size(), vmax, st));
        }
        prof_begin(ctx, B.precision == 0 ? 1 : 3, tk);
        CKL(launch_adjoint(B.precision, c == 1, B.n_ant_max, B.desc.p, P.dpl.p, P.pl.C, ctx->partial_a.p, st,
                           B.nst[1][c]));
        prof_end(ctx, tk, B.solver ? 0.0 : B.pairs_class[c], 0.0);
        prof_begin(ctx, 5, tk);
        CKL(launch_adj_finish(B.desc.p, P.dpl.p, std::min(B.fin_grid, std::max(1, P.pl.n_blocks)),
                              ctx->partial_a.p, st));
        prof_end(ctx, tk, 0.0, B.fin_bytes[1]);
    }
    return SL1M_OK;
}

// One operator application (operator-mode batch): forward or adjoint.
int batch_op(sl1m_ctx* ctx, Batch& B, int op)
{
    for (int c = 0; c < 2; ++c) RET(launch_op_class(ctx, B, op, c));
    return SL1M_OK;
}

// One tick of every solve of a solver-mode batch: adjoint, adjoint finish,
// forward, forward finish (per gains class), then the phase machine.
static int enqueue_tick(sl1m_ctx* ctx, Batch& B)
{
    for (int c = 0; c < 2; ++c) RET(launch_op_class(ctx, B, 1, c));
    for (int c = 0; c < 2; ++c) RET(launch_op_class(ctx, B, 0, c));
    // while profiling (ticks are launched directly then, never captured) the
    // scalars kernel counts the pairs the tick evaluated
    double* ev = (ctx->prof && B.solver && ctx->evals_dev.p) ? ctx->evals_dev.p + 2 * (B.precision != 0) : nullptr;
    CKL(launch_scalars(B.desc.p, B.n_probs_dev.p, B.sc_grid, ev, ctx->stream));
    if (B.has_mfista) {
        ProfTok tk;
        prof_begin(ctx, 6, tk);
        for (int c = 0; c < 2; ++c) {
            if (!B.has_class[c]) continue;
            const int nb = B.plan[0][c].pl.n_blocks + B.plan[1][c].pl.n_blocks;
            CKL(launch_mfista_mix(B.desc.p, B.plan[0][c].dpl.p, B.plan[1][c].dpl.p,
                                  std::min(B.fin_grid, std::max(1, nb)), ctx->stream));
        }
        prof_end(ctx, tk, 0.0, 0.0);
    }
    return SL1M_OK;
}

// n ticks; replayed from a captured CUDA graph unless profiling (events per
// kernel) or graphs are off.
int batch_ticks(sl1m_ctx* ctx, Batch& B, int n)
{
    bool hm = false;
    if (B.solver)
        for (const sl1m_problem* p : B.probs) hm = hm || p->algo == 1;
    if (hm != B.has_mfista) {
        B.has_mfista = hm;
        B.graph_ok = false;
    }
    if (!ctx->use_graphs || ctx->prof) {
        for (int i = 0; i < n; ++i) RET(enqueue_tick(ctx, B));
        return SL1M_OK;
    }
    // The captured tick bakes in the context's partial-sum scratch, which a
    // larger batch (another problem's solve or operator call, the autotuner)
    // may have reallocated since: capture again rather than replay with a
    // freed buffer.  The scratch only grows, so it still fits this batch.
    if (B.graph_ok && (B.cap_partial[0] != ctx->partial_f.p || B.cap_partial[1] != ctx->partial_a.p))
        B.graph_ok = false;
    if (!B.graph_ok) {
        if (B.gexec) {
            cudaGraphExecDestroy(B.gexec);
            B.gexec = nullptr;
        }
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        const long long l0 = ctx->n_launch;
        const int rc = enqueue_tick(ctx, B);
        const cudaError_t ec = cudaStreamEndCapture(ctx->stream, &g);
        if (rc != SL1M_OK || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (rc != SL1M_OK) return rc;
            CK(ec);
        }
        const cudaError_t ei = cudaGraphInstantiate(&B.gexec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) B.gexec = nullptr;
        CK(ei);
        B.graph_ok = true;
        B.cap_partial[0] = ctx->partial_f.p;
        B.cap_partial[1] = ctx->partial_a.p;
        B.tick_launches = ctx->n_launch - l0;
        ctx->n_launch = l0;
    }
    for (int i = 0; i < n; ++i) {
        CK(cudaGraphLaunch(B.gexec, ctx->stream));
        ctx->n_launch += B.tick_launches;
    }
    return SL1M_OK;
}

// A gains kernel's bounded wait for a bulk copy gave up (the flag was read
// on the context's stream before its last synchronisation): the results of
// the launches since the previous check are invalid.
static int check_wait_fault(sl1m_ctx* ctx, unsigned fault)
{
    if (!fault) return SL1M_OK;
    CK(wait_fault_clear(ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return sl1m_fail(ctx, SL1M_ERR_CUDA, "a bulk copy into shared memory did not complete within the kernel's "
                                         "bounded wait; the results of this call are invalid");
}

int batch_phases(sl1m_ctx* ctx, Batch& B, std::vector<int>& out)
{
    const int np = (int)B.probs.size();
    out.resize(np);
    CKL(launch_phases(B.desc.p, B.n_probs_dev.p, std::max(1, std::min(64, (np + 127) / 128)), B.phases_dev.p,
                      ctx->stream));
    CK(cudaMemcpyAsync(out.data(), B.phases_dev.p, sizeof(int) * np, cudaMemcpyDeviceToHost, ctx->stream));
    unsigned fault = 0;
    CK(wait_fault_read(&fault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return check_wait_fault(ctx, fault);
}

// Operator-mode batch of a single problem (cached per precision).
static int op_prepare(sl1m_problem* prob, int precision, Batch** out)
{
    sl1m_ctx* ctx = prob->ctx;
    RET(prob->rebuild(ctx->stream));
    auto& B = prob->op_batch[precision];
    if (!B) B = std::make_unique<Batch>();
    ProblemDev& D = *prob->dev;
    CK(D.x_sorted.reserve(prob->hp.pix.n_pad, ctx->stream));
    CK(D.fwd_sorted.reserve(prob->hp.vis.n_pad, ctx->stream));
    CK(D.r_sorted.reserve(prob->hp.vis.n_pad, ctx->stream));
    CK(D.adj_sorted.reserve(prob->hp.pix.n_pad, ctx->stream));
    DevProblem d = prob->hp;
    d.st = nullptr;
    d.x = D.x_sorted.p;
    d.r = D.r_sorted.p;
    d.fwd_out = D.fwd_sorted.p;
    d.adj_out = D.adj_sorted.p;
    if (B->probs.empty() || memcmp(&B->hdesc[0], &d, sizeof d) != 0)
        RET(batch_set(ctx, *B, {prob}, {d}, precision, false));
    *out = B.get();
    return SL1M_OK;
}

// Run a single solve (or the power iteration alone) to completion.
static int run_single(sl1m_problem* prob, int precision, int max_ticks, SolveState& s)
{
    sl1m_ctx* ctx = prob->ctx;
    auto& B = prob->solve_batch[precision];
    if (!B) B = std::make_unique<Batch>();
    const DevProblem d = prob->solver_desc();
    if (B->probs.empty() || memcmp(&B->hdesc[0], &d, sizeof d) != 0)
        RET(batch_set(ctx, *B, {prob}, {d}, precision, true));
    const int check = 8;
    std::vector<int> ph;
    int issued = 0;
    while (issued < max_ticks) {
        const int n = std::min(check, max_ticks - issued);
        RET(batch_ticks(ctx, *B, n));
        issued += n;
        RET(batch_phases(ctx, *B, ph));
        if (ph[0] == PH_DONE || ph[0] == PH_IDLE) break;
    }
    return prob->read_state(s, ctx->stream);
}

// ================================================================ C ABI
extern "C" {

int sl1m_version(void) { return 200; }

const char* sl1m_status_string(int s)
{
    switch (s) {
    case SL1M_OK: return "ok";
    case SL1M_ERR_ARG: return "invalid argument";
    case SL1M_ERR_OOM: return "out of memory";
    case SL1M_ERR_CUDA: return "CUDA error";
    case SL1M_ERR_NONFINITE: return "non-finite value";
    case SL1M_ERR_TIMEOUT: return "timeout";
    case SL1M_ERR_BUSY: return "busy (admission refused)";
    case SL1M_ERR_STATE: return "problem incomplete";
    default: return "unknown status";
    }
}

int sl1m_create(sl1m_ctx** out, int device, void* cuda_stream)
{
    if (!out) return SL1M_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return SL1M_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return SL1M_ERR_CUDA;
    auto* c = new (std::nothrow) sl1m_ctx();
    if (!c) return SL1M_ERR_OOM;
    c->device = device;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { delete c; return SL1M_ERR_CUDA; }
    c->num_sms = prop.multiProcessorCount;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
        c->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return SL1M_ERR_CUDA;
        }
        c->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&c->upstream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return SL1M_ERR_CUDA;
    }
    *out = c;
    return SL1M_OK;
}

int sl1m_destroy(sl1m_ctx* ctx)
{
    if (!ctx) return SL1M_ERR_ARG;
    cudaSetDevice(ctx->device);
    server_destroy(ctx);
    cudaStreamSynchronize(ctx->stream);
    for (auto* p : ctx->problems) delete p;
    ctx->problems.clear();
    delete ctx;
    return SL1M_OK;
}

// A copy per calling thread, so that a message the server thread writes
// meanwhile cannot invalidate the pointer returned here.
const char* sl1m_last_error(const sl1m_ctx* ctx)
{
    if (!ctx) return "null context";
    thread_local std::string copy;
    std::lock_guard<std::mutex> lk(ctx->err_mu);
    copy = ctx->err;
    return copy.c_str();
}

#define NOT_WHILE_SERVING(ctx)                                                                   \
    do {                                                                                         \
        if ((ctx)->server) return sl1m_fail(ctx, SL1M_ERR_BUSY, "a server is running on this context"); \
    } while (0)

int sl1m_problem_create(sl1m_ctx* ctx, sl1m_problem** out)
{
    if (!ctx || !out) return sl1m_fail(ctx, SL1M_ERR_ARG, "null argument");
    auto* p = new (std::nothrow) sl1m_problem();
    if (!p) return sl1m_fail(ctx, SL1M_ERR_OOM, "host allocation failed");
    p->ctx = ctx;
    memset(&p->hp, 0, sizeof p->hp);
    ctx->problems.push_back(p);
    *out = p;
    return SL1M_OK;
}

int sl1m_problem_destroy(sl1m_problem* prob)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    if (prob->in_server) return sl1m_fail(ctx, SL1M_ERR_BUSY, "problem is queued on the server");
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    ctx->problems.erase(std::remove(ctx->problems.begin(), ctx->problems.end(), prob), ctx->problems.end());
    delete prob;
    return SL1M_OK;
}

static bool all_finite(const double* a, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

#define NOT_QUEUED(prob)                                                                           \
    do {                                                                                           \
        if ((prob)->in_server) return sl1m_fail((prob)->ctx, SL1M_ERR_BUSY, "problem is queued on the server"); \
    } while (0)

int sl1m_set_visibilities(sl1m_problem* prob, int64_t n_vis, const double* uvw, const double* vis,
                          const double* weights, const int32_t* ant_pair)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    NOT_QUEUED(prob);
    if (n_vis <= 0 || !uvw) return sl1m_fail(ctx, SL1M_ERR_ARG, "n_vis must be > 0 and uvw non-null");
    if (n_vis > (int64_t)1 << 30) return sl1m_fail(ctx, SL1M_ERR_ARG, "n_vis too large");
    if (!all_finite(uvw, 3 * n_vis)) return sl1m_fail(ctx, SL1M_ERR_ARG, "non-finite uvw");
    if (vis && !all_finite(vis, 2 * n_vis)) return sl1m_fail(ctx, SL1M_ERR_ARG, "non-finite visibilities");
    if (weights) {
        for (int64_t k = 0; k < n_vis; ++k)
            if (!std::isfinite(weights[k]) || weights[k] < 0)
                return sl1m_fail(ctx, SL1M_ERR_ARG, "weights must be finite and >= 0");
    }
    if (ant_pair) {
        for (int64_t k = 0; k < 2 * n_vis; ++k)
            if (ant_pair[k] < 0) return sl1m_fail(ctx, SL1M_ERR_ARG, "negative antenna index");
    }
    prob->n_vis = n_vis;
    prob->uvw.assign(uvw, uvw + 3 * n_vis);
    if (vis) prob->vis.assign(vis, vis + 2 * n_vis);
    else prob->vis.assign(2 * n_vis, 0.0);
    if (weights) prob->weights.assign(weights, weights + n_vis);
    else prob->weights.clear();
    if (ant_pair) prob->ant.assign(ant_pair, ant_pair + 2 * n_vis);
    else prob->ant.clear();
    prob->dirty = true;
    return SL1M_OK;
}

int sl1m_set_vis_data(sl1m_problem* prob, const double* vis)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    NOT_QUEUED(prob);
    if (!vis || prob->n_vis <= 0) return sl1m_fail(ctx, SL1M_ERR_ARG, "no visibilities set");
    if (!all_finite(vis, 2 * prob->n_vis)) return sl1m_fail(ctx, SL1M_ERR_ARG, "non-finite visibilities");
    prob->vis.assign(vis, vis + 2 * prob->n_vis);
    if (!prob->dirty && prob->dev) {
        cudaSetDevice(ctx->device);
        std::vector<double2> Vs(prob->hp.vis.n_pad, make_double2(0.0, 0.0));
        for (int i = 0; i < prob->hp.vis.n_pad; ++i) {
            const int o = prob->vis_orig[i];
            if (o >= 0) Vs[i] = make_double2(vis[2 * o], vis[2 * o + 1]);
        }
        // same size: copy in place so descriptors and captured graphs stay valid
        CK(cudaMemcpyAsync(prob->dev->V.p, Vs.data(), sizeof(double2) * Vs.size(), cudaMemcpyHostToDevice,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        ctx->h2d += (long long)sizeof(double2) * Vs.size();
    }
    return SL1M_OK;
}

int sl1m_set_pixels(sl1m_problem* prob, int64_t n_pix, const double* lm, const double* sigma,
                    const int32_t* kind)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    NOT_QUEUED(prob);
    if (n_pix <= 0 || !lm) return sl1m_fail(ctx, SL1M_ERR_ARG, "n_pix must be > 0 and lm non-null");
    if (n_pix > (int64_t)1 << 30) return sl1m_fail(ctx, SL1M_ERR_ARG, "n_pix too large");
    for (int64_t j = 0; j < n_pix; ++j) {
        const double l = lm[2 * j], m = lm[2 * j + 1];
        if (!std::isfinite(l) || !std::isfinite(m) || !(l * l + m * m < 1.0))
            return sl1m_fail(ctx, SL1M_ERR_ARG, "pixel %lld outside the sky (l^2+m^2 >= 1)", (long long)j);
        const int k = kind ? kind[j] : 0;
        if (k < 0 || k > 2) return sl1m_fail(ctx, SL1M_ERR_ARG, "bad pixel kind %d", k);
        const double s = sigma ? sigma[j] : 0.0;
        if (!std::isfinite(s) || s < 0) return sl1m_fail(ctx, SL1M_ERR_ARG, "sigma must be finite and >= 0");
        if (k != 0 && !(s > 0)) return sl1m_fail(ctx, SL1M_ERR_ARG, "Gaussian pixel needs sigma > 0");
    }
    prob->n_pix = n_pix;
    prob->lm.assign(lm, lm + 2 * n_pix);
    if (sigma) prob->sigma.assign(sigma, sigma + n_pix);
    else prob->sigma.clear();
    if (kind) {
        prob->kind.assign(kind, kind + n_pix);
        if (!prob->sigma.empty())            // Dirac pixels ignore sigma: one class for all
            for (int64_t j = 0; j < n_pix; ++j)
                if (prob->kind[j] == 0) prob->sigma[j] = 0.0;
    } else {
        prob->kind.clear();
        prob->sigma.clear();
    }
    if (prob->n_ant > 0 && (int64_t)prob->gains.size() != 2 * n_pix * prob->n_ant) {
        prob->n_ant = 0;
        prob->gains.clear();
    }
    prob->dirty = true;
    return SL1M_OK;
}

int sl1m_set_gains(sl1m_problem* prob, int32_t n_ant, const double* Gn)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    NOT_QUEUED(prob);
    if (!Gn || n_ant == 0) {
        prob->n_ant = 0;
        prob->gains.clear();
        prob->dirty = true;
        return SL1M_OK;
    }
    if (n_ant < 0 || n_ant > 300) return sl1m_fail(ctx, SL1M_ERR_ARG, "n_ant must be in [1, 300]");
    if (prob->n_pix <= 0) return sl1m_fail(ctx, SL1M_ERR_STATE, "set pixels before gains");
    const size_t cnt = (size_t)2 * prob->n_pix * n_ant;
    if (!all_finite(Gn, cnt)) return sl1m_fail(ctx, SL1M_ERR_ARG, "non-finite gains");
    prob->n_ant = n_ant;
    prob->gains.assign(Gn, Gn + cnt);
    prob->dirty = true;
    return SL1M_OK;
}

static int check_prec(sl1m_ctx* ctx, int precision)
{
    if (precision != SL1M_FP64 && precision != SL1M_MIXED)
        return sl1m_fail(ctx, SL1M_ERR_ARG, "precision must be SL1M_FP64 or SL1M_MIXED");
    return SL1M_OK;
}

int sl1m_forward_dev(sl1m_problem* prob, const double* x_dev, double* vis_out_dev, int precision)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    NOT_WHILE_SERVING(ctx);
    if (!x_dev || !vis_out_dev) return sl1m_fail(ctx, SL1M_ERR_ARG, "null pointer");
    RET(check_prec(ctx, precision));
    CK(cudaSetDevice(ctx->device));
    Batch* B;
    RET(op_prepare(prob, precision, &B));
    ProblemDev& D = *prob->dev;
    CKL(launch_gather_real(x_dev, D.x_sorted.p, prob->hp.pix.orig, prob->hp.pix.n_pad, 1.0, ctx->stream));
    RET(batch_op(ctx, *B, 0));
    CKL(launch_scatter_cplx(D.fwd_sorted.p, (double2*)vis_out_dev, prob->hp.vis.orig, prob->hp.vis.n_pad,
                            ctx->stream));
    return SL1M_OK;
}

int sl1m_adjoint_dev(sl1m_problem* prob, const double* r_dev, double* img_out_dev, int precision)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    NOT_WHILE_SERVING(ctx);
    if (!r_dev || !img_out_dev) return sl1m_fail(ctx, SL1M_ERR_ARG, "null pointer");
    RET(check_prec(ctx, precision));
    CK(cudaSetDevice(ctx->device));
    Batch* B;
    RET(op_prepare(prob, precision, &B));
    ProblemDev& D = *prob->dev;
    CKL(launch_gather_cplx((const double2*)r_dev, D.r_sorted.p, prob->hp.vis.orig, prob->hp.vis.n_pad,
                           ctx->stream));
    RET(batch_op(ctx, *B, 1));
    CKL(launch_scatter_real(D.adj_sorted.p, img_out_dev, prob->hp.pix.orig, prob->hp.pix.n_pad, ctx->stream));
    return SL1M_OK;
}

int sl1m_forward(sl1m_problem* prob, const double* x, double* vis_out, int precision)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    NOT_WHILE_SERVING(ctx);
    if (!x || !vis_out) return sl1m_fail(ctx, SL1M_ERR_ARG, "null pointer");
    if (!all_finite(x, prob->n_pix > 0 ? prob->n_pix : 0)) return sl1m_fail(ctx, SL1M_ERR_ARG, "non-finite x");
    CK(cudaSetDevice(ctx->device));
    RET(prob->rebuild(ctx->stream));
    ProblemDev& D = *prob->dev;
    CK(D.x_user.reserve(prob->n_pix, ctx->stream));
    CK(D.vis_user.reserve(prob->n_vis, ctx->stream));
    CK(cudaMemcpyAsync(D.x_user.p, x, sizeof(double) * prob->n_pix, cudaMemcpyHostToDevice, ctx->stream));
    RET(sl1m_forward_dev(prob, D.x_user.p, (double*)D.vis_user.p, precision));
    CK(cudaMemcpyAsync(vis_out, D.vis_user.p, sizeof(double2) * prob->n_vis, cudaMemcpyDeviceToHost, ctx->stream));
    unsigned fault = 0;
    CK(wait_fault_read(&fault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    RET(check_wait_fault(ctx, fault));
    ctx->h2d += (long long)sizeof(double) * prob->n_pix;
    ctx->d2h += (long long)sizeof(double2) * prob->n_vis;
    return SL1M_OK;
}

int sl1m_adjoint(sl1m_problem* prob, const double* r, double* img_out, int precision)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    NOT_WHILE_SERVING(ctx);
    if (!r || !img_out) return sl1m_fail(ctx, SL1M_ERR_ARG, "null pointer");
    if (!all_finite(r, prob->n_vis > 0 ? 2 * prob->n_vis : 0)) return sl1m_fail(ctx, SL1M_ERR_ARG, "non-finite r");
    CK(cudaSetDevice(ctx->device));
    RET(prob->rebuild(ctx->stream));
    ProblemDev& D = *prob->dev;
    CK(D.r_user.reserve(prob->n_vis, ctx->stream));
    CK(D.img_user.reserve(prob->n_pix, ctx->stream));
    CK(cudaMemcpyAsync(D.r_user.p, r, sizeof(double2) * prob->n_vis, cudaMemcpyHostToDevice, ctx->stream));
    RET(sl1m_adjoint_dev(prob, (const double*)D.r_user.p, D.img_user.p, precision));
    CK(cudaMemcpyAsync(img_out, D.img_user.p, sizeof(double) * prob->n_pix, cudaMemcpyDeviceToHost, ctx->stream));
    unsigned fault = 0;
    CK(wait_fault_read(&fault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    RET(check_wait_fault(ctx, fault));
    ctx->h2d += (long long)sizeof(double2) * prob->n_vis;
    ctx->d2h += (long long)sizeof(double) * prob->n_pix;
    return SL1M_OK;
}

int sl1m_dirty_image(sl1m_problem* prob, int precision, double* img_out, double* lambda_max_out)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    NOT_WHILE_SERVING(ctx);
    if (!img_out && !lambda_max_out) return sl1m_fail(ctx, SL1M_ERR_ARG, "null pointer");
    RET(check_prec(ctx, precision));
    CK(cudaSetDevice(ctx->device));
    Batch* B;
    RET(op_prepare(prob, precision, &B));
    ProblemDev& D = *prob->dev;
    cudaStream_t st = ctx->stream;
    CKL(launch_weighted_vis(prob->hp.V, prob->hp.vis.d, D.r_sorted.p, prob->hp.vis.n_pad, st));
    RET(batch_op(ctx, *B, 1));
    CK(D.img_user.reserve(prob->n_pix, st));
    CKL(launch_scatter_real(D.adj_sorted.p, D.img_user.p, prob->hp.pix.orig, prob->hp.pix.n_pad, st));
    std::vector<double> img(prob->n_pix);
    CK(cudaMemcpyAsync(img.data(), D.img_user.p, sizeof(double) * prob->n_pix, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    ctx->d2h += (long long)sizeof(double) * prob->n_pix;
    if (img_out) std::copy(img.begin(), img.end(), img_out);
    if (lambda_max_out) *lambda_max_out = *std::max_element(img.begin(), img.end());
    return SL1M_OK;
}

int sl1m_max_eig(sl1m_problem* prob, int max_iter, double tol, int precision, double* L_out, int* iters_out)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    NOT_WHILE_SERVING(ctx);
    if (!L_out || max_iter <= 0 || !(tol >= 0)) return sl1m_fail(ctx, SL1M_ERR_ARG, "bad arguments");
    RET(check_prec(ctx, precision));
    CK(cudaSetDevice(ctx->device));
    RET(prob->rebuild(ctx->stream));
    sl1m_solve_opts o;
    memset(&o, 0, sizeof o);
    o.power_max_iter = max_iter;
    o.power_tol = tol > 0 ? tol : 1e-300;
    RET(prob->init_solve(&o, 0.0, true, ctx->stream));
    SolveState s;
    RET(run_single(prob, precision, max_iter + 2, s));
    if (s.nonfinite) return sl1m_fail(ctx, SL1M_ERR_NONFINITE, "non-finite value in power iteration");
    if (!(s.mu > 0.0)) return sl1m_fail(ctx, SL1M_ERR_ARG, "operator is zero (all weights zero?)");
    *L_out = s.L > 0 ? s.L : s.mu;
    if (iters_out) *iters_out = s.pit;
    return SL1M_OK;
}

static int check_opts(sl1m_ctx* ctx, const sl1m_solve_opts* o)
{
    if (!(o->lambda >= 0) || !std::isfinite(o->lambda) || !(o->L >= 0) || !std::isfinite(o->L) ||
        o->max_iter < 0 || !(o->rel_tol >= 0) || o->power_max_iter < 0 || !(o->power_tol >= 0))
        return sl1m_fail(ctx, SL1M_ERR_ARG, "bad solver options");
    return check_prec(ctx, o->precision);
}

int sl1m_solve(sl1m_problem* prob, const sl1m_solve_opts* o, double* img_out, sl1m_solve_stats* stats)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    NOT_WHILE_SERVING(ctx);
    if (!o || !img_out) return sl1m_fail(ctx, SL1M_ERR_ARG, "null pointer");
    RET(check_opts(ctx, o));
    if (o->x0 && !all_finite(o->x0, prob->n_pix)) return sl1m_fail(ctx, SL1M_ERR_ARG, "non-finite x0");
    const auto t0 = std::chrono::steady_clock::now();
    CK(cudaSetDevice(ctx->device));
    RET(prob->rebuild(ctx->stream));
    RET(prob->init_solve(o, o->L, false, ctx->stream));
    const int pmax = o->power_max_iter > 0 ? o->power_max_iter : 50;
    SolveState s;
    RET(run_single(prob, o->precision, o->max_iter + (o->L > 0 ? 0 : pmax + 1) + 2, s));
    RET(prob->fetch_image(img_out, ctx->stream));
    if (stats) {
        stats->iters = s.k;
        stats->converged = s.converged;
        stats->E = s.E;
        stats->E_paper = s.resid2 + o->lambda * s.l1;
        stats->resid2 = s.resid2;
        stats->l1 = s.l1;
        stats->nnz = s.nnz;
        stats->L = s.L;
        stats->power_iters = s.pit;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (s.nonfinite) return sl1m_fail(ctx, SL1M_ERR_NONFINITE, "non-finite value during the solve");
    if (s.phase != PH_DONE) return sl1m_fail(ctx, SL1M_ERR_STATE, "solve did not finish");
    return SL1M_OK;
}

int sl1m_autotune(sl1m_problem* prob, int precision, int32_t* nst_out, int32_t* ctas_per_sm_out,
                  int32_t* npoly_out)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    NOT_WHILE_SERVING(ctx);
    RET(check_prec(ctx, precision));
    CK(cudaSetDevice(ctx->device));
    Batch* Bop;
    RET(op_prepare(prob, precision, &Bop));
    ProblemDev& D = *prob->dev;
    cudaStream_t st = ctx->stream;
    CK(cudaMemsetAsync(D.x_sorted.p, 0, sizeof(double) * prob->hp.pix.n_pad, st));
    CK(cudaMemsetAsync(D.r_sorted.p, 0, sizeof(double2) * prob->hp.vis.n_pad, st));
    const bool gains = prob->n_ant > 0;
    const DevProblem& d = Bop->hdesc[0];
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int rc = SL1M_OK;
    for (int op = 0; op < 2 && rc == SL1M_OK; ++op) {
        const std::vector<int> nb = {op == 0 ? d.vis.n_blk : d.pix.n_blk};
        const std::vector<int> ns = {op == 0 ? d.pix.n_gran : d.vis.n_gran};
        const std::vector<const UnitCost*> uc = {&prob->unit_cost(precision, op)};
        const long long units = (long long)nb[0] * ns[0];
        // stage 1: streamed granules per stage x CTAs per SM; stage 2: at the
        // best of those, the share of pairs whose sincos runs on the FMA pipe
        std::vector<int> cands = {NST_DEFAULT};
        const bool mixed_plain = precision == SL1M_MIXED && !gains;
        if (mixed_plain) cands = op == 0 ? std::vector<int>{2, 4, 8} : std::vector<int>{2, 4};
        float best = 1e30f;
        int bcode = NST_DEFAULT, bk = 0;
        const auto time_shape = [&](int code, int k) -> float {
            if (mixed_plain) code = shape_for(code, prob->has_gauss);
            DevPlan P;
            if (build_plan(nb, ns, ctx->num_sms * k, P, st, &uc) != cudaSuccess) { rc = SL1M_ERR_CUDA; return 0.f; }
            const size_t need = (size_t)std::max(1, P.pl.n_slots) * BLK;
            if ((op == 0 ? ctx->partial_f.reserve(need, st) : ctx->partial_a.reserve(need, st)) != cudaSuccess) {
                rc = SL1M_ERR_OOM;
                return 0.f;
            }
            // each timed launch follows a launch of the other operator, as in a
            // solver tick: a forward does not find the pixel stream the previous
            // forward left in L2, and shapes are ranked as a solve runs them
            float ms = 0.f;
            for (int rep = 0; rep < 4; ++rep) {
                const int rb = batch_op(ctx, *Bop, 1 - op);
                if (rb != SL1M_OK) { rc = rb; return 0.f; }
                cudaEventRecord(e0, st);
                cudaError_t e = op == 0 ? launch_forward(precision, gains, prob->n_ant, Bop->desc.p, P.dpl.p, P.pl.C,
                                                         ctx->partial_f.p, st, code)
                                        : launch_adjoint(precision, gains, prob->n_ant, Bop->desc.p, P.dpl.p, P.pl.C,
                                                         ctx->partial_a.p, st, code);
                if (e != cudaSuccess) { rc = SL1M_ERR_CUDA; return 0.f; }
                ctx->n_launch += 1;
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) { rc = SL1M_ERR_CUDA; return 0.f; }
                float m = 0.f;
                cudaEventElapsedTime(&m, e0, e1);
                if (rep > 0) ms += m;                // the first is a warm-up
            }
            return ms;
        };
        std::vector<int> kbest(cands.size(), 1);   // per stage count: its fastest grid at npoly 0
        for (size_t ci = 0; ci < cands.size(); ++ci) {
            const int nst = cands[ci];
            const int occ = occupancy((precision == SL1M_FP64 ? 0 : 2) + op, gains, std::max(1, prob->n_ant),
                                      mixed_plain ? shape_for(nst, prob->has_gauss) : nst);
            float bn = 1e30f;
            for (int k = 1; k <= occ && rc == SL1M_OK; ++k) {
                const float ms = time_shape(nst, k);
                if (rc == SL1M_OK && ms < bn) { bn = ms; kbest[ci] = k; }
                if (rc == SL1M_OK && ms < best) { best = ms; bcode = nst; bk = k; }
            }
        }
        // then npoly 1 and 2 at every stage count (with its grid): the stage
        // count that is fastest at npoly 0 need not be the fastest at npoly 1
        for (size_t ci = 0; mixed_plain && ci < cands.size() && rc == SL1M_OK; ++ci) {
            for (int npoly = 1; npoly <= 2 && rc == SL1M_OK; ++npoly) {
                const int code = shape_code(cands[ci], npoly);
                const int k = std::min(kbest[ci], occupancy(2 + op, false, 1, shape_for(code, prob->has_gauss)));
                const float ms = time_shape(code, k);
                if (rc == SL1M_OK && ms < best) { best = ms; bcode = code; bk = k; }
            }
        }
        if (rc != SL1M_OK) break;
        ctx->tune[tune_key(precision, op, gains, prob->has_gauss, units)] = {bcode, bk};
        if (nst_out) nst_out[op] = shape_nst(bcode);
        if (ctas_per_sm_out) ctas_per_sm_out[op] = bk;
        if (npoly_out) npoly_out[op] = shape_npoly(bcode);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // cached batches of this problem were built with the old choice
    for (auto& b : prob->op_batch) b.reset();
    for (auto& b : prob->solve_batch) b.reset();
    if (rc != SL1M_OK) return sl1m_fail(ctx, rc, "autotune failed");
    return SL1M_OK;
}

int sl1m_set_tile_shape(sl1m_problem* prob, int precision, int op, int nst, int ctas_per_sm, int npoly)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    NOT_WHILE_SERVING(ctx);
    RET(check_prec(ctx, precision));
    const bool gains = prob->n_ant > 0;
    if (op < 0 || op > 1 || ctas_per_sm < 1 || npoly < 0 || npoly > 2)
        return sl1m_fail(ctx, SL1M_ERR_ARG, "bad tile shape (op %d, ctas/SM %d, npoly %d)", op, ctas_per_sm, npoly);
    if (!(nst == 2 || nst == 4 || (nst == 8 && op == 0)))
        return sl1m_fail(ctx, SL1M_ERR_ARG, "nst must be 2, 4 or 8 (the adjoint: 2 or 4)");
    if ((gains || precision == SL1M_FP64) && (nst != NST_DEFAULT || npoly != 0))
        return sl1m_fail(ctx, SL1M_ERR_ARG, "with gains or in FP64 only the CTAs per SM can be set");
    RET(prob->rebuild(ctx->stream));
    const DevProblem& d = prob->hp;
    const long long units = op == 0 ? (long long)d.vis.n_blk * d.pix.n_gran : (long long)d.pix.n_blk * d.vis.n_gran;
    const int code = shape_code(nst, npoly);
    const int occ = occupancy((precision == SL1M_FP64 ? 0 : 2) + op, gains, std::max(1, prob->n_ant), code);
    if (ctas_per_sm > occ)
        return sl1m_fail(ctx, SL1M_ERR_ARG, "%d CTAs per SM do not fit (at most %d)", ctas_per_sm, occ);
    ctx->tune[tune_key(precision, op, gains, prob->has_gauss, units)] = {code, ctas_per_sm};
    for (auto& b : prob->op_batch) b.reset();
    for (auto& b : prob->solve_batch) b.reset();
    return SL1M_OK;
}

int sl1m_profile_enable(sl1m_ctx* ctx, int on)
{
    if (!ctx) return SL1M_ERR_ARG;
    if (on && !ctx->evals_dev.p) {
        CK(cudaSetDevice(ctx->device));
        CK(ctx->evals_dev.alloc(4));
        CK(cudaMemsetAsync(ctx->evals_dev.p, 0, 4 * sizeof(double), ctx->stream));
    }
    ctx->prof = on != 0;
    return SL1M_OK;
}

int sl1m_profile_reset(sl1m_ctx* ctx)
{
    if (!ctx) return SL1M_ERR_ARG;
    cudaSetDevice(ctx->device);
    ctx->drain_profile();
    for (int i = 0; i < NPROF; ++i) {
        ctx->prof_ms[i] = 0;
        ctx->prof_n[i] = 0;
        ctx->prof_pairs[i] = 0;
        ctx->prof_bytes[i] = 0;
    }
    return SL1M_OK;
}

int sl1m_profile_read(sl1m_ctx* ctx, int kid, double* ms, int64_t* launches, double* pairs, double* bytes)
{
    if (!ctx || kid < 0 || kid >= NPROF) return sl1m_fail(ctx, SL1M_ERR_ARG, "bad kernel id");
    cudaSetDevice(ctx->device);
    ctx->drain_profile();
    if (ms) *ms = ctx->prof_ms[kid];
    if (launches) *launches = ctx->prof_n[kid];
    if (pairs) *pairs = ctx->prof_pairs[kid];
    if (bytes) *bytes = ctx->prof_bytes[kid];
    return SL1M_OK;
}

int sl1m_plan_preview(int32_t n_probs, const int32_t* owned_blocks, const int32_t* streamed_granules,
                      int32_t max_ctas, const float* unit_costs, int32_t* n_ctas, int64_t* n_units,
                      int32_t* n_slots, int32_t* blk_first_cta, int32_t* blk_n_ctas, int32_t* blk_first_slot,
                      int64_t* cta_first_unit)
{
    if (n_probs <= 0 || !owned_blocks || !streamed_granules || max_ctas <= 0) return SL1M_ERR_ARG;
    std::vector<int> nb(n_probs), ns(n_probs);
    for (int p = 0; p < n_probs; ++p) {
        if (owned_blocks[p] < 0 || streamed_granules[p] < 0) return SL1M_ERR_ARG;
        nb[p] = owned_blocks[p];
        ns[p] = streamed_granules[p];
    }
    std::vector<UnitCost> uc(n_probs);
    std::vector<const UnitCost*> ucp(n_probs);
    if (unit_costs) {
        long long off = 0;
        for (int p = 0; p < n_probs; ++p) {
            const long long up = (long long)nb[p] * ns[p];
            for (long long k = 0; k < up; ++k)
                if (!(unit_costs[off + k] > 0.f) || !std::isfinite(unit_costs[off + k])) return SL1M_ERR_ARG;
            uc[p].unit.assign(unit_costs + off, unit_costs + off + up);
            ucp[p] = &uc[p];
            off += up;
        }
    }
    HostPlan H;
    plan_host(nb, ns, max_ctas, H, unit_costs ? &ucp : nullptr);
    if (n_ctas) *n_ctas = H.C;
    if (n_units) *n_units = H.U;
    if (n_slots) *n_slots = H.n_slots;
    for (int b = 0; b < H.n_blocks; ++b) {
        if (blk_first_cta) blk_first_cta[b] = H.clo[b];
        if (blk_n_ctas) blk_n_ctas[b] = H.ncon[b];
        if (blk_first_slot) blk_first_slot[b] = H.poff[b];
    }
    if (cta_first_unit)
        for (int c = 0; c <= H.C; ++c)
            cta_first_unit[c] = H.cta_u0.empty() ? (H.U * c) / H.C : H.cta_u0[c];
    return SL1M_OK;
}

int sl1m_granule_order(int64_t n, const double* xy, int32_t* order, int64_t* n_pad)
{
    if (n <= 0 || !xy || n > ((int64_t)1 << 30)) return SL1M_ERR_ARG;
    std::vector<int> members(n);
    for (int64_t i = 0; i < n; ++i) members[i] = (int)i;
    std::vector<int> ord;
    kd_append(ord, std::move(members), xy, xy + 1, 2);
    if (n_pad) *n_pad = (int64_t)ord.size();
    if (order) std::copy(ord.begin(), ord.end(), order);
    return SL1M_OK;
}

int sl1m_granule_layout(int64_t n, const double* xyzw, const int32_t* order, int64_t n_pad, float* hi,
                        float* lo, float* off, float* offlo, float* cen_hi, float* cen_lo, float* ext)
{
    if (n <= 0 || !xyzw || !order || n > ((int64_t)1 << 30) || n_pad < n || n_pad % G != 0 ||
        n_pad > ((int64_t)1 << 31) - G)
        return SL1M_ERR_ARG;
    std::vector<char> seen((size_t)n, 0);
    std::vector<int> ord((size_t)n_pad);
    for (int64_t i = 0; i < n_pad; ++i) {
        const int32_t o = order[i];
        if (o < -1 || o >= n) return SL1M_ERR_ARG;
        if (o >= 0) {
            if (seen[(size_t)o]) return SL1M_ERR_ARG;
            seen[(size_t)o] = 1;
        }
        ord[(size_t)i] = o;
    }
    std::vector<d4> xyz((size_t)n);
    for (int64_t i = 0; i < n; ++i)
        xyz[(size_t)i] = make_d4(xyzw[4 * i], xyzw[4 * i + 1], xyzw[4 * i + 2], xyzw[4 * i + 3]);
    HostSide H;
    layout_side(ord, xyz, (int)n, H);
    auto put = [](float* dst, const float4* src, size_t cnt) {
        if (dst) std::memcpy(dst, src, cnt * sizeof(float4));
    };
    put(hi, H.hi.data(), H.hi.size());
    put(lo, H.lo.data(), H.lo.size());
    put(off, H.off.data(), H.off.size());
    put(offlo, H.offlo.data(), H.offlo.size());
    put(cen_hi, H.cen_hi.data(), H.cen_hi.size());
    put(cen_lo, H.cen_lo.data(), H.cen_lo.size());
    put(ext, H.ext.data(), H.ext.size());
    return SL1M_OK;
}

int sl1m_counters(sl1m_ctx* ctx, int64_t* launches, int64_t* h2d_bytes, int64_t* d2h_bytes)
{
    if (!ctx) return SL1M_ERR_ARG;
    if (launches) *launches = ctx->n_launch;
    if (h2d_bytes) *h2d_bytes = ctx->h2d;
    if (d2h_bytes) *d2h_bytes = ctx->d2h;
    return SL1M_OK;
}

int sl1m_counters_reset(sl1m_ctx* ctx)
{
    if (!ctx) return SL1M_ERR_ARG;
    ctx->n_launch = ctx->h2d = ctx->d2h = 0;
    return SL1M_OK;
}

int sl1m_problem_bytes(const sl1m_problem* prob, int64_t* bytes)
{
    if (!prob || !bytes) return SL1M_ERR_ARG;
    *bytes = prob->dev ? (int64_t)prob->dev_bytes() : 0;
    return SL1M_OK;
}

int sl1m_selftest_bounded_wait(sl1m_ctx* ctx, int64_t* waited_ns, int64_t* limit_ns)
{
    if (!ctx) return SL1M_ERR_ARG;
    NOT_WHILE_SERVING(ctx);
    CK(cudaSetDevice(ctx->device));
    constexpr int NB = 2;
    DBuf<unsigned long long> w;
    CK(w.alloc(NB));
    CK(cudaMemsetAsync(w.p, 0, sizeof(unsigned long long) * NB, ctx->stream));
    CKL(launch_wait_selftest(w.p, NB, ctx->stream));
    unsigned long long hw[NB] = {0, 0};
    CK(cudaMemcpyAsync(hw, w.p, sizeof hw, cudaMemcpyDeviceToHost, ctx->stream));
    unsigned fault = 0;
    CK(wait_fault_read(&fault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (waited_ns) *waited_ns = (int64_t)std::min(hw[0], hw[1]);
    if (limit_ns) *limit_ns = (int64_t)wait_limit_ns();
    return check_wait_fault(ctx, fault);
}

int sl1m_exact_tile_share(const sl1m_problem* prob, double* share, int64_t* n_tiles)
{
    if (!prob || !share) return SL1M_ERR_ARG;
    if (prob->dirty || !prob->dev)
        return sl1m_fail(prob->ctx, SL1M_ERR_STATE, "problem not laid out on the device yet");
    // the test the mixed kernels make per tile: the granules' extents bound
    // the FP32 product term D = (X - Xc).(Y - Yc) above D_MAX turns
    long long n_ex = 0;
    for (const float4& v : prob->gext_vis)
        for (const float4& p : prob->gext_pix) n_ex += v.x * p.x + v.y * p.y + v.z * p.z > D_MAX;
    const long long n = (long long)prob->gext_vis.size() * (long long)prob->gext_pix.size();
    *share = n > 0 ? (double)n_ex / (double)n : 0.0;
    if (n_tiles) *n_tiles = n;
    return SL1M_OK;
}

}  // extern "C"
