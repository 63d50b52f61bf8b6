// sl1m_host.cpp -- host side of libsl1m: contexts, problem layout in HBM,
// stream-K launch plans, the operator calls, the power iteration for L and
// the FISTA driver (Hardy 2013, Sect. 2-3).  See include/sl1m.h for the ABI.
#include "sl1m.h"

#include <algorithm>
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
// median.  Only the last run can be shorter than G.
static void kd_rec(std::vector<int>& idx, size_t lo, size_t hi, const double* x, const double* y,
                   size_t stride)
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
    kd_rec(idx, lo, lo + left, x, y, stride);
    kd_rec(idx, lo + left, hi, x, y, stride);
}

// Append `members` (caller indices) in k-d order, padded with -1 to a
// multiple of G.
static void kd_append(std::vector<int>& order, std::vector<int> members, const double* x,
                      const double* y, size_t stride)
{
    kd_rec(members, 0, members.size(), x, y, stride);
    order.insert(order.end(), members.begin(), members.end());
    while (order.size() % G) order.push_back(-1);
}

struct HostSide {
    int n = 0, n_pad = 0, n_gran = 0, n_blk = 0;
    std::vector<float4> hi, lo, off, offlo, cen_hi, cen_lo, ext;
    std::vector<d4> d;
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
    for (int g = 0; g < S.n_gran; ++g) {
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
void plan_host(const std::vector<int>& nb, const std::vector<int>& ns, int Cmax, HostPlan& H)
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
    auto cta_of = [&](long long x) { return (int)(((x + 1) * C + U - 1) / U - 1); };
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
                       DevPlan& D, cudaStream_t st)
{
    HostPlan H;
    plan_host(nb, ns, Cmax, H);
    cudaError_t err;
    auto up = [&](DBuf<int>& b, const std::vector<int>& v) {
        return b.upload(v.data(), std::max<size_t>(1, v.size()), st, v.empty());
    };
    if ((err = D.u0.upload(H.u0.data(), H.u0.size(), st))) return err;
    if ((err = up(D.b0, H.b0))) return err;
    if ((err = up(D.poff, H.poff))) return err;
    if ((err = up(D.clo, H.clo))) return err;
    if ((err = up(D.ncon, H.ncon))) return err;
    D.pl.n_probs = (int)nb.size();
    D.pl.C = H.C;
    D.pl.U = H.U;
    D.pl.prob_u0 = D.u0.p;
    D.pl.prob_b0 = D.b0.p;
    D.pl.blk_poff = D.poff.p;
    D.pl.blk_clo = D.clo.p;
    D.pl.blk_ncon = D.ncon.p;
    D.pl.n_blocks = H.n_blocks;
    D.pl.n_slots = H.n_slots;
    return cudaSuccess;
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
    if (own_stream && stream) cudaStreamDestroy(stream);
}

// ============================================================== problem

struct ProblemDev {
    DevSide vis, pix;
    DBuf<int2> ant;
    DBuf<double2> V;
    DBuf<float4> pgauss;
    DBuf<d4> pgauss64;
    DBuf<float> gsig;
    DBuf<int> gkind;
    DBuf<float2> gains32;
    DBuf<double2> gains64;
    // operator scratch
    DBuf<double> x_user, x_sorted, adj_sorted, img_user;
    DBuf<double2> r_user, r_sorted, fwd_sorted, vis_user;
    // solver
    DBuf<double> I0, I1, y, xv, blk_r2, blk_l1, blk_z2;
    DBuf<double2> AI0, AI1, rr;
    DBuf<int> blk_nnz, blk_badv, blk_badp;
    DBuf<SolveState> st;
    DBuf<SolveBufs> bufs;
    DBuf<DevProblem> desc;
};

struct sl1m_problem_impl {};

int sl1m_problem::rebuild()
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
    cudaStream_t st = ctx->stream;
    if (!dev) dev = std::make_unique<ProblemDev>();
    ProblemDev& D = *dev;
    // ---- visibilities: k-d order on (u, v)
    {
        std::vector<int> members(n_vis);
        for (int64_t k = 0; k < n_vis; ++k) members[k] = (int)k;
        std::vector<int> order;
        kd_append(order, std::move(members), uvw.data(), uvw.data() + 1, 3);
        std::vector<d4> xyz(n_vis);
        for (int64_t k = 0; k < n_vis; ++k)
            xyz[k] = make_d4(uvw[3 * k], uvw[3 * k + 1], uvw[3 * k + 2],
                                  weights.empty() ? 1.0 : weights[k]);
        HostSide H;
        layout_side(order, xyz, (int)n_vis, H);
        CK(upload_side(H, D.vis, hp.vis, st));
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
        vis_orig = H.orig;
    }
    // ---- pixels: classes of equal (kind, sigma), each in k-d order on (l, m)
    {
        std::vector<std::pair<std::pair<int, double>, int>> cls(n_pix);
        for (int64_t j = 0; j < n_pix; ++j)
            cls[j] = {{kind.empty() ? 0 : kind[j], sigma.empty() ? 0.0 : sigma[j]}, (int)j};
        std::stable_sort(cls.begin(), cls.end(),
                         [](const auto& a, const auto& b) { return a.first < b.first; });
        std::vector<int> order;
        std::vector<std::pair<int, float>> gran_cls;
        size_t i = 0;
        while (i < cls.size()) {
            size_t j = i;
            std::vector<int> members;
            while (j < cls.size() && cls[j].first == cls[i].first) members.push_back(cls[j++].second);
            const size_t before = order.size();
            kd_append(order, std::move(members), lm.data(), lm.data() + 1, 2);
            for (size_t g = before / G; g < order.size() / G; ++g)
                gran_cls.push_back({cls[i].first.first, (float)cls[i].first.second});
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
        std::vector<int> gk(H.n_gran);
        for (int g = 0; g < H.n_gran; ++g) { gk[g] = gran_cls[g].first; gs[g] = gran_cls[g].second; }
        CK(D.gsig.upload(gs.data(), gs.size(), st));
        CK(D.gkind.upload(gk.data(), gk.size(), st));
        pix_orig = H.orig;
        has_gauss = false;
        for (int g = 0; g < H.n_gran; ++g) has_gauss |= gk[g] != DIRAC;
        // gains in sorted pixel order
        if (n_ant > 0) {
            std::vector<float2> g32((size_t)H.n_pad * n_ant, make_float2(0.f, 0.f));
            std::vector<double2> g64((size_t)H.n_pad * n_ant, make_double2(0.0, 0.0));
            for (int t = 0; t < H.n_pad; ++t) {
                const int o = H.orig[t];
                if (o < 0) continue;
                for (int a = 0; a < n_ant; ++a) {
                    const double re = gains[((size_t)o * n_ant + a) * 2], im = gains[((size_t)o * n_ant + a) * 2 + 1];
                    g32[(size_t)t * n_ant + a] = make_float2((float)re, (float)im);
                    g64[(size_t)t * n_ant + a] = make_double2(re, im);
                }
            }
            CK(D.gains32.upload(g32.data(), g32.size(), st));
            CK(D.gains64.upload(g64.data(), g64.size(), st));
        } else {
            D.gains32.free();
            D.gains64.free();
        }
    }
    hp.ant = D.ant.p;
    hp.V = D.V.p;
    hp.pgauss = D.pgauss.p;
    hp.pgauss64 = D.pgauss64.p;
    hp.gsig = D.gsig.p;
    hp.gkind = D.gkind.p;
    hp.gains32 = n_ant > 0 ? D.gains32.p : nullptr;
    hp.gains64 = n_ant > 0 ? D.gains64.p : nullptr;
    hp.n_ant = n_ant;
    hp.active = 1;
    ctx->h2d += (long long)dev_bytes();
    plans.clear();
    solver_ready = false;
    desc_valid = false;
    dirty = false;
    return SL1M_OK;
}

// Plan for (op 0 = forward / 1 = adjoint, precision) of this single problem.
int sl1m_problem::plan(int op, int precision, const Plan** out)
{
    const bool gains = n_ant > 0;
    const int key = op * 4 + precision * 2 + (gains ? 1 : 0);
    auto it = plans.find(key);
    if (it == plans.end()) {
        const int which = (precision == 0 ? 0 : 2) + op;
        const int occ = occupancy(which, gains, n_ant);
        auto D = std::make_unique<DevPlan>();
        std::vector<int> nb(1), ns(1);
        nb[0] = op == 0 ? hp.vis.n_blk : hp.pix.n_blk;
        ns[0] = op == 0 ? hp.pix.n_gran : hp.vis.n_gran;
        CK(build_plan(nb, ns, ctx->num_sms * occ, *D, ctx->stream));
        it = plans.emplace(key, std::move(D)).first;
    }
    *out = &it->second->pl;
    const size_t need = (size_t)std::max(1, it->second->pl.n_slots) * BLK;
    if (op == 0) CK(ctx->partial_f.reserve(need, ctx->stream));
    else CK(ctx->partial_a.reserve(need, ctx->stream));
    return SL1M_OK;
}

// Copy the descriptor to the device only when it changed since the last
// launch (a solve keeps one descriptor for all its iterations).
int sl1m_problem::upload_desc()
{
    if (desc_valid && memcmp(&hp, &last_desc, sizeof hp) == 0) return SL1M_OK;
    CK(dev->desc.reserve(1, ctx->stream));
    CK(cudaMemcpyAsync(dev->desc.p, &hp, sizeof hp, cudaMemcpyHostToDevice, ctx->stream));
    memcpy(&last_desc, &hp, sizeof hp);
    desc_valid = true;
    return SL1M_OK;
}

double sl1m_problem::pairs() const { return (double)n_vis * (double)n_pix; }

// Forward on sorted device input x_sorted (already gathered) -> fwd_sorted.
int sl1m_problem::run_forward(int precision, int fin_mode, const SolveBufs* bufs_dev)
{
    const Plan* pl;
    RET(plan(0, precision, &pl));
    RET(upload_desc());
    ProfTok tk;
    prof_begin(ctx, precision == 0 ? 0 : 2, tk);
    CKL(launch_forward(precision, n_ant > 0, n_ant, dev->desc.p, *pl, ctx->partial_f.p, ctx->stream));
    prof_end(ctx, tk, pairs(), 0.0);
    prof_begin(ctx, 4, tk);
    CKL(launch_fwd_finish(dev->desc.p, bufs_dev, *pl, ctx->partial_f.p, fin_mode, ctx->stream));
    // finish bytes: partial slots + per-vis state traffic
    const double vb = (double)hp.vis.n_pad;
    const double fb = (double)pl->n_slots * BLK * 16.0 + vb * (fin_mode == FIN_SOLVE ? 16 * 5 + 32 : 16 + 32);
    prof_end(ctx, tk, 0.0, fb);
    return SL1M_OK;
}

int sl1m_problem::run_adjoint(int precision, int fin_mode, const SolveBufs* bufs_dev)
{
    const Plan* pl;
    RET(plan(1, precision, &pl));
    RET(upload_desc());
    ProfTok tk;
    prof_begin(ctx, precision == 0 ? 1 : 3, tk);
    CKL(launch_adjoint(precision, n_ant > 0, dev->desc.p, *pl, ctx->partial_a.p, ctx->stream));
    prof_end(ctx, tk, pairs(), 0.0);
    prof_begin(ctx, 5, tk);
    CKL(launch_adj_finish(dev->desc.p, bufs_dev, *pl, ctx->partial_a.p, fin_mode, ctx->stream));
    const double pb = (double)hp.pix.n_pad;
    const double ab = (double)pl->n_slots * BLK * 8.0 + pb * (fin_mode == FIN_SOLVE ? 8 * 5 + 4 : 8);
    prof_end(ctx, tk, 0.0, ab);
    return SL1M_OK;
}

int sl1m_problem::ensure_solver()
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
    b.st = D.st.p;
    hbufs = b;
    CK(D.bufs.upload(&b, 1, ctx->stream));
    CK(cudaMemsetAsync(D.blk_badp.p, 0, sizeof(int) * std::max(1, hp.pix.n_blk), ctx->stream));
    CK(cudaMemsetAsync(D.blk_badv.p, 0, sizeof(int) * std::max(1, hp.vis.n_blk), ctx->stream));
    solver_ready = true;
    return SL1M_OK;
}

void sl1m_problem::reset_operands()
{
    hp.x = nullptr;
    hp.xpp[0] = hp.xpp[1] = nullptr;
    hp.xsel = nullptr;
    hp.xscale = nullptr;
    hp.r = nullptr;
    hp.done = nullptr;
    hp.fwd_out = nullptr;
    hp.adj_out = nullptr;
}

// Power iteration on sorted device vectors; st must be allocated.
int sl1m_problem::power(int precision, int max_iter, double tol, double* L, int* iters)
{
    RET(ensure_solver());
    ProblemDev& D = *dev;
    SolveState s0;
    memset(&s0, 0, sizeof s0);
    s0.inv_mu = 1.0;
    s0.pmax = max_iter;
    s0.ptol = tol;
    CK(cudaMemcpyAsync(D.st.p, &s0, sizeof s0, cudaMemcpyHostToDevice, ctx->stream));
    CKL(launch_fill_valid(D.xv.p, hp.pix.orig, hp.pix.n_pad, 1.0 / std::sqrt((double)n_pix), ctx->stream));
    reset_operands();
    hp.x = D.xv.p;
    hp.xscale = &D.st.p->inv_mu;
    hp.r = D.rr.p;
    hp.done = &D.st.p->pdone;
    const int check = 8;
    SolveState sh;
    for (int it = 0; it < max_iter; it += check) {
        for (int q = 0; q < check && it + q < max_iter; ++q) {
            RET(run_forward(precision, FIN_POWER, D.bufs.p));
            RET(run_adjoint(precision, FIN_POWER, D.bufs.p));
            CKL(launch_scalars(D.bufs.p, D.desc.p, 1, FIN_POWER, ctx->stream));
        }
        CK(cudaMemcpyAsync(&sh, D.st.p, sizeof sh, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (sh.pdone) break;
    }
    reset_operands();
    if (sh.nonfinite) return sl1m_fail(ctx, SL1M_ERR_NONFINITE, "non-finite value in power iteration");
    if (!(sh.mu > 0.0)) return sl1m_fail(ctx, SL1M_ERR_ARG, "operator is zero (all weights zero?)");
    *L = sh.mu;
    if (iters) *iters = sh.pit;
    return SL1M_OK;
}

// ================================================================ C ABI

extern "C" {

int sl1m_version(void) { return 100; }

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
    *out = c;
    return SL1M_OK;
}

int sl1m_destroy(sl1m_ctx* ctx)
{
    if (!ctx) return SL1M_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto* p : ctx->problems) delete p;
    ctx->problems.clear();
    delete ctx;
    return SL1M_OK;
}

const char* sl1m_last_error(const sl1m_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

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

int sl1m_set_visibilities(sl1m_problem* prob, int64_t n_vis, const double* uvw, const double* vis,
                          const double* weights, const int32_t* ant_pair)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
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
        CK(prob->dev->V.upload(Vs.data(), Vs.size(), ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return SL1M_OK;
}

int sl1m_set_pixels(sl1m_problem* prob, int64_t n_pix, const double* lm, const double* sigma,
                    const int32_t* kind)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
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
        // Dirac pixels ignore sigma: one class for all of them
        if (!prob->sigma.empty())
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
    if (!Gn || n_ant == 0) {
        prob->n_ant = 0;
        prob->gains.clear();
        prob->dirty = true;
        return SL1M_OK;
    }
    if (n_ant < 0 || n_ant > 400) return sl1m_fail(ctx, SL1M_ERR_ARG, "n_ant must be in [1, 400]");
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
    if (!x_dev || !vis_out_dev) return sl1m_fail(ctx, SL1M_ERR_ARG, "null pointer");
    RET(check_prec(ctx, precision));
    CK(cudaSetDevice(ctx->device));
    RET(prob->rebuild());
    ProblemDev& D = *prob->dev;
    CK(D.x_sorted.reserve(prob->hp.pix.n_pad, ctx->stream));
    CK(D.fwd_sorted.reserve(prob->hp.vis.n_pad, ctx->stream));
    CKL(launch_gather_real(x_dev, D.x_sorted.p, prob->hp.pix.orig, prob->hp.pix.n_pad, 1.0, ctx->stream));
    prob->reset_operands();
    prob->hp.x = D.x_sorted.p;
    prob->hp.fwd_out = D.fwd_sorted.p;
    RET(prob->run_forward(precision, FIN_OP, nullptr));
    CKL(launch_scatter_cplx(D.fwd_sorted.p, (double2*)vis_out_dev, prob->hp.vis.orig, prob->hp.vis.n_pad,
                           ctx->stream));
    prob->reset_operands();
    return SL1M_OK;
}

int sl1m_adjoint_dev(sl1m_problem* prob, const double* r_dev, double* img_out_dev, int precision)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    if (!r_dev || !img_out_dev) return sl1m_fail(ctx, SL1M_ERR_ARG, "null pointer");
    RET(check_prec(ctx, precision));
    CK(cudaSetDevice(ctx->device));
    RET(prob->rebuild());
    ProblemDev& D = *prob->dev;
    CK(D.r_sorted.reserve(prob->hp.vis.n_pad, ctx->stream));
    CK(D.adj_sorted.reserve(prob->hp.pix.n_pad, ctx->stream));
    CKL(launch_gather_cplx((const double2*)r_dev, D.r_sorted.p, prob->hp.vis.orig, prob->hp.vis.n_pad,
                          ctx->stream));
    prob->reset_operands();
    prob->hp.r = D.r_sorted.p;
    prob->hp.adj_out = D.adj_sorted.p;
    RET(prob->run_adjoint(precision, FIN_OP, nullptr));
    CKL(launch_scatter_real(D.adj_sorted.p, img_out_dev, prob->hp.pix.orig, prob->hp.pix.n_pad, ctx->stream));
    prob->reset_operands();
    return SL1M_OK;
}

int sl1m_forward(sl1m_problem* prob, const double* x, double* vis_out, int precision)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    if (!x || !vis_out) return sl1m_fail(ctx, SL1M_ERR_ARG, "null pointer");
    if (!all_finite(x, prob->n_pix > 0 ? prob->n_pix : 0)) return sl1m_fail(ctx, SL1M_ERR_ARG, "non-finite x");
    CK(cudaSetDevice(ctx->device));
    RET(prob->rebuild());
    ProblemDev& D = *prob->dev;
    CK(D.x_user.reserve(prob->n_pix, ctx->stream));
    CK(D.vis_user.reserve(prob->n_vis, ctx->stream));
    CK(cudaMemcpyAsync(D.x_user.p, x, sizeof(double) * prob->n_pix, cudaMemcpyHostToDevice, ctx->stream));
    RET(sl1m_forward_dev(prob, D.x_user.p, (double*)D.vis_user.p, precision));
    CK(cudaMemcpyAsync(vis_out, D.vis_user.p, sizeof(double2) * prob->n_vis, cudaMemcpyDeviceToHost, ctx->stream));
    ctx->h2d += (long long)sizeof(double) * prob->n_pix;
    ctx->d2h += (long long)sizeof(double2) * prob->n_vis;
    CK(cudaStreamSynchronize(ctx->stream));
    return SL1M_OK;
}

int sl1m_adjoint(sl1m_problem* prob, const double* r, double* img_out, int precision)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    if (!r || !img_out) return sl1m_fail(ctx, SL1M_ERR_ARG, "null pointer");
    if (!all_finite(r, prob->n_vis > 0 ? 2 * prob->n_vis : 0)) return sl1m_fail(ctx, SL1M_ERR_ARG, "non-finite r");
    CK(cudaSetDevice(ctx->device));
    RET(prob->rebuild());
    ProblemDev& D = *prob->dev;
    CK(D.r_user.reserve(prob->n_vis, ctx->stream));
    CK(D.img_user.reserve(prob->n_pix, ctx->stream));
    CK(cudaMemcpyAsync(D.r_user.p, r, sizeof(double2) * prob->n_vis, cudaMemcpyHostToDevice, ctx->stream));
    RET(sl1m_adjoint_dev(prob, (const double*)D.r_user.p, D.img_user.p, precision));
    CK(cudaMemcpyAsync(img_out, D.img_user.p, sizeof(double) * prob->n_pix, cudaMemcpyDeviceToHost, ctx->stream));
    ctx->h2d += (long long)sizeof(double2) * prob->n_vis;
    ctx->d2h += (long long)sizeof(double) * prob->n_pix;
    CK(cudaStreamSynchronize(ctx->stream));
    return SL1M_OK;
}

int sl1m_max_eig(sl1m_problem* prob, int max_iter, double tol, int precision, double* L_out, int* iters_out)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    if (!L_out || max_iter <= 0 || !(tol >= 0)) return sl1m_fail(ctx, SL1M_ERR_ARG, "bad arguments");
    RET(check_prec(ctx, precision));
    CK(cudaSetDevice(ctx->device));
    RET(prob->rebuild());
    return prob->power(precision, max_iter, tol, L_out, iters_out);
}

int sl1m_solve(sl1m_problem* prob, const sl1m_solve_opts* o, double* img_out, sl1m_solve_stats* stats)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    if (!o || !img_out) return sl1m_fail(ctx, SL1M_ERR_ARG, "null pointer");
    if (!(o->lambda >= 0) || !std::isfinite(o->lambda) || !(o->L >= 0) || !std::isfinite(o->L) ||
        o->max_iter < 0 || !(o->rel_tol >= 0))
        return sl1m_fail(ctx, SL1M_ERR_ARG, "bad solver options");
    RET(check_prec(ctx, o->precision));
    const auto t0 = std::chrono::steady_clock::now();
    CK(cudaSetDevice(ctx->device));
    RET(prob->rebuild());
    RET(prob->ensure_solver());
    ProblemDev& D = *prob->dev;
    const int prec = o->precision;
    double L = o->L;
    int pits = 0;
    if (L == 0.0) {
        RET(prob->power(prec, o->power_max_iter > 0 ? o->power_max_iter : 50,
                        o->power_tol > 0 ? o->power_tol : 1e-6, &L, &pits));
    }
    // Step 0: y_1 = I_0 = x0 (or 0), t_1 = 1
    double l1_0 = 0.0;
    if (o->x0) {
        if (!all_finite(o->x0, prob->n_pix)) return sl1m_fail(ctx, SL1M_ERR_ARG, "non-finite x0");
        CK(D.x_user.reserve(prob->n_pix, ctx->stream));
        CK(cudaMemcpyAsync(D.x_user.p, o->x0, sizeof(double) * prob->n_pix, cudaMemcpyHostToDevice, ctx->stream));
        CKL(launch_gather_real(D.x_user.p, D.I0.p, prob->hp.pix.orig, prob->hp.pix.n_pad, 1.0, ctx->stream));
        for (int64_t j = 0; j < prob->n_pix; ++j) l1_0 += o->x0[j];
        ctx->h2d += (long long)sizeof(double) * prob->n_pix;
    } else {
        CK(cudaMemsetAsync(D.I0.p, 0, sizeof(double) * prob->hp.pix.n_pad, ctx->stream));
    }
    CK(cudaMemcpyAsync(D.y.p, D.I0.p, sizeof(double) * prob->hp.pix.n_pad, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(D.I1.p, D.I0.p, sizeof(double) * prob->hp.pix.n_pad, cudaMemcpyDeviceToDevice, ctx->stream));
    SolveState s0;
    memset(&s0, 0, sizeof s0);
    s0.lambda = o->lambda;
    s0.L = L;
    s0.tol = o->rel_tol;
    s0.t = 1.0;
    s0.l1 = l1_0;
    s0.max_iter = o->max_iter;
    s0.inv_mu = 1.0;
    CK(cudaMemcpyAsync(D.st.p, &s0, sizeof s0, cudaMemcpyHostToDevice, ctx->stream));
    // A I_0, r_1 = W (A y_1 - V), E_0
    prob->reset_operands();
    prob->hp.x = D.I0.p;
    RET(prob->run_forward(prec, FIN_INIT, D.bufs.p));
    CKL(launch_scalars(D.bufs.p, D.desc.p, 1, FIN_INIT, ctx->stream));
    // iterations
    prob->reset_operands();
    prob->hp.xpp[0] = D.I0.p;
    prob->hp.xpp[1] = D.I1.p;
    prob->hp.xsel = &D.st.p->parity;
    prob->hp.r = D.rr.p;
    prob->hp.done = &D.st.p->done;
    SolveState sh;
    memset(&sh, 0, sizeof sh);
    const int check = 8;
    int issued = 0;
    bool finished = o->max_iter == 0;
    while (!finished) {
        for (int q = 0; q < check && issued < o->max_iter; ++q, ++issued) {
            RET(prob->run_adjoint(prec, FIN_SOLVE, D.bufs.p));
            RET(prob->run_forward(prec, FIN_SOLVE, D.bufs.p));
            CKL(launch_scalars(D.bufs.p, D.desc.p, 1, FIN_SOLVE, ctx->stream));
        }
        CK(cudaMemcpyAsync(&sh, D.st.p, sizeof sh, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        finished = sh.done || issued >= o->max_iter;
    }
    CK(cudaMemcpyAsync(&sh, D.st.p, sizeof sh, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    // result: I_k lives in I[k & 1]
    double* Ik = (sh.k & 1) ? D.I1.p : D.I0.p;
    CK(D.img_user.reserve(prob->n_pix, ctx->stream));
    CKL(launch_scatter_real(Ik, D.img_user.p, prob->hp.pix.orig, prob->hp.pix.n_pad, ctx->stream));
    CK(cudaMemcpyAsync(img_out, D.img_user.p, sizeof(double) * prob->n_pix, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->d2h += (long long)sizeof(double) * prob->n_pix;
    prob->reset_operands();
    if (stats) {
        stats->iters = sh.k;
        stats->converged = sh.converged;
        stats->E = sh.E;
        stats->E_paper = sh.resid2 + o->lambda * sh.l1;
        stats->resid2 = sh.resid2;
        stats->l1 = sh.l1;
        stats->nnz = sh.nnz;
        stats->L = L;
        stats->power_iters = pits;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (sh.nonfinite) return sl1m_fail(ctx, SL1M_ERR_NONFINITE, "non-finite value during the solve");
    return SL1M_OK;
}

int sl1m_profile_enable(sl1m_ctx* ctx, int on)
{
    if (!ctx) return SL1M_ERR_ARG;
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
                      int32_t max_ctas, int32_t* n_ctas, int64_t* n_units, int32_t* n_slots,
                      int32_t* blk_first_cta, int32_t* blk_n_ctas, int32_t* blk_first_slot)
{
    if (n_probs <= 0 || !owned_blocks || !streamed_granules || max_ctas <= 0) return SL1M_ERR_ARG;
    std::vector<int> nb(n_probs), ns(n_probs);
    for (int p = 0; p < n_probs; ++p) {
        if (owned_blocks[p] < 0 || streamed_granules[p] < 0) return SL1M_ERR_ARG;
        nb[p] = owned_blocks[p];
        ns[p] = streamed_granules[p];
    }
    HostPlan H;
    plan_host(nb, ns, max_ctas, H);
    if (n_ctas) *n_ctas = H.C;
    if (n_units) *n_units = H.U;
    if (n_slots) *n_slots = H.n_slots;
    for (int b = 0; b < H.n_blocks; ++b) {
        if (blk_first_cta) blk_first_cta[b] = H.clo[b];
        if (blk_n_ctas) blk_n_ctas[b] = H.ncon[b];
        if (blk_first_slot) blk_first_slot[b] = H.poff[b];
    }
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

}  // extern "C"

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
    b += D.ant.bytes() + D.V.bytes() + D.pgauss.bytes() + D.pgauss64.bytes() + D.gsig.bytes() +
         D.gkind.bytes() + D.gains32.bytes() + D.gains64.bytes();
    b += D.x_user.bytes() + D.x_sorted.bytes() + D.adj_sorted.bytes() + D.img_user.bytes() +
         D.r_user.bytes() + D.r_sorted.bytes() + D.fwd_sorted.bytes() + D.vis_user.bytes();
    b += D.I0.bytes() + D.I1.bytes() + D.y.bytes() + D.xv.bytes() + D.blk_r2.bytes() + D.blk_l1.bytes() +
         D.blk_z2.bytes() + D.AI0.bytes() + D.AI1.bytes() + D.rr.bytes() + D.blk_nnz.bytes() +
         D.blk_badv.bytes() + D.blk_badp.bytes() + D.st.bytes() + D.bufs.bytes() + D.desc.bytes();
    return b;
}

sl1m_problem::~sl1m_problem() = default;
