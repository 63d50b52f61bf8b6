// sl1m_server.cpp -- continuous-batching solve server of libsl1m.
//
// Independent solves share the forward and adjoint launches of a Batch: a
// request loop on a host thread admits queued requests (by slot count and a
// device-memory budget), lays out each admitted problem on an upload stream
// while the previous round's ticks run, replays the captured tick graph
// `ticks_per_round` times, reads the phase of every solve, and retires the
// finished ones (image to the caller's order, stats, latency).  Every solve
// keeps its own state on the device (phase machine of the scalars kernel).
//
// Only the request loop changes `active` and the counters, and it does so
// under `mu`, which the caller-side calls (submit, poll, wait, info) take to
// read them; the loop reads its own list without the lock.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "sl1m_host.h"
#include "sl1m_kernels.h"

using namespace sl1m;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct Request {
    uint64_t ticket = 0;
    sl1m_problem* prob = nullptr;
    sl1m_solve_opts opts{};
    std::vector<double> x0;
    double t_submit = 0, t_end = 0;
    int status = SL1M_OK;
    bool done = false;
    std::vector<double> img;
    sl1m_solve_stats stats{};
    size_t bytes = 0;
};

struct Server {
    sl1m_ctx* ctx = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::vector<Request*> active;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    size_t budget = 0, in_use = 0;
    int max_slots = 64, ticks_per_round = 4, precision = SL1M_MIXED;
    int admission = SL1M_ADMIT_TWO_LANES;
    double max_pairs = 4e9;
    bool stop = false, running = false;
    long long finished = 0, max_active = 0, ticks = 0, rounds = 0;
    Batch batch;
};

// Retire one request: image in the caller's order, stats, latency.
static void retire(Server& S, Request* r, int status)
{
    sl1m_problem* p = r->prob;
    if (status == SL1M_OK) {
        SolveState st;
        r->img.resize(p->n_pix);
        status = p->fetch_image(r->img.data(), S.ctx->stream);
        if (status == SL1M_OK) status = p->read_state(st, S.ctx->stream);
        if (status == SL1M_OK) {
            r->stats.iters = st.k;
            r->stats.converged = st.converged;
            r->stats.E = st.E;
            r->stats.E_paper = st.resid2 + r->opts.lambda * st.l1;
            r->stats.resid2 = st.resid2;
            r->stats.l1 = st.l1;
            r->stats.nnz = st.nnz;
            r->stats.L = st.L;
            r->stats.power_iters = st.pit;
            if (st.nonfinite) status = SL1M_ERR_NONFINITE;
        }
    }
    r->t_end = now_s();
    r->stats.seconds = r->t_end - r->t_submit;
    std::lock_guard<std::mutex> lk(S.mu);
    r->status = status;
    r->done = true;
    S.in_use -= std::min(S.in_use, r->bytes);
    S.finished += 1;
    S.cv_done.notify_all();
}

// Admission by memory (wait for running solves to free theirs) and by work in
// flight (N_v N_p summed over running solves: enough to fill the GPU, no
// more, since every running solve adds its pairs to every tick).

// SL1M_ADMIT_ARRIVAL: strictly in arrival order; the first request that does
// not fit stops admission (one request is always admitted when none runs).
static void admit_in_arrival_order(Server& S, std::vector<Request*>& admit)
{
    double work = 0.0;
    for (Request* r : S.active) work += r->prob->pairs();
    while (!S.pending.empty() && (int)(S.active.size() + admit.size()) < S.max_slots) {
        Request* r = S.pending.front();
        const size_t need = r->prob->estimate_bytes();
        const bool first = S.active.empty() && admit.empty();
        if (S.in_use + need > S.budget && !first) break;
        if (work + r->prob->pairs() > S.max_pairs && !first) break;
        work += r->prob->pairs();
        S.pending.pop_front();
        r->bytes = need;
        S.in_use += need;
        admit.push_back(r);
    }
}

// SL1M_ADMIT_TWO_LANES: requests of at most scale / 16 pairs ("small") and
// the others ("large") are admitted in arrival order within their lane, each
// lane against its own work budget: large ones against max_pairs (one large
// request is always admitted when no large one runs), small ones against
// scale / 4 more.  scale is max_pairs, or the pairs of the largest running
// request when one alone exceeds max_pairs: such a request fills the GPU by
// itself for a long time, and a request of a sixteenth of its size shares
// its ticks instead of waiting for it to end.  A small request never waits
// behind a large one that does not fit, and a large one never waits for small
// ones to drain; small ones add at most a quarter to a tick's work.
static void admit_two_lanes(Server& S, std::vector<Request*>& admit)
{
    double scale = S.max_pairs;
    for (Request* r : S.active) scale = std::max(scale, r->prob->pairs());
    const double small_max = scale / 16.0, small_budget = scale / 4.0;
    double work_large = 0.0, work_small = 0.0;
    bool any_large = false;
    for (Request* r : S.active) {
        const double w = r->prob->pairs();
        if (w <= small_max) work_small += w;
        else {
            work_large += w;
            any_large = true;
        }
    }
    bool large_blocked = false, small_blocked = false;
    for (auto it = S.pending.begin(); it != S.pending.end() && !(large_blocked && small_blocked);) {
        if ((int)(S.active.size() + admit.size()) >= S.max_slots) break;
        Request* r = *it;
        const double w = r->prob->pairs();
        const bool small = w <= small_max;
        if (small ? small_blocked : large_blocked) {
            ++it;
            continue;
        }
        const size_t need = r->prob->estimate_bytes();
        const bool first = S.active.empty() && admit.empty();
        const bool mem_ok = S.in_use + need <= S.budget || first;
        const bool work_ok = small ? (work_small + w <= small_budget || first)
                                   : (work_large + w <= S.max_pairs || !any_large);
        if (!mem_ok && !small) break;            // memory for the oldest large one first
        if (!mem_ok || !work_ok) {               // keep arrival order within the lane
            (small ? small_blocked : large_blocked) = true;
            ++it;
            continue;
        }
        if (small) work_small += w;
        else {
            work_large += w;
            any_large = true;
        }
        it = S.pending.erase(it);
        r->bytes = need;
        S.in_use += need;
        admit.push_back(r);
    }
}

static void server_loop(Server* Sp)
{
    Server& S = *Sp;
    sl1m_ctx* ctx = S.ctx;
    cudaSetDevice(ctx->device);
    std::vector<int> phases;
    while (true) {
        std::vector<Request*> admit;
        {
            std::unique_lock<std::mutex> lk(S.mu);
            while (!S.stop && S.pending.empty() && S.active.empty()) S.cv_work.wait(lk);
            if (S.stop && S.pending.empty() && S.active.empty()) break;
            if (S.admission == SL1M_ADMIT_ARRIVAL) admit_in_arrival_order(S, admit);
            else admit_two_lanes(S, admit);
        }
        // ticks of the running solves (asynchronous) ...
        if (!S.active.empty()) {
            const int rc = batch_ticks(ctx, S.batch, S.ticks_per_round);
            if (rc != SL1M_OK) {
                for (Request* r : S.active) retire(S, r, rc);
                std::lock_guard<std::mutex> lk(S.mu);
                S.active.clear();
            } else {
                std::lock_guard<std::mutex> lk(S.mu);
                S.ticks += S.ticks_per_round;
            }
        }
        // ... while the newcomers are laid out on the upload stream
        std::vector<Request*> joined;
        for (Request* r : admit) {
            sl1m_problem* p = r->prob;
            int rc = p->rebuild(ctx->upstream);
            if (rc == SL1M_OK) rc = p->init_solve(&r->opts, r->opts.L, false, ctx->upstream);
            if (rc != SL1M_OK) retire(S, r, rc);
            else joined.push_back(r);
        }
        bool changed = !joined.empty();
        if (!S.active.empty()) {
            if (batch_phases(ctx, S.batch, phases) != SL1M_OK) phases.assign(S.active.size(), PH_DONE);
            std::vector<Request*> keep;
            for (size_t i = 0; i < S.active.size(); ++i) {
                if (phases[i] == PH_DONE || phases[i] == PH_IDLE) {
                    retire(S, S.active[i], SL1M_OK);
                    changed = true;
                } else {
                    keep.push_back(S.active[i]);
                }
            }
            std::lock_guard<std::mutex> lk(S.mu);
            S.active.swap(keep);
        }
        {
            std::lock_guard<std::mutex> lk(S.mu);
            S.rounds += 1;
        }
        if (changed) {
            {
                std::lock_guard<std::mutex> lk(S.mu);
                for (Request* r : joined) S.active.push_back(r);
                S.max_active = std::max<long long>(S.max_active, (long long)S.active.size());
            }
            if (!S.active.empty()) {
                std::vector<sl1m_problem*> probs;
                std::vector<DevProblem> descs;
                for (Request* r : S.active) {
                    probs.push_back(r->prob);
                    descs.push_back(r->prob->solver_desc());
                }
                const int rc = batch_set(ctx, S.batch, probs, descs, S.precision, true);
                if (rc != SL1M_OK) {
                    for (Request* r : S.active) retire(S, r, rc);
                    std::lock_guard<std::mutex> lk(S.mu);
                    S.active.clear();
                }
            }
        }
    }
    std::lock_guard<std::mutex> lk(S.mu);
    S.running = false;
}

static void destroy_one(Server* S)
{
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    for (auto& kv : S->reqs)
        if (kv.second->prob) kv.second->prob->in_server = false;
    delete S;
}

void server_destroy(sl1m_ctx* ctx)
{
    if (ctx->server) destroy_one(ctx->server);
    if (ctx->server_done) destroy_one(ctx->server_done);
    ctx->server = ctx->server_done = nullptr;
}

static Server* any_server(sl1m_ctx* ctx) { return ctx->server ? ctx->server : ctx->server_done; }

extern "C" {

int sl1m_server_start(sl1m_ctx* ctx, const sl1m_server_opts* opts)
{
    if (!ctx) return SL1M_ERR_ARG;
    if (ctx->server) return sl1m_fail(ctx, SL1M_ERR_STATE, "server already running");
    server_destroy(ctx);
    cudaSetDevice(ctx->device);
    auto* S = new (std::nothrow) Server();
    if (!S) return sl1m_fail(ctx, SL1M_ERR_OOM, "host allocation failed");
    S->ctx = ctx;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    S->budget = (opts && opts->mem_budget_bytes > 0) ? (size_t)opts->mem_budget_bytes : (size_t)(0.8 * free_b);
    S->max_slots = (opts && opts->max_slots > 0) ? opts->max_slots : 64;
    S->max_slots = std::min(S->max_slots, MAX_PROBS);
    S->ticks_per_round = (opts && opts->ticks_per_round > 0) ? opts->ticks_per_round : 4;
    S->max_pairs = (opts && opts->max_pairs_per_tick > 0) ? opts->max_pairs_per_tick : 4e9;
    S->admission = opts ? opts->admission : SL1M_ADMIT_TWO_LANES;
    if (S->admission != SL1M_ADMIT_TWO_LANES && S->admission != SL1M_ADMIT_ARRIVAL) {
        delete S;
        return sl1m_fail(ctx, SL1M_ERR_ARG, "bad admission policy");
    }
    S->precision = opts ? opts->precision : SL1M_MIXED;
    if (S->precision != SL1M_MIXED && S->precision != SL1M_FP64) {
        delete S;
        return sl1m_fail(ctx, SL1M_ERR_ARG, "bad server precision");
    }
    S->running = true;
    ctx->server = S;
    S->th = std::thread(server_loop, S);
    return SL1M_OK;
}

int sl1m_server_submit(sl1m_ctx* ctx, sl1m_problem* prob, const sl1m_solve_opts* o, uint64_t* ticket)
{
    if (!ctx || !prob || !o || !ticket) return sl1m_fail(ctx, SL1M_ERR_ARG, "null argument");
    Server* S = ctx->server;
    if (!S) return sl1m_fail(ctx, SL1M_ERR_STATE, "no server running");
    if (prob->ctx != ctx) return sl1m_fail(ctx, SL1M_ERR_ARG, "problem belongs to another context");
    if (prob->in_server) return sl1m_fail(ctx, SL1M_ERR_BUSY, "problem already queued");
    if (prob->n_vis <= 0 || prob->n_pix <= 0) return sl1m_fail(ctx, SL1M_ERR_STATE, "problem incomplete");
    if (!(o->lambda >= 0) || !(o->L >= 0) || o->max_iter < 0 || !(o->rel_tol >= 0))
        return sl1m_fail(ctx, SL1M_ERR_ARG, "bad solver options");
    if (prob->estimate_bytes() > S->budget)
        return sl1m_fail(ctx, SL1M_ERR_BUSY, "problem exceeds the server memory budget");
    auto r = std::make_unique<Request>();
    r->prob = prob;
    r->opts = *o;
    r->opts.precision = S->precision;
    if (o->x0) {
        r->x0.assign(o->x0, o->x0 + prob->n_pix);
        r->opts.x0 = r->x0.data();
    }
    r->t_submit = now_s();
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->running || S->stop) return sl1m_fail(ctx, SL1M_ERR_STATE, "no server running");
    r->ticket = S->next_ticket++;
    *ticket = r->ticket;
    prob->in_server = true;
    S->pending.push_back(r.get());
    S->reqs[r->ticket] = std::move(r);
    S->cv_work.notify_all();
    return SL1M_OK;
}

int sl1m_server_poll(sl1m_ctx* ctx, uint64_t ticket, int* done)
{
    if (!ctx || !done) return sl1m_fail(ctx, SL1M_ERR_ARG, "null argument");
    Server* S = any_server(ctx);
    if (!S) return sl1m_fail(ctx, SL1M_ERR_STATE, "no server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return sl1m_fail(ctx, SL1M_ERR_ARG, "unknown ticket");
    *done = it->second->done ? 1 : 0;
    return SL1M_OK;
}

int sl1m_server_wait(sl1m_ctx* ctx, uint64_t ticket, double timeout_s, double* img_out, sl1m_solve_stats* stats)
{
    if (!ctx) return SL1M_ERR_ARG;
    Server* S = any_server(ctx);
    if (!S) return sl1m_fail(ctx, SL1M_ERR_STATE, "no server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return sl1m_fail(ctx, SL1M_ERR_ARG, "unknown ticket");
    Request* r = it->second.get();
    auto ready = [&] { return r->done; };
    if (timeout_s < 0) S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready))
        return sl1m_fail(ctx, SL1M_ERR_TIMEOUT, "request %llu not finished after %.3f s",
                         (unsigned long long)ticket, timeout_s);
    const int status = r->status;
    if (img_out && status == SL1M_OK) std::copy(r->img.begin(), r->img.end(), img_out);
    if (stats) *stats = r->stats;
    r->prob->in_server = false;
    S->reqs.erase(it);
    if (status != SL1M_OK) return sl1m_fail(ctx, status, "request failed: %s", sl1m_status_string(status));
    return SL1M_OK;
}

int sl1m_server_stop(sl1m_ctx* ctx)
{
    if (!ctx) return SL1M_ERR_ARG;
    Server* S = ctx->server;
    if (!S) return sl1m_fail(ctx, SL1M_ERR_STATE, "no server");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    // keep the Server (finished results stay collectable); calls other than
    // the server's are allowed again
    if (ctx->server_done) destroy_one(ctx->server_done);
    ctx->server_done = S;
    ctx->server = nullptr;
    return SL1M_OK;
}

int sl1m_server_info(sl1m_ctx* ctx, sl1m_server_info_t* info)
{
    if (!ctx || !info) return SL1M_ERR_ARG;
    Server* S = any_server(ctx);
    if (!S) return sl1m_fail(ctx, SL1M_ERR_STATE, "no server");
    std::lock_guard<std::mutex> lk(S->mu);
    info->queued = (int64_t)S->pending.size();
    info->active = (int64_t)S->active.size();
    info->finished = S->finished;
    info->max_active = S->max_active;
    info->bytes_in_use = (int64_t)S->in_use;
    info->bytes_budget = (int64_t)S->budget;
    info->ticks = S->ticks;
    info->rounds = S->rounds;
    return SL1M_OK;
}

}  // extern "C"
