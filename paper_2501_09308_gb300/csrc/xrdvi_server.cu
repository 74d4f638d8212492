// Continuous-batching fit server (xrdvi_server_*): host runtime around the
// fit kernels.
//
// Requests (a problem + fit options) enter a FIFO queue.  An admission thread
// takes the head request whenever its device footprint fits into the budget
// next to the resident fits (admission by HBM footprint) and a slot is free,
// and creates its context (validation, tables, upload) from one
// stream-ordered memory pool.  An engine thread advances every resident fit
// together by one batched step (xrdvi::multi_plan_launch_step): sampling,
// window ranges and the gradient are single launches whose work lists span
// all resident fits, whatever their K, N and peak counts; the profile and
// likelihood launches are shared by the fits too small to fill the GPU alone,
// while a fit with enough work of its own runs its own kernels inside the
// step.  Fits that run a variant outside the batched step (shared shapes,
// angle-dependent width, fitted background, naive sums, importance weights)
// take their own kernels between those launches.  Fits join and leave the batch between slices of a few steps, so
// requests that arrive while others run start within a slice.  A reaper
// thread draws the posterior of each finished fit, copies its results and
// frees it.  All device work runs on one stream in submission order; a fit's
// whole state stays on the device from creation to posterior; each fit's work
// items and reductions are those of its standalone kernels, so its result is
// the same alone and in the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/xrdvi.h"
#include "xrdvi_internal.h"


namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    std::vector<int32_t> off;
    std::vector<float> pos, inten, x, y, bg;
    xrdvi_config cfg{};
    xrdvi_request_opts opts{};
    size_t footprint = 0;
    double t_submit = 0, t_admit = -1, t_done = -1;
    bool done = false;
    xrdvi_status status = XRDVI_OK;
    std::string error;
    std::vector<double> pi, combo_logp;
    std::vector<uint64_t> combos;
    std::vector<float> loc, raw;
    double final_elbo = 0, log_evidence = 0, ess = 0, coverage_log = 0, elbo_tail_mean = 0;
};

// A resident fit: its request, its context and the steps enqueued so far.
struct Fit {
    std::shared_ptr<Request> r;
    xrdvi_ctx *c = nullptr;
    int steps = 0;
    bool batched = false;
};

size_t a256(size_t n) { return (n + 511) & ~static_cast<size_t>(511); }  // pool granularity allowance

constexpr int kSliceSteps = 8;   // SVI steps between changes of the batch

#define XR_TRY_STATUS(expr)                  \
    do {                                     \
        const xrdvi_status _s = (expr);      \
        if (_s != XRDVI_OK) return _s;       \
    } while (0)

}  // namespace

struct xrdvi_server {
    int device = 0, sm_count = 0;
    size_t budget = 0;
    int slots = 0;
    cudaMemPool_t pool = nullptr;
    cudaStream_t stream = nullptr;          // every fit's device work, in submission order
    xrdvi::MultiStepPlan *plan = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_engine, cv_reap;
    std::deque<std::shared_ptr<Request>> queue;    // waiting for admission
    std::vector<Fit *> ready;                      // created, waiting to join the batch
    std::deque<Fit *> finished;                    // all steps enqueued, waiting for the posterior
    std::unordered_map<uint64_t, std::shared_ptr<Request>> table;
    size_t in_use = 0, peak = 0;
    int64_t resident = 0, completed = 0;
    uint64_t next_id = 1;
    bool stopping = false, admit_done = false, engine_done = false;
    std::thread admit_thread, engine_thread, reap_thread;
    Clock::time_point t0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
    void admit_loop();
    void engine_loop();
    void reap_loop();
    void finish(Request &r);   // under mu: release the request's budget and slot, mark it done
};

void xrdvi_server::finish(Request &r) {
    in_use -= r.footprint;
    --resident;
    ++completed;
    r.t_done = now();
    r.done = true;
}

void xrdvi_server::admit_loop() {
    cudaSetDevice(device);
    for (;;) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] {
                return stopping || (!queue.empty() && queue.front()->footprint <= budget - in_use && resident < slots);
            });
            if (stopping) {
                admit_done = true;
                cv_engine.notify_all();
                return;
            }
            r = queue.front();
            queue.pop_front();
            in_use += r->footprint;
            peak = std::max(peak, in_use);
            ++resident;
            r->t_admit = now();
        }
        xrdvi_peaks pk{static_cast<int32_t>(r->off.size() - 1), r->off.data(), r->pos.data(), r->inten.data()};
        xrdvi_pattern pt{static_cast<int32_t>(r->x.size()), r->x.data(), r->y.data(), r->bg.data()};
        xrdvi_ctx *c = nullptr;
        xrdvi_status s;
        {
            xrdvi::NvtxRange nvtx("server admit");
            s = xrdvi::create_context(&pk, &pt, &r->cfg, pool, stream, &c);
        }
        std::lock_guard<std::mutex> lk(mu);
        if (s != XRDVI_OK) {
            r->status = s;
            r->error = xrdvi_last_error();
            finish(*r);
            cv_done.notify_all();
            cv_work.notify_all();
            continue;
        }
        Fit *f = new Fit();
        f->r = r;
        f->c = c;
        f->batched = xrdvi::ctx_multi_eligible(c);
        ready.push_back(f);
        cv_engine.notify_all();
    }
}

void xrdvi_server::engine_loop() {
    cudaSetDevice(device);
    std::vector<Fit *> members;
    bool dirty = true;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
    bool ev_live[2] = {false, false};
    int slot = 0;
    std::vector<xrdvi::FitStep> fs;
    std::vector<xrdvi_ctx *> solo;
    // the batch's steps are replayed from graphs captured (on a private
    // stream) whenever the batch changes: one of a whole slice, one of a step
    cudaStream_t cap = nullptr;
    cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    cudaGraphExec_t g_slice = nullptr, g_one = nullptr;
    auto drop_graphs = [&] {
        if (g_slice) cudaGraphExecDestroy(g_slice);
        if (g_one) cudaGraphExecDestroy(g_one);
        g_slice = g_one = nullptr;
    };
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            if (members.empty())
                cv_engine.wait(lk, [&] { return !ready.empty() || (stopping && admit_done); });
            if (!ready.empty()) {
                for (Fit *f : ready) members.push_back(f);
                ready.clear();
                dirty = true;
            }
            if (members.empty() && stopping && admit_done) break;
        }
        // fits with nothing to run go straight to the reaper
        for (size_t i = 0; i < members.size();) {
            if (members[i]->steps >= members[i]->r->opts.iters) {
                std::lock_guard<std::mutex> lk(mu);
                finished.push_back(members[i]);
                cv_reap.notify_all();
                dirty = true;   // the captured steps must no longer include it
                members.erase(members.begin() + i);
            } else {
                ++i;
            }
        }
        if (members.empty()) continue;
        if (dirty) {
            fs.clear();
            solo.clear();
            for (Fit *f : members) {
                if (f->batched) {
                    xrdvi::FitStep st;
                    xrdvi::ctx_fit_step(f->c, &st);
                    fs.push_back(st);
                } else {
                    solo.push_back(f->c);
                }
            }
            if (!fs.empty()) xrdvi::multi_plan_set(plan, fs.data(), static_cast<int>(fs.size()), sm_count, stream);
            drop_graphs();
            const xrdvi::MultiStepPlan *pl = fs.empty() ? nullptr : plan;
            if (xrdvi::capture_batch_steps(pl, solo.data(), static_cast<int>(solo.size()), kSliceSteps, cap,
                                           &g_slice) != XRDVI_OK ||
                xrdvi::capture_batch_steps(pl, solo.data(), static_cast<int>(solo.size()), 1, cap, &g_one) !=
                    XRDVI_OK)
                drop_graphs();   // launched kernel by kernel instead
            dirty = false;
        }
        xrdvi::NvtxRange nvtx("server slice");
        int n = kSliceSteps;
        for (Fit *f : members) n = std::min(n, f->r->opts.iters - f->steps);
        if (n == kSliceSteps && g_slice) {
            cudaGraphLaunch(g_slice, stream);
        } else if (g_one) {
            for (int i = 0; i < n; ++i) cudaGraphLaunch(g_one, stream);
        } else {
            for (int i = 0; i < n; ++i) {
                if (!fs.empty()) xrdvi::multi_plan_launch_step(plan, stream);
                for (xrdvi_ctx *c : solo) xrdvi::ctx_enqueue_steps(c, 1, stream);
            }
        }
        for (Fit *f : members) {
            f->steps += n;
            xrdvi::ctx_advance(f->c, n);
        }
        cudaEventRecord(ev[slot], stream);
        ev_live[slot] = true;
        // at most two slices in flight: new arrivals join within about a slice
        if (ev_live[slot ^ 1]) cudaEventSynchronize(ev[slot ^ 1]);
        slot ^= 1;
    }
    cudaStreamSynchronize(stream);
    drop_graphs();
    if (cap) cudaStreamDestroy(cap);
    for (int i = 0; i < 2; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    std::lock_guard<std::mutex> lk(mu);
    engine_done = true;
    cv_reap.notify_all();
}

void xrdvi_server::reap_loop() {
    cudaSetDevice(device);
    for (;;) {
        Fit *f = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_reap.wait(lk, [&] { return !finished.empty() || engine_done; });
            if (finished.empty()) return;
            f = finished.front();
            finished.pop_front();
        }
        xrdvi::NvtxRange nvtx("server posterior");
        Request &r = *f->r;
        xrdvi_ctx *c = f->c;
        const int K = static_cast<int>(r.off.size()) - 1, W = (K + 63) / 64;
        xrdvi_status s = XRDVI_OK;
        if (r.opts.iters > 0) {
            // the device keeps the last kTraceCap estimates: the tail mean covers at most those
            const int tail = std::min(std::max(1, r.opts.iters / 4), xrdvi::kTraceCap);
            std::vector<double> trace(tail);
            s = xrdvi::ctx_read_trace(c, tail, trace.data());
            r.final_elbo = trace[tail - 1];
            double acc = 0.0;
            for (int i = 0; i < tail; ++i) acc += trace[i];
            r.elbo_tail_mean = acc / tail;
        }
        if (s == XRDVI_OK && r.opts.S_post > 0) {
            r.pi.resize(K);
            r.combos.resize(static_cast<size_t>(r.opts.top_m) * W);
            r.combo_logp.resize(r.opts.top_m);
            s = xrdvi_posterior(c, r.opts.S_post, r.opts.post_seed, r.opts.top_m, r.pi.data(), r.combos.data(),
                                r.combo_logp.data(), &r.log_evidence, &r.ess, &r.coverage_log);
        }
        if (s == XRDVI_OK) {
            r.loc.resize(K * 5);
            r.raw.resize(K * 5);
            s = xrdvi_get_params(c, r.loc.data(), r.raw.data());
        }
        if (s != XRDVI_OK) r.error = xrdvi_last_error();
        r.status = s;
        xrdvi_destroy(c);   // stream-ordered frees
        delete f;
        {
            std::lock_guard<std::mutex> lk(mu);
            finish(r);
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

extern "C" size_t xrdvi_footprint_bytes(int32_t K, int32_t N, int32_t M_total, int32_t S, int32_t S_post,
                                        int32_t top_m) {
    using namespace xrdvi;
    if (K < 1 || N < 1 || M_total < 1 || S < 1 || S_post < 0 || top_m < 0) return 0;
    const size_t T = (static_cast<size_t>(N) + kTile - 1) / kTile, Npad = T * kTile;
    // phase chunks: the rule of choose_chunks with an upper bound on resident
    // warps (up to 160 SMs x 4 blocks x 8 warps), so C is never underestimated
    auto chunks = [&](size_t s) {
        const size_t resident = 160 * 4 * kWarps, items = s * T;
        size_t c = (kItemsPerWarp * resident + items - 1) / items;
        c = std::min<size_t>(c, kMaxChunks);
        c = std::min<size_t>(c, static_cast<size_t>(K));
        return std::max<size_t>(c, 1);
    };
    auto ws = [&](size_t s, bool fit) {
        const size_t sk = s * K, C = chunks(s);
        size_t b = 0;
        b += a256(sk * 5 * 4) * 2 + a256(sk * sizeof(PhaseConst)) + a256(s * 8) * 2 + a256(s * Npad * 4) +
             a256(s * T * 8) + a256(C * s * Npad * 4) + a256(sk * T * 8) + a256(kCounters * 4);
        b += fit ? a256(sk * T * kGradSums * 4) + a256(static_cast<size_t>(K) * kGradBlocks * kGredVals * 8) +
                       a256(static_cast<size_t>(K) * 4)
                 : a256(s * 8);
        // far field: range ends, node sums (and node weights of g in a fit, both levels)
        b += a256(sk * T * 4) * 2 + a256(kMaxChunks * s * T * kFarNodes * 4) * 2 + a256(s * T * kFarNodes * 4) * 2;
        return b;
    };
    size_t b = a256(M_total * 4) * 2 + a256((K + 1) * 4) + a256(N * 4) * 3 + a256(K * 8);
    b += a256(T * kFarNodes * kTile * 4) + a256(T * kFarNodes * 4) * 2;   // far-field tables
    b += a256(T * kFarNodes * kFarNodes * 4) * 2 + a256(T * kFarNodes * 4) * 2 + a256(T * 4);   // second level
    b += ws(S, true);
    b += a256(K * 20) * 2 + a256(K * 40) * 3 + a256(8) * 2 + a256(kTraceCap * 8) + a256(4) * 2;
    if (S_post > 0) {
        const size_t W = (K + 63) / 64, capM = std::max(top_m, 64);
        b += ws(S_post, false);
        b += a256(S_post * 8) + a256(static_cast<size_t>(S_post) * K) + a256(K * 8) + a256(32) +
             a256(capM * W * 8) + a256(capM * 8) + a256(K * 4) + a256(K * 8) + a256((2 * capM + 2) * 8) +
             a256((2 * capM + 2) * 4) + a256((2 * capM + 2) * W * 8) + a256((2 * capM + 2) * 4);
    }
    return b;
}

extern "C" {

xrdvi_status xrdvi_server_create(size_t hbm_budget, int32_t max_slots, xrdvi_server **out) {
    if (!out) return xrdvi::report_error(XRDVI_EINVAL, "null output pointer");
    *out = nullptr;
    if (max_slots < 1 || max_slots > xrdvi::kMaxBatch)
        return xrdvi::report_error(XRDVI_EINVAL, "max_slots must be in [1, 64]");
    if (hbm_budget == 0) return xrdvi::report_error(XRDVI_EINVAL, "hbm_budget must be positive");
    auto srv = std::make_unique<xrdvi_server>();
    cudaError_t e = cudaGetDevice(&srv->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&srv->sm_count, cudaDevAttrMultiProcessorCount, srv->device);
    if (e != cudaSuccess) return xrdvi::report_error(XRDVI_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = srv->device;
    e = cudaMemPoolCreate(&srv->pool, &props);
    if (e != cudaSuccess) return xrdvi::report_error(XRDVI_ECUDA, std::string("cudaMemPoolCreate: ") + cudaGetErrorString(e));
    uint64_t keep = UINT64_MAX;  // keep released memory reserved for the next fits
    cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    e = cudaStreamCreateWithFlags(&srv->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        srv->plan = xrdvi::multi_plan_create(max_slots);
        if (!srv->plan) e = cudaErrorMemoryAllocation;
    }
    if (e != cudaSuccess) {
        if (srv->stream) cudaStreamDestroy(srv->stream);
        cudaMemPoolDestroy(srv->pool);
        return xrdvi::report_error(XRDVI_ECUDA, std::string("server set-up: ") + cudaGetErrorString(e));
    }
    srv->budget = hbm_budget;
    srv->slots = max_slots;
    srv->t0 = Clock::now();
    xrdvi_server *p = srv.get();
    srv->admit_thread = std::thread([p] { p->admit_loop(); });
    srv->engine_thread = std::thread([p] { p->engine_loop(); });
    srv->reap_thread = std::thread([p] { p->reap_loop(); });
    *out = srv.release();
    return XRDVI_OK;
}

xrdvi_status xrdvi_server_submit(xrdvi_server *srv, const xrdvi_peaks *pk, const xrdvi_pattern *pt,
                                 const xrdvi_config *cfg, const xrdvi_request_opts *opts, uint64_t *req_id) {
    if (!srv || !pk || !pt || !cfg || !opts || !req_id) return xrdvi::report_error(XRDVI_EINVAL, "null argument");
    if (opts->iters < 0 || opts->S_post < 0 || opts->S_post > 65536 || (opts->S_post > 0 && (opts->top_m < 1 || opts->top_m > 4096)))
        return xrdvi::report_error(XRDVI_EINVAL, "bad request options");
    if (!pk->offsets || pk->K < 1 || pk->K > xrdvi::kMaxK || !pt->x_deg || pt->N < 1)
        return xrdvi::report_error(XRDVI_EINVAL, "bad problem sizes");
    auto r = std::make_shared<Request>();
    const int K = pk->K, N = pt->N, M = pk->offsets[K];
    if (M < 1 || M > xrdvi::kMaxPeaks) return xrdvi::report_error(XRDVI_EINVAL, "bad peak count");
    r->off.assign(pk->offsets, pk->offsets + K + 1);
    r->pos.assign(pk->pos_deg, pk->pos_deg + M);
    r->inten.assign(pk->rel_int, pk->rel_int + M);
    r->x.assign(pt->x_deg, pt->x_deg + N);
    r->y.assign(pt->y_counts, pt->y_counts + N);
    r->bg.assign(pt->bg, pt->bg + N);
    r->cfg = *cfg;
    r->opts = *opts;
    r->footprint = xrdvi_footprint_bytes(K, N, M, cfg->S, opts->S_post, opts->top_m);
    if (r->footprint > srv->budget)
        return xrdvi::report_error(XRDVI_ENOMEM, "request needs " + std::to_string(r->footprint) +
                                                      " bytes, more than the server's budget");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stopping) return xrdvi::report_error(XRDVI_EBUSY, "server is shutting down");
        r->id = srv->next_id++;
        r->t_submit = srv->now();
        srv->table[r->id] = r;
        srv->queue.push_back(r);
        *req_id = r->id;
    }
    srv->cv_work.notify_all();
    return XRDVI_OK;
}

xrdvi_status xrdvi_server_poll(xrdvi_server *srv, uint64_t req_id, int32_t timeout_ms, xrdvi_result *res) {
    if (!srv || !res) return xrdvi::report_error(XRDVI_EINVAL, "null argument");
    std::shared_ptr<Request> r;
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        auto it = srv->table.find(req_id);
        if (it == srv->table.end()) return xrdvi::report_error(XRDVI_EINVAL, "unknown or already collected request");
        r = it->second;
        const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(timeout_ms, 0));
        if (!srv->cv_done.wait_until(lk, deadline, [&] { return r->done; }))
            return xrdvi::report_error(XRDVI_ETIMEOUT, "request not finished yet");
        srv->table.erase(it);
    }
    const int K = static_cast<int>(r->off.size()) - 1;
    res->status = r->status;
    res->K = K;
    res->t_submit = r->t_submit;
    res->t_admit = r->t_admit;
    res->t_done = r->t_done;
    res->final_elbo = r->final_elbo;
    res->log_evidence = r->log_evidence;
    res->ess = r->ess;
    res->coverage_log = r->coverage_log;
    res->elbo_tail_mean = r->elbo_tail_mean;
    res->footprint_bytes = r->footprint;
    if (res->pi && !r->pi.empty()) std::memcpy(res->pi, r->pi.data(), r->pi.size() * 8);
    if (res->combos && !r->combos.empty()) std::memcpy(res->combos, r->combos.data(), r->combos.size() * 8);
    if (res->combo_logp && !r->combo_logp.empty())
        std::memcpy(res->combo_logp, r->combo_logp.data(), r->combo_logp.size() * 8);
    if (res->loc && !r->loc.empty()) std::memcpy(res->loc, r->loc.data(), r->loc.size() * 4);
    if (res->raw && !r->raw.empty()) std::memcpy(res->raw, r->raw.data(), r->raw.size() * 4);
    if (r->status != XRDVI_OK) xrdvi::report_error(static_cast<xrdvi_status>(r->status), r->error);
    return XRDVI_OK;
}

xrdvi_status xrdvi_server_cancel(xrdvi_server *srv, uint64_t req_id) {
    if (!srv) return xrdvi::report_error(XRDVI_EINVAL, "null argument");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = std::find_if(srv->queue.begin(), srv->queue.end(),
                               [&](const std::shared_ptr<Request> &r) { return r->id == req_id; });
        if (it == srv->queue.end()) return xrdvi::report_error(XRDVI_EBUSY, "request is not queued (running or done)");
        (*it)->status = XRDVI_ECANCELED;
        (*it)->error = "cancelled before it ran";
        (*it)->t_done = srv->now();
        (*it)->done = true;
        srv->queue.erase(it);
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();  // the next request may fit now
    return XRDVI_OK;
}

xrdvi_status xrdvi_server_get_stats(xrdvi_server *srv, xrdvi_server_stats *st) {
    if (!srv || !st) return xrdvi::report_error(XRDVI_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    st->queued = static_cast<int64_t>(srv->queue.size());
    st->running = srv->resident;
    st->completed = srv->completed;
    st->bytes_in_use = srv->in_use;
    st->peak_bytes = srv->peak;
    st->budget = srv->budget;
    st->slots = srv->slots;
    return XRDVI_OK;
}

void xrdvi_server_destroy(xrdvi_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
        for (auto &r : srv->queue) {
            r->status = XRDVI_ECANCELED;
            r->error = "server destroyed before the request ran";
            r->t_done = srv->now();
            r->done = true;
        }
        srv->queue.clear();
    }
    srv->cv_work.notify_all();
    srv->cv_engine.notify_all();
    srv->cv_done.notify_all();
    srv->admit_thread.join();    // a context being created joins the batch first
    srv->engine_thread.join();   // running fits finish their steps
    srv->reap_thread.join();     // and their posteriors
    cudaStreamSynchronize(srv->stream);
    xrdvi::multi_plan_destroy(srv->plan);
    cudaStreamDestroy(srv->stream);
    cudaMemPoolDestroy(srv->pool);
    delete srv;
}

size_t xrdvi_enumerate_footprint_bytes(int32_t K, int32_t N, int32_t M_total, int32_t S, int32_t nsub) {
    // a fit workspace of nsub*S samples plus per-sub-model state
    if (nsub < 1) return 0;
    const size_t base = xrdvi_footprint_bytes(K, N, M_total, S * nsub, 0, 0);
    if (base == 0) return 0;
    const size_t kb = static_cast<size_t>(K) * nsub;
    return base + a256(kb * 20) * 2 + a256(kb * 40) * 3 + a256(kb * xrdvi::kGradBlocks * xrdvi::kGredVals * 8) +
           a256(kb * 4) +
           a256(static_cast<size_t>(nsub) * 8) * 3 + a256(static_cast<size_t>(nsub) * 4);
}

xrdvi_status xrdvi_enumerate(const xrdvi_peaks *pk, const xrdvi_pattern *pt, const xrdvi_config *cfg,
                             int32_t iters, size_t hbm_budget, double *elbo_c, double *logp_c) {
    using xrdvi::report_error;
    if (!pk || !pt || !cfg || !logp_c) return report_error(XRDVI_EINVAL, "null argument");
    if (pk->K < 1 || pk->K > 16) return report_error(XRDVI_EINVAL, "enumeration needs K in [1, 16]");
    if (iters < 1) return report_error(XRDVI_EINVAL, "iters must be >= 1");
    XR_TRY_STATUS(xrdvi::validate_problem(pk, pt, cfg));
    const int K = pk->K, n = (1 << K) - 1, S = cfg->S, M = pk->offsets[K];
    // sub-models per batch: as many as the sample limit and the budget allow
    int Bmax = std::min(n, xrdvi::kMaxS / S);
    while (Bmax > 1 && xrdvi_enumerate_footprint_bytes(K, pt->N, M, S, Bmax) > hbm_budget) Bmax = (Bmax + 1) / 2;
    if (Bmax < 1 || xrdvi_enumerate_footprint_bytes(K, pt->N, M, S, Bmax) > hbm_budget)
        return report_error(XRDVI_ENOMEM, "one sub-model fit needs more than hbm_budget");
    const int tail = std::max(1, iters / 4);
    std::vector<double> score(n, 0.0);
    std::vector<uint32_t> masks;
    for (int first = 1; first <= n; first += Bmax) {
        const int nb = std::min(Bmax, n - first + 1);
        masks.resize(nb);
        for (int i = 0; i < nb; ++i) masks[i] = static_cast<uint32_t>(first + i);
        xrdvi_ctx *c = nullptr;
        XR_TRY_STATUS(xrdvi::create_batch_context(pk, pt, cfg, nb, masks.data(), nullptr, nullptr, &c));
        xrdvi_status st = xrdvi::batch_set_tail(c, iters - tail);
        if (st == XRDVI_OK) st = xrdvi_fit(c, iters, nullptr);
        if (st == XRDVI_OK) st = xrdvi::batch_tail_sums(c, score.data() + (first - 1));
        xrdvi_destroy(c);
        if (st != XRDVI_OK) return st;
    }
    for (double &v : score) {
        v /= tail;
        if (!std::isfinite(v)) return report_error(XRDVI_ENONFINITE, "enumeration: a sub-model ELBO is not finite");
    }
    // normalisation on the device (FP64 log-sum-exp)
    double *d = nullptr;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocAsync(&d, sizeof(double) * 2 * n, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, score.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        xrdvi::launch_enum_lse(d, n, d + n, s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(logp_c, d + n, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
    if (d) cudaFreeAsync(d, s);
    const cudaError_t e2 = s ? cudaStreamSynchronize(s) : cudaSuccess;
    if (s) cudaStreamDestroy(s);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return report_error(XRDVI_ECUDA, std::string("enumeration: ") + cudaGetErrorString(e));
    if (elbo_c) std::memcpy(elbo_c, score.data(), sizeof(double) * n);
    return XRDVI_OK;
}

}  // extern "C"
