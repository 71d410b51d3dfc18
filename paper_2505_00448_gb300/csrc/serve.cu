// Serving loop over the resident cohort (Sec. 1: on-the-fly, real-time
// analyses of a cohort that stays in memory).
//
// A scheduler thread owns `slots` execution slots, each with its own CUDA
// stream, workspace, mask staging and pinned output staging. Requests (test,
// options, sample mask, variable subsets, host outputs) wait in a FIFO queue and
// are admitted continuously: whenever a slot is idle and the request's device
// memory estimate fits in the budget next to what the other slots hold, it is
// launched on that slot's stream, so the kernels of several requests overlap on
// the device. A request finishes when its device-to-host copies complete (an
// event per slot); its latency is measured from submission to that moment.
// The presort of the continuous variables (shared, read-only) is built once at
// start. Results do not depend on what else runs: every kernel reduces in a
// fixed order.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>

#include "napg_internal.cuh"

namespace napg {

using Clock = std::chrono::steady_clock;

// A request that has waited this long stops smaller requests from overtaking it.
constexpr double kMaxOvertakeMs = 200.0;
constexpr size_t kMaxQueued = 1 << 16;

struct ServeReq {
    uint64_t ticket = 0;
    int32_t test = 0;
    napg_options opt{};
    std::vector<uint8_t> mask;
    bool has_mask = false;
    std::vector<int32_t> va, vb;
    bool symmetric = true;
    double *stat = nullptr, *pval = nullptr;
    int32_t *n = nullptr;
    int64_t cnt = 0;
    size_t est = 0;
    Clock::time_point t_submit;
    bool done = false;
    int32_t status = NAPG_OK;
    double latency_ms = 0.0;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    Workspace ws;
    uint8_t *mask = nullptr;
    size_t mask_cap = 0;
    double *h_stat = nullptr, *h_p = nullptr;   // pinned staging
    int32_t *h_n = nullptr;
    size_t h_cap = 0;
    uint32_t *h_err = nullptr;                   // pinned copy of the device error word
    std::shared_ptr<ServeReq> req;
};

struct ServeState {
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<ServeReq>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<ServeReq>> tickets;
    std::vector<Slot> slots;
    size_t budget = 0;
    bool stopping = false;
    uint64_t next_ticket = 1;
};

// Device bytes a request needs beyond the resident cohort (an upper estimate
// of the workspace run_on_stream grows for it, plus its mask).
size_t request_bytes(const Cohort &c, int32_t test, const napg_options &opt, const std::vector<int32_t> &va,
                     const std::vector<int32_t> &vb, bool symmetric) {
    const double S = (double)c.S, W = (double)c.W, Sp = std::ceil(S / 64.0) * 64.0;
    const double na = (double)va.size(), nb = symmetric ? na : (double)vb.size();
    const double pairs = na * nb;
    double R = 0.0;
    if (test != NAPG_PEARSON && test != NAPG_SPEARMAN)
        for (int32_t v : va) R += c.nlev[v];
    const bool mixed = opt.precision == NAPG_MIXED;
    auto pad128 = [](double x) { return std::ceil(x / 128.0) * 128.0; };
    double b = S + 20.0 * pairs + 4.0 * (na + nb) * W + 84.0 * pairs + 64.0 * (na + nb) + 4096.0;
    switch (test) {
        case NAPG_PEARSON: {
            double nu = na;
            if (!symmetric) {
                nu = na + nb;                       // union of the lists
                b += 20.0 * nu * nu + 84.0 * nu * nu;
            }
            b += 28.0 * nu * nu;
            b += mixed ? 10.0 * pad128(nu) * Sp + 16.0 * nu : 8.0 * nu * Sp;
        } break;
        case NAPG_SPEARMAN: b += 32.0 * pairs; break;
        case NAPG_CHI2: {
            double RR = R;
            if (!symmetric) {
                RR = R;
                for (int32_t v : vb) RR += c.nlev[v];
                b += 104.0 * (na + nb) * (na + nb);
            }
            b += 4.0 * RR * W + 4.0 * RR * RR + (mixed ? 2.0 * pad128(RR) * Sp : 0.0);
        } break;
        case NAPG_ANOVA:
        case NAPG_TTEST:
            b += 4.0 * R * W + 20.0 * R * nb;
            b += mixed ? 10.0 * pad128(nb) * Sp + 2.0 * pad128(R) * Sp : 8.0 * nb * Sp;
            break;
        default:  // MWU, KRUSKAL
            b += 4.0 * R * W + 12.0 * R * nb + 8.0 * pairs + 64.0 * S;
            break;
    }
    return (size_t)(b * 1.1);
}

// Admission plan (host logic only). Queue entries in arrival order with their
// memory estimates and ages; slots with their held memory and whether busy.
// Each idle slot takes the first queued request whose estimate fits next to
// what the other slots hold; a request older than kMaxOvertakeMs blocks later
// ones from overtaking it. assign[k] = queue index given to slot k, or -1.
void plan_admission(const size_t *est, const double *age_ms, int32_t nq, const size_t *slot_mem,
                    const int32_t *slot_busy, int32_t nslots, size_t budget, int32_t *assign) {
    std::vector<size_t> mem(slot_mem, slot_mem + nslots);
    std::vector<char> taken(nq, 0);
    for (int32_t k = 0; k < nslots; ++k) assign[k] = -1;
    for (int32_t k = 0; k < nslots; ++k) {
        if (slot_busy[k]) continue;
        size_t others = 0;
        for (int32_t j = 0; j < nslots; ++j)
            if (j != k) others += mem[j];
        for (int32_t q = 0; q < nq; ++q) {
            if (taken[q]) continue;
            const size_t need = std::max(mem[k], est[q]);
            if (others + need <= budget) {
                assign[k] = q;
                taken[q] = 1;
                mem[k] = need;
                break;
            }
            if (age_ms[q] >= kMaxOvertakeMs) break;   // the oldest waiting request goes first
        }
    }
}

static napg_status slot_grow(napg_ctx *ctx, Slot &s, int64_t cnt, int64_t S) {
    if (s.mask_cap < (size_t)S) {
        if (s.mask) cudaFree(s.mask);
        s.mask = nullptr;
        s.mask_cap = 0;
        NAPG_CU(ctx, cudaMalloc(&s.mask, (size_t)S));
        s.mask_cap = (size_t)S;
    }
    if (s.h_cap < (size_t)cnt) {
        if (s.h_stat) cudaFreeHost(s.h_stat);
        if (s.h_p) cudaFreeHost(s.h_p);
        if (s.h_n) cudaFreeHost(s.h_n);
        s.h_stat = s.h_p = nullptr;
        s.h_n = nullptr;
        s.h_cap = 0;
        NAPG_CU(ctx, cudaMallocHost(&s.h_stat, sizeof(double) * (size_t)cnt));
        NAPG_CU(ctx, cudaMallocHost(&s.h_p, sizeof(double) * (size_t)cnt));
        NAPG_CU(ctx, cudaMallocHost(&s.h_n, sizeof(int32_t) * (size_t)cnt));
        s.h_cap = (size_t)cnt;
    }
    return NAPG_OK;
}

// enqueue request r on slot s (scheduler thread)
static napg_status slot_launch(napg_ctx *ctx, Slot &s, ServeReq &r) {
    const Cohort &c = ctx->coh;
    NAPG_ST(slot_grow(ctx, s, r.cnt, c.S));
    if (r.has_mask) NAPG_CU(ctx, cudaMemcpyAsync(s.mask, r.mask.data(), (size_t)c.S, cudaMemcpyHostToDevice, s.st));
    napg_status st_ = NAPG_OK;
    double *ds = (double *)ws_get(ctx, s.ws, Workspace::kOutStat, sizeof(double) * (size_t)r.cnt, &st_);
    double *dp = (double *)ws_get(ctx, s.ws, Workspace::kOutP, sizeof(double) * (size_t)r.cnt, &st_);
    int32_t *dn = (int32_t *)ws_get(ctx, s.ws, Workspace::kOutN, sizeof(int32_t) * (size_t)r.cnt, &st_);
    if (st_) return st_;
    RunArgs a{};
    a.test = r.test;
    a.opt = r.opt;
    a.mask = r.has_mask ? s.mask : nullptr;
    a.mask_on_device = true;
    a.va = r.va.data();
    a.na = (int32_t)r.va.size();
    a.vb = r.symmetric ? nullptr : r.vb.data();
    a.nb = r.symmetric ? a.na : (int32_t)r.vb.size();
    a.stat = ds;
    a.pval = r.pval ? dp : nullptr;
    a.n = dn;
    NAPG_ST(run_on_stream(ctx, s.ws, s.st, a));
    if (r.stat || r.test == NAPG_MWU)
        NAPG_CU(ctx, cudaMemcpyAsync(s.h_stat, ds, sizeof(double) * (size_t)r.cnt, cudaMemcpyDeviceToHost, s.st));
    if (r.pval) NAPG_CU(ctx, cudaMemcpyAsync(s.h_p, dp, sizeof(double) * (size_t)r.cnt, cudaMemcpyDeviceToHost, s.st));
    if (r.n) NAPG_CU(ctx, cudaMemcpyAsync(s.h_n, dn, sizeof(int32_t) * (size_t)r.cnt, cudaMemcpyDeviceToHost, s.st));
    NAPG_CU(ctx, cudaMemcpyAsync(s.h_err, ctx->dev_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s.st));
    NAPG_CU(ctx, cudaEventRecord(s.ev, s.st));
    return NAPG_OK;
}

static void finish(ServeState &S, ServeReq &r, int32_t status) {
    r.status = status;
    r.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r.t_submit).count();
    r.done = true;
    (void)S;
}

static void scheduler(napg_ctx *ctx) {
    ServeState &S = *ctx->serve;
    cudaSetDevice(ctx->device);
    const int32_t ns = (int32_t)S.slots.size();
    std::vector<size_t> est, mem(ns);
    std::vector<double> age;
    std::vector<int32_t> busy(ns), assign(ns);
    while (true) {
        bool progressed = false;
        // completions
        for (int32_t k = 0; k < ns; ++k) {
            Slot &s = S.slots[k];
            if (!s.req) continue;
            const cudaError_t q = cudaEventQuery(s.ev);
            if (q == cudaErrorNotReady) continue;
            ServeReq &r = *s.req;
            int32_t status = NAPG_OK;
            if (q != cudaSuccess) {
                status = NAPG_E_CUDA;
                (void)cudaGetLastError();
            } else {
                if (r.stat) std::copy(s.h_stat, s.h_stat + r.cnt, r.stat);
                if (r.pval) std::copy(s.h_p, s.h_p + r.cnt, r.pval);
                if (r.n) std::copy(s.h_n, s.h_n + r.cnt, r.n);
                if (*(volatile uint32_t *)s.h_err & kErrTimeout) status = NAPG_E_TIMEOUT;
                else if (*(volatile uint32_t *)s.h_err & kErrExactLimit) status = NAPG_E_UNSUPPORTED;
            }
            {
                std::lock_guard<std::mutex> lk(S.mu);
                finish(S, r, status);
            }
            S.cv.notify_all();
            s.req.reset();
            progressed = true;
        }
        // admissions
        std::vector<std::shared_ptr<ServeReq>> picked(ns);
        {
            std::lock_guard<std::mutex> lk(S.mu);
            bool any_running = false;
            for (auto &s : S.slots) any_running |= (bool)s.req;
            if (S.stopping && S.queue.empty() && !any_running) break;
            const int32_t nq = (int32_t)std::min<size_t>(S.queue.size(), 4096);
            if (nq > 0) {
                est.resize(nq);
                age.resize(nq);
                const auto now = Clock::now();
                for (int32_t q = 0; q < nq; ++q) {
                    est[q] = S.queue[q]->est;
                    age[q] = std::chrono::duration<double, std::milli>(now - S.queue[q]->t_submit).count();
                }
                for (int32_t k = 0; k < ns; ++k) {
                    mem[k] = S.slots[k].ws.total();
                    busy[k] = S.slots[k].req ? 1 : 0;
                }
                plan_admission(est.data(), age.data(), nq, mem.data(), busy.data(), ns, S.budget, assign.data());
                std::vector<char> drop(nq, 0);
                for (int32_t k = 0; k < ns; ++k)
                    if (assign[k] >= 0) {
                        picked[k] = S.queue[assign[k]];
                        drop[assign[k]] = 1;
                    }
                std::deque<std::shared_ptr<ServeReq>> rest;
                for (int32_t q = 0; q < (int32_t)S.queue.size(); ++q)
                    if (q >= nq || !drop[q]) rest.push_back(S.queue[q]);
                S.queue.swap(rest);
            }
        }
        for (int32_t k = 0; k < ns; ++k) {
            if (!picked[k]) continue;
            Slot &s = S.slots[k];
            napg_status rc = slot_launch(ctx, s, *picked[k]);
            if (rc != NAPG_OK) {
                cudaStreamSynchronize(s.st);
                {
                    std::lock_guard<std::mutex> lk(S.mu);
                    finish(S, *picked[k], rc);
                }
                S.cv.notify_all();
            } else {
                s.req = picked[k];
            }
            progressed = true;
        }
        if (!progressed) {
            std::unique_lock<std::mutex> lk(S.mu);
            S.cv.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

static void free_serve(napg_ctx *ctx) {
    ServeState *S = ctx->serve;
    if (!S) return;
    for (auto &s : S->slots) {
        if (s.st) cudaStreamSynchronize(s.st);
        for (int i = 0; i < Workspace::kNumSlots; ++i)
            if (s.ws.ptr[i]) cudaFree(s.ws.ptr[i]);
        if (s.mask) cudaFree(s.mask);
        if (s.h_stat) cudaFreeHost(s.h_stat);
        if (s.h_p) cudaFreeHost(s.h_p);
        if (s.h_n) cudaFreeHost(s.h_n);
        if (s.h_err) cudaFreeHost(s.h_err);
        if (s.ev) cudaEventDestroy(s.ev);
        if (s.st) cudaStreamDestroy(s.st);
    }
    delete S;
    ctx->serve = nullptr;
}

}  // namespace napg

using namespace napg;

extern "C" {

napg_status napg_serve_start(napg_ctx *ctx, size_t mem_budget, int32_t slots) {
    if (!ctx || slots < 1 || slots > 64) return NAPG_E_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    if (ctx->serve) return fail(ctx, NAPG_E_BUSY, "serving already started");
    if (!ctx->coh.loaded) return fail(ctx, NAPG_E_ARG, "no cohort loaded");
    NAPG_CU(ctx, cudaSetDevice(ctx->device));
    // the shared presort, built before any slot reads it
    if (ctx->coh.n_cont > 0 && ctx->coh.S <= kMaxRankSamples) {
        NAPG_ST(ensure_presort(ctx, ctx->coh, ctx->ws, ctx->stream));
        NAPG_CU(ctx, cudaStreamSynchronize(ctx->stream));
    }
    if (mem_budget == 0) {
        size_t fr = 0, tot = 0;
        NAPG_CU(ctx, cudaMemGetInfo(&fr, &tot));
        mem_budget = (size_t)(0.8 * (double)fr);
    }
    NAPG_CU(ctx, cudaMemsetAsync(ctx->dev_err, 0, sizeof(uint32_t), ctx->stream));
    *ctx->host_err = 0;
    NAPG_CU(ctx, cudaStreamSynchronize(ctx->stream));
    auto *S = new ServeState();
    S->budget = mem_budget;
    S->slots.resize(slots);
    for (auto &s : S->slots) {
        if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&s.h_err, sizeof(uint32_t)) != cudaSuccess) {
            ctx->serve = S;
            free_serve(ctx);
            return cuda_fail(ctx, cudaGetLastError(), "serve slot");
        }
    }
    ctx->serve = S;
    S->th = std::thread(scheduler, ctx);
    return NAPG_OK;
}

napg_status napg_serve_submit(napg_ctx *ctx, const napg_request *req, uint64_t *ticket) {
    if (!ctx || !req || !ticket) return NAPG_E_ARG;
    ServeState *S = ctx->serve;
    if (!S) return fail(ctx, NAPG_E_ARG, "serving not started");
    auto r = std::make_shared<ServeReq>();
    r->test = req->test;
    r->opt = req->opt;
    if (req->n_a < 0 || (req->n_a > 0 && !req->vars_a)) return fail(ctx, NAPG_E_ARG, "bad vars_a");
    r->va.assign(req->vars_a, req->vars_a + req->n_a);
    r->symmetric = req->vars_b == nullptr;
    if (!r->symmetric) {
        if (req->n_b < 0) return fail(ctx, NAPG_E_ARG, "bad vars_b");
        r->vb.assign(req->vars_b, req->vars_b + req->n_b);
    }
    RunArgs a{};
    a.test = r->test;
    a.opt = r->opt;
    a.va = r->va.data();
    a.na = (int32_t)r->va.size();
    a.vb = r->symmetric ? nullptr : r->vb.data();
    a.nb = r->symmetric ? a.na : (int32_t)r->vb.size();
    bool sym = false;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        NAPG_ST(check_run_vars(ctx, a, &sym));
    }
    const Cohort &c = ctx->coh;
    if (req->sample_mask) {
        r->has_mask = true;
        r->mask.assign(req->sample_mask, req->sample_mask + c.S);
    }
    r->stat = req->stat;
    r->pval = req->pval;
    r->n = req->n;
    r->cnt = (int64_t)a.na * a.nb;
    r->est = request_bytes(c, r->test, r->opt, r->va, r->vb, r->symmetric);
    if (r->est > S->budget) return fail(ctx, NAPG_E_UNSUPPORTED, "request larger than the serving memory budget");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stopping) return fail(ctx, NAPG_E_BUSY, "serving is stopping");
        if (S->queue.size() >= kMaxQueued) return fail(ctx, NAPG_E_BUSY, "serving queue full");
        r->ticket = S->next_ticket++;
        r->t_submit = Clock::now();
        S->tickets[r->ticket] = r;
        S->queue.push_back(r);
        *ticket = r->ticket;
    }
    S->cv.notify_all();
    return NAPG_OK;
}

napg_status napg_serve_poll(napg_ctx *ctx, uint64_t ticket, int32_t *done, double *latency_ms, int32_t *status_out) {
    if (!ctx || !done) return NAPG_E_ARG;
    ServeState *S = ctx->serve;
    if (!S) return fail(ctx, NAPG_E_ARG, "serving not started");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return fail(ctx, NAPG_E_ARG, "unknown ticket");
    const ServeReq &r = *it->second;
    *done = r.done ? 1 : 0;
    if (latency_ms) *latency_ms = r.done ? r.latency_ms : 0.0;
    if (status_out) *status_out = r.done ? r.status : NAPG_OK;
    if (r.done) S->tickets.erase(it);      // a finished ticket is reported once
    return NAPG_OK;
}

napg_status napg_serve_stop(napg_ctx *ctx) {
    if (!ctx) return NAPG_E_ARG;
    ServeState *S = ctx->serve;
    if (!S) return NAPG_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    free_serve(ctx);
    return NAPG_OK;
}

// the admission policy on its own (no GPU), for checking it
napg_status napg_serve_plan(const uint64_t *est, const double *age_ms, int32_t nq, const uint64_t *slot_mem,
                            const int32_t *slot_busy, int32_t nslots, uint64_t budget, int32_t *assign) {
    if (nq < 0 || nslots < 0 || (nq > 0 && (!est || !age_ms)) || (nslots > 0 && (!slot_mem || !slot_busy || !assign)))
        return NAPG_E_ARG;
    std::vector<size_t> e(est, est + nq), m(slot_mem, slot_mem + nslots);
    plan_admission(e.data(), age_ms, nq, m.data(), slot_busy, nslots, (size_t)budget, assign);
    return NAPG_OK;
}

}  // extern "C"
