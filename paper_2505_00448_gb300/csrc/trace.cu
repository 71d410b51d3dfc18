// Stage tracing (CUDA events) and the library-wide kernel launch counter.
#include <atomic>
#include <cstdio>

#include "napg_internal.cuh"

namespace napg {

static std::atomic<uint64_t> g_launches{0};

void count_launch(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
// launches recorded into a CUDA graph run later, when the graph is launched
void uncount_launches(uint64_t k) { g_launches.fetch_sub(k, std::memory_order_relaxed); }

static cudaEvent_t take_event(Tracer &t) {
    if (!t.pool.empty()) {
        cudaEvent_t e = t.pool.back();
        t.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

Stage::Stage(Tracer &t, cudaStream_t s, const char *n) : tr(&t), st(s), name(n) {
    if (!t.on) { tr = nullptr; return; }
    std::lock_guard<std::mutex> lk(t.mu);
    a = take_event(t);
    cudaEventRecord(a, st);
    l0 = launches_so_far();
}

void Stage::end() {
    if (!tr) return;
    std::lock_guard<std::mutex> lk(tr->mu);
    cudaEvent_t b = take_event(*tr);
    cudaEventRecord(b, st);
    tr->pending.push_back({name, a, b, launches_so_far() - l0});
    tr = nullptr;
}

}  // namespace napg

using namespace napg;

extern "C" {

napg_status napg_trace_enable(napg_ctx *ctx, int32_t on) {
    if (!ctx) return NAPG_E_ARG;
    ctx->trace.on = on != 0;
    return NAPG_OK;
}

napg_status napg_trace_read(napg_ctx *ctx, char *buf, size_t cap) {
    if (!ctx || !buf || cap == 0) return NAPG_E_ARG;
    Tracer &t = ctx->trace;
    std::lock_guard<std::mutex> lk(t.mu);
    for (auto &r : t.pending) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventSynchronize(trace)");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        bool found = false;
        for (auto &g : t.agg)
            if (g.first == r.name) { g.second.ms += ms; g.second.launches += r.launches; found = true; break; }
        if (!found) {
            Tracer::Agg a;
            a.ms = ms;
            a.launches = r.launches;
            t.agg.push_back({r.name, a});
        }
        t.pool.push_back(r.a);
        t.pool.push_back(r.b);
    }
    t.pending.clear();
    std::string out = "{\"stages\": {";
    bool first = true;
    char tmp[256];
    for (auto &g : t.agg) {
        snprintf(tmp, sizeof(tmp), "%s\"%s\": {\"launches\": %llu, \"ms\": %.6f}", first ? "" : ", ", g.first.c_str(),
                 (unsigned long long)g.second.launches, g.second.ms);
        out += tmp;
        first = false;
    }
    snprintf(tmp, sizeof(tmp), "}, \"kernel_launches\": %llu}", (unsigned long long)launches_so_far());
    out += tmp;
    t.agg.clear();
    const size_t n = std::min(cap - 1, out.size());
    memcpy(buf, out.data(), n);
    buf[n] = '\0';
    return NAPG_OK;
}

uint64_t napg_kernel_launches(void) { return launches_so_far(); }

}  // extern "C"
