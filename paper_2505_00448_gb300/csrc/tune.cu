// Autotuner: picks a launch shape per problem shape by timing the candidates
// once (CUDA events on the run's own stream) and keeping the fastest for the
// rest of the context's life. Candidates of one kind give identical results,
// so the tuning run's outputs stand. A shape near a recorded one (same kind, K
// within a factor of 2, rows within a factor of 4) takes its choice without
// timing.
// While a stream is being captured into a graph nothing can be timed: the
// choice recorded for the closest shape (same kind and rows, nearest K) is
// used, else the first candidate.
#include <cstdio>
#include <cmath>
#include <cstring>
#include <string>

#include "napg_internal.cuh"

namespace napg {

static const char *kind_name(int k) {
    switch (k) {
        case kTuneStackMask: return "stacked_mask";
        case kTuneStackOneHot: return "stacked_onehot";
        case kTuneSpearman: return "spearman_threads";
        case kTuneRankGroups: return "rank_groups_threads";
        case kTuneStackOneHotNS1: return "stacked_onehot_counts_sums";
        case kTuneStackSquares: return "stacked_observed_squares";
        case kTuneSxy: return "sxy_stage_samples";
        default: return "unknown";
    }
}

napg_status tuned_launch(napg_ctx *ctx, const TuneKey &key, int ncand, const std::function<napg_status(int)> &run,
                         cudaStream_t st) {
    Tuner &T = ctx->tune;
    int choice = -1;
    {
        std::lock_guard<std::mutex> lk(T.mu);
        auto pin = T.pinned.find(key.kind);
        if (pin != T.pinned.end()) choice = pin->second;
    }
    if (choice >= 0) {
        if (choice >= ncand) return fail(ctx, NAPG_E_ARG, "pinned launch shape out of range");
        return run(choice);
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        (void)cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;   // be safe: no timing
    }
    {
        std::lock_guard<std::mutex> lk(T.mu);
        auto it = T.best.find(key);
        auto ld = [](int64_t x, int64_t y) { return std::fabs(std::log((double)(x + 1) / (double)(y + 1))); };
        if (it != T.best.end()) {
            choice = it->second.choice;
        } else if (cs != cudaStreamCaptureStatusNone || !T.on || ncand < 2) {
            // nearest recorded shape of the same kind and rows
            double bestd = 1e300;
            for (auto &kv : T.best)
                if (kv.first.kind == key.kind && kv.first.a == key.a && kv.first.b == key.b) {
                    const double d = ld(kv.first.c, key.c);
                    if (d < bestd) { bestd = d; choice = kv.second.choice; }
                }
            if (choice < 0) choice = 0;
        } else {
            // a recorded shape of the same kind close to this one (K within a
            // factor of 2, rows within a factor of 4) decides without timing: a
            // stream of requests or sample contexts of varied sizes times a few
            // size classes, not every one
            double bestd = 1e300;
            for (auto &kv : T.best)
                if (kv.first.kind == key.kind && ld(kv.first.c, key.c) <= std::log(2.0) &&
                    ld(kv.first.a, key.a) <= std::log(4.0) && ld(kv.first.b, key.b) <= std::log(4.0)) {
                    const double d = ld(kv.first.a, key.a) + ld(kv.first.b, key.b) + ld(kv.first.c, key.c);
                    if (d < bestd) { bestd = d; choice = kv.second.choice; }
                }
        }
    }
    if (choice >= 0) return run(choice);
    // time every candidate once; outputs of the last run stand (all equal)
    std::vector<float> ms(ncand, 0.f);
    cudaEvent_t e0, e1;
    NAPG_CU(ctx, cudaEventCreate(&e0));
    NAPG_CU(ctx, cudaEventCreate(&e1));
    napg_status rc = NAPG_OK;
    for (int c = 0; c < ncand && rc == NAPG_OK; ++c) {
        if (cudaEventRecord(e0, st) != cudaSuccess) { rc = NAPG_E_CUDA; break; }
        rc = run(c);
        if (rc != NAPG_OK) break;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { rc = NAPG_E_CUDA; break; }
        cudaEventElapsedTime(&ms[c], e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != NAPG_OK) {
        (void)cudaGetLastError();
        return rc == NAPG_E_CUDA ? fail(ctx, NAPG_E_CUDA, "autotuning run failed") : rc;
    }
    int best = 0;
    for (int c = 1; c < ncand; ++c)
        if (ms[c] < ms[best]) best = c;
    {
        std::lock_guard<std::mutex> lk(T.mu);
        T.best[key] = TuneRec{best, ms};
    }
    // leave the outputs of the chosen shape in place when it was not the last one run
    if (best != ncand - 1) return run(best);
    return NAPG_OK;
}

}  // namespace napg

using namespace napg;

extern "C" {

napg_status napg_tune_enable(napg_ctx *ctx, int32_t on) {
    if (!ctx) return NAPG_E_ARG;
    std::lock_guard<std::mutex> lk(ctx->tune.mu);
    ctx->tune.on = on != 0;
    return NAPG_OK;
}

napg_status napg_tune_pin(napg_ctx *ctx, const char *kind, int32_t choice) {
    if (!ctx || !kind || choice < -1 || choice > 3) return NAPG_E_ARG;
    int k = 0;
    for (int c = 1; c <= kTuneKindMax; ++c)
        if (strcmp(kind_name(c), kind) == 0) k = c;
    if (!k) return fail(ctx, NAPG_E_ARG, std::string("unknown launch-shape kind: ") + kind);
    std::lock_guard<std::mutex> lk(ctx->tune.mu);
    if (choice < 0) ctx->tune.pinned.erase(k);
    else ctx->tune.pinned[k] = choice;
    return NAPG_OK;
}

napg_status napg_tune_read(napg_ctx *ctx, char *buf, size_t cap) {
    if (!ctx || !buf || cap == 0) return NAPG_E_ARG;
    std::lock_guard<std::mutex> lk(ctx->tune.mu);
    std::string out = "[";
    bool first = true;
    for (auto &kv : ctx->tune.best) {
        char tmp[256];
        snprintf(tmp, sizeof(tmp), "%s{\"kind\": \"%s\", \"rows_a\": %lld, \"rows_b\": %lld, \"k\": %lld, \"choice\": %d, \"ms\": [",
                 first ? "" : ", ", kind_name(kv.first.kind), (long long)kv.first.a, (long long)kv.first.b,
                 (long long)kv.first.c, kv.second.choice);
        out += tmp;
        for (size_t i = 0; i < kv.second.ms.size(); ++i) {
            snprintf(tmp, sizeof(tmp), "%s%.4f", i ? ", " : "", kv.second.ms[i]);
            out += tmp;
        }
        out += "]}";
        first = false;
    }
    out += "]";
    if (out.size() + 1 > cap) return fail(ctx, NAPG_E_ARG, "buffer too small");
    memcpy(buf, out.c_str(), out.size() + 1);
    return NAPG_OK;
}

}  // extern "C"
