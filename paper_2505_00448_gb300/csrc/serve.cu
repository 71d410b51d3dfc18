// Serving loop: not built yet in this file.
#include "napg_internal.cuh"

extern "C" {
napg_status napg_serve_start(napg_ctx *ctx, size_t, int32_t) { return napg::fail(ctx, NAPG_E_UNSUPPORTED, "serving not built"); }
napg_status napg_serve_submit(napg_ctx *ctx, const napg_request *, uint64_t *) { return napg::fail(ctx, NAPG_E_UNSUPPORTED, "serving not built"); }
napg_status napg_serve_poll(napg_ctx *ctx, uint64_t, int32_t *, double *, int32_t *) { return napg::fail(ctx, NAPG_E_UNSUPPORTED, "serving not built"); }
napg_status napg_serve_stop(napg_ctx *ctx) { (void)ctx; return NAPG_OK; }
}
