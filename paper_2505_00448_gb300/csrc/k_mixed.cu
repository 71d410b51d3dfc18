// Mixed-precision (tcgen05) moment contractions: not built yet in this file.
#include "napg_internal.cuh"

namespace napg {

napg_status mixed_pearson(napg_ctx *ctx, Workspace &, cudaStream_t, const int32_t *, int32_t, const uint32_t *, double *,
                          double *, double *, int32_t *, double *) {
    return fail(ctx, NAPG_E_UNSUPPORTED, "NAPG_MIXED is not available in this build");
}
napg_status mixed_groupsum(napg_ctx *ctx, Workspace &, cudaStream_t, const uint32_t *, int32_t, const int32_t *, int32_t,
                           const uint32_t *, int32_t *, double *, double *, double *) {
    return fail(ctx, NAPG_E_UNSUPPORTED, "NAPG_MIXED is not available in this build");
}
napg_status mixed_contingency(napg_ctx *ctx, Workspace &, cudaStream_t, const uint32_t *, int32_t, int32_t *) {
    return fail(ctx, NAPG_E_UNSUPPORTED, "NAPG_MIXED is not available in this build");
}

}  // namespace napg
