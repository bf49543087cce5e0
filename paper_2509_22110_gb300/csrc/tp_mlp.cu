// tp_mlp.cu - learned far field (placeholder until the network kernels land)
#include "tp_internal.cuh"
void tp_mlp_release(tp_ctx*) {}
extern "C" tp_status tp_far_model_load(tp_ctx* ctx, const char*) {
    return tp_set_err(ctx, TP_E_MODEL, "far-field model not available in this build");
}
