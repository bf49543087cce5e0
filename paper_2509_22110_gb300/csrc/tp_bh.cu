// tp_bh.cu - Barnes-Hut traversal (placeholder until the traversal kernels land)
#include "tp_internal.cuh"
tp_status tp_launch_bh(tp_ctx* ctx, const tp_params*, bool) {
    return tp_set_err(ctx, TP_E_STATE, "Barnes-Hut not available in this build");
}
