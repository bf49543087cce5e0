// tp_lbvh.cu - cluster tree (placeholder until the LBVH kernels land)
#include "tp_internal.cuh"
tp_status tp_launch_tree_build(tp_ctx* ctx, int, int) {
    return tp_set_err(ctx, TP_E_STATE, "tree build not available in this build");
}
