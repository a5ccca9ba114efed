// P2M and M2P launches of every compiled Taylor order, float arithmetic.
#include "farfield.cuh"

namespace lspr {

int p2m_orders_f32(lspr_ctx *ctx, int B) {
    LSPR_DISPATCH_P(p2m_launch, float, B, ctx, B);
    return LSPR_OK;
}

int m2p_orders_f32(lspr_ctx *ctx, double *acc, int *counter, int B) {
    if (B > 1 && (ctx->tensor_cores & 1)) {
        const int rc = m2p_tc_launch(ctx, acc, counter, B);
        if (rc != LSPR_E_STATE) return rc;
    }
    LSPR_DISPATCH_P(m2p_launch, float, B, ctx, acc, counter, B);
    return LSPR_OK;
}

}  // namespace lspr
