// Check of the bounded barrier wait that every pipeline wait of the tensor-core kernels uses:
// one thread waits on a shared-memory mbarrier that nothing arrives on.  The wait must give up
// after its limit (about one second), raise the abort flag, and leave the context usable.  No
// fault, trap or endless loop is involved: the wait is the product kernels' own helper.
#include "lspr_internal.cuh"
#include "tcgen05.cuh"

namespace lspr {

namespace {

__global__ void wait_timeout_kernel(int *out) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ volatile int abort_flag;
    if (threadIdx.x != 0) return;
    abort_flag = 0;
    tc::bar_init(tc::smem_addr(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const uint64_t t0 = tc::now_ns();
    const bool ok = tc::bar_wait(tc::smem_addr(&bar), 0u, &abort_flag);   // nobody arrives
    const uint64_t t1 = tc::now_ns();
    out[0] = ok ? 1 : 0;
    out[1] = abort_flag;
    out[2] = (int)((t1 - t0) / 1000000ull);   // milliseconds waited
}

}  // namespace

int selftest_wait_timeout(lspr_ctx *ctx, int32_t *result) {
    DArr<int> &buf = ctx->counters;   // 8 ints, cleared per product; free between calls
    LSPR_TRY(ctx, buf.ensure(8));
    LSPR_TRY(ctx, cudaMemsetAsync(buf.p, 0, 3 * sizeof(int), ctx->stream));
    ++ctx->n_launches;
    wait_timeout_kernel<<<1, 32, 0, ctx->stream>>>(buf.p);
    LSPR_TRY(ctx, cudaGetLastError());
    int h[3] = {0, 0, 0};
    LSPR_TRY(ctx, cudaMemcpyAsync(h, buf.p, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    LSPR_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    result[0] = h[0];
    result[1] = h[1];
    result[2] = h[2];
    return LSPR_OK;
}

}  // namespace lspr
