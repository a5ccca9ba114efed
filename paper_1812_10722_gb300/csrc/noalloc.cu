// Allocation-free variant of the direct FP32 matrix-vector product.
//
// lspr_matvec allocates its per-call scratch (source weights, far-field
// accumulators, staging) on first use.  Some callers cannot allow that: code that
// runs inside a host application whose device memory is owned by another
// allocator (a framework's caching pool, a fixed memory budget), and
// latency-critical loops in which cudaMalloc/cudaFree would stall, since those
// calls can synchronise the whole device.  For them this entry point does the
// same direct FP32 product with its scratch in one file-scope device array of
// fixed size and never calls cudaMalloc, cudaFree or an allocating library routine.
//
// Set-up: the first call on a device, with that device current, resolves the
// array's device address with cudaGetSymbolAddress and caches it for the device
// (the host-side name of the array is not a device address).  The CUDA runtime
// creates the array when it loads this library's device code onto the device; with
// lazy module loading (the runtime's default) that happens during this first
// lookup, so the first call may allocate the array itself (about 1.5 MiB) and the
// calls after it do not.  Make that first call before any stream capture begins
// and before the phase in which the caller cannot allow allocation.  The cached
// address belongs to the device's primary context (the one the runtime API uses):
// it does not survive cudaDeviceReset, and a context whose stream lives in another
// CUDA context must not use this entry point.
//
// Sharing: every call on a device uses the same array and leaves its contents
// behind; each call clears the accumulators it needs before use.  Calls that
// overlap on the GPU (different streams, or different contexts on one device)
// race on the array and must be serialised by the caller.
#include <mutex>

#include "lspr_internal.cuh"

namespace lspr {

constexpr int64_t kNoAllocMaxPanels = 16384;
constexpr int64_t kNoAllocMaxSources = 4 * kNoAllocMaxPanels;   // far rule with at most 4 points
// [source weights: kNoAllocMaxSources float4][accumulators: kNoAllocMaxPanels x 4 double]
constexpr size_t kNoAllocWeightBytes = kNoAllocMaxSources * sizeof(float4);
constexpr size_t kNoAllocBytes = kNoAllocWeightBytes + kNoAllocMaxPanels * 4 * sizeof(double);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[kMaxDevices] = {nullptr};

static cudaError_t noalloc_scratch(int device, void **out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[device] = p;
    }
    *out = g_noalloc_ptr[device];
    return cudaSuccess;
}

// Block rows of Eq. matrix_lspr from the far-field accumulators and the FP64
// near-singular CSR, with s passed by value (one warp per row).
__global__ void noalloc_assemble_kernel(int64_t N, const double *__restrict__ acc, const int64_t *__restrict__ ptr,
                                        const int *__restrict__ col, const double *__restrict__ dV,
                                        const double *__restrict__ dK, const double2 *__restrict__ x, double2 s,
                                        double2 *y) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    double vr = 0, vi = 0, kr = 0, ki = 0;
    for (int64_t e = ptr[i] + lane; e < ptr[i + 1]; e += 32) {
        const int j = col[e];
        const double a = dV[e], b = dK[e];
        const double2 ph = x[j], dp = x[N + j];
        vr += a * dp.x;
        vi += a * dp.y;
        kr += b * ph.x;
        ki += b * ph.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        vr += __shfl_xor_sync(0xffffffffu, vr, o);
        vi += __shfl_xor_sync(0xffffffffu, vi, o);
        kr += __shfl_xor_sync(0xffffffffu, kr, o);
        ki += __shfl_xor_sync(0xffffffffu, ki, o);
    }
    if (lane != 0) return;
    const double Vr = acc[4 * i] + vr, Vi = acc[4 * i + 1] + vi;
    const double Kr = acc[4 * i + 2] + kr, Ki = acc[4 * i + 3] + ki;
    const double2 ph = x[i];
    const double svr = s.x * Vr - s.y * Vi, svi = s.x * Vi + s.y * Vr;
    y[i] = make_double2(0.5 * ph.x + Kr - Vr, 0.5 * ph.y + Ki - Vi);
    y[N + i] = make_double2(0.5 * ph.x - Kr + svr, 0.5 * ph.y - Ki + svi);
}

}  // namespace lspr

using namespace lspr;

extern "C" int lspr_matvec_direct_fp32_noalloc(lspr_ctx *c, const double *x, double *y, double s_re, double s_im) {
    if (!c || !x || !y) return LSPR_E_ARG;
    if (!c->mesh.ready) return LSPR_E_STATE;
    const Mesh &m = c->mesh;
    if (m.S != 1) {
        c->last_error = "lspr_matvec_direct_fp32_noalloc: one surface only";
        return LSPR_E_STATE;
    }
    if (m.N > kNoAllocMaxPanels || m.Ns > kNoAllocMaxSources) {
        c->last_error = "lspr_matvec_direct_fp32_noalloc: mesh exceeds the fixed scratch (16384 panels, 65536 sources)";
        return LSPR_E_ARG;
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return LSPR_E_CUDA;
    void *base = nullptr;
    LSPR_TRY(c, noalloc_scratch(c->device, &base));
    float4 *w = (float4 *)base;
    double *acc = (double *)((unsigned char *)base + kNoAllocWeightBytes);
    cudaStream_t st = c->stream;
    LSPR_TRY(c, cudaMemsetAsync(acc, 0, sizeof(double) * 4 * m.N, st));
    ++c->n_launches;
    LSPR_TRY_ST(launch_weights_fp32_raw(st, m.Ns, m.N, c->wo.spos64.p, c->wo.src_panel.p, (const double2 *)x, w));
    ++c->n_launches;
    LSPR_TRY_ST(launch_p2p_fp32_raw(st, c->direct.items.p, c->direct.n, c->wo.tgt32.p, m.N, c->wo.spos32.p,
                                    c->wo.snrm32.p, w, acc));
    ++c->n_launches;
    noalloc_assemble_kernel<<<grid_for(m.N * 32, 256), 256, 0, st>>>(m.N, acc, m.near_ptr.p, m.near_col.p,
                                                                     m.near_dV.p, m.near_dK.p, (const double2 *)x,
                                                                     make_double2(s_re, s_im), (double2 *)y);
    LSPR_TRY(c, cudaGetLastError());
    return LSPR_OK;
}
