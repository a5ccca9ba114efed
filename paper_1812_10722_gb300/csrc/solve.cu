// Operator assembly, GMRES and observables.
//   assemble_kernel   near-singular / singular correction (CSR SpMV, FP64) fused with
//                     the 2x2 block operator of Eq. matrix_lspr:
//                       y_top = phi/2 + K phi - V dphi,  y_bot = phi/2 - K phi + s V dphi
//   solve             right-hand side, the GMRES of gmres_graph.cu (B complex systems in
//                     lockstep, Sec. II.D-E), iterative refinement with a float-float or
//                     FP64 residual
//   dipole / sigma    p = -eps_out sum_j A_j (c_j dphi2s/dn_j - phi_j n_j),
//                     dphi2s/dn = s dphi1s/dn - ((eps_out - eps_in)/eps_out) dphi_inc/dn,
//                     sigma = Im(k^2 e.p / (eps_out |E0|)) / Re k, k = 2 pi sqrt(eps_out)/lambda
//                     (Eqs. dipole_def_gauss_i_final with outward normals, cext_fwa)
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>

#include "cplx.cuh"
#include "lspr_internal.cuh"

namespace lspr {

// principal square root
__device__ __forceinline__ double2 csqrt_p(double2 z) {
    const double r = sqrt(z.x * z.x + z.y * z.y);
    const double re = sqrt(fmax(0.0, 0.5 * (r + z.x)));
    double im = sqrt(fmax(0.0, 0.5 * (r - z.x)));
    if (z.y < 0) im = -im;
    return make_double2(re, im);
}

// ------------------------------------------------------------------ assembly
// RAW = true writes the layer potentials (V dphi, K phi) instead of the block rows.
// kRowLanes lanes per (row, right-hand side) read the row's near entries coalesced
// (rows hold ~25 entries); groups are ordered row-major so the B right-hand sides of a
// row reuse its CSR entries from cache.  acc is [panel][B][4], x and y are [B][2N].
constexpr int kRowLanes = 8;
template <bool RAW>
__global__ void assemble_kernel(int64_t N, int B, const double *__restrict__ acc, const int64_t *__restrict__ ptr,
                                const int *__restrict__ col, const double *__restrict__ dV,
                                const double *__restrict__ dK, const double2 *__restrict__ x, const double2 *s,
                                double2 *y, double2 *Vd, double2 *Kp, const int *inv) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t grp = g / kRowLanes;
    const int lane = (int)(g % kRowLanes);
    const int64_t i = grp / B;
    const int b = (int)(grp - i * B);
    // the far part of system b sits in slot inv[b] of acc (identity without a map); rows
    // of converged systems (slot -1) are left untouched
    const int slot = i < N ? (inv ? inv[b] : b) : -1;
    const bool valid = i < N && slot >= 0;
    const double2 *xb = x + (int64_t)b * 2 * N;
    double vr = 0, vi = 0, kr = 0, ki = 0;
    if (valid) {
        for (int64_t e = ptr[i] + lane; e < ptr[i + 1]; e += kRowLanes) {
            const int j = col[e];
            const double a = dV[e], c = dK[e];
            const double2 ph = xb[j], dp = xb[N + j];
            vr += a * dp.x;
            vi += a * dp.y;
            kr += c * ph.x;
            ki += c * ph.y;
        }
    }
#pragma unroll
    for (int o = kRowLanes / 2; o > 0; o >>= 1) {
        vr += __shfl_xor_sync(0xffffffffu, vr, o, kRowLanes);
        vi += __shfl_xor_sync(0xffffffffu, vi, o, kRowLanes);
        kr += __shfl_xor_sync(0xffffffffu, kr, o, kRowLanes);
        ki += __shfl_xor_sync(0xffffffffu, ki, o, kRowLanes);
    }
    if (!valid || lane != 0) return;
    const double *ai = acc + 4 * (i * B + slot);
    const double2 V = make_double2(ai[0] + vr, ai[1] + vi);
    const double2 K = make_double2(ai[2] + kr, ai[3] + ki);
    if (RAW) {
        Vd[(int64_t)b * N + i] = V;
        Kp[(int64_t)b * N + i] = K;
        return;
    }
    const double2 ph = xb[i];
    const double2 sv = cmul(s[b], V);
    double2 *yb = y + (int64_t)b * 2 * N;
    yb[i] = make_double2(0.5 * ph.x + K.x - V.x, 0.5 * ph.y + K.y - V.y);
    yb[N + i] = make_double2(0.5 * ph.x - K.x + sv.x, 0.5 * ph.y - K.y + sv.y);
}

// Several right-hand sides: x [B][2N] is transposed to xt [2N][B] once per product, so
// that the gathers of the near-field SpMV and of the source weights read the B values of
// a panel contiguously (32 x 32 tiles through shared memory, both sides coalesced).
__device__ __forceinline__ void put(double2 &o, double2 v) { o = v; }
__device__ __forceinline__ void put(float2 &o, double2 v) { o = make_float2((float)v.x, (float)v.y); }
template <class T>
__global__ void transpose_kernel(int B, int64_t n2, const double2 *__restrict__ x, T *__restrict__ xt) {
    __shared__ double2 tile[32][33];
    const int64_t k0 = (int64_t)blockIdx.x * 32;
    const int b0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {   // rows b, columns k
        const int b = b0 + r;
        const int64_t k = k0 + threadIdx.x;
        if (b < B && k < n2) tile[r][threadIdx.x] = x[(int64_t)b * n2 + k];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {   // rows k, columns b
        const int64_t k = k0 + r;
        const int b = b0 + threadIdx.x;
        if (b < B && k < n2) put(xt[k * B + b], tile[threadIdx.x][r]);
    }
}

// The block rows for several right-hand sides from xt [2N][B]: L lanes per row (a power
// of two, L <= 32), lane r handling b = r, r + L, ...; the row's CSR entries are read by
// all lanes of the group (one transaction) and the gathers of x are contiguous in b.
__global__ void assemble_rhs_kernel(int64_t N, int B, int L, const double *__restrict__ acc,
                                    const int64_t *__restrict__ ptr, const int *__restrict__ col,
                                    const double *__restrict__ dV, const double *__restrict__ dK,
                                    const double2 *__restrict__ xt, const double2 *s, double2 *y, const int *inv) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = g / L;
    const int r = (int)(g - i * L);
    if (i >= N) return;
    const int64_t e0 = ptr[i], e1 = ptr[i + 1];
    for (int b = r; b < B; b += L) {
        const int slot = inv ? inv[b] : b;
        if (slot < 0) continue;   // converged system: row left untouched
        double vr = 0, vi = 0, kr = 0, ki = 0;
        for (int64_t e = e0; e < e1; ++e) {
            const int64_t j = col[e];
            const double a = dV[e], c = dK[e];
            const double2 ph = xt[j * B + b], dp = xt[(N + j) * B + b];
            vr += a * dp.x;
            vi += a * dp.y;
            kr += c * ph.x;
            ki += c * ph.y;
        }
        const double *ai = acc + 4 * (i * B + slot);
        const double2 V = make_double2(ai[0] + vr, ai[1] + vi);
        const double2 K = make_double2(ai[2] + kr, ai[3] + ki);
        const double2 ph = xt[i * B + b];
        const double2 sv = cmul(s[b], V);
        double2 *yb = y + (int64_t)b * 2 * N;
        yb[i] = make_double2(0.5 * ph.x + K.x - V.x, 0.5 * ph.y + K.y - V.y);
        yb[N + i] = make_double2(0.5 * ph.x - K.x + sv.x, 0.5 * ph.y - K.y + sv.y);
    }
}

// The same for FP32 products, in FP32 arithmetic from the FP32 transposed copy and the FP32
// near values (the far field of this mode is FP32; FP64 arithmetic would run at 1/64 of the
// FP32 rate on this GPU and bound the kernel)
__global__ void assemble_rhs_f32_kernel(int64_t N, int B, int L, const double *__restrict__ acc,
                                        const int64_t *__restrict__ ptr, const int *__restrict__ col,
                                        const float2 *__restrict__ dVK, const float2 *__restrict__ xt,
                                        const double2 *s, double2 *y, const int *inv) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = g / L;
    const int r = (int)(g - i * L);
    if (i >= N) return;
    const int64_t e0 = ptr[i], e1 = ptr[i + 1];
    for (int b = r; b < B; b += L) {
        const int slot = inv ? inv[b] : b;
        if (slot < 0) continue;   // converged system: row left untouched
        float vr = 0.f, vi = 0.f, kr = 0.f, ki = 0.f;
        for (int64_t e = e0; e < e1; ++e) {
            const int64_t j = col[e];
            const float2 c = dVK[e];
            const float2 ph = xt[j * B + b], dp = xt[(N + j) * B + b];
            vr = fmaf(c.x, dp.x, vr);
            vi = fmaf(c.x, dp.y, vi);
            kr = fmaf(c.y, ph.x, kr);
            ki = fmaf(c.y, ph.y, ki);
        }
        const double *ai = acc + 4 * (i * B + slot);
        const float Vr = (float)ai[0] + vr, Vi = (float)ai[1] + vi;
        const float Kr = (float)ai[2] + kr, Ki = (float)ai[3] + ki;
        const float2 ph = xt[i * B + b];
        const float sr = (float)s[b].x, si = (float)s[b].y;
        const float svr = sr * Vr - si * Vi, svi = sr * Vi + si * Vr;
        double2 *yb = y + (int64_t)b * 2 * N;
        yb[i] = make_double2(0.5f * ph.x + Kr - Vr, 0.5f * ph.y + Ki - Vi);
        yb[N + i] = make_double2(0.5f * ph.x - Kr + svr, 0.5f * ph.y - Ki + svi);
    }
}

// Several surfaces, Eq. matrix_multi: the block rows of panel i on surface s for channel
// sets (b, t) of the far field (acc [panel][B S][4]) and the near corrections, the latter
// split by the source panel's surface t:
//   y_top = phi/2 + (K phi)_s - (V dphi)_s,  y_bot = phi/2 - sum_t (K phi)_t + sum_t s_bt (V dphi)_t
// One thread per (row, right-hand side); s is [B][S].  RAW: write the layer potentials per
// source surface instead, Vd[t][i] = (V dphi)_t and Kp[t][i] = (K phi)_t (B = 1).
template <bool RAW>
__global__ void assemble_surf_kernel(int64_t N, int B, int S, const int *__restrict__ surf,
                                     const double *__restrict__ acc, const int64_t *__restrict__ ptr,
                                     const int *__restrict__ col, const double *__restrict__ dV,
                                     const double *__restrict__ dK, const double2 *__restrict__ x,
                                     const double2 *__restrict__ s, double2 *y, double2 *Vd, double2 *Kp,
                                     const int *inv) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= N * B) return;
    const int64_t i = g / B;
    const int b = (int)(g - i * B);
    // the far part of system b sits in sets k S .. k S + S - 1, k = inv[b] (identity without
    // a map); rows of converged systems (k = -1) are left untouched
    const int k = inv ? inv[b] : b;
    if (k < 0) return;
    const int si = surf[i];
    const double2 *xb = x + (int64_t)b * 2 * N;
    double2 Ks = make_double2(0, 0), Vs = make_double2(0, 0), Ka = make_double2(0, 0), Vw = make_double2(0, 0);
    for (int t = 0; t < S; ++t) {
        const double *a = acc + 4 * ((i * B + k) * S + t);
        double2 V = make_double2(a[0], a[1]), K = make_double2(a[2], a[3]);
        if (RAW) {   // near corrections of surface t added below
            Vd[(int64_t)t * N + i] = V;
            Kp[(int64_t)t * N + i] = K;
            continue;
        }
        Ka = cadd(Ka, K);
        Vw = cadd(Vw, cmul(s[b * S + t], V));
        if (t == si) {
            Ks = K;
            Vs = V;
        }
    }
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        const int j = col[e];
        const int t = surf[j];
        const double2 dv = cscale(xb[N + j], dV[e]), dk = cscale(xb[j], dK[e]);
        if (RAW) {
            Vd[(int64_t)t * N + i] = cadd(Vd[(int64_t)t * N + i], dv);
            Kp[(int64_t)t * N + i] = cadd(Kp[(int64_t)t * N + i], dk);
            continue;
        }
        Ka = cadd(Ka, dk);
        Vw = cadd(Vw, cmul(s[b * S + t], dv));
        if (t == si) {
            Ks = cadd(Ks, dk);
            Vs = cadd(Vs, dv);
        }
    }
    if (RAW) return;
    const double2 ph = xb[i];
    double2 *yb = y + (int64_t)b * 2 * N;
    yb[i] = make_double2(0.5 * ph.x + Ks.x - Vs.x, 0.5 * ph.y + Ks.y - Vs.y);
    yb[N + i] = make_double2(0.5 * ph.x - Ka.x + Vw.x, 0.5 * ph.y - Ka.y + Vw.y);
}

// far-field parts of B right-hand sides x [B][2N] into ctx->acc [panel][B S][4] (S surfaces:
// channel set b S + t holds the potentials of surface t's sources); with B > 1 the
// transposed copy xt of x is formed first (the block assembly reads it too)
static int far_part(lspr_ctx *ctx, int mode, const double2 *x, int B) {
    const int prec = mode_prec(mode);
    const bool tree = mode_tree(mode);
    const int64_t N = ctx->mesh.N;
    const int S = ctx->mesh.S;
    const int BS = B * S;
    if (tree && !ctx->tree.ready) return LSPR_E_STATE;
    LSPR_TRY(ctx, ctx->acc.ensure(4 * N * BS));
    LSPR_TRY(ctx, ctx->counters.ensure(8));
    LSPR_TRY(ctx, cudaMemsetAsync(ctx->acc.p, 0, sizeof(double) * 4 * N * BS, ctx->stream));
    LSPR_TRY(ctx, cudaMemsetAsync(ctx->counters.p, 0, sizeof(int) * 8, ctx->stream));
    const double2 *xt = nullptr;
    const float2 *xtf = nullptr;
    const dim3 tg(grid_for(2 * N, 32), grid_for(B, 32)), tb(32, 8);
    if (B > 1 && prec == PREC_F32) {
        LSPR_TRY(ctx, ctx->xtf.ensure((size_t)B * 2 * N));
        ++ctx->n_launches;
        transpose_kernel<float2><<<tg, tb, 0, ctx->stream>>>(B, 2 * N, x, ctx->xtf.p);
        xtf = ctx->xtf.p;
    } else if (B > 1) {
        LSPR_TRY(ctx, ctx->xt.ensure((size_t)B * 2 * N));
        ++ctx->n_launches;
        transpose_kernel<double2><<<tg, tb, 0, ctx->stream>>>(B, 2 * N, x, ctx->xt.p);
        xt = ctx->xt.p;
    }
    LSPR_TRY_ST(launch_weights(ctx, prec, x, xt, N, B, S, xtf));
    if (tree && ctx->timing.enabled) {
        // kernel timing: every far-field kernel on the main stream, one after another, so that
        // the events around a launch measure that kernel alone (no overlap, no waiting)
        LSPR_TRY_ST(launch_p2p(ctx, prec, ctx->tree.p2p_items.p, ctx->tree.n_p2p_items, ctx->acc.p, ctx->stream,
                               ctx->counters.p, BS));
        LSPR_TRY_ST(launch_p2m(ctx, prec, BS));
        LSPR_TRY_ST(launch_m2p(ctx, prec, ctx->acc.p, ctx->counters.p + 1, BS));
    } else if (tree) {
        // P2P on the side stream overlaps P2M -> M2P on the main stream; both add into acc
        LSPR_TRY(ctx, cudaEventRecord(ctx->ev_fork, ctx->stream));
        LSPR_TRY(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
        LSPR_TRY_ST(launch_p2p(ctx, prec, ctx->tree.p2p_items.p, ctx->tree.n_p2p_items, ctx->acc.p, ctx->side,
                               ctx->counters.p, BS));
        LSPR_TRY(ctx, cudaEventRecord(ctx->ev_join, ctx->side));
        LSPR_TRY_ST(launch_p2m(ctx, prec, BS));
        LSPR_TRY_ST(launch_m2p(ctx, prec, ctx->acc.p, ctx->counters.p + 1, BS));
        LSPR_TRY(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
    } else {
        LSPR_TRY_ST(launch_p2p(ctx, prec, ctx->direct.items.p, ctx->direct.n, ctx->acc.p, ctx->stream,
                               ctx->counters.p, BS));
    }
    ctx->matvec_count += B;
    return LSPR_OK;
}

int apply_operator(lspr_ctx *ctx, int mode, const double2 *x, double2 *y, const double2 *s, int B) {
    const Mesh &m = ctx->mesh;
    const int64_t N = m.N;
    LSPR_TRY_ST(far_part(ctx, mode, x, B));
    cudaEvent_t ev;
    timer_begin(ctx, T_NEAR, &ev);
    ++ctx->n_launches;
    if (m.S > 1) {
        assemble_surf_kernel<false><<<grid_for(N * B, 128), 128, 0, ctx->stream>>>(
            N, B, m.S, m.surf.p, ctx->acc.p, m.near_ptr.p, m.near_col.p, m.near_dV.p, m.near_dK.p, x, s, y, nullptr,
            nullptr, ctx->rhs_inv);
    } else if (B == 1) {
        assemble_kernel<false><<<grid_for(N * kRowLanes, 256), 256, 0, ctx->stream>>>(
            N, B, ctx->acc.p, m.near_ptr.p, m.near_col.p, m.near_dV.p, m.near_dK.p, x, s, y, nullptr, nullptr,
            ctx->rhs_inv);
    } else {
        int L = 1;
        while (L < B && L < 32) L *= 2;
        if (mode_prec(mode) == PREC_F32)
            assemble_rhs_f32_kernel<<<grid_for(N * L, 256), 256, 0, ctx->stream>>>(
                N, B, L, ctx->acc.p, m.near_ptr.p, m.near_col.p, m.near_f32.p, ctx->xtf.p, s, y, ctx->rhs_inv);
        else
            assemble_rhs_kernel<<<grid_for(N * L, 256), 256, 0, ctx->stream>>>(N, B, L, ctx->acc.p, m.near_ptr.p,
                                                                              m.near_col.p, m.near_dV.p, m.near_dK.p,
                                                                              ctx->xt.p, s, y, ctx->rhs_inv);
    }
    timer_end(ctx, T_NEAR, ev);
    LSPR_TRY(ctx, cudaGetLastError());
    return LSPR_OK;
}

int layer_potentials(lspr_ctx *ctx, int mode, const double2 *x, double2 *Vd, double2 *Kp) {
    const Mesh &m = ctx->mesh;
    LSPR_TRY_ST(far_part(ctx, mode, x, 1));
    ++ctx->n_launches;
    if (m.S > 1)
        assemble_surf_kernel<true><<<grid_for(m.N, 128), 128, 0, ctx->stream>>>(
            m.N, 1, m.S, m.surf.p, ctx->acc.p, m.near_ptr.p, m.near_col.p, m.near_dV.p, m.near_dK.p, x, nullptr,
            nullptr, Vd, Kp, nullptr);
    else
        assemble_kernel<true><<<grid_for(m.N * kRowLanes, 256), 256, 0, ctx->stream>>>(
            m.N, 1, ctx->acc.p, m.near_ptr.p, m.near_col.p, m.near_dV.p, m.near_dK.p, x, nullptr, nullptr, Vd, Kp,
            nullptr);
    LSPR_TRY(ctx, cudaGetLastError());
    return LSPR_OK;
}

// --------------------------------------------------------------------- GMRES
constexpr int kRedThreads = 256;
constexpr int kChunk = 1024;   // elements per partial-sum block

__global__ void norm_partial_kernel(int B, int64_t n2, const double2 *__restrict__ w, int64_t wstride, double *part,
                                    int nchunks, const int *active) {
    __shared__ double red[kRedThreads];
    const int chunk = blockIdx.x, b = blockIdx.y;
    if (active && !active[b]) return;
    double s = 0;
    const int64_t beg = (int64_t)chunk * kChunk, end = min(n2, beg + kChunk);
    for (int64_t k = beg + threadIdx.x; k < end; k += blockDim.x) s += cabs2(w[b * wstride + k]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)b * nchunks + chunk] = red[0];
}

__global__ void norm_final_kernel(int B, int nchunks, const double *part, double *out, const int *active) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B || (active && !active[b])) return;
    double s = 0;
    for (int c = 0; c < nchunks; ++c) s += part[(int64_t)b * nchunks + c];
    out[b] = sqrt(s);
}

__global__ void add_kernel(int B, int64_t n2, double2 *x, const double2 *d, double sign) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (k >= n2) return;
    const double2 a = x[(int64_t)b * n2 + k], c = d[(int64_t)b * n2 + k];
    x[(int64_t)b * n2 + k] = make_double2(a.x + sign * c.x, a.y + sign * c.y);
}

// r_b = b_b - y_b (update = 0) or r_b -= y_b (update = 1) for the systems with inv[b] >= 0
__global__ void resid_combine_kernel(int B, int64_t n2, double2 *r, const double2 *bv, const double2 *y,
                                     const int *inv, int update) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (k >= n2 || inv[b] < 0) return;
    const int64_t o = (int64_t)b * n2 + k;
    r[o] = update ? csub(r[o], y[o]) : csub(bv[o], y[o]);
}

// ------------------------------------------------------------------ RHS
__global__ void dphi_inc_kernel(int64_t N, const double *nx, const double *ny, const double *nz, double E0x,
                                double E0y, double E0z, double2 *x) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    x[i] = make_double2(0, 0);
    x[N + i] = make_double2(-(E0x * nx[i] + E0y * ny[i] + E0z * nz[i]), 0.0);
}

// b[b] = [0 ; sum_t ((eps_out - eps_bt)/eps_out) (V dphi_inc)_t], Vinc [S][N], eps_in [B][S]
__global__ void rhs_kernel(int B, int S, int64_t N, const double2 *__restrict__ Vinc, const double2 *eps_in,
                           double2 eps_out, double2 *rhs) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (i >= N) return;
    double2 acc = make_double2(0, 0);
    for (int t = 0; t < S; ++t) {
        const double2 f = cdiv(csub(eps_out, eps_in[b * S + t]), eps_out);
        acc = cadd(acc, cmul(f, Vinc[(int64_t)t * N + i]));
    }
    rhs[(int64_t)b * 2 * N + i] = make_double2(0, 0);
    rhs[(int64_t)b * 2 * N + N + i] = acc;
}

// Point charges inside the surfaces (Eqs. integral_eq_lspr_system, matrix_multi: the interior
// row of a surface holding charges carries (1 / (4 pi eps_t)) sum_k q_k / |r - r_k|).
// coul[i] = sum over the charges of panel i's surface of q_k / |c_i - r_k| (FP64; the charges
// pass through shared memory in tiles of the block size).
constexpr int kCoulThreads = 128;
__global__ void __launch_bounds__(kCoulThreads)
    coulomb_kernel(int64_t N, int64_t nq, const double *__restrict__ cx, const double *__restrict__ cy,
                   const double *__restrict__ cz, const int *__restrict__ surf, const dbl4 *__restrict__ charges,
                   const int *__restrict__ qsurf, double *__restrict__ coul) {
    __shared__ dbl4 sq[kCoulThreads];
    __shared__ int ss[kCoulThreads];
    const int64_t i = blockIdx.x * (int64_t)kCoulThreads + threadIdx.x;
    const bool live = i < N;
    const double x = live ? cx[i] : 0.0, y = live ? cy[i] : 0.0, z = live ? cz[i] : 0.0;
    const int t = live ? surf[i] : -1;
    double phi = 0.0;
    for (int64_t k0 = 0; k0 < nq; k0 += kCoulThreads) {
        __syncthreads();
        if (k0 + threadIdx.x < nq) {
            sq[threadIdx.x] = charges[k0 + threadIdx.x];
            ss[threadIdx.x] = qsurf[k0 + threadIdx.x];
        }
        __syncthreads();
        const int cnt = (int)min((int64_t)kCoulThreads, nq - k0);
        for (int k = 0; k < cnt; ++k) {
            if (ss[k] != t) continue;
            const double dx = x - sq[k].x, dy = y - sq[k].y, dz = z - sq[k].z;
            phi += sq[k].w / sqrt(dx * dx + dy * dy + dz * dz);
        }
    }
    if (live) coul[i] = phi;
}

// rhs top row of panel i += coul[i] / (4 pi eps_t), eps_t = eps_in[b][surf[i]]
__global__ void charge_rhs_kernel(int B, int S, int64_t N, const double *__restrict__ coul,
                                  const int *__restrict__ surf, const double2 *eps_in, double2 *rhs) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (i >= N) return;
    const double2 e = eps_in[b * S + surf[i]];
    const double2 f = cdiv(make_double2(coul[i] / (4.0 * M_PI), 0.0), e);
    rhs[(int64_t)b * 2 * N + i] = cadd(rhs[(int64_t)b * 2 * N + i], f);
}

// ---------------------------------------------------------- dipole + sigma
// dipole of surface 0 (the particle; eps_in [B][S], its permittivity eps_in[b][0])
__global__ void dipole_partial_kernel(int B, int S, int64_t N, const int *__restrict__ surf,
                                      const double2 *__restrict__ x, const double2 *eps_in,
                                      double2 eps_out, const double *cx, const double *cy, const double *cz,
                                      const double *nx, const double *ny, const double *nz, const double *area,
                                      double E0x, double E0y, double E0z, double *part, int nchunks) {
    __shared__ double red[6][kRedThreads];
    const int chunk = blockIdx.x, b = blockIdx.y;
    const double2 s = cdiv(eps_in[b * S], eps_out);
    const double2 f = cdiv(csub(eps_out, eps_in[b * S]), eps_out);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const int64_t beg = (int64_t)chunk * kChunk, end = min(N, beg + kChunk);
    for (int64_t j = beg + threadIdx.x; j < end; j += blockDim.x) {
        if (surf[j] != 0) continue;
        const double2 ph = x[(int64_t)b * 2 * N + j], dp = x[(int64_t)b * 2 * N + N + j];
        const double dinc = -(E0x * nx[j] + E0y * ny[j] + E0z * nz[j]);
        const double2 d2 = csub(cmul(s, dp), cscale(f, dinc));
        const double A = area[j];
        const double c[3] = {cx[j], cy[j], cz[j]}, n[3] = {nx[j], ny[j], nz[j]};
        for (int d = 0; d < 3; ++d) {
            acc[2 * d] += A * (c[d] * d2.x - ph.x * n[d]);
            acc[2 * d + 1] += A * (c[d] * d2.y - ph.y * n[d]);
        }
    }
    for (int q = 0; q < 6; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < 6; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 6; ++q) part[((int64_t)b * nchunks + chunk) * 6 + q] = red[q][0];
}

// out[b] = (p_x, p_y, p_z as complex, sigma): 7 doubles per wavelength
__global__ void dipole_final_kernel(int B, int nchunks, const double *part, double2 eps_out, double E0x, double E0y,
                                    double E0z, const double *lambda, double *out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int c = 0; c < nchunks; ++c)
        for (int q = 0; q < 6; ++q) s[q] += part[((int64_t)b * nchunks + c) * 6 + q];
    double2 p[3];
    for (int d = 0; d < 3; ++d) {
        const double2 v = cmul(make_double2(-eps_out.x, -eps_out.y), make_double2(s[2 * d], s[2 * d + 1]));
        p[d] = v;
        out[b * 7 + 2 * d] = v.x;
        out[b * 7 + 2 * d + 1] = v.y;
    }
    const double E = sqrt(E0x * E0x + E0y * E0y + E0z * E0z);
    const double2 ep = cscale(cadd(cadd(cscale(p[0], E0x), cscale(p[1], E0y)), cscale(p[2], E0z)), 1.0 / E);
    const double2 k = cscale(csqrt_p(eps_out), 2.0 * M_PI / lambda[b]);
    const double2 q = cdiv(cmul(cmul(k, k), ep), cscale(eps_out, E));
    out[b * 7 + 6] = q.y / k.x;
}

// ------------------------------------------------------------------ driver
int solve_impl(lspr_ctx *ctx, const double *eps_in, double eps_out_re, double eps_out_im, const double *E0,
               const double *lambda_nm, int B, const lspr_solve_opts &o, double *dipole_out, double *sigma_out,
               lspr_solve_stats *stt) {
    const Mesh &me = ctx->mesh;
    const int64_t N = me.N, n2 = 2 * N;
    cudaStream_t st = ctx->stream;
    const int mode = o.mode;
    const bool tree = mode_tree(mode);
    const double2 eout = make_double2(eps_out_re, eps_out_im);
    const int S = me.S;   // eps_in is [B][S]
    // the tensor-core far field's group lists before any product (a recorded Arnoldi cycle
    // launches the kernels without the host code that would form them)
    if (tree && mode == LSPR_TREE_FP32 && B * S > 1 && (ctx->tensor_cores & 3))
        LSPR_TRY_ST(tree_tc_lists(ctx, (ctx->tensor_cores & 2) != 0));
    LSPR_TRY(ctx, ctx->gm_eps.ensure((size_t)B * S));
    LSPR_TRY(ctx, ctx->gm_s.ensure((size_t)B * S));
    LSPR_TRY(ctx, ctx->gm_b.ensure((size_t)B * n2));
    LSPR_TRY(ctx, ctx->gm_x.ensure((size_t)B * n2));
    LSPR_TRY(ctx, ctx->gm_r.ensure((size_t)B * n2));
    LSPR_TRY(ctx, ctx->gm_vinc.ensure(n2 + 2 * (size_t)S * N));
    LSPR_TRY(ctx, ctx->gm_out.ensure((size_t)B * 8 + B));
    std::vector<double2> he((size_t)B * S), hs((size_t)B * S);
    for (int q = 0; q < B * S; ++q) {
        he[q] = make_double2(eps_in[2 * q], eps_in[2 * q + 1]);
        const double d = eps_out_re * eps_out_re + eps_out_im * eps_out_im;
        hs[q] = make_double2((he[q].x * eps_out_re + he[q].y * eps_out_im) / d,
                             (he[q].y * eps_out_re - he[q].x * eps_out_im) / d);
    }
    LSPR_TRY(ctx, cudaMemcpyAsync(ctx->gm_eps.p, he.data(), sizeof(double2) * B * S, cudaMemcpyHostToDevice, st));
    LSPR_TRY(ctx, cudaMemcpyAsync(ctx->gm_s.p, hs.data(), sizeof(double2) * B * S, cudaMemcpyHostToDevice, st));
    // right-hand side V (dphi_inc/dn) with the operator of the solve's mode: dphi_inc/dn
    // is smooth and the sum has no cancellation, so FP32 evaluation (FP64 accumulation)
    // leaves ~1e-7 relative error in b
    double2 *xin = ctx->gm_vinc.p, *Vinc = ctx->gm_vinc.p + n2;
    ++ctx->n_launches;
    dphi_inc_kernel<<<grid_for(N, 256), 256, 0, st>>>(N, me.nx.p, me.ny.p, me.nz.p, E0[0], E0[1], E0[2], xin);
    LSPR_TRY_ST(layer_potentials(ctx, mode, xin, Vinc, Vinc + (size_t)S * N));
    ++ctx->n_launches;
    rhs_kernel<<<dim3(grid_for(N, 256), B), 256, 0, st>>>(B, S, N, Vinc, ctx->gm_eps.p, eout, ctx->gm_b.p);
    if (ctx->nq > 0) {   // point charges on their surfaces' interior rows
        if (ctx->max_charge_surf >= S) {
            ctx->last_error = "a charge's surface index is not a surface of the mesh";
            return LSPR_E_ARG;
        }
        LSPR_TRY(ctx, ctx->coul.ensure(N));
        ++ctx->n_launches;
        coulomb_kernel<<<grid_for(N, kCoulThreads), kCoulThreads, 0, st>>>(N, ctx->nq, me.cx.p, me.cy.p, me.cz.p,
                                                                            me.surf.p, ctx->charges.p,
                                                                            ctx->charge_surf.p, ctx->coul.p);
        ++ctx->n_launches;
        charge_rhs_kernel<<<dim3(grid_for(N, 256), B), 256, 0, st>>>(B, S, N, ctx->coul.p, me.surf.p, ctx->gm_eps.p,
                                                                     ctx->gm_b.p);
    }
    LSPR_TRY(ctx, cudaMemsetAsync(ctx->gm_x.p, 0, sizeof(double2) * B * n2, st));
    // ||b||
    const int nch = (int)((n2 + kChunk - 1) / kChunk);
    LSPR_TRY(ctx, ctx->gm_dpart.ensure((size_t)B * nch));
    LSPR_TRY(ctx, ctx->gm_bnorm.ensure(B));
    ++ctx->n_launches;
    norm_partial_kernel<<<dim3(nch, B), kRedThreads, 0, st>>>(B, n2, ctx->gm_b.p, n2, ctx->gm_dpart.p, nch, nullptr);
    ++ctx->n_launches;
    norm_final_kernel<<<grid_for(B, 64), 64, 0, st>>>(B, nch, ctx->gm_dpart.p, ctx->gm_bnorm.p, nullptr);
    LSPR_TRY(ctx, cudaGetLastError());
    std::vector<double> bnorm(B);
    LSPR_TRY(ctx, cudaMemcpyAsync(bnorm.data(), ctx->gm_bnorm.p, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
    LSPR_TRY(ctx, cudaStreamSynchronize(st));
    for (auto &v : bnorm)
        if (!(v > 0)) v = 1.0;

    std::vector<int> iters(B, 0);
    std::vector<double> relres(B, 1.0);
    const int m = std::max(1, std::min(o.restart, kMaxRestart));
    const bool refine = o.refine && (mode == LSPR_TREE_FP32 || mode == LSPR_DIRECT_FP32);
    if (!refine) {
        LSPR_TRY_ST(gmres_graph_solve(ctx, mode, B, m, o.maxiter, o.tol, ctx->gm_s.p, ctx->gm_b.p, ctx->gm_x.p,
                                      true, false, iters, relres, bnorm));
    } else {
        // Iterative refinement (per system b): the residual r_b = b_b - A x_b is formed with a
        // high-precision operator of the same kind (tree or direct); the correction solves
        // A d_b = r_b with the FP32-mode GMRES to the relative tolerance that brings r_b to
        // 0.3 tol ||b_b|| (between 1e-4 and 0.5 of ||r_b||; systems that met tol take no steps).
        // refine == 2: native FP64 residual; otherwise float-float (about 48 significant bits
        // at a fraction of the cost of FP64 on this GPU).
        // Once a system's residual is small (||r_b|| <= kUpdateRatio tol ||b_b||), its next
        // residual is updated instead, r_b <- r_b - A d_b with the FP32 operator: the update
        // differs from the high-precision residual by (A_hi - A_32) d_b, whose norm is at most
        // the FP32 operator's relative error (<= 1e-5 measured bound, ~5e-7 typical) times
        // ||A d_b|| ~ ||r_b||, i.e. <= 1e-2 tol ||b_b||.  The products of a cycle run on the
        // systems that need them only (packed into the first right-hand-side slots), so that
        // the few systems near the resonance whose first correction leaves a larger residual
        // do not make every system pay for another high-precision product.
        constexpr double kUpdateRatio = 1e3;
        // the first correction stops at 3e-4 of ||b||: near the resonance its FP32 recurrence
        // estimate is optimistic by an order of magnitude, so going further buys little (1e-4:
        // 30.6, 3e-4: 31.8, 1e-3: 31.8 lambda-solves/s on the 64-wavelength sweep, the same
        // accuracy)
        constexpr double kFirstInner = 3e-4;
        const int mode_hi = o.refine == 2 ? (tree ? LSPR_TREE_FP64 : LSPR_DIRECT_FP64)
                                          : (tree ? LSPR_TREE_FF : LSPR_DIRECT_FF);
        std::vector<int> it2(B, 0);
        std::vector<double> rr2(B, 1.0), rn(B, 0.0);
        DArr<double2> &dx = ctx->gm_dx;
        LSPR_TRY(ctx, dx.ensure((size_t)B * n2));
        LSPR_TRY(ctx, ctx->gm_z.ensure((size_t)B * n2));
        LSPR_TRY(ctx, ctx->gm_rmap.ensure(2 * (size_t)B + 2));
        const int max_cycles = 12;
        int used = 0;
        std::vector<char> upd(B, 0);   // r_b holds the updated residual of the current x_b
        std::vector<char> fin(B, 0);   // system b met tol
        std::vector<int> map(2 * (size_t)B + 2);
        auto norm_of_r = [&]() -> int {
            ++ctx->n_launches;
            norm_partial_kernel<<<dim3(nch, B), kRedThreads, 0, st>>>(B, n2, ctx->gm_r.p, n2, ctx->gm_dpart.p, nch,
                                                                      nullptr);
            ++ctx->n_launches;
            norm_final_kernel<<<grid_for(B, 64), 64, 0, st>>>(B, nch, ctx->gm_dpart.p, ctx->gm_bnorm.p, nullptr);
            LSPR_TRY(ctx, cudaGetLastError());
            LSPR_TRY(ctx, cudaMemcpyAsync(rn.data(), ctx->gm_bnorm.p, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
            LSPR_TRY(ctx, cudaStreamSynchronize(st));
            return LSPR_OK;
        };
        // r_b = b_b - A_md xin_b (update = 0) or r_b -= A_md xin_b (update = 1) for the systems
        // with sel[b], through gm_z; the other systems' r_b are untouched
        auto subset_residual = [&](int md, const double2 *xin, const std::vector<char> &sel, int update) -> int {
            int n = 0;
            for (int b = 0; b < B; ++b) {
                if (sel[b]) {
                    map[n] = b;
                    map[B + b] = n++;
                } else {
                    map[B + b] = -1;
                }
            }
            if (n == 0) return LSPR_OK;
            for (int q = n; q < B; ++q) map[q] = 0;
            map[2 * B] = n;
            map[2 * B + 1] = n * S;
            LSPR_TRY(ctx, cudaMemcpyAsync(ctx->gm_rmap.p, map.data(), sizeof(int) * map.size(), cudaMemcpyHostToDevice,
                                          st));
            ctx->rhs_map = ctx->gm_rmap.p;
            ctx->rhs_inv = ctx->gm_rmap.p + B;
            ctx->rhs_nact = ctx->gm_rmap.p + 2 * B + 1;
            ctx->timing_sets = n * S;
            const int rc = apply_operator(ctx, md, xin, ctx->gm_z.p, ctx->gm_s.p, B);
            ctx->rhs_map = ctx->rhs_inv = ctx->rhs_nact = nullptr;
            ctx->timing_sets = -1;
            LSPR_TRY_ST(rc);
            ctx->matvec_count += n - B;   // products of the selected systems only
            ++ctx->n_launches;
            resid_combine_kernel<<<dim3(grid_for(n2, 256), B), 256, 0, st>>>(B, n2, ctx->gm_r.p, ctx->gm_b.p,
                                                                             ctx->gm_z.p, ctx->gm_rmap.p + B, update);
            LSPR_TRY(ctx, cudaGetLastError());
            LSPR_TRY(ctx, cudaStreamSynchronize(st));   // map is reused by the next call
            return LSPR_OK;
        };
        for (int cycle = 0;; ++cycle) {
            if (cycle == 0) {   // x = 0: r = b
                LSPR_TRY(ctx, cudaMemcpyAsync(ctx->gm_r.p, ctx->gm_b.p, sizeof(double2) * B * n2,
                                              cudaMemcpyDeviceToDevice, st));
                for (int b = 0; b < B; ++b) rn[b] = bnorm[b];
            } else {
                std::vector<char> sel(B);
                for (int b = 0; b < B; ++b) sel[b] = !upd[b] && !fin[b];
                LSPR_TRY_ST(subset_residual(mode_hi, ctx->gm_x.p, sel, 0));
                LSPR_TRY_ST(norm_of_r());
            }
            bool done = true;
            double worst = 0.0;
            for (int b = 0; b < B; ++b) {
                relres[b] = rn[b] / bnorm[b];
                fin[b] = relres[b] <= o.tol;
                done = done && fin[b];
                worst = std::max(worst, relres[b]);
            }
            if (done || cycle == max_cycles || used >= o.maxiter || !std::isfinite(worst)) break;
            // per-system inner tolerance through the reference norms: GMRES stops system b when
            // its residual estimate is <= 1 x rnorm[b] = inner_b ||r_b||
            std::vector<double> rnorm(B);
            for (int b = 0; b < B; ++b) {
                const double inner =
                    fin[b] ? 2.0 : std::min(0.5, std::max(cycle == 0 ? kFirstInner : 1e-4, 0.3 * o.tol / relres[b]));
                rnorm[b] = rn[b] > 0 ? inner * rn[b] : 1.0;
            }
            LSPR_TRY(ctx, cudaMemsetAsync(dx.p, 0, sizeof(double2) * B * n2, st));
            // the caller forms the next residual itself: the inner solve may stop on its
            // recurrence estimate
            LSPR_TRY_ST(gmres_graph_solve(ctx, mode, B, m, std::max(1, o.maxiter - used), 1.0, ctx->gm_s.p,
                                          ctx->gm_r.p, dx.p, true, true, it2, rr2, rnorm));
            ++ctx->n_launches;
            add_kernel<<<dim3(grid_for(n2, 256), B), 256, 0, st>>>(B, n2, ctx->gm_x.p, dx.p, 1.0);
            int mx = 0;
            for (int b = 0; b < B; ++b) {
                iters[b] += it2[b];
                mx = std::max(mx, it2[b]);
            }
            used += mx;
            // r_b <- r_b - A_32 d_b for the systems whose residual was small (the next cycle forms
            // the others' high-precision residuals and every norm)
            for (int b = 0; b < B; ++b) upd[b] = !fin[b] && relres[b] <= kUpdateRatio * o.tol;
            LSPR_TRY_ST(subset_residual(mode, dx.p, upd, 1));
        }
        LSPR_TRY(ctx, cudaStreamSynchronize(st));
    }
    // dipole and sigma
    const int nchN = (int)((N + kChunk - 1) / kChunk);
    DArr<double> &part = ctx->gm_dippart, &lam = ctx->gm_lambda;
    LSPR_TRY(ctx, part.ensure((size_t)B * nchN * 6));
    LSPR_TRY(ctx, lam.ensure(B));
    LSPR_TRY(ctx, cudaMemcpyAsync(lam.p, lambda_nm, sizeof(double) * B, cudaMemcpyHostToDevice, st));
    ++ctx->n_launches;
    dipole_partial_kernel<<<dim3(nchN, B), kRedThreads, 0, st>>>(B, me.S, N, me.surf.p, ctx->gm_x.p, ctx->gm_eps.p,
                                                                 eout, me.cx.p,
                                                                 me.cy.p, me.cz.p, me.nx.p, me.ny.p, me.nz.p,
                                                                 me.area.p, E0[0], E0[1], E0[2], part.p, nchN);
    ++ctx->n_launches;
    dipole_final_kernel<<<grid_for(B, 64), 64, 0, st>>>(B, nchN, part.p, eout, E0[0], E0[1], E0[2], lam.p,
                                                         ctx->gm_out.p);
    LSPR_TRY(ctx, cudaGetLastError());
    std::vector<double> out((size_t)B * 7);
    LSPR_TRY(ctx, cudaMemcpyAsync(out.data(), ctx->gm_out.p, sizeof(double) * 7 * B, cudaMemcpyDeviceToHost, st));
    LSPR_TRY(ctx, cudaStreamSynchronize(st));
    int rc = LSPR_OK;
    for (int b = 0; b < B; ++b) {
        for (int q = 0; q < 6; ++q) dipole_out[6 * b + q] = out[7 * b + q];
        sigma_out[b] = out[7 * b + 6];
        const bool ok = relres[b] <= o.tol;
        if (!ok) rc = LSPR_E_NOT_CONVERGED;
        if (stt) {
            if (stt->iterations) stt->iterations[b] = iters[b];
            if (stt->residual) stt->residual[b] = relres[b];
            if (stt->status) stt->status[b] = ok ? LSPR_OK : LSPR_E_NOT_CONVERGED;
        }
    }
    return rc;
}

}  // namespace lspr
