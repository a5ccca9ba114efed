// Far-field kernels of the matrix-vector product (Sec. II.D, Eq. summation):
// sources are the far-rule Gauss nodes y_j with weights q_j = w_j A_j dphi_j / (4 pi)
// (single layer) and mu_j = w_j A_j phi_j / (4 pi) (double layer); targets are the
// panel centroids x_i.  For every target
//     Vd_i = sum_j q_j / |x_i - y_j|,   Kp_i = sum_j mu_j (x_i - y_j).n_j / |x_i - y_j|^3
// over all sources except those of panel i itself (its singular integral is
// added exactly by the near-field correction).  Complex weights are carried as
// two real channels (the paper's real/imaginary split of the treecode work).
//
// Several right-hand sides (wavelengths) share one geometry: the kernels generate G,
// dG/dn (P2P), the monomials (P2M) or the Taylor coefficients (M2P) once per pair,
// source or (target, box) and apply them to a chunk of NB right-hand sides.
// Layouts for B right-hand sides: weights [source][B], accumulators [panel][B][4],
// moments [box][term][B].
//
//   p2p_kernel  direct sums of a 64-target block against a contiguous source range
//   p2m_kernel  Cartesian Taylor moments of a leaf about its centre c, shifted into
//               every accepted ancestor box:
//                 M^V_k = sum_j q_j (c - y_j)^k
//                 M^K_k = sum_j mu_j * (-sum_d n_{j,d} k_d (c - y_j)^(k - e_d))
//   m2p_kernel  Vd_i += sum_{|k|<=P} a_k(x_i - c) M^V_k (same for K), with
//               a_k(R) = D^k (1/|R|) / k! from the recurrence
//               n |R|^2 a_k + (2n-1) sum_d R_d a_(k-e_d) + (n-1) sum_d a_(k-2e_d) = 0,
//               n = |k|, a_0 = 1/|R|.
// Partial sums are formed in the kernel's precision (FP32 or FP64) per work
// item and accumulated in FP64 with atomics.
#include <algorithm>

#include "farfield.cuh"

namespace lspr {

// ----------------------------------------------------------------- weights
// w[s][slot] = w_s A_s / (4 pi) * (dphi_b, phi_b) at the source's panel, b = map[slot]
// (identity without a map; only the first *nact slots are formed when nact is given);
// x is [B][2N] complex
template <typename T4>
// Several surfaces (S > 1): channel set slot = b * S + t carries the weights of the sources
// of surface t only (zero elsewhere), so that each surface's layer potentials come out
// separately; BS = B * S sets per source.
__global__ void weights_kernel(int64_t Ns, int64_t N, int B, int S, const dbl4 *__restrict__ spos64,
                               const int *__restrict__ src_panel, const int *__restrict__ surf,
                               const double2 *__restrict__ x, const double2 *__restrict__ xt, T4 *__restrict__ w,
                               const int *map, const int *nact) {
    const int BS = B * S;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= Ns * BS) return;
    const int64_t s = g / BS;
    const int slot = (int)(g - s * BS);
    if (nact && slot >= *nact) return;
    const int p = src_panel[s];
    // set slot = k S + t: surface t of the k-th running system (map: k -> system)
    const int k = slot / S, t = slot - k * S;
    const int b = map ? map[k] : k;
    const int bs = b * S + t;
    if (S > 1 && surf[p] != bs - b * S) {
        w[g] = zero4<T4>();
        return;
    }
    const double wa = spos64[s].w * kInv4Pi;
    // x [B][2N], or its transposed copy xt [2N][B] when given
    const double2 phi = xt ? xt[(int64_t)p * B + b] : x[(int64_t)b * 2 * N + p];
    const double2 dphi = xt ? xt[(N + p) * B + b] : x[(int64_t)b * 2 * N + N + p];
    T4 o;
    o.x = wa * dphi.x;
    o.y = wa * dphi.y;
    o.z = wa * phi.x;
    o.w = wa * phi.y;
    w[g] = o;
}

// The same for FP32 products of several right-hand sides from the FP32 transposed copy
// xt [2N][B], in FP32 arithmetic (the weights feed FP32 kernels; FP64 arithmetic would run
// at 1/64 of the FP32 rate on this GPU)
__global__ void weights_f32t_kernel(int64_t Ns, int64_t N, int B, int S, const float4 *__restrict__ spos32,
                                    const int *__restrict__ src_panel, const int *__restrict__ surf,
                                    const float2 *__restrict__ xt, float4 *__restrict__ w, const int *map,
                                    const int *nact) {
    const int BS = B * S;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= Ns * BS) return;
    const int64_t s = g / BS;
    const int slot = (int)(g - s * BS);
    if (nact && slot >= *nact) return;
    const int p = src_panel[s];
    const int k = slot / S, t = slot - k * S;
    const int b = map ? map[k] : k;
    if (S > 1 && surf[p] != t) {
        w[g] = zero4<float4>();
        return;
    }
    const float wa = spos32[s].w * (float)kInv4Pi;
    const float2 phi = xt[(int64_t)p * B + b], dphi = xt[(N + p) * B + b];
    w[g] = make_float4(wa * dphi.x, wa * dphi.y, wa * phi.x, wa * phi.y);
}

// item.w = 1 iff some source of [item.y, item.z) belongs to a panel of the item's target block
__global__ void item_flags_kernel(int4 *items, int64_t nitems, const int *__restrict__ src_tblock) {
    const int64_t it = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (it >= nitems) return;
    int4 item = items[it];
    int hit = 0;
    for (int s = item.y + lane; s < item.z; s += 32) hit |= src_tblock[s] == item.x;
    hit = __any_sync(0xffffffffu, hit);
    if (lane == 0) items[it].w = hit;
}

// FP64 -> float-float copies (moments accumulated in FP64, geometry)
__global__ void to_ff_kernel(int64_t n, const dbl4 *__restrict__ a, ff4 *__restrict__ b, int id_in_w) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const dbl4 v = a[i];
    ff4 o;
    o.x = ffloat(v.x);
    o.y = ffloat(v.y);
    o.z = ffloat(v.z);
    o.w = id_in_w ? ffloat(__int_as_float((int)v.w), 0.f) : ffloat(v.w);
    b[i] = o;
}

// --------------------------------------------------------------- launchers
int launch_weights(lspr_ctx *ctx, int prec, const double2 *x, const double2 *xt, int64_t N, int B, int S,
                   const float2 *xtf) {
    const int64_t Ns = ctx->mesh.Ns;
    const int BS = B * S;
    const unsigned grid = grid_for(Ns * BS, 256);
    cudaEvent_t ev;
    timer_begin(ctx, T_WEIGHTS, &ev);
    ++ctx->n_launches;
    if (prec == PREC_F64) {
        LSPR_TRY(ctx, ctx->w64.ensure(Ns * BS));
        weights_kernel<dbl4><<<grid, 256, 0, ctx->stream>>>(Ns, N, B, S, ctx->wo.spos64.p, ctx->wo.src_panel.p, ctx->mesh.surf.p, x, xt,
                                                            ctx->w64.p, ctx->rhs_map, ctx->rhs_nact);
    } else if (prec == PREC_FF) {
        LSPR_TRY(ctx, ctx->w_ff.ensure(Ns * BS));
        weights_kernel<ff4><<<grid, 256, 0, ctx->stream>>>(Ns, N, B, S, ctx->wo.spos64.p, ctx->wo.src_panel.p, ctx->mesh.surf.p, x, xt,
                                                           ctx->w_ff.p, ctx->rhs_map, ctx->rhs_nact);
    } else if (xtf) {
        LSPR_TRY(ctx, ctx->w32.ensure(Ns * BS));
        weights_f32t_kernel<<<grid, 256, 0, ctx->stream>>>(Ns, N, B, S, ctx->wo.spos32.p, ctx->wo.src_panel.p,
                                                           ctx->mesh.surf.p, xtf, ctx->w32.p, ctx->rhs_map,
                                                           ctx->rhs_nact);
    } else {
        LSPR_TRY(ctx, ctx->w32.ensure(Ns * BS));
        weights_kernel<float4><<<grid, 256, 0, ctx->stream>>>(Ns, N, B, S, ctx->wo.spos64.p, ctx->wo.src_panel.p, ctx->mesh.surf.p, x, xt,
                                                              ctx->w32.p, ctx->rhs_map, ctx->rhs_nact);
    }
    timer_end(ctx, T_WEIGHTS, ev);
    LSPR_TRY(ctx, cudaGetLastError());
    return LSPR_OK;
}

// float-float copies of the work-order geometry (after every change of work order)
int launch_ff_geometry(lspr_ctx *ctx) {
    const Mesh &m = ctx->mesh;
    WorkOrder &w = ctx->wo;
    LSPR_TRY(ctx, w.spos_ff.ensure(m.Ns));
    LSPR_TRY(ctx, w.snrm_ff.ensure(m.Ns));
    LSPR_TRY(ctx, w.tgt_ff.ensure(m.N));
    ctx->n_launches += 3;
    to_ff_kernel<<<grid_for(m.Ns, 256), 256, 0, ctx->stream>>>(m.Ns, w.spos64.p, w.spos_ff.p, 0);
    to_ff_kernel<<<grid_for(m.Ns, 256), 256, 0, ctx->stream>>>(m.Ns, w.snrm64.p, w.snrm_ff.p, 1);
    to_ff_kernel<<<grid_for(m.N, 256), 256, 0, ctx->stream>>>(m.N, w.tgt64.p, w.tgt_ff.p, 1);
    LSPR_TRY(ctx, cudaGetLastError());
    return LSPR_OK;
}

int launch_ff_boxes(lspr_ctx *ctx) {
    Tree &tr = ctx->tree;
    LSPR_TRY(ctx, tr.box_c_ff.ensure(tr.nboxes));
    ++ctx->n_launches;
    to_ff_kernel<<<grid_for(tr.nboxes, 256), 256, 0, ctx->stream>>>(tr.nboxes, tr.box_c64.p, tr.box_c_ff.p, 0);
    LSPR_TRY(ctx, cudaGetLastError());
    return LSPR_OK;
}

static int slot_of(int prec, int f32, int f64, int ff) { return prec == PREC_F64 ? f64 : (prec == PREC_FF ? ff : f32); }

int launch_p2p(lspr_ctx *ctx, int prec, const int4 *items, int64_t nitems, double *acc, cudaStream_t st,
               int *counter, int B) {
    if (nitems == 0) return LSPR_OK;
    cudaEvent_t ev;
    const int slot = slot_of(prec, T_P2P, T_P2P64, T_P2PFF);
    timer_begin_on(ctx, slot, &ev, st);
    ++ctx->n_launches;
    if (prec == PREC_F64) {
        if (B == 1) p2p_launch<double, 1>(ctx, items, nitems, B, acc, st, counter);
        else p2p_launch<double, batch_chunk<double>(2)>(ctx, items, nitems, B, acc, st, counter);
    } else if (prec == PREC_FF) {
        if (B == 1) p2p_launch<ffloat, 1>(ctx, items, nitems, B, acc, st, counter);
        else LSPR_TRY_ST(p2p_ff_multi(ctx, items, nitems, B, acc, st, counter));
    } else if (B > 1 && (ctx->tensor_cores & 2) && items == ctx->tree.p2p_items.p) {
        // the tensor-core P2P for products of at least tc_p2p_min_rhs right-hand sides in use, the
        // FP32 pipe below: decided on the host when every slot is in use, else on the device from
        // the count of running systems (both kernels are launched; the one not chosen returns at once)
        const int mn = std::max(2, ctx->tc_p2p_min_rhs);
        if (!ctx->rhs_nact) {
            if (B >= mn) LSPR_TRY_ST(p2p_tc_launch(ctx, acc, st, counter, B, 0));
            else p2p_launch<float, batch_chunk<float>(2)>(ctx, items, nitems, B, acc, st, counter);
        } else {
            LSPR_TRY_ST(p2p_tc_launch(ctx, acc, st, counter, B, mn));
            p2p_launch<float, batch_chunk<float>(2)>(ctx, items, nitems, B, acc, st, counter, mn);
        }
    } else {
        if (B == 1) p2p1_launch(ctx, items, nitems, acc, st, counter);
        else p2p_launch<float, batch_chunk<float>(2)>(ctx, items, nitems, B, acc, st, counter);
    }
    timer_end_on(ctx, slot, ev, st);
    timer_rhs(ctx, slot, B);
    LSPR_TRY(ctx, cudaGetLastError());
    return LSPR_OK;
}

int launch_item_flags(lspr_ctx *ctx, int4 *items, int64_t nitems) {
    if (nitems == 0) return LSPR_OK;
    ++ctx->n_launches;
    item_flags_kernel<<<grid_for(nitems * 32, 256), 256, 0, ctx->stream>>>(items, nitems, ctx->wo.src_tblock.p);
    LSPR_TRY(ctx, cudaGetLastError());
    return LSPR_OK;
}

int launch_p2m(lspr_ctx *ctx, int prec, int B) {
    Tree &tr = ctx->tree;
    if (tr.n_p2m_items == 0) return LSPR_OK;
    const int64_t nm = tr.nboxes * tr.NT * B;
    cudaEvent_t ev;
    const int slot = slot_of(prec, T_P2M, T_P2M64, T_P2MFF);
    timer_begin(ctx, slot, &ev);
    ++ctx->n_launches;
    if (prec == PREC_F32) {
        LSPR_TRY(ctx, tr.mom32.ensure(nm));
        LSPR_TRY(ctx, cudaMemsetAsync(tr.mom32.p, 0, sizeof(float4) * nm, ctx->stream));
        LSPR_TRY_ST(p2m_orders_f32(ctx, B));
    } else {
        LSPR_TRY(ctx, tr.mom64.ensure(nm));
        LSPR_TRY(ctx, cudaMemsetAsync(tr.mom64.p, 0, sizeof(dbl4) * nm, ctx->stream));
        if (prec == PREC_F64) {
            LSPR_TRY_ST(p2m_orders_f64(ctx, B));
        } else {
            LSPR_TRY_ST(p2m_orders_ff(ctx, B));
            LSPR_TRY(ctx, tr.mom_ff.ensure(nm));
            ++ctx->n_launches;
            to_ff_kernel<<<grid_for(nm, 256), 256, 0, ctx->stream>>>(nm, tr.mom64.p, tr.mom_ff.p, 0);
        }
    }
    timer_end(ctx, slot, ev);
    timer_rhs(ctx, slot, B);
    LSPR_TRY(ctx, cudaGetLastError());
    return LSPR_OK;
}

int launch_m2p(lspr_ctx *ctx, int prec, double *acc, int *counter, int B) {
    Tree &tr = ctx->tree;
    if (tr.n_m2p_items == 0) return LSPR_OK;
    cudaEvent_t ev;
    const int slot = slot_of(prec, T_M2P, T_M2P64, T_M2PFF);
    timer_begin(ctx, slot, &ev);
    ++ctx->n_launches;
    if (prec == PREC_F64) {
        LSPR_TRY_ST(m2p_orders_f64(ctx, acc, counter, B));
    } else if (prec == PREC_FF) {
        LSPR_TRY_ST(m2p_orders_ff(ctx, acc, counter, B));
    } else {
        LSPR_TRY_ST(m2p_orders_f32(ctx, acc, counter, B));
    }
    timer_end(ctx, slot, ev);
    timer_rhs(ctx, slot, B);
    LSPR_TRY(ctx, cudaGetLastError());
    return LSPR_OK;
}

// Launchers on explicit buffers (no context-owned scratch), one right-hand side: used
// by the allocation-free matvec entry point.
int launch_weights_fp32_raw(cudaStream_t st, int64_t Ns, int64_t N, const dbl4 *spos64, const int *src_panel,
                            const double2 *x, float4 *w) {
    weights_kernel<float4><<<grid_for(Ns, 256), 256, 0, st>>>(Ns, N, 1, 1, spos64, src_panel, nullptr, x, nullptr, w, nullptr,
                                                               nullptr);
    return cudaGetLastError() == cudaSuccess ? LSPR_OK : LSPR_E_CUDA;
}

int launch_p2p_fp32_raw(cudaStream_t st, const int4 *items, int64_t nitems, const float4 *tgt, int64_t ntgt,
                        const float4 *spos, const float4 *snrm, const float4 *w, double *acc) {
    if (nitems == 0) return LSPR_OK;
    p2p_kernel<float, 1, false><<<grid_for(nitems, p2p_warps(1)), p2p_warps(1) * 32, 0, st>>>(
        items, nitems, 1, 1, tgt, ntgt, spos, snrm, w, acc, nullptr, nullptr, 1 << 30);
    return cudaGetLastError() == cudaSuccess ? LSPR_OK : LSPR_E_CUDA;
}

}  // namespace lspr