// C ABI entry points (declared in include/lspr.h).  Argument checking, context
// ownership and status mapping live here; the numerical work is in mesh.cu,
// tree.cu, farfield.cu and solve.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <new>
#include <vector>

#include "lspr_internal.cuh"

namespace lspr {

void timer_begin(lspr_ctx *ctx, int slot, cudaEvent_t *ev) { timer_begin_on(ctx, slot, ev, ctx->stream); }

void timer_end(lspr_ctx *ctx, int slot, cudaEvent_t ev) { timer_end_on(ctx, slot, ev, ctx->stream); }

void timer_begin_on(lspr_ctx *ctx, int slot, cudaEvent_t *ev, cudaStream_t st) {
    (void)slot;
    *ev = nullptr;
    Timing &t = ctx->timing;
    if (!t.enabled) return;
    if (t.used + 2 > t.pool.size()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            t.pool.push_back(e);
        }
    }
    *ev = t.pool[t.used++];
    cudaEventRecord(*ev, st);
}

void timer_end_on(lspr_ctx *ctx, int slot, cudaEvent_t ev, cudaStream_t st) {
    Timing &t = ctx->timing;
    if (!t.enabled || !ev) return;
    if (t.used + 1 > t.pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        t.pool.push_back(e);
    }
    cudaEvent_t e2 = t.pool[t.used++];
    cudaEventRecord(e2, st);
    t.pending.push_back({slot, {ev, e2}});
    if (t.used > 4096) timer_collect(ctx);
}

void timer_collect(lspr_ctx *ctx) {
    Timing &t = ctx->timing;
    if (t.pending.empty()) {
        t.used = 0;
        return;
    }
    cudaStreamSynchronize(ctx->stream);
    if (ctx->side) cudaStreamSynchronize(ctx->side);
    for (auto &p : t.pending) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess) {
            t.ms[p.first] += ms;
            t.launches[p.first] += 1;
        }
    }
    t.pending.clear();
    t.used = 0;
}

}  // namespace lspr

namespace lspr {

// LSPR_E_TIMEOUT if a bounded device wait ran out since the last status that reported one
// (the stream is synchronised by the caller); otherwise rc
int timeout_status(lspr_ctx *c, int rc) {
    int count = 0;
    if (cudaMemcpy(&count, c->dev_err.p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_status(c, cudaGetLastError(), "reading the device error count");
    if (count == c->dev_err_seen) return rc;
    c->dev_err_seen = count;
    c->last_error = "a bounded device wait ran out: the product is incomplete";
    return (rc == LSPR_OK || rc == LSPR_E_NOT_CONVERGED) ? LSPR_E_TIMEOUT : rc;
}

}  // namespace lspr

using namespace lspr;

extern "C" {

const char *lspr_status_string(int s) {
    switch (s) {
    case LSPR_OK: return "ok";
    case LSPR_E_ARG: return "invalid argument";
    case LSPR_E_STATE: return "call out of order (mesh or tree missing)";
    case LSPR_E_CUDA: return "CUDA error";
    case LSPR_E_OOM: return "device memory exhausted";
    case LSPR_E_NOT_CONVERGED: return "GMRES did not reach the tolerance";
    case LSPR_E_TIMEOUT: return "device wait exceeded its bound";
    case LSPR_E_MESH: return "degenerate or non-finite mesh";
    default: return "unknown status";
    }
}

const char *lspr_version(void) { return "lspr-gb300 0.1 (sm_103a)"; }

const char *lspr_last_error(lspr_ctx *c) { return c ? c->last_error.c_str() : ""; }

int lspr_create(lspr_ctx **out, int device, void *cuda_stream) {
    if (!out) return LSPR_E_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return n == 0 ? LSPR_E_CUDA : LSPR_E_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return LSPR_E_CUDA;
    lspr_ctx *c = new (std::nothrow) lspr_ctx();
    if (!c) return LSPR_E_OOM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        c->dev_err.ensure(2) != cudaSuccess || cudaMemset(c->dev_err.p, 0, 2 * sizeof(int)) != cudaSuccess) {
        lspr_destroy(c);
        return LSPR_E_CUDA;
    }
    *out = c;
    return LSPR_OK;
}

int lspr_destroy(lspr_ctx *c) {
    if (!c) return LSPR_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->side) cudaStreamSynchronize(c->side);
    if (c->gstream) cudaStreamSynchronize(c->gstream);
    for (GraphCache &g : c->gcache) g.reset();
    for (cudaEvent_t e : c->timing.pool) cudaEventDestroy(e);
    for (cudaEvent_t e : {c->ev_fork, c->ev_join, c->ev_g0, c->ev_g1})
        if (e) cudaEventDestroy(e);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    delete c;   // device arrays free themselves
    return LSPR_OK;
}

int lspr_mesh_upload(lspr_ctx *c, const double *verts, int64_t nv, const int32_t *tris, int64_t ntri,
                     const int32_t *surf_id, int32_t nsurf, const lspr_quad_opts *q, int32_t on_device) {
    if (!c || !verts || !tris || !q || nv < 3 || ntri < 1 || nsurf < 1 || nsurf > kMaxSurfaces) return LSPR_E_ARG;
    if (nsurf > 1 && !surf_id) return LSPR_E_ARG;
    if (ntri > (int64_t)1 << 28 || nv > (int64_t)1 << 30) return LSPR_E_ARG;
    cudaSetDevice(c->device);
    return mesh_build(c, verts, nv, tris, ntri, nsurf > 1 ? surf_id : nullptr, nsurf, on_device, *q);
}

int lspr_tree_build(lspr_ctx *c, double theta, int32_t P, int32_t Ncrit) {
    if (!c) return LSPR_E_ARG;
    if (!c->mesh.ready) return LSPR_E_STATE;
    if (!(theta > 0.0 && theta < 1.0) || P < 1 || P > kMaxP || Ncrit < 1) return LSPR_E_ARG;
    cudaSetDevice(c->device);
    return tree_build(c, theta, P, Ncrit);
}

int lspr_matvec(lspr_ctx *c, const double *x, double *y, int32_t B, const double *eps_ratio, int32_t mode,
                int32_t on_device) {
    if (!c || !x || !y || !eps_ratio || B < 1 || mode < 0 || mode > 5) return LSPR_E_ARG;
    if (!c->mesh.ready) return LSPR_E_STATE;
    if (mode_tree(mode) && !c->tree.ready) return LSPR_E_STATE;
    cudaSetDevice(c->device);
    const int64_t n2 = 2 * c->mesh.N;
    const double2 *xd = (const double2 *)x;
    double2 *yd = (double2 *)y;
    const double2 *sd = (const double2 *)eps_ratio;
    if (!on_device) {
        LSPR_TRY(c, c->xbuf.ensure((size_t)B * n2));
        LSPR_TRY(c, c->ybuf.ensure((size_t)B * n2));
        const int S = c->mesh.S;   // eps_ratio is [B][S]
        LSPR_TRY(c, c->sbuf.ensure((size_t)B * S));
        LSPR_TRY(c, cudaMemcpyAsync(c->xbuf.p, x, sizeof(double2) * B * n2, cudaMemcpyHostToDevice, c->stream));
        LSPR_TRY(c, cudaMemcpyAsync(c->sbuf.p, eps_ratio, sizeof(double2) * B * S, cudaMemcpyHostToDevice,
                                    c->stream));
        xd = c->xbuf.p;
        yd = c->ybuf.p;
        sd = c->sbuf.p;
    }
    LSPR_TRY_ST(apply_operator(c, mode, xd, yd, sd, B));
    if (!on_device)
        LSPR_TRY(c, cudaMemcpyAsync(y, yd, sizeof(double2) * B * n2, cudaMemcpyDeviceToHost, c->stream));
    LSPR_TRY(c, cudaStreamSynchronize(c->stream));
    timer_collect(c);
    return timeout_status(c, LSPR_OK);
}

int lspr_solve(lspr_ctx *c, const double *eps_in, double eps_out_re, double eps_out_im, const double *E0,
               const double *lambda_nm, int32_t B, const lspr_solve_opts *o, double *dipole_out,
               double *sigma_ext_out, lspr_solve_stats *st) {
    if (!c || !eps_in || !E0 || !lambda_nm || !o || !dipole_out || !sigma_ext_out || B < 1) return LSPR_E_ARG;
    if (o->mode < 0 || o->mode > 5 || !(o->tol > 0) || o->restart < 1 || o->maxiter < 1) return LSPR_E_ARG;
    if (o->refine < 0 || o->refine > 2) return LSPR_E_ARG;
    if (!(E0[0] * E0[0] + E0[1] * E0[1] + E0[2] * E0[2] > 0)) return LSPR_E_ARG;
    if (!c->mesh.ready) return LSPR_E_STATE;
    if (mode_tree(o->mode) && !c->tree.ready) return LSPR_E_STATE;
    cudaSetDevice(c->device);
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t mv0 = c->matvec_count;
    int rc = solve_impl(c, eps_in, eps_out_re, eps_out_im, E0, lambda_nm, B, *o, dipole_out, sigma_ext_out, st);
    timer_collect(c);
    if (cudaStreamSynchronize(c->stream) == cudaSuccess) rc = timeout_status(c, rc);
    if (st) {
        st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        st->matvecs = c->matvec_count - mv0;
    }
    return rc;
}

int lspr_get_info(lspr_ctx *c, int64_t *n_panels, int64_t *n_sources, int64_t *n_near, int64_t *n_boxes,
                  int64_t *n_p2p_items, int64_t *n_m2p_pairs, int64_t *n_p2p_pairs) {
    if (!c) return LSPR_E_ARG;
    if (n_panels) *n_panels = c->mesh.N;
    if (n_sources) *n_sources = c->mesh.Ns;
    if (n_near) *n_near = c->mesh.nnz;
    if (n_boxes) *n_boxes = c->tree.ready ? c->tree.nboxes : 0;
    if (n_p2p_items) *n_p2p_items = c->tree.ready ? c->tree.n_p2p_items : 0;
    if (n_m2p_pairs) *n_m2p_pairs = c->tree.ready ? c->tree.n_m2p_pairs : 0;
    if (n_p2p_pairs) *n_p2p_pairs = c->tree.ready ? c->tree.p2p_pairs : 0;
    return LSPR_OK;
}

int lspr_get_tc_info(lspr_ctx *c, int64_t *m2p_units, int64_t *m2p_group_boxes, int64_t *p2p_group_sources,
                     int64_t *p2p_stages) {
    if (!c) return LSPR_E_ARG;
    const Tree &tr = c->tree;
    const bool m = tr.ready && tr.tc_built, p = tr.ready && tr.tcp_built;
    if (m2p_units) *m2p_units = m ? tr.n_tc_items : 0;
    if (m2p_group_boxes) *m2p_group_boxes = m ? tr.n_tc_pairs : 0;
    if (p2p_group_sources) *p2p_group_sources = p ? tr.n_tcp_sources : 0;
    if (p2p_stages) *p2p_stages = p ? tr.n_tcp_stages : 0;
    return LSPR_OK;
}

int lspr_launch_count(lspr_ctx *c, int64_t *count) {
    if (!c || !count) return LSPR_E_ARG;
    *count = c->n_launches;
    return LSPR_OK;
}

int lspr_set_graphs(lspr_ctx *c, int32_t enable) {
    if (!c) return LSPR_E_ARG;
    c->use_graphs = enable != 0;
    return LSPR_OK;
}

int lspr_set_tensor_cores(lspr_ctx *c, int32_t enable) {
    if (!c) return LSPR_E_ARG;
    c->tensor_cores = enable & 3;
    return LSPR_OK;
}

int lspr_set_charges(lspr_ctx *c, const double *charges, int64_t nq, const int32_t *surf_q) {
    if (!c || nq < 0 || (nq > 0 && (!charges || !surf_q))) return LSPR_E_ARG;
    int mx = -1;
    for (int64_t k = 0; k < nq; ++k) {
        if (surf_q[k] < 0) return LSPR_E_ARG;
        mx = std::max(mx, (int)surf_q[k]);
    }
    c->nq = 0;
    c->max_charge_surf = -1;
    if (nq == 0) return LSPR_OK;
    std::vector<dbl4> h((size_t)nq);
    for (int64_t k = 0; k < nq; ++k)
        h[k] = make_dbl4(charges[4 * k], charges[4 * k + 1], charges[4 * k + 2], charges[4 * k + 3]);
    LSPR_TRY(c, c->charges.ensure(nq));
    LSPR_TRY(c, c->charge_surf.ensure(nq));
    LSPR_TRY(c, cudaMemcpyAsync(c->charges.p, h.data(), sizeof(dbl4) * nq, cudaMemcpyHostToDevice, c->stream));
    LSPR_TRY(c, cudaMemcpyAsync(c->charge_surf.p, surf_q, sizeof(int32_t) * nq, cudaMemcpyHostToDevice, c->stream));
    LSPR_TRY(c, cudaStreamSynchronize(c->stream));
    c->nq = nq;
    c->max_charge_surf = mx;
    return LSPR_OK;
}

int lspr_selftest_wait_timeout(lspr_ctx *c, int32_t *result) {
    if (!c || !result) return LSPR_E_ARG;
    return lspr::selftest_wait_timeout(c, result);
}

int lspr_device_errors(lspr_ctx *c, int32_t *count) {
    if (!c || !count) return LSPR_E_ARG;
    *count = 0;
    if (!c->dev_err.p) return LSPR_OK;
    LSPR_TRY(c, cudaStreamSynchronize(c->stream));
    LSPR_TRY(c, cudaMemcpy(count, c->dev_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost));
    return LSPR_OK;
}

int lspr_selftest_gate_waits(lspr_ctx *c, int32_t enable) {
    if (!c) return LSPR_E_ARG;
    const int v = enable ? 1 : 0;
    LSPR_TRY(c, cudaMemcpyAsync(c->dev_err.p + 1, &v, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    LSPR_TRY(c, cudaStreamSynchronize(c->stream));
    return LSPR_OK;
}

int lspr_graph_stats(lspr_ctx *c, int64_t *cycles, int64_t *recordings) {
    if (!c) return LSPR_E_ARG;
    if (cycles) *cycles = c->graph_cycles;
    if (recordings) *recordings = c->graph_recordings;
    return LSPR_OK;
}

int lspr_set_timing(lspr_ctx *c, int32_t enable) {
    if (!c) return LSPR_E_ARG;
    timer_collect(c);
    c->timing.enabled = enable != 0;
    for (int k = 0; k < kTimerSlots; ++k) {
        c->timing.ms[k] = 0;
        c->timing.launches[k] = 0;
        c->timing.rhs[k] = 0;
    }
    return LSPR_OK;
}

int lspr_get_timing_rhs(lspr_ctx *c, int64_t *rhs) {
    if (!c || !rhs) return LSPR_E_ARG;
    for (int k = 0; k < kTimerSlots; ++k) rhs[k] = c->timing.rhs[k];
    return LSPR_OK;
}

int lspr_get_arnoldi_stats(lspr_ctx *c, int64_t *out) {
    if (!c || !out) return LSPR_E_ARG;
    unsigned long long h[4] = {0, 0, 0, 0};
    if (c->arn.stats.p) {
        cudaSetDevice(c->device);
        LSPR_TRY(c, cudaMemcpyAsync(h, c->arn.stats.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        LSPR_TRY(c, cudaStreamSynchronize(c->stream));
    }
    for (int k = 0; k < 4; ++k) out[k] = (int64_t)h[k];
    return LSPR_OK;
}

int lspr_get_timing(lspr_ctx *c, double *ms, int64_t *launches) {
    if (!c) return LSPR_E_ARG;
    timer_collect(c);
    for (int k = 0; k < kTimerSlots; ++k) {
        if (ms) ms[k] = c->timing.ms[k];
        if (launches) launches[k] = c->timing.launches[k];
    }
    return LSPR_OK;
}

}  // extern "C"
