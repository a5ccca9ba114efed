// Autotuners.
//
// lspr_autotune: the treecode parameters (theta, P, Ncrit) of Sec. II.D under an accuracy bound
// on sigma_ext: a grid search in which every candidate is built and solved, its sigma_ext
// compared with a reference solve, and the cheapest qualifying candidate kept.  The accuracy of
// a (theta, P, Ncrit) choice is measured, not predicted: the deviation of sigma_ext is not
// monotone in theta, P or Ncrit (the acceptance criterion changes which boxes are expanded, and
// the solve amplifies operator errors near the resonance).  The cost is either the time of the
// tuning solve or, for a batch of many right-hand sides, a model built from measured product
// times at the batch's size (the tuning wavelengths are few, and a tree that is fastest for four
// right-hand sides is not the fastest for sixty-four), which also picks the P2P path.
//
// lspr_tune_solver: the GMRES restart length and the P2P path for the whole batch, each pair
// timed with a full solve.
#include <algorithm>
#include <cmath>
#include <vector>

#include "lspr_internal.cuh"

using namespace lspr;

namespace {

struct Trial {
    double theta;
    int P, Ncrit;
};

// one solve of the tuning wavelengths; sigma receives its results, iters its Arnoldi steps
int tuning_solve(lspr_ctx *c, const double *eps_in, double eo_re, double eo_im, const double *E0, const double *lam,
                 int B, const lspr_solve_opts &so, std::vector<double> &sigma, std::vector<int32_t> &iters) {
    std::vector<double> dip(6 * (size_t)B), res((size_t)B);
    std::vector<int32_t> status((size_t)B);
    sigma.assign(B, 0.0);
    iters.assign(B, 0);
    lspr_solve_stats st{iters.data(), res.data(), status.data(), 0.0, 0};
    return solve_impl(c, eps_in, eo_re, eo_im, E0, lam, B, so, dip.data(), sigma.data(), &st);
}

// builds the tree and solves once untimed (recording of graphs, first-use set-up) and once
// timed; sigma receives the second solve's results
int run_trial(lspr_ctx *c, const Trial &t, const double *eps_in, double eo_re, double eo_im, const double *E0,
              const double *lam, int B, const lspr_solve_opts &so, std::vector<double> &sigma,
              std::vector<int32_t> &iters, double &ms) {
    int rc = tree_build(c, t.theta, t.P, t.Ncrit);
    if (rc != LSPR_OK) return rc;
    rc = tuning_solve(c, eps_in, eo_re, eo_im, E0, lam, B, so, sigma, iters);
    if (rc != LSPR_OK) return rc;
    cudaEvent_t e0, e1;
    LSPR_TRY(c, cudaEventCreate(&e0));
    LSPR_TRY(c, cudaEventCreate(&e1));
    cudaEventRecord(e0, c->stream);
    rc = tuning_solve(c, eps_in, eo_re, eo_im, E0, lam, B, so, sigma, iters);
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float f = 0.f;
    cudaEventElapsedTime(&f, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ms = f;
    return rc;
}

// time of one product of the given mode on the batch buffers (CUDA events on the stream)
int time_product(lspr_ctx *c, int mode, int Bt, const double2 *x, double2 *y, const double2 *s, double &ms) {
    cudaEvent_t e0, e1;
    LSPR_TRY(c, cudaEventCreate(&e0));
    LSPR_TRY(c, cudaEventCreate(&e1));
    cudaEventRecord(e0, c->stream);
    int rc = apply_operator(c, mode, x, y, s, Bt);
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float f = 0.f;
    cudaEventElapsedTime(&f, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ms = f;
    return rc;
}

// modelled cost of the current tree for Bt right-hand sides: (steps + 4) x FP32 product + one
// residual product; the faster P2P path is left in c->tensor_cores
struct ProductBufs {
    DArr<double2> x, y, s;
};
int model_cost(lspr_ctx *c, int mode, int res_mode, int Bt, int steps, ProductBufs &pb, int base_mask, double &cost,
               double &t_main, double &t_res, int &mask) {
    const int S = c->mesh.S;
    const int64_t n2 = 2 * c->mesh.N;
    LSPR_TRY(c, pb.x.ensure((size_t)Bt * n2));
    LSPR_TRY(c, pb.y.ensure((size_t)Bt * n2));
    LSPR_TRY(c, pb.s.ensure((size_t)Bt * S));
    LSPR_TRY(c, cudaMemsetAsync(pb.x.p, 0, sizeof(double2) * Bt * n2, c->stream));
    std::vector<double2> sh((size_t)Bt * S, make_double2(-2.0, 0.1));
    LSPR_TRY(c, cudaMemcpyAsync(pb.s.p, sh.data(), sizeof(double2) * sh.size(), cudaMemcpyHostToDevice, c->stream));
    std::vector<int> masks{base_mask & ~2};
    if (Bt >= 2 && mode_prec(mode) == PREC_F32) masks.push_back(base_mask | 2);
    t_main = 1e30;
    for (int mk : masks) {
        c->tensor_cores = mk;
        double t = 0.0;
        LSPR_TRY_ST(apply_operator(c, mode, pb.x.p, pb.y.p, pb.s.p, Bt));   // first use: lists, buffers
        LSPR_TRY_ST(time_product(c, mode, Bt, pb.x.p, pb.y.p, pb.s.p, t));
        if (t < t_main) {
            t_main = t;
            mask = mk;
        }
    }
    c->tensor_cores = mask;
    t_res = 0.0;
    if (res_mode >= 0) LSPR_TRY_ST(time_product(c, res_mode, Bt, pb.x.p, pb.y.p, pb.s.p, t_res));
    cost = (steps + 4) * t_main + t_res;
    return LSPR_OK;
}

}  // namespace

extern "C" {

int lspr_autotune(lspr_ctx *c, const double *eps_in, double eps_out_re, double eps_out_im, const double *E0,
                  const double *lambda_nm, int32_t B, const lspr_tune_opts *o, lspr_tune_result *res) {
    if (!c || !eps_in || !E0 || !lambda_nm || !o || !res || B < 1) return LSPR_E_ARG;
    if (!(o->target_rel_err > 0) || !(o->tol > 0) || o->restart < 1) return LSPR_E_ARG;
    if (o->mode != LSPR_TREE_FP32 && o->mode != LSPR_TREE_FP64 && o->mode != LSPR_TREE_FF) return LSPR_E_ARG;
    if (o->refine < 0 || o->refine > 2 || o->grid < 0 || o->grid > 1 || o->time_rhs < 0) return LSPR_E_ARG;
    if (!c->mesh.ready) return LSPR_E_STATE;
    cudaSetDevice(c->device);
    lspr_solve_opts so;
    so.tol = o->tol;
    so.restart = o->restart;
    so.maxiter = 5000;
    so.mode = o->mode;
    so.refine = o->refine;
    const bool model = o->time_rhs > 0;
    const int res_mode = (o->mode == LSPR_TREE_FP32 && o->refine) ? (o->refine == 1 ? LSPR_TREE_FF : LSPR_TREE_FP64)
                                                                   : -1;
    const int base_mask = c->tensor_cores;
    ProductBufs pb;
    // reference: the most accurate compiled order at a tight acceptance criterion
    const Trial ref = {0.3, kMaxP, 256};
    std::vector<double> sref;
    std::vector<int32_t> its;
    double ref_ms = 0.0, ref_main = 0.0, ref_res = 0.0;
    int ref_mask = base_mask;
    int rc = run_trial(c, ref, eps_in, eps_out_re, eps_out_im, E0, lambda_nm, B, so, sref, its, ref_ms);
    if (rc != LSPR_OK) return rc;
    const int steps = *std::max_element(its.begin(), its.end());
    if (model) {
        rc = model_cost(c, o->mode, res_mode, o->time_rhs, steps, pb, base_mask, ref_ms, ref_main, ref_res, ref_mask);
        if (rc != LSPR_OK) return rc;
    }
    const double bound = 0.5 * o->target_rel_err;
    Trial best = ref;
    double best_ms = ref_ms, best_err = 0.0, best_main = ref_main, best_res = ref_res;
    int best_mask = ref_mask;
    int n = 0, ok = 0;
    std::vector<Trial> grid;
    if (o->grid == 0) {
        for (int P = 4; P <= kMaxP; ++P)
            for (double theta : {0.3, 0.4, 0.5, 0.6})
                for (int Ncrit : {128, 256, 512}) grid.push_back({theta, P, Ncrit});
    } else {
        for (int P = 5; P <= 7; ++P)
            for (double theta : {0.4, 0.5})
                for (int Ncrit : {256, 512}) grid.push_back({theta, P, Ncrit});
    }
    for (const Trial &t : grid) {
        if (t.theta == ref.theta && t.P == ref.P && t.Ncrit == ref.Ncrit) continue;
        std::vector<double> s;
        std::vector<int32_t> ti;
        double ms = 0.0, t_main = 0.0, t_res = 0.0;
        int mask = base_mask;
        ++n;
        if (model) {
            c->tensor_cores = base_mask;
            rc = tree_build(c, t.theta, t.P, t.Ncrit);
            if (rc == LSPR_OK) rc = tuning_solve(c, eps_in, eps_out_re, eps_out_im, E0, lambda_nm, B, so, s, ti);
        } else {
            rc = run_trial(c, t, eps_in, eps_out_re, eps_out_im, E0, lambda_nm, B, so, s, ti, ms);
        }
        if (rc == LSPR_E_NOT_CONVERGED) continue;
        if (rc != LSPR_OK) return rc;
        double err = 0.0;
        for (int b = 0; b < B; ++b) err = std::max(err, std::fabs(s[b] - sref[b]) / std::fabs(sref[b]));
        if (!(err <= bound)) continue;
        ++ok;
        if (model) {
            rc = model_cost(c, o->mode, res_mode, o->time_rhs, steps, pb, base_mask, ms, t_main, t_res, mask);
            if (rc != LSPR_OK) return rc;
        }
        if (ms < best_ms) {
            best = t;
            best_ms = ms;
            best_err = err;
            best_main = t_main;
            best_res = t_res;
            best_mask = mask;
        }
    }
    c->tensor_cores = model ? best_mask : base_mask;
    rc = tree_build(c, best.theta, best.P, best.Ncrit);
    if (rc != LSPR_OK) return rc;
    res->theta = best.theta;
    res->P = best.P;
    res->Ncrit = best.Ncrit;
    res->rel_err = best_err;
    res->ms = best_ms;
    res->ref_ms = ref_ms;
    res->candidates = n + 1;
    res->qualified = ok;
    res->tensor_cores = c->tensor_cores;
    res->iterations = steps;
    res->product_ms = best_main;
    res->residual_product_ms = best_res;
    LSPR_TRY(c, cudaStreamSynchronize(c->stream));
    return timeout_status(c, LSPR_OK);
}

int lspr_tune_solver(lspr_ctx *c, const double *eps_in, double eps_out_re, double eps_out_im, const double *E0,
                     const double *lambda_nm, int32_t B, const lspr_solve_opts *o, const int32_t *restarts,
                     int32_t n_restarts, int32_t *restart, int32_t *tensor_cores, double *ms) {
    if (!c || !eps_in || !E0 || !lambda_nm || !o || !restarts || !restart || !tensor_cores || !ms || B < 1 ||
        n_restarts < 1)
        return LSPR_E_ARG;
    for (int k = 0; k < n_restarts; ++k)
        if (restarts[k] < 1 || restarts[k] > 512) return LSPR_E_ARG;
    if (o->mode < 0 || o->mode > 5 || !(o->tol > 0) || o->maxiter < 1 || o->refine < 0 || o->refine > 2)
        return LSPR_E_ARG;
    if (!c->mesh.ready) return LSPR_E_STATE;
    if (mode_tree(o->mode) && !c->tree.ready) return LSPR_E_STATE;
    cudaSetDevice(c->device);
    const int base = c->tensor_cores;
    std::vector<int> masks{base & ~2};
    if (B >= 2 && mode_prec(o->mode) == PREC_F32) masks.push_back(base | 2);
    double best = 1e300;
    int best_m = -1, best_mask = base;
    std::vector<double> dip(6 * (size_t)B), sig((size_t)B), res((size_t)B);
    std::vector<int32_t> its((size_t)B), status((size_t)B);
    for (int mk : masks)
        for (int k = 0; k < n_restarts; ++k) {
            c->tensor_cores = mk;
            lspr_solve_opts so = *o;
            so.restart = restarts[k];
            lspr_solve_stats st{its.data(), res.data(), status.data(), 0.0, 0};
            cudaEvent_t e0, e1;
            LSPR_TRY(c, cudaEventCreate(&e0));
            LSPR_TRY(c, cudaEventCreate(&e1));
            cudaEventRecord(e0, c->stream);
            int rc = solve_impl(c, eps_in, eps_out_re, eps_out_im, E0, lambda_nm, B, so, dip.data(), sig.data(), &st);
            cudaEventRecord(e1, c->stream);
            cudaEventSynchronize(e1);
            float f = 0.f;
            cudaEventElapsedTime(&f, e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (rc == LSPR_E_NOT_CONVERGED) continue;
            if (rc != LSPR_OK) {
                c->tensor_cores = base;
                return rc;
            }
            if (f < best) {
                best = f;
                best_m = restarts[k];
                best_mask = mk;
            }
        }
    c->tensor_cores = best_m > 0 ? best_mask : base;
    if (best_m < 0) return LSPR_E_NOT_CONVERGED;
    *restart = best_m;
    *tensor_cores = best_mask;
    *ms = best;
    LSPR_TRY(c, cudaStreamSynchronize(c->stream));
    return timeout_status(c, LSPR_OK);
}

}  // extern "C"
