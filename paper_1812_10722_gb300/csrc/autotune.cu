// Autotuner of the treecode parameters (theta, P, Ncrit) of Sec. II.D under an accuracy
// bound on sigma_ext: a grid search in which every candidate is built and solved, its
// sigma_ext compared with a reference solve, and the fastest qualifying candidate kept.
// The accuracy of a (theta, P, Ncrit) choice is measured, not predicted: the deviation
// of sigma_ext is not monotone in theta, P or Ncrit (the acceptance criterion changes
// which boxes are expanded, and the solve amplifies operator errors near the resonance).
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

// builds the tree, solves once untimed (recording of graphs, first-use set-up) and once
// timed; sigma receives the second solve's results
int run_trial(lspr_ctx *c, const Trial &t, const double *eps_in, double eo_re, double eo_im, const double *E0,
              const double *lam, int B, const lspr_solve_opts &so, std::vector<double> &sigma, double &ms) {
    int rc = tree_build(c, t.theta, t.P, t.Ncrit);
    if (rc != LSPR_OK) return rc;
    std::vector<double> dip(6 * (size_t)B);
    sigma.assign(B, 0.0);
    rc = solve_impl(c, eps_in, eo_re, eo_im, E0, lam, B, so, dip.data(), sigma.data(), nullptr);
    if (rc != LSPR_OK) return rc;
    cudaEvent_t e0, e1;
    LSPR_TRY(c, cudaEventCreate(&e0));
    LSPR_TRY(c, cudaEventCreate(&e1));
    cudaEventRecord(e0, c->stream);
    rc = solve_impl(c, eps_in, eo_re, eo_im, E0, lam, B, so, dip.data(), sigma.data(), nullptr);
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float f = 0.f;
    cudaEventElapsedTime(&f, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ms = f;
    return rc;
}

}  // namespace

extern "C" {

int lspr_autotune(lspr_ctx *c, const double *eps_in, double eps_out_re, double eps_out_im, const double *E0,
                  const double *lambda_nm, int32_t B, const lspr_tune_opts *o, lspr_tune_result *res) {
    if (!c || !eps_in || !E0 || !lambda_nm || !o || !res || B < 1) return LSPR_E_ARG;
    if (!(o->target_rel_err > 0) || !(o->tol > 0) || o->restart < 1) return LSPR_E_ARG;
    if (o->mode != LSPR_TREE_FP32 && o->mode != LSPR_TREE_FP64 && o->mode != LSPR_TREE_FF) return LSPR_E_ARG;
    if (o->refine < 0 || o->refine > 2 || o->grid < 0 || o->grid > 1) return LSPR_E_ARG;
    if (!c->mesh.ready) return LSPR_E_STATE;
    cudaSetDevice(c->device);
    lspr_solve_opts so;
    so.tol = o->tol;
    so.restart = o->restart;
    so.maxiter = 5000;
    so.mode = o->mode;
    so.refine = o->refine;
    // reference: the most accurate compiled order at a tight acceptance criterion
    const Trial ref = {0.3, kMaxP, 256};
    std::vector<double> sref;
    double ref_ms = 0.0;
    int rc = run_trial(c, ref, eps_in, eps_out_re, eps_out_im, E0, lambda_nm, B, so, sref, ref_ms);
    if (rc != LSPR_OK) return rc;
    const double bound = 0.5 * o->target_rel_err;
    Trial best = ref;
    double best_ms = ref_ms, best_err = 0.0;
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
                double ms = 0.0;
                rc = run_trial(c, t, eps_in, eps_out_re, eps_out_im, E0, lambda_nm, B, so, s, ms);
                ++n;
                if (rc == LSPR_E_NOT_CONVERGED) continue;
                if (rc != LSPR_OK) return rc;
                double err = 0.0;
                for (int b = 0; b < B; ++b) err = std::max(err, std::fabs(s[b] - sref[b]) / std::fabs(sref[b]));
                if (!(err <= bound)) continue;
                ++ok;
                if (ms < best_ms) {
                    best = t;
                    best_ms = ms;
                    best_err = err;
                }
            }
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
    LSPR_TRY(c, cudaStreamSynchronize(c->stream));
    return timeout_status(c, LSPR_OK);
}

}  // extern "C"
