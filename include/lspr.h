/*
 * lspr.h -- C ABI of the GB300 (sm_103a) quasistatic LSPR boundary-element library.
 *
 * Method: Clementi, Cooper & Barba, "Computational nanoplasmonics in the
 * quasistatic limit for biosensing applications" (arXiv:1812.10722).
 *   - interface problem and its boundary integral equations: Sec. II.A, II.C,
 *     Eqs. electrostatic_scatter, integral_eq_lspr
 *   - flat-panel collocation and the 2x2 block system: Eqs. layers_disc,
 *     matrix_lspr, layers_element
 *   - singular / near-singular / far quadrature: Sec. II.C "Integral evaluation"
 *   - treecode (octree, N_crit, MAC theta, Cartesian Taylor order P): Sec. II.D
 *   - complex GMRES: Sec. II.D-II.E
 *   - dipole and extinction cross-section: Eqs. dipole_def_gauss_i_final,
 *     scat_efield_long_range, scat_efield_fwa, cext_fwa
 *
 * Conventions shared by every entry point
 *   - Lengths in nm, cross-sections in nm^2.  Triangles are counter-clockwise
 *     seen from outside, so (v1-v0)x(v2-v0) is the outward normal.
 *   - A complex number is two doubles (re, im); complex arrays are interleaved.
 *   - The unknown vector of one wavelength is [phi_1 .. phi_N, dphi_1 .. dphi_N]
 *     (potential and its normal derivative inside the particle, one value per
 *     panel); B right-hand sides are stored one after another ([B][2N] complex).
 *   - Every call returns an lspr_status; no exception or abort crosses the ABI.
 *     On an error the context stays valid unless the status is LSPR_E_CUDA
 *     after a sticky device error.
 *   - A context is bound to one device and one CUDA stream and is not
 *     thread-safe; separate contexts are independent.  All device memory the
 *     library needs is owned by the context and freed by lspr_destroy.
 */
#ifndef LSPR_H
#define LSPR_H

#include <stdint.h>

#if defined(__GNUC__)
#define LSPR_API __attribute__((visibility("default")))
#else
#define LSPR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LSPR_OK = 0,
    LSPR_E_ARG = 1,            /* invalid argument (null pointer, size, unsupported option) */
    LSPR_E_STATE = 2,          /* call out of order (no mesh, no tree) */
    LSPR_E_CUDA = 3,           /* a CUDA runtime call failed */
    LSPR_E_OOM = 4,            /* device memory exhausted */
    LSPR_E_NOT_CONVERGED = 5,  /* at least one wavelength missed the GMRES tolerance (see stats) */
    LSPR_E_TIMEOUT = 6,        /* a device-side wait exceeded its bound */
    LSPR_E_MESH = 7            /* degenerate or non-finite mesh */
} lspr_status;

typedef struct lspr_ctx lspr_ctx;

/* Matrix-vector product modes (lspr_matvec, lspr_solve_opts.mode). */
enum {
    LSPR_DIRECT_FP64 = 0,  /* all pairs, FP64 arithmetic */
    LSPR_DIRECT_FP32 = 1,  /* all pairs, FP32 arithmetic, FP64 accumulation across tiles */
    LSPR_TREE_FP64 = 2,    /* treecode (needs lspr_tree_build), FP64 */
    LSPR_TREE_FP32 = 3,    /* treecode, FP32 P2P/P2M/M2P, FP64 accumulation and corrections */
    LSPR_DIRECT_FF = 4,    /* all pairs, float-float arithmetic (hi + lo FP32 pair, ~48 bits) */
    LSPR_TREE_FF = 5       /* treecode in float-float arithmetic */
};

/* Quadrature options, Sec. II.C "Integral evaluation" (paper's Tables 1 and 4). */
typedef struct {
    int32_t K;          /* points per far panel: 1, 3 or 4 */
    int32_t K_fine;     /* points per near-singular panel: 19, 25 or 37 */
    int32_t N_k;        /* Gauss-Legendre points per edge for the singular (self) panel, 1..32 */
    double threshold;   /* near-singular iff L_j / |c_i - c_j| >= threshold, L_j = sqrt(2 A_j) */
} lspr_quad_opts;

/* Solver options. */
typedef struct {
    double tol;         /* relative residual ||b - A x|| / ||b|| per wavelength */
    int32_t restart;    /* GMRES restart length m (1..512) */
    int32_t maxiter;    /* total Arnoldi steps per wavelength */
    int32_t mode;       /* matvec mode of the Krylov iteration (LSPR_DIRECT_* / LSPR_TREE_*) */
    int32_t refine;     /* FP32 modes only: 0 plain solve; 1 iterative refinement with the residual
                           in float-float arithmetic; 2 the same with a native FP64 residual */
} lspr_solve_opts;

/* Per-solve statistics; arrays hold B entries and are owned by the caller (may be null). */
typedef struct {
    int32_t *iterations;       /* Arnoldi steps taken per wavelength */
    double *residual;          /* final relative residual per wavelength */
    int32_t *status;           /* LSPR_OK or LSPR_E_NOT_CONVERGED per wavelength */
    double seconds;            /* wall time of the call */
    int64_t matvecs;           /* operator applications (all wavelengths) */
} lspr_solve_stats;

/* Text for a status code (static storage). */
LSPR_API const char *lspr_status_string(int status);

/* Text of the last CUDA or argument error recorded by the context ("" if none);
 * valid until the next call on the context. */
LSPR_API const char *lspr_last_error(lspr_ctx *ctx);

/* Library version string (static storage). */
LSPR_API const char *lspr_version(void);

/* Create a context on CUDA device `device`; all work is queued on `cuda_stream`
 * (a cudaStream_t, or null for the legacy default stream).  *out receives the
 * context.  Errors: LSPR_E_ARG (null out, bad device), LSPR_E_CUDA. */
LSPR_API int lspr_create(lspr_ctx **out, int device, void *cuda_stream);

/* Free every device and host resource of the context.  Null is accepted. */
LSPR_API int lspr_destroy(lspr_ctx *ctx);

/* Upload a triangle mesh and precompute everything that depends only on the
 * geometry and the quadrature (Sec. II.C):
 *   - panel centroids (collocation points), unit outward normals, areas, L = sqrt(2A)
 *   - Gauss-node sources of the far rule (K per panel, weight w_g * A)
 *   - singular self integrals V_ii (semi-analytical: radial part exact, N_k-point
 *     Gauss-Legendre in the angle on each edge), K_ii = 0 on a flat panel
 *   - the near-singular list (L_j/|c_i - c_j| >= threshold) and, per near pair,
 *     the FP64 correction (K_fine rule minus K rule) of V_ij and K_ij
 * verts: [nv][3] doubles; tris: [ntri][3] vertex indices (int32); surf_id: [ntri]
 * surface index in [0, nsurf), 1 <= nsurf <= 16 (may be null when nsurf == 1).
 * Surfaces are closed and disjoint (Eq. integral_eq_lspr_system): surface 0 is the
 * particle whose dipole gives sigma_ext, the others analytes in the same host.
 * on_device = 0: host pointers; 1: device pointers on the context's device.
 * The library copies the data; the caller keeps ownership.  Invalidates any tree.
 * Errors: LSPR_E_ARG (sizes, rules, indices out of range), LSPR_E_MESH
 * (zero-area or non-finite panel), LSPR_E_OOM, LSPR_E_CUDA. */
LSPR_API int lspr_mesh_upload(lspr_ctx *ctx, const double *verts, int64_t nv, const int32_t *tris, int64_t ntri,
                     const int32_t *surf_id, int32_t nsurf, const lspr_quad_opts *q, int32_t on_device);

/* Build the treecode structures of Sec. II.D on the device: Morton keys of the
 * Gauss-node sources and the collocation targets, radix sort, an octree whose
 * leaves hold at most Ncrit sources (or sit at the maximum depth of 10 levels),
 * box centres and radii r_b, and per block of 64 targets the interaction lists:
 * a box is accepted for the Taylor expansion of order P when r_b < theta * r,
 * r the distance from the box centre to the nearest point of the target block's
 * bounding box (and the box is clear of every target's near-singular region);
 * leaves that fail are summed directly.  Supported P: 1..8; theta in (0, 1).
 * Errors: LSPR_E_STATE (no mesh), LSPR_E_ARG, LSPR_E_OOM, LSPR_E_CUDA. */
LSPR_API int lspr_tree_build(lspr_ctx *ctx, double theta, int32_t P, int32_t Ncrit);

/* y[b] = A(s_b) x[b] for b < B, A the block operator of Eq. matrix_lspr:
 *   y_top = phi/2 + K phi - V dphi,   y_bot = phi/2 - K phi + s_b V dphi,
 * with s_b = eps_ratio[b] = eps_in/eps_out (complex).  x, y: [B][2N] complex.
 * Several surfaces (Eq. matrix_multi): for panel i on surface s,
 *   y_top = phi/2 + (K phi)_s - (V dphi)_s,
 *   y_bot = phi/2 - sum_t (K phi)_t + sum_t s_bt (V dphi)_t,
 * (.)_t the layer potential of surface t's panels, eps_ratio [B][nsurf] complex.
 * on_device = 0: x, y, eps_ratio are host pointers; 1: device pointers.  The
 * call is complete (stream synchronised) on return.
 * Errors: LSPR_E_STATE (no mesh; tree mode without a tree), LSPR_E_ARG, LSPR_E_CUDA,
 * LSPR_E_TIMEOUT (a bounded device wait ran out: y is written but incomplete). */
LSPR_API int lspr_matvec(lspr_ctx *ctx, const double *x, double *y, int32_t B, const double *eps_ratio,
                int32_t mode, int32_t on_device);

/* Solve the interface problem for B wavelengths and return the induced dipole
 * and the extinction cross-section of each (host pointers):
 *   eps_in   [B][nsurf] complex  permittivity of every surface per wavelength
 *   eps_out                host permittivity (re, im)
 *   E0       [3]           incident field amplitude (direction = polarisation)
 *   lambda_nm[B]           vacuum wavelengths
 *   dipole_out [B][3] complex, sigma_ext_out [B] (nm^2): caller-allocated.
 * The right-hand side V((eps_out-eps_in)/eps_out dphi_inc/dn), dphi_inc/dn = -E0.n,
 * is formed with the operator of the matvec mode of `o` (FP64 accumulation in every
 * mode); GMRES (right 2x2 block-Jacobi preconditioner; Krylov basis and Gram-Schmidt in
 * float-float, ~48 significant bits, rotations and solution in FP64) runs in
 * that mode, and with o->refine in an FP32 mode the residual of a refinement cycle
 * is formed with the float-float (refine 1) or FP64 (refine 2) operator of the same
 * kind, or, once it is below 1e3 tol ||b||, updated with the FP32 product of the last
 * correction (the update's deviation from the high-precision residual is at most the
 * FP32 operator's relative error times the previous residual); the dipole is
 * p = -eps_out * sum_j A_j (c_j dphi2s/dn_j - phi_j n_j) over the panels and
 * sigma_ext = Im(k^2 e.p / (eps_out |E0|)) / Re k with k = 2 pi sqrt(eps_out) / lambda
 * (E0 = 0 is allowed, e.g. for the response to point charges alone: the dipole is then the
 * result and sigma_ext, a ratio to |E0|, is not finite).  The dipole is taken about the
 * coordinate origin: when point charges give surface 0 a net charge, the exterior field has a
 * monopole part and the dipole moment depends on that choice of origin.
 * Returns LSPR_E_NOT_CONVERGED if any wavelength missed tol (results are still
 * written), LSPR_E_TIMEOUT if a bounded device wait ran out during the solve (results are
 * written but not trustworthy).  st may be null. */
LSPR_API int lspr_solve(lspr_ctx *ctx, const double *eps_in, double eps_out_re, double eps_out_im, const double *E0,
               const double *lambda_nm, int32_t B, const lspr_solve_opts *o, double *dipole_out,
               double *sigma_ext_out, lspr_solve_stats *st);

/* Autotuner of the treecode parameters (theta, P, Ncrit) for the current mesh: every
 * candidate of a fixed grid (P 4..8, theta 0.3..0.6, Ncrit 128/256/512, or the coarse grid) is built and
 * solved for the given wavelengths, its sigma_ext compared with a reference solve
 * (treecode P = 8, theta = 0.3, whose own deviation from the direct FP64 solution is
 * ~2e-6 on the sphere workloads), and the fastest candidate whose largest relative
 * sigma_ext deviation stays within half of target_rel_err is chosen; its tree is left
 * built in the context.  Solve times are CUDA-event times on the context's stream.
 * If no candidate qualifies, the reference parameters are chosen.  Errors as
 * lspr_solve (a candidate whose solve does not converge is skipped). */
typedef struct {
    double target_rel_err;   /* allowed sigma_ext deviation from the FP64 solution, e.g. 1e-4 */
    double tol;              /* GMRES tolerance of the tuning solves */
    int32_t restart;         /* GMRES restart of the tuning solves */
    int32_t mode;            /* tree matvec mode timed (LSPR_TREE_FP32 or LSPR_TREE_FP64) */
    int32_t refine;          /* refinement of the timed solves (as lspr_solve_opts.refine) */
    int32_t grid;            /* 0: the full grid (60 candidates); 1: a coarse grid for large meshes
                                (P 5..7, theta 0.4/0.5, Ncrit 256/512: 12 candidates) */
    int32_t time_rhs;        /* 0: a candidate's cost is the time of its tuning solve; > 0: it is
                                modelled for a batch of time_rhs right-hand sides as
                                (reference Arnoldi steps + 4) x the time of one FP32 product of
                                that many right-hand sides (the faster of the tensor-core P2P and
                                the FP32-pipe P2P when time_rhs >= 2) + the time of one product of
                                the refinement residual's mode */
    int32_t pad_;
} lspr_tune_opts;

typedef struct {
    double theta;            /* chosen parameters */
    int32_t P, Ncrit;
    double rel_err;          /* largest sigma_ext deviation of the choice from the reference */
    double ms;               /* solve time of the choice (all wavelengths) */
    double ref_ms;           /* solve time of the reference parameters */
    int32_t candidates;      /* candidates built and solved */
    int32_t qualified;       /* candidates within the accuracy bound */
    int32_t tensor_cores;    /* the tensor-core mask left set (lspr_set_tensor_cores): with time_rhs,
                                bit 1 is set iff the tensor-core P2P was the faster */
    int32_t iterations;      /* Arnoldi steps of the reference solve (largest over the wavelengths) */
    double product_ms;       /* time_rhs > 0: the chosen candidate's FP32 product time */
    double residual_product_ms;   /* time_rhs > 0: its refinement-residual product time */
} lspr_tune_result;

LSPR_API int lspr_autotune(lspr_ctx *ctx, const double *eps_in, double eps_out_re, double eps_out_im,
                           const double *E0, const double *lambda_nm, int32_t B, const lspr_tune_opts *o,
                           lspr_tune_result *res);

/* Autotuner of the solver's execution for the current tree and a whole batch (the wavelengths
 * that will be solved together): every pair of a GMRES restart length from restarts[0 ..
 * n_restarts) and a P2P path (FP32 pipe; tensor cores, for B >= 2) is timed with one full solve
 * (o->mode, o->tol, o->refine; o->restart is ignored) with CUDA events on the context's stream.
 * The fastest pair whose wavelengths all converge is applied (its tensor-core mask is left set)
 * and returned: *restart, *tensor_cores (the mask) and *ms (its solve time).  The tree and the
 * accuracy are not changed (the restart length and the P2P path move sigma_ext only within the
 * solve tolerance and the FP32-level rounding).  Errors as lspr_solve; LSPR_E_ARG for an empty
 * or out-of-range restart list (1..512). */
LSPR_API int lspr_tune_solver(lspr_ctx *ctx, const double *eps_in, double eps_out_re, double eps_out_im,
                              const double *E0, const double *lambda_nm, int32_t B, const lspr_solve_opts *o,
                              const int32_t *restarts, int32_t n_restarts, int32_t *restart,
                              int32_t *tensor_cores, double *ms);

/* Sizes of the current geometry and tree (any pointer may be null):
 * panels, sources, near pairs (including self), boxes, P2P source-range items,
 * M2P (target block, box) pairs, and the P2P target-source pairs per matvec. */
LSPR_API int lspr_get_info(lspr_ctx *ctx, int64_t *n_panels, int64_t *n_sources, int64_t *n_near, int64_t *n_boxes,
                  int64_t *n_p2p_items, int64_t *n_m2p_pairs, int64_t *n_p2p_pairs);

/* Sizes of the tensor-core work lists of the current tree (0 until the first product of
 * several right-hand sides forms them; any pointer may be null): M2P work units (a group of
 * four consecutive 64-target blocks and a stretch of its box list), (group, box) entries of
 * the groups' united box lists, source entries of the P2P groups' united source ranges, and
 * the P2P pipeline stages (8 sources of one range each) that one unit of right-hand sides
 * takes.  LSPR_E_ARG: null context. */
LSPR_API int lspr_get_tc_info(lspr_ctx *ctx, int64_t *m2p_units, int64_t *m2p_group_boxes,
                              int64_t *p2p_group_sources, int64_t *p2p_stages);

/* Kernel timing on the context's stream while enabled (lspr_set_timing(ctx, 1) clears
 * the counters).  While enabled, the treecode's P2P runs on the context's stream after
 * P2M and M2P instead of beside them on a second stream, so that the events around each
 * launch time that kernel alone.  Milliseconds summed over launches and launch counts, arrays of 16:
 * [0] P2P FP32, [1] M2P FP32, [2] P2M FP32, [3] near correction + block assembly,
 * [4] GMRES vector kernels, [5] tree build, [6] mesh + near precompute, [7] other,
 * [8] P2P FP64, [9] M2P FP64, [10] P2M FP64, [11] source weights,
 * [12] P2P float-float, [13] M2P float-float, [14] P2M float-float, [15] unused.
 * Every timed launch is bracketed by CUDA events on the stream it runs on. */
LSPR_API int lspr_set_timing(lspr_ctx *ctx, int32_t enable);
/* Number of CUDA kernels the context has launched since lspr_create. */
LSPR_API int lspr_launch_count(lspr_ctx *ctx, int64_t *count);
LSPR_API int lspr_get_timing(lspr_ctx *ctx, double *ms, int64_t *launches);
/* Right-hand sides (channel sets: wavelengths x surfaces) summed over the timed launches of the
 * far-field slots ([0]-[2], [8]-[10], [12]-[14]; 0 elsewhere), so that the algorithmic work of
 * the timed launches can be counted exactly.  rhs: array of 16.  LSPR_E_ARG: null pointer. */
LSPR_API int lspr_get_timing_rhs(lspr_ctx *ctx, int64_t *rhs);
/* Work counters of the Arnoldi steps since the context was created (GMRES, Sec. II.D-E), summed
 * over steps and running systems: out[0] = sum of (j + 1), the basis vectors one Gram-Schmidt
 * pass reads at step j; out[1] = system-steps; out[2] = sum of (j + 1) over the system-steps
 * that took the second pass; out[3] = those system-steps.  The basis traffic of the vector
 * kernels follows from them (16 bytes per complex entry).  out: array of 4.  LSPR_E_ARG: null
 * pointer.  The counters are read from the device (the call synchronises the context's
 * stream). */
LSPR_API int lspr_get_arnoldi_stats(lspr_ctx *ctx, int64_t *out);

/* GMRES of lspr_solve runs each Arnoldi cycle as one CUDA graph launch: a graph
 * loop whose body is one Arnoldi step (preconditioner, product, two Gram-Schmidt
 * passes, Givens rotation and stop test on the device), so the host takes part once
 * per restart cycle instead of once per step.  The graph of a configuration (buffer
 * sizes, mode, B, restart) is recorded on first use and reused, also across mesh and
 * tree rebuilds of the same sizes.  lspr_set_graphs(ctx, 0) selects host-driven cycles
 * (the same kernels launched by the host, which reads the loop condition after each
 * step); kernel timing (lspr_set_timing) also uses them, since timing events cannot sit
 * inside a graph loop.  If recording fails the context falls back to host-driven
 * cycles. */
LSPR_API int lspr_set_graphs(lspr_ctx *ctx, int32_t enable);
/* Tensor cores for the FP32 far field of several right-hand sides (B >= 2), as a mask:
 * bit 0 (default on): the M2P contraction on tcgen05 (TF32 operands split into high and low
 * parts, FP32 accumulation in tensor memory; about 2x the FP32-pipe kernel at 16 right-hand
 * sides, 4x at 64); bit 1 (default off; lspr_tune_solver sets it where it pays): the tree P2P
 * on tcgen05 (same split; 2.3x the FP32-pipe kernel at 64 right-hand sides) for products with
 * at least 24 right-hand sides (channel sets) in use, the FP32-pipe P2P below that (inside a
 * solve the count falls as wavelengths converge, and the choice is then made on the device).
 * 0 selects the FP32-pipe kernels of the same sums.  Bits above 1 are ignored.
 * LSPR_E_ARG: null context. */
LSPR_API int lspr_set_tensor_cores(lspr_ctx *ctx, int32_t enable);
/* Bounded waits inside device kernels that ran out since lspr_create (the tensor-core
 * far-field kernels' pipeline barriers, about one second each): a kernel whose wait runs out
 * stops its block, drains its copies and MMAs in flight, frees its tensor memory and counts
 * here; the product it computed is incomplete, and the lspr_matvec, lspr_solve or
 * lspr_autotune call that launched it returns LSPR_E_TIMEOUT (results are still written).
 * Synchronises the context's stream.  LSPR_E_ARG: null pointer. */
LSPR_API int lspr_device_errors(lspr_ctx *ctx, int32_t *count);
/* Check of that failure path inside the real product kernels: while enabled, every launch of a
 * tensor-core far-field kernel first waits, with the pipelines' bounded wait, on a barrier that
 * nothing arrives on; the wait gives up after its limit (about one second) before any copy or
 * MMA is issued, the kernel returns without doing its work, the device error count grows and
 * the call returns LSPR_E_TIMEOUT.  No fault, trap or endless loop is involved, and the context
 * stays usable: disable it and the next product is complete.  Synchronises the context's
 * stream.  LSPR_E_ARG: null context. */
LSPR_API int lspr_selftest_gate_waits(lspr_ctx *ctx, int32_t enable);
/* Point charges inside the surfaces (Eqs. integral_eq_lspr_system, matrix_multi: the interior
 * row of an analyte surface carries (1 / (4 pi eps_t)) sum_k q_k / |r - r_k|, r the collocation
 * point, eps_t the surface's permittivity of each wavelength in lspr_solve).  charges: [nq][4]
 * host doubles (x, y, z in nm, q in the units of the incident field E0 times nm^2, so that both
 * right-hand-side terms are potentials); surf_q: [nq] host int32, the surface holding each
 * charge.  The library copies them; they apply to every later lspr_solve until replaced, and
 * nq = 0 removes them.  A surface index >= the mesh's surface count makes lspr_solve return
 * LSPR_E_ARG.  LSPR_E_ARG: null context, nq < 0, null arrays with nq > 0, negative index. */
LSPR_API int lspr_set_charges(lspr_ctx *ctx, const double *charges, int64_t nq, const int32_t *surf_q);
/* Diagnostic of that failure path: one device thread waits, with the kernels' bounded wait, on
 * a barrier that nothing arrives on.  result[0] = 1 if the wait reported success (a fault of
 * the mechanism), result[1] = the abort flag it raised (1 expected), result[2] = milliseconds
 * it waited (about 1000).  Synchronises the context's stream; the context stays usable.
 * result: 3 int32 on the host.  LSPR_E_ARG: null pointer. */
LSPR_API int lspr_selftest_wait_timeout(lspr_ctx *ctx, int32_t *result);
/* Graph cycles launched and graphs recorded since lspr_create (either pointer may be null). */
LSPR_API int lspr_graph_stats(lspr_ctx *ctx, int64_t *cycles, int64_t *recordings);

/* Allocation-free direct FP32 product y = A(s) x (the LSPR_DIRECT_FP32 product of
 * lspr_matvec for one right-hand side).  The paper has no counterpart: this is a
 * service for callers that must not allocate device memory during the call, such
 * as code embedded in an application whose device memory belongs to another
 * allocator or that has a fixed budget, and latency-critical loops where
 * cudaMalloc/cudaFree would stall (they can synchronise the device).  The call
 * uses no cudaMalloc, cudaFree or allocating library routine: its scratch
 * (source weights and accumulators) is one fixed device array of 1.5 MiB inside
 * the library, which every GPU that loads the library's device code keeps until
 * exit (with lazy module loading the runtime creates it at the first call's
 * address lookup, so that first call may allocate it; later calls do not).
 *   ctx        context with an uploaded mesh of at most 16384 panels and 65536
 *              far-rule sources (larger meshes: LSPR_E_ARG)
 *   x, y       device pointers on the context's device, [2N] complex each
 *   s          eps_in / eps_out (re, im)
 * The work is queued on the context's stream and is not synchronised on return.
 * The first call on a device looks up the array's device address and caches it
 * for that device's primary context (make it before any stream capture; the
 * cache does not survive cudaDeviceReset).  All calls on a device share the array
 * and leave their contents in it; calls that overlap on the GPU race and must be
 * serialised.  A tree build does not change the product (its Morton reordering of
 * the sources and targets is taken into account).
 * Errors: LSPR_E_ARG, LSPR_E_STATE (no mesh, or a mesh of several surfaces), LSPR_E_CUDA. */
LSPR_API int lspr_matvec_direct_fp32_noalloc(lspr_ctx *ctx, const double *x, double *y, double s_re, double s_im);

#ifdef __cplusplus
}
#endif

#endif /* LSPR_H */
