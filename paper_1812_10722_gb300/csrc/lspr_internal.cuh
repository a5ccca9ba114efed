// Internal declarations of the sm_103a LSPR boundary-element library.
// Layout of device data (all owned by one lspr_ctx):
//   panels    FP64 structure-of-arrays in input order (centroid, normal, area, L, V_ii)
//   sources   Gauss nodes of the far rule, "work order" (input order until a tree
//             is built, Morton order afterwards): position+weight (x,y,z,w_g*A),
//             normal (nx,ny,nz,panel id as int bits) in FP64 and FP32 copies
//   targets   collocation points in work order (x,y,z,panel id as int bits)
//   near CSR  per panel row: the self entry first, then every near-singular panel,
//             with FP64 corrections dV, dK (fine rule minus far rule; self: V_ii, 0)
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ffloat.cuh"
#include "lspr.h"

// 32-byte aligned four-double vector (CUDA's double4 is deprecated)
struct __align__(32) dbl4 {
    double x, y, z, w;
};
__host__ __device__ inline dbl4 make_dbl4(double x, double y, double z, double w) { return dbl4{x, y, z, w}; }

namespace lspr {

// arithmetic of the far-field kernels
enum Prec { PREC_F32 = 0, PREC_F64 = 1, PREC_FF = 2 };
inline int mode_prec(int mode) {
    return (mode == LSPR_DIRECT_FP64 || mode == LSPR_TREE_FP64) ? PREC_F64
           : (mode == LSPR_DIRECT_FF || mode == LSPR_TREE_FF)   ? PREC_FF
                                                                : PREC_F32;
}
inline bool mode_tree(int mode) { return mode == LSPR_TREE_FP64 || mode == LSPR_TREE_FP32 || mode == LSPR_TREE_FF; }

constexpr double kInv4Pi = 0.079577471545947667884;   // 1 / (4 pi)
constexpr int kTargetBlock = 64;                       // targets per interaction block (2 per lane)
constexpr int kTcGroup = 4;        // target blocks per tensor-core M2P group (256 targets)
constexpr int kTcGroupSeg = 32;    // boxes per tensor-core M2P work unit at most
constexpr int kTcP2PSrc = 2048;    // sources per tensor-core P2P work unit at most
constexpr int kMaxP = 8;                               // highest Taylor order compiled
constexpr int kMaxDepth = 10;                          // octree levels below the root (10 bits per axis)
constexpr int kMaxNk = 32;
constexpr int kMaxSurfaces = 16;                       // particle + analyte surfaces

// number of multi-indices with |k| <= P
__host__ __device__ constexpr int n_terms(int P) { return (P + 1) * (P + 2) * (P + 3) / 6; }

// ---------------------------------------------------------------- device arrays
// Counts device allocations made through DArr: captured CUDA graphs embed buffer
// addresses and are re-recorded when this number has changed since their recording.
inline std::atomic<uint64_t> g_alloc_generation{0};

template <class T>
struct DArr {
    T *p = nullptr;
    size_t n = 0;      // elements allocated
    DArr() = default;
    DArr(const DArr &) = delete;
    DArr &operator=(const DArr &) = delete;
    ~DArr() { release(); }
    cudaError_t ensure(size_t count) {
        if (count <= n && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        size_t c = count ? count : 1;
        cudaError_t e = cudaMalloc((void **)&p, c * sizeof(T));
        if (e == cudaSuccess) n = c;
        ++g_alloc_generation;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

// Typed view of a context-owned scratch buffer: the temporaries of the mesh and tree
// builds reuse device memory from call to call instead of allocating and freeing it
// (cudaFree synchronises the device).  Temporaries that are live at the same time use
// different slots.
template <class T>
struct Tmp {
    DArr<unsigned char> *buf;
    T *p = nullptr;
    size_t n = 0;
    explicit Tmp(DArr<unsigned char> &b) : buf(&b) {}
    cudaError_t ensure(size_t count) {
        const cudaError_t e = buf->ensure((count ? count : 1) * sizeof(T));
        if (e == cudaSuccess) {
            p = (T *)buf->p;
            n = count;
        }
        return e;
    }
};
constexpr int kScratchSlots = 16;

struct Mesh {
    bool ready = false;
    int64_t N = 0, nv = 0, Ns = 0;
    int K = 4, Kf = 19, Nk = 9;
    double thr = 0.5;
    double Lmax = 0, rho_max = 0;         // largest L and largest centroid-to-node distance
    DArr<double> verts;                   // [nv*3]
    DArr<int> tris;                       // [N*3]
    DArr<double> cx, cy, cz, nx, ny, nz, area, L, Vself;   // [N]
    int S = 1;                            // surfaces (surface 0: the particle)
    DArr<int> surf;                       // [N] surface of each panel
    // natural-order sources (s = K*i + g) and targets (i)
    DArr<dbl4> src_pos64, src_nrm64;
    DArr<dbl4> tgt64;
    // near CSR
    DArr<int64_t> near_ptr;               // [N+1]
    DArr<int> near_col;                   // [nnz]
    DArr<double> near_dV, near_dK;        // [nnz]
    DArr<float2> near_f32;                // [nnz] (dV, dK) in FP32, for FP32 products
    int64_t nnz = 0;
};

struct WorkOrder {   // sources/targets in the order the far-field kernels walk them
    DArr<dbl4> spos64, snrm64;
    DArr<float4> spos32, snrm32;
    DArr<dbl4> tgt64;
    DArr<float4> tgt32;
    DArr<int> src_panel;   // [Ns]
    DArr<int> tgt_panel;   // [N]
    DArr<ff4> spos_ff, snrm_ff, tgt_ff;   // float-float copies
    DArr<int> tgt_pos;     // [N] work-order position of each panel's target
    DArr<int> src_tblock;  // [Ns] target block holding the source's own panel
};

struct Tree {
    bool ready = false;
    double theta = 0.5;
    int P = 6, Ncrit = 300, NT = 84;
    int64_t nboxes = 0, ntblocks = 0;
    int64_t n_p2p_items = 0, n_m2p_items = 0, n_m2p_pairs = 0, n_p2m_items = 0;
    int64_t p2p_pairs = 0;
    // boxes
    DArr<int> box_beg, box_end, box_child, box_nchild, box_level, box_used;
    DArr<unsigned> box_key;
    DArr<dbl4> box_c64;   // centre (x,y,z), radius r_b
    DArr<float4> box_c32;
    // lists
    DArr<int4> p2p_items;    // (target block, source begin, source end, 0)
    DArr<int4> m2p_items;    // (target block, list begin, list end, 0)
    DArr<int> m2p_list;      // box ids
    // the M2P lists of groups of kTcGroup consecutive target blocks (tensor-core M2P): the
    // union of the blocks' lists, sorted by box, with a mask of the blocks that accepted each
    // box, cut into segments
    DArr<int4> tc_items;     // (group, list begin, list end, 0)
    DArr<int2> tc_list;      // (box id, block mask)
    int64_t n_tc_items = 0, n_tc_pairs = 0;
    // the P2P source ranges of the same groups (tensor-core P2P): the union of the blocks'
    // ranges cut at every range end, each piece with the mask of the blocks that sum it
    DArr<int4> tcp_items;    // (group, interval begin, interval end, 0)
    DArr<int4> tcp_ivl;      // (source begin, source end, block mask, 0)
    int64_t n_tcp_items = 0, n_tcp_ivl = 0, n_tcp_sources = 0, n_tcp_stages = 0;   // stages of 8 sources
    bool tc_built = false, tcp_built = false;   // the group lists above match the tree
    DArr<int4> p2m_items;    // (leaf, source begin, source end, 0): leaves under an accepted box
    DArr<int> box_parent;    // parent box (-1 for the root)
    // moments [box][NT] x (Vre, Vim, Kre, Kim)
    DArr<float4> mom32;
    DArr<dbl4> mom64;        // FP64 moments; also the accumulation buffer of the float-float ones
    DArr<ff4> mom_ff, box_c_ff;
};

struct DirectItems {
    int64_t n = 0;
    DArr<int4> items;
};

// An instantiated Arnoldi-cycle graph and what it was recorded for
struct GraphCache {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t key[24] = {0};
    uint64_t use = 0;        // last use, for replacement
    int64_t per_step = 0;    // kernels launched per Arnoldi step (body of the loop)
    int64_t outer = 0;       // kernels launched once per cycle
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        use = 0;
    }
    ~GraphCache() { reset(); }
};

// device state of the Arnoldi cycles of B systems with restart length m
struct ArnoldiBufs {
    DArr<double2> h;        // [B][m+1]  coefficients of one Gram-Schmidt pass
    DArr<double2> hcol;     // [B][m+1]  Hessenberg column being built
    DArr<double2> part;     // [B][m+1][chunks] partial inner products
    DArr<double> npart;     // [B][blocks] partial squared norms
    DArr<double> nrm;       // [B] norm of the new basis vector / of the residual
    DArr<double> npart0;    // [B][chunks] partial squared norms of A z before orthogonalisation
    DArr<double> nrm0;      // [B] ||A z|| before orthogonalisation
    DArr<int> reorth;       // [B] 1: the step takes the second Gram-Schmidt pass
    DArr<double2> H;        // [B][m+1][m] rotated Hessenberg matrix (R)
    DArr<double> cs;        // [B][m] Givens cosines
    DArr<double2> sn;       // [B][m] Givens sines
    DArr<double2> g;        // [B][m+1] rotated right-hand side beta e_1
    DArr<double2> y;        // [B][m] update coefficients
    DArr<double> res;       // [B] residual estimate |g_{j+1}|
    DArr<double> bn;        // [B] reference norm of the relative residual
    DArr<double> par;       // [2] tolerance, iteration limit
    DArr<unsigned> tick;    // [2B] last-block tickets
    DArr<int> ctl;          // [1 + 3B] current column j, active[B], jb[B], iters[B]
    DArr<int> rmap;         // [2B + 2] running systems packed first: slot -> b, b -> slot, count, sets
    DArr<float4> hff;       // [B][m+1]  h in float-float (re.hi, im.hi, re.lo, im.lo)
    DArr<float4> yff;       // [B][m]    update coefficients in float-float
    DArr<float2> ninv;      // [B] 1 / ||w|| in float-float
    DArr<double> vinv;      // [N] 1 / V_ii (preconditioner)
    DArr<double2> pq;       // [B][S] 1 / (1 + s) (preconditioner)
    DArr<int> go;           // host-driven cycles: the loop condition
    DArr<unsigned long long> stats;   // [4] work counters (lspr_get_arnoldi_stats)
};

constexpr int kTimerSlots = 16;

struct Timing {
    bool enabled = false;
    double ms[kTimerSlots] = {0};
    int64_t launches[kTimerSlots] = {0};
    int64_t rhs[kTimerSlots] = {0};    // right-hand sides (channel sets) summed over the launches
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    size_t used = 0;
};

enum TimerSlot {
    T_P2P = 0, T_M2P = 1, T_P2M = 2, T_NEAR = 3, T_GMRES = 4, T_TREE = 5, T_MESH = 6, T_OTHER = 7,
    T_P2P64 = 8, T_M2P64 = 9, T_P2M64 = 10, T_WEIGHTS = 11, T_P2PFF = 12, T_M2PFF = 13, T_P2MFF = 14
};

}  // namespace lspr

struct lspr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;       // second stream: P2P overlaps P2M -> M2P
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    lspr::DArr<int> counters;          // work-item counters of the persistent kernels
    int num_sms = 0;
    lspr::Mesh mesh;
    lspr::WorkOrder wo;
    lspr::Tree tree;
    lspr::DirectItems direct;
    lspr::Timing timing;
    // per-matvec scratch
    lspr::DArr<double> acc;            // [B][N][4]: V re/im, K re/im (far part)
    lspr::DArr<float4> w32;            // [Ns] source weights
    lspr::DArr<dbl4> w64;
    lspr::DArr<ff4> w_ff;
    lspr::DArr<double2> xbuf, ybuf;    // staging for host matvec
    lspr::DArr<double2> xt;            // [2N][B] transposed right-hand sides of a product
    lspr::DArr<float2> xtf;            // [2N][B] the same in FP32 (FP32 products)
    lspr::DArr<double2> sbuf;
    // solver scratch
    lspr::DArr<float4> gm_V;   // Krylov basis, float-float complex entries
    lspr::DArr<double2> gm_w, gm_z, gm_x, gm_b, gm_r;
    lspr::DArr<double> gm_bnorm, gm_dpart;
    lspr::DArr<double2> gm_s, gm_vinc, gm_eps;
    lspr::DArr<double> gm_out;         // dipole + sigma results
    lspr::DArr<double2> gm_dx;         // refinement correction
    lspr::DArr<int> gm_rmap;           // [2B + 2] systems of a refinement product (packing map)
    lspr::DArr<double> gm_dippart, gm_lambda;
    lspr::DArr<unsigned char> scratch[lspr::kScratchSlots];   // see lspr::Tmp
    // device-driven Arnoldi cycles (a CUDA graph per configuration, gmres_graph.cu)
    bool use_graphs = true;
    int tensor_cores = 1;              // tcgen05 for B >= 2 in FP32: bit 0 M2P, bit 1 P2P
    int tc_p2p_min_rhs = 24;           // the tensor-core P2P takes products of at least this many
                                       // right-hand sides in use; fewer take the FP32-pipe P2P
    lspr::DArr<unsigned char> tc_img;  // split moments in tensor-core operand layout
    lspr::DArr<int> dev_err;           // [0] bounded device waits that ran out (never reset);
                                       // [1] failure-path check: tensor-core kernels give up at once
    int dev_err_seen = 0;              // [0] as last reported by a status (LSPR_E_TIMEOUT)
    // point charges inside the surfaces (lspr_set_charges): (x, y, z, q) and the surface of each
    lspr::DArr<dbl4> charges;
    lspr::DArr<int> charge_surf;
    int64_t nq = 0;
    int max_charge_surf = -1;
    lspr::DArr<double> coul;           // [N] sum_k q_k / |c_i - r_k| over the charges of i's surface
    cudaStream_t gstream = nullptr;    // private recording/launch stream
    cudaEvent_t ev_g0 = nullptr, ev_g1 = nullptr;
    lspr::GraphCache gcache[2];
    lspr::ArnoldiBufs arn;
    // right-hand sides in use while recording an Arnoldi step (null: all B): slot -> system
    // map, system -> slot map (-1: converged), and the number of channel sets in use (running
    // systems x surfaces); the far-field kernels work on the first *rhs_nact sets only
    const int *rhs_map = nullptr, *rhs_inv = nullptr, *rhs_nact = nullptr;
    int timing_sets = -1;   // host copy of *rhs_nact for the per-launch work count of timing
    int64_t graph_cycles = 0, graph_recordings = 0;
    // last error text
    std::string last_error;
    int64_t matvec_count = 0;
    int64_t n_launches = 0;            // kernels launched by this context
};

namespace lspr {

// -------------------------------------------------------------- error helpers
int cuda_status(lspr_ctx *ctx, cudaError_t e, const char *what);
// LSPR_E_TIMEOUT in place of rc (LSPR_OK or LSPR_E_NOT_CONVERGED) when a bounded device wait ran
// out since the last status that reported one; call with the context's stream synchronised
int timeout_status(lspr_ctx *ctx, int rc);
#define LSPR_TRY(ctx, expr)                                              \
    do {                                                                 \
        cudaError_t e__ = (expr);                                        \
        if (e__ != cudaSuccess) return ::lspr::cuda_status(ctx, e__, #expr); \
    } while (0)
#define LSPR_TRY_ST(expr)             \
    do {                              \
        int s__ = (expr);             \
        if (s__ != LSPR_OK) return s__; \
    } while (0)

// timing helpers (no-ops unless enabled)
void timer_begin(lspr_ctx *ctx, int slot, cudaEvent_t *ev);
void timer_end(lspr_ctx *ctx, int slot, cudaEvent_t ev);
void timer_begin_on(lspr_ctx *ctx, int slot, cudaEvent_t *ev, cudaStream_t st);
void timer_end_on(lspr_ctx *ctx, int slot, cudaEvent_t ev, cudaStream_t st);
void timer_collect(lspr_ctx *ctx);
// channel sets a timed far-field launch works on: the packed count when the host knows it
// (timing_sets >= 0: host-driven Arnoldi steps and refinement products), else all B
inline void timer_rhs(lspr_ctx *ctx, int slot, int64_t B) {
    if (ctx->timing.enabled) ctx->timing.rhs[slot] += ctx->timing_sets >= 0 ? std::min<int64_t>(ctx->timing_sets, B) : B;
}

inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

// ------------------------------------------------------------ mesh.cu
// surf: [ntri] surface index of each panel in [0, nsurf) (null: one surface)
int mesh_build(lspr_ctx *ctx, const double *verts, int64_t nv, const int *tris, int64_t ntri, const int *surf,
               int nsurf, int on_device,
               const lspr_quad_opts &q);
// natural-order work arrays (direct mode)
int workorder_natural(lspr_ctx *ctx);

// ------------------------------------------------------------ tree.cu
// A kernel's dynamic shared memory above 48 KB is opted into on every device it runs on:
// set[d] holds the size already allowed on device d (devices past the table set it each call).
constexpr int kSmemDevices = 64;
template <class K>
inline cudaError_t allow_smem(K kernel, int bytes, int device, int *set) {
    const bool tracked = device >= 0 && device < kSmemDevices;
    if (tracked && set[device] >= bytes) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && tracked) set[device] = bytes;
    return e;
}

int tree_build(lspr_ctx *ctx, double theta, int P, int Ncrit);
int tree_tc_lists(lspr_ctx *ctx, bool p2p);
int selftest_wait_timeout(lspr_ctx *ctx, int32_t *result);
// stable LSD radix sort of (keys, vals) on the context's stream (bits: key width)
int radix_sort(lspr_ctx *ctx, unsigned *keys, int *vals, unsigned *ktmp, int *vals_tmp, int64_t n, int bits, int *hist,
               int *offs);
int64_t radix_sort_scratch_ints(int64_t n);   // ints needed by each of hist and offs
// 10-bit coordinate -> every third bit (Morton interleave helper)
__device__ __forceinline__ unsigned spread10(unsigned v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// ------------------------------------------------------------ farfield.cu
// accumulate far parts (coarse rule everywhere except own panel) into acc[N][4]
// B right-hand sides: weights [source][B], accumulators acc [panel][B][4]
int launch_p2p(lspr_ctx *ctx, int prec, const int4 *items, int64_t nitems, double *acc, cudaStream_t st,
               int *counter, int B);
int launch_p2m(lspr_ctx *ctx, int prec, int B);
int launch_m2p(lspr_ctx *ctx, int prec, double *acc, int *counter, int B);
// float-float copies of the work-order geometry / box centres
int launch_ff_geometry(lspr_ctx *ctx);
int launch_ff_boxes(lspr_ctx *ctx);
// item.w = 1 where a P2P item may contain sources of its own target block's panels
int launch_item_flags(lspr_ctx *ctx, int4 *items, int64_t nitems);
// xt: x transposed to [2N][B] (B > 1), or null
// S > 1 surfaces: B x S channel sets, weights of set (b, t) masked to the sources of surface t
// x [B][2N]; xt: its transposed FP64 copy [2N][B] or null; xtf: its transposed FP32 copy
// (FP32 products of several right-hand sides) or null
int launch_weights(lspr_ctx *ctx, int prec, const double2 *x, const double2 *xt, int64_t N, int B, int S,
                   const float2 *xtf = nullptr);
int launch_weights_fp32_raw(cudaStream_t st, int64_t Ns, int64_t N, const dbl4 *spos64, const int *src_panel,
                            const double2 *x, float4 *w);
int launch_p2p_fp32_raw(cudaStream_t st, const int4 *items, int64_t nitems, const float4 *tgt, int64_t ntgt,
                        const float4 *spos, const float4 *snrm, const float4 *w, double *acc);

// ------------------------------------------------------------ solve.cu
// y = A(s) x for one right-hand side, x and y device [2N] complex
int apply_operator(lspr_ctx *ctx, int mode, const double2 *x, double2 *y, const double2 *s, int B);
// layer potentials without the block assembly: out[i] = (V dphi)_i, (K phi)_i
// per source surface t (S of them): Vd[t * N + i] = (V dphi)_t, Kp[t * N + i] = (K phi)_t
int layer_potentials(lspr_ctx *ctx, int mode, const double2 *x, double2 *Vd, double2 *Kp);
int solve_impl(lspr_ctx *ctx, const double *eps_in, double eps_out_re, double eps_out_im, const double *E0,
               const double *lambda_nm, int B, const lspr_solve_opts &o, double *dipole_out, double *sigma_out,
               lspr_solve_stats *st);

// ------------------------------------------------------------ gmres_graph.cu
constexpr int kMaxRestart = 512;   // longest Arnoldi cycle (restart length m)
// Restarted GMRES(m) for B systems A(s_b) x_b = b_b whose Arnoldi cycles each run as one
// CUDA graph launch (a device-side loop over the steps), or host-driven launches of the
// same kernels without graphs or with per-kernel timing.  x_zero: x holds zeros on entry
// (the first residual is b without a matrix-vector product).  trust_estimate: return
// after a cycle whose recurrence residual estimates meet tol, without the explicit
// residual (for inner solves whose caller forms the residual itself).  iters/relres
// receive the steps taken and the last relative residual (explicit or estimated) per
// system.
int gmres_graph_solve(lspr_ctx *ctx, int mode, int B, int m, int maxiter, double tol, const double2 *s_d,
                      const double2 *b_d, double2 *x_d, bool x_zero, bool trust_estimate, std::vector<int> &iters,
                      std::vector<double> &relres, const std::vector<double> &bnorm);

}  // namespace lspr
