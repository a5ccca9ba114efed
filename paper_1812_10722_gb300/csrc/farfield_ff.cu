// P2M and M2P launches of every compiled Taylor order, float-float arithmetic.
//
// The float-float M2P evaluates the same recurrence as the FP32/FP64 kernels,
//   n |R|^2 a_k + (2n-1) sum_d R_d a_(k-e_d) + (n-1) sum_d a_(k-2e_d) = 0,  a_0 = 1/|R|,
// but rolled: one code path serves every order P <= kMaxP, walking a table of the terms
// (degree-ordered, so the terms of order P are a prefix of the table) and keeping each
// lane's coefficients a_k in shared memory.  Fully unrolled, the float-float recurrence
// is ~10^4 instructions per (target, box) and overflows the instruction cache.
#include "farfield.cuh"

namespace lspr {

namespace {

// right-hand sides per float-float P2P work unit: 95.9 ms per 64-right-hand-side product on the
// 81920-panel sphere's tree (theta 0.4, P 7, Ncrit 512) against 120.6 ms for chunks of 4 and
// 281.6 ms for the two-targets-per-lane kernel with chunks of 2; chunks of 16 spill (162
// registers at 8)
constexpr int kFfP2PChunk = 8;

// one term k of the table: distances u - index(k - e_d) and u - index(k - 2 e_d) to the term's
// own index u (0: absent), and the recurrence weights -(2n-1)/n and -(n-1)/n as float-float pairs
struct FfTerm {
    unsigned char d1[3], d2[3];
    short pad;
    float c1h, c1l, c2h, c2l;
};
struct FfTermTable {
    FfTerm t[n_terms(kMaxP)];
};

constexpr FfTermTable make_ff_terms() {
    FfTermTable tab{};
    constexpr MultiIndex<kMaxP> mi{};
    for (int u = 0; u < n_terms(kMaxP); ++u) {
        for (int d = 0; d < 3; ++d) {
            tab.t[u].d1[d] = (unsigned char)(mi.m1[u][d] >= 0 ? u - mi.m1[u][d] : 0);
            tab.t[u].d2[d] = (unsigned char)(mi.m2[u][d] >= 0 ? u - mi.m2[u][d] : 0);
        }
        const double n = mi.deg[u];
        const double c1 = u ? -(2.0 * n - 1.0) / n : 0.0, c2 = u ? -(n - 1.0) / n : 0.0;
        tab.t[u].c1h = (float)c1;
        tab.t[u].c1l = (float)(c1 - (double)(float)c1);
        tab.t[u].c2h = (float)c2;
        tab.t[u].c2l = (float)(c2 - (double)(float)c2);
    }
    return tab;
}
static_assert(n_terms(kMaxP) - n_terms(kMaxP - 3) <= 255, "term distances must fit the table's bytes");

__constant__ FfTermTable c_ff_terms = make_ff_terms();

// The recurrence of a degree-n term reads terms of degrees n-1 and n-2 only, so each lane keeps
// its coefficients in a ring of W slots (term u in slot u mod W), W = the terms of the three
// highest degrees P-2, P-1, P (85 instead of 120 at P = 7): every term read is among the W
// written last.
__host__ __device__ inline int ff_ring(int P) {
    return P < 2 ? n_terms(P) : n_terms(P) - n_terms(P - 3);
}

// Shared memory of a block: one part (TP terms) of a box's staged moments for its chunk of
// right-hand sides (TP x NB, shared by the block's two warps) and each warp's coefficient ring
// (2 x W x 32)
__host__ __device__ inline size_t ff_m2p_smem(int TP, int W, int NB) {
    return (size_t)TP * NB * sizeof(ff4) + 2 * (size_t)W * 32 * sizeof(ffloat);
}

// Work units and accumulation as in m2p_kernel; NT = n_terms(P) at run time.  A block of two
// warps takes a unit: warp h the targets 32 h .. 32 h + 31 of the 64-target block, both on the
// same boxes, so each box's moments are staged once for the two, in parts of TP terms (the
// launcher picks TP so that more blocks fit per SM).  The recurrence is rolled (each lane's
// coefficients live in its column of the warp's ring), and the contraction accumulates with
// ff_mac.
template <int NB>
__global__ void __launch_bounds__(64)
    m2p_ff_kernel(const int4 *__restrict__ items, int64_t nitems, int nbc, int B, int NT,
                  const ff4 *__restrict__ tgt, int64_t ntgt, const int *__restrict__ list,
                  const ff4 *__restrict__ box_c, const ff4 *__restrict__ mom, double *__restrict__ acc, int *counter,
                  const int *nact, int W, int TP) {
    extern __shared__ __align__(16) unsigned char ff_smem[];
    __shared__ int64_t unit;
    const int h = threadIdx.x >> 5, lane = threadIdx.x & 31;
    ff4 *sm = (ff4 *)ff_smem;
    ffloat *sa = (ffloat *)(sm + TP * NB) + (size_t)h * W * 32;   // sa[(t mod W) * 32 + lane]
    const int Bact = nact ? *nact : B;   // right-hand sides in use (the first Bact slots)
    nbc = (Bact + NB - 1) / NB;
    const int64_t units = nitems * nbc;
    while (true) {
        if (threadIdx.x == 0) unit = atomicAdd(counter, 1);
        __syncthreads();
        const int64_t it = unit;
        __syncthreads();   // every thread has read the unit before thread 0 takes the next one
        if (it >= units) return;
        const int64_t ii = it / nbc;
        const int b0 = (int)(it - ii * nbc) * NB, nb = min(NB, Bact - b0);
        const int4 item = __ldg(items + ii);
        const int64_t ti = (int64_t)item.x * kTargetBlock + lane + 32 * h;
        const ff4 q = ti < ntgt ? tgt[ti] : tgt[0];
        ffloat a[NB][4];
#pragma unroll
        for (int j = 0; j < NB; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) a[j][c] = ffloat(0.f, 0.f);
#pragma unroll 1
        for (int l = item.y; l < item.z; ++l) {
            const int b = __ldg(list + l);
            const ff4 c = box_c[b];
            // terms t0 .. t0 + TP - 1 of the box's moments into sm (the whole block, at the same t)
            auto stage = [&](int t0) {
                __syncthreads();   // the previous part's moments are no longer read
                const int nq = min(TP, NT - t0) * NB;
                for (int q2 = threadIdx.x; q2 < nq; q2 += 64) {
                    const int t = q2 / NB, j = q2 - t * NB;
                    sm[q2] = j < nb ? mom[((int64_t)b * NT + t0 + t) * B + b0 + j] : zero4<ff4>();
                }
                __syncthreads();
            };
            stage(0);
            const ffloat R[3] = {q.x - c.x, q.y - c.y, q.z - c.z};
            const ffloat r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
            const ffloat a0 = rsq(r2);
            const ffloat ir2 = a0 * a0;
            sa[lane] = a0;
            int su = 0;   // slot of term t
            int tpart = 0;   // first term of the staged part
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                const ff4 m = sm[j];
                ff_mac(a[j][0], a0, m.x);
                ff_mac(a[j][1], a0, m.y);
                ff_mac(a[j][2], a0, m.z);
                ff_mac(a[j][3], a0, m.w);
            }
#pragma unroll 1
            for (int t = 1; t < NT; ++t) {
                if (t == tpart + TP) stage(tpart = t);
                const FfTerm &e = c_ff_terms.t[t];
                su = su + 1 == W ? 0 : su + 1;
                ffloat s1(0.f, 0.f), s2(0.f, 0.f);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (e.d1[d]) {
                        const int sl = su - e.d1[d];
                        s1 += R[d] * sa[(sl < 0 ? sl + W : sl) * 32 + lane];
                    }
                    if (e.d2[d]) {
                        const int sl = su - e.d2[d];
                        s2 += sa[(sl < 0 ? sl + W : sl) * 32 + lane];
                    }
                }
                const ffloat at = (ffloat(e.c1h, e.c1l) * s1 + ffloat(e.c2h, e.c2l) * s2) * ir2;
                sa[su * 32 + lane] = at;
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    const ff4 m = sm[(t - tpart) * NB + j];
                    ff_mac(a[j][0], at, m.x);
                    ff_mac(a[j][1], at, m.y);
                    ff_mac(a[j][2], at, m.z);
                    ff_mac(a[j][3], at, m.w);
                }
            }
        }
        if (ti < ntgt) {
            const int64_t tp = panel_of(q.w);
#pragma unroll
            for (int j = 0; j < NB; ++j)
                if (j < nb)
                    atomic_add4(acc + 4 * (tp * B + b0 + j), (double)a[j][0], (double)a[j][1], (double)a[j][2],
                                (double)a[j][3]);
        }
    }
}

template <int NB>
int m2p_ff_launch(lspr_ctx *ctx, double *acc, int *counter, int B) {
    static int occ = 0, occ_nt = -1, tp_sel = 0;
    static int smem_set[kSmemDevices] = {};
    Tree &tr = ctx->tree;
    const int NT = n_terms(tr.P), W = ff_ring(tr.P);
    LSPR_TRY(ctx, allow_smem(m2p_ff_kernel<NB>, (int)ff_m2p_smem(NT, W, NB), ctx->device, smem_set));
    if (occ_nt != NT) {
        // the fewest parts (1 to 3) of a box's moments that give the most resident blocks per SM
        // (P 7, 8 right-hand sides: three parts of 40 terms, 53.8 KB, four blocks instead of three)
        occ = 0;
        tp_sel = NT;
        for (int parts = 1; parts <= 3; ++parts) {
            const int tp = (NT + parts - 1) / parts;
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, m2p_ff_kernel<NB>, 64,
                                                              ff_m2p_smem(tp, W, NB)) != cudaSuccess) {
                (void)cudaGetLastError();
                per_sm = 0;
            }
            if (per_sm > occ) {
                occ = per_sm;
                tp_sel = tp;
            }
        }
        if (occ < 1) {
            occ = 1;
            tp_sel = NT;
        }
        occ_nt = NT;
    }
    const size_t smem = ff_m2p_smem(tp_sel, W, NB);
    const int nbc = (B + NB - 1) / NB;
    const unsigned grid =
        (unsigned)std::min<int64_t>(tr.n_m2p_items * nbc, (int64_t)occ * std::max(1, ctx->num_sms));
    m2p_ff_kernel<NB><<<grid, 64, smem, ctx->stream>>>(
        tr.m2p_items.p, tr.n_m2p_items, nbc, B, NT, Views<ffloat>::tgt(ctx), ctx->mesh.N, tr.m2p_list.p,
        Views<ffloat>::bc(ctx), Views<ffloat>::mom(ctx), acc, counter, ctx->rhs_nact, W, tp_sel);
    return LSPR_OK;
}

// Float-float P2P of several right-hand sides, one target per lane: a warp takes (item, half
// of its 64-target block, chunk of NB right-hand sides), so G and dG/dn of a pair (~170 FP32
// instructions in float-float) serve NB right-hand sides (4 ff_mac each) instead of the two of
// the two-targets-per-lane kernel.  Sources are staged per warp in chunks of 32 and read by
// broadcast; sums and the own-panel rule are those of p2p_kernel.
constexpr int kFfP2PWarps = 4;
template <int NB>
__global__ void __launch_bounds__(kFfP2PWarps * 32)
    p2p_ff1_kernel(const int4 *__restrict__ items, int64_t nitems, int B, const ff4 *__restrict__ tgt, int64_t ntgt,
                   const ff4 *__restrict__ spos, const ff4 *__restrict__ snrm, const ff4 *__restrict__ sw,
                   double *__restrict__ acc, int *counter, const int *nact) {
    __shared__ ff4 sh[kFfP2PWarps][2][32];
    __shared__ ff4 shw[kFfP2PWarps][32][NB];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Bact = nact ? *nact : B;
    const int nbc = (Bact + NB - 1) / NB;
    const int64_t units = nitems * 2 * nbc;
    while (true) {
        int v = 0;
        if (lane == 0) v = atomicAdd(counter, 1);
        const int64_t it = __shfl_sync(0xffffffffu, v, 0);
        if (it >= units) return;
        const int64_t ii = it / (2 * nbc);
        const int rem = (int)(it - ii * 2 * nbc), h = rem / nbc;
        const int b0 = (rem - h * nbc) * NB, nb = min(NB, Bact - b0);
        const int4 item = __ldg(items + ii);
        const int64_t t = (int64_t)item.x * kTargetBlock + 32 * h + lane;
        const ff4 q = t < ntgt ? tgt[t] : tgt[0];
        const int tp = panel_of(q.w);
        ffloat a[NB][4];
#pragma unroll
        for (int k = 0; k < NB; ++k)
#pragma unroll
            for (int c = 0; c < 4; ++c) a[k][c] = ffloat(0.f, 0.f);
        for (int base = item.y; base < item.z; base += 32) {
            const int s = base + lane;
            if (s < item.z) {
                sh[warp][0][lane] = spos[s];
                sh[warp][1][lane] = snrm[s];
#pragma unroll
                for (int k = 0; k < NB; ++k) shw[warp][lane][k] = k < nb ? sw[(int64_t)s * B + b0 + k] : zero4<ff4>();
            }
            __syncwarp();
            const int cnt = min(32, item.z - base);
#pragma unroll 2
            for (int kk = 0; kk < cnt; ++kk) {
                const ff4 p = sh[warp][0][kk], n = sh[warp][1][kk];
                const ffloat dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
                ffloat r = rsq(dx * dx + dy * dy + dz * dz);
                if (item.w && panel_of(n.w) == tp) r = ffloat(0.f, 0.f);
                const ffloat tk = (dx * n.x + dy * n.y + dz * n.z) * (r * r) * r;
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    const ff4 w = shw[warp][kk][k];
                    ff_mac(a[k][0], r, w.x);
                    ff_mac(a[k][1], r, w.y);
                    ff_mac(a[k][2], tk, w.z);
                    ff_mac(a[k][3], tk, w.w);
                }
            }
            __syncwarp();
        }
        if (t < ntgt) {
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (k < nb)
                    atomic_add4(acc + 4 * ((int64_t)tp * B + b0 + k), (double)a[k][0], (double)a[k][1],
                                (double)a[k][2], (double)a[k][3]);
        }
    }
}

template <int NB>
int p2p_ff1_launch(lspr_ctx *ctx, const int4 *items, int64_t nitems, int B, double *acc, cudaStream_t st,
                   int *counter) {
    static int occ = 0;
    const int nbc = (B + NB - 1) / NB;
    const unsigned grid = std::min<unsigned>(grid_for(nitems * 2 * nbc, kFfP2PWarps),
                                             persistent_grid(ctx, p2p_ff1_kernel<NB>, kFfP2PWarps * 32, &occ));
    p2p_ff1_kernel<NB><<<grid, kFfP2PWarps * 32, 0, st>>>(items, nitems, B, Views<ffloat>::tgt(ctx), ctx->mesh.N,
                                                          Views<ffloat>::spos(ctx), Views<ffloat>::snrm(ctx),
                                                          Views<ffloat>::w(ctx), acc, counter, ctx->rhs_nact);
    return LSPR_OK;
}

}  // namespace

int p2p_ff_multi(lspr_ctx *ctx, const int4 *items, int64_t nitems, int B, double *acc, cudaStream_t st, int *counter) {
    return p2p_ff1_launch<kFfP2PChunk>(ctx, items, nitems, B, acc, st, counter);
}

int p2m_orders_ff(lspr_ctx *ctx, int B) {
    LSPR_DISPATCH_P(p2m_launch, ffloat, B, ctx, B);
    return LSPR_OK;
}

int m2p_orders_ff(lspr_ctx *ctx, double *acc, int *counter, int B) {
    if (ctx->tree.P < 1 || ctx->tree.P > kMaxP) return LSPR_E_ARG;
    // chunks of 8 right-hand sides: the recurrence is shared by more of them (24.8 / 29.5 / 28.5 ms
    // for chunks of 8 / 4 / 16 at 16 right-hand sides, 20480 panels, P = 7)
    return B == 1 ? m2p_ff_launch<1>(ctx, acc, counter, B) : m2p_ff_launch<8>(ctx, acc, counter, B);
}

}  // namespace lspr
