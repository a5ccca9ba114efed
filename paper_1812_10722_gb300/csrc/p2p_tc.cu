// P2P of several right-hand sides on the fifth-generation tensor cores (tcgen05).
//
// The direct far-rule sum of a target x over sources y_s with weights w_s (per right-hand
// side: V re, V im from the single layer, K re, K im from the double layer),
//   D[4 j + c][x] += G(x, y_s) w_s[j].c (c = 0, 1),  dG/dn(x, y_s) w_s[j].c (c = 2, 3),
// is a matrix product once the kernel values are laid out as an operand: K = 16 per stage,
// columns 0..7 hold G of eight sources and columns 8..15 their dG/dn; A (the weights) has the
// V channels in columns 0..7 and the K channels in columns 8..15 (the other half is zero), B
// (the kernel tile, generated in registers by one thread per target) has the 256 targets of a
// group of four target blocks as N.  The group walks the union of its blocks' P2P source
// ranges; a target whose block does not sum a range gets zero kernel values there, and a
// target's own panel is skipped (its exact integral is in the near correction), as in
// p2p_kernel.  Operands are split into TF32 high and low parts: with 16 right-hand sides the
// high and low weights are the two halves of one 128-row operand (two MMAs per K step give
// all four products, the epilogue adds both halves), with 32 the three 3xTF32 products.
//
// Roles (persistent, one CTA per SM): warps 0-7 generate both operands of every stage and
// drain each unit's accumulator behind the next unit's first stage; warp 8 (one lane) fetches
// work units into a small ring; warp 9 (one lane) issues the MMAs into one of two 256-column
// TMEM accumulators.  Every wait is bounded as in the tensor-core M2P.
//
// Opt-in (lspr_set_tensor_cores bit 1): on this GPU the generation of the kernel tile (one
// thread per target, 8 warps) bounds it, and a group's union of source ranges holds about
// 1.7x the pairs of its blocks' own lists, so at 16 right-hand sides it is slower than
// p2p_kernel (1.40 ms against 0.94 ms per product on the 20480-panel sphere).
#include "farfield.cuh"
#include "tcgen05.cuh"

namespace lspr {

namespace {

using namespace tc;

constexpr int kSrc = 8;                        // sources per stage
constexpr int kKC = 2 * kSrc;                  // K per stage: G then dG/dn of the sources
constexpr int kTcN = kTcGroup * kTargetBlock;  // targets per work unit (the MMA's N)
constexpr int kChunkSBO = (kKC / 4) * 128;     // bytes per 8-row group of a stage operand
constexpr int kGenWarps = kTcN / 32;           // one thread per target
constexpr int kProdWarp = kGenWarps, kMmaWarp = kGenWarps + 1;
constexpr int kTcThreads = 32 * (kGenWarps + 2);
constexpr int kUnitRing = 4;
constexpr int kRingConsumers = kGenWarps + 1;  // lane 0 of each consumer warp
constexpr uint32_t kTmemCols = 2 * kTcN;       // two accumulators
static_assert(kTmemCols <= 512 && kTcN <= 256, "one MMA spans the group");

template <int RC>
struct P2PShape {
    static constexpr int ROWS = 4 * RC;
    static constexpr bool STACKED = ROWS == 64;           // hi and lo weights as one operand
    static constexpr uint32_t IDESC = idesc_tf32(128, kTcN);
    static constexpr int A_CH = (ROWS / 8) * kChunkSBO;   // one split part of the weights
    static constexpr int B_CH = (kTcN / 8) * kChunkSBO;   // one split part of the kernel tile
    static constexpr int STAGE = 2 * A_CH + 2 * B_CH;     // A_hi | A_lo | B_hi | B_lo
    static constexpr int NS = (200 * 1024) / STAGE;
    static constexpr int SMEM = NS * STAGE;
    static_assert(ROWS == 64 || ROWS == 128, "unit of 16 or 32 right-hand sides");
    static_assert(kSrc * RC <= kTcN, "one weight per generating thread");
};

__device__ __forceinline__ int core_off(int r, int k) {
    return (r >> 3) * kChunkSBO + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ float4 f4_hi(const float4 v) {
    return make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
}
__device__ __forceinline__ float4 f4_sub(const float4 a, const float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}

template <int RC>
__global__ void __launch_bounds__(kTcThreads, 1)
    p2p_tc_kernel(const int4 *__restrict__ items, int64_t nitems, const int4 *__restrict__ ivl, int B,
                  const float4 *__restrict__ tgt, int64_t ntgt, const float4 *__restrict__ spos,
                  const float4 *__restrict__ snrm, const float4 *__restrict__ sw, double *__restrict__ acc,
                  int *counter, int *error, const int *nact) {
    using S = P2PShape<RC>;
    constexpr int NS = S::NS;
    extern __shared__ __align__(128) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t full_s[NS], empty_s[NS];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], ring_full[kUnitRing], ring_empty[kUnitRing], drain, gate;
    __shared__ int64_t ring[kUnitRing];
    __shared__ uint32_t tslot;
    __shared__ volatile int abort_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = smem_addr(tc_smem);
    // the weight operand's structural zeros (V rows in the dG/dn columns, K rows in the G
    // columns) are never written afterwards
    for (int i = tid; i < S::SMEM / 16; i += kTcThreads) ((float4 *)tc_smem)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            bar_init(smem_addr(&full_s[s]), kTcN);   // one arrival per generating thread
            bar_init(smem_addr(&empty_s[s]), 1);     // the MMAs' commit
        }
        for (int a = 0; a < 2; ++a) {
            bar_init(smem_addr(&acc_full[a]), 1);
            bar_init(smem_addr(&acc_empty[a]), kGenWarps);
        }
        for (int r = 0; r < kUnitRing; ++r) {
            bar_init(smem_addr(&ring_full[r]), 1);
            bar_init(smem_addr(&ring_empty[r]), kRingConsumers);
        }
        bar_init(smem_addr(&drain), 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // failure-path check (error[1] set by the host): a bounded wait on a barrier that nothing
        // arrives on runs out before any copy or MMA is issued, and the block returns without work
        if (__ldcg(error + 1)) {
            bar_init(smem_addr(&gate), 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            bar_wait(smem_addr(&gate), 0u, &abort_s);   // phase 0 never completes: no arrival
        }
    }
    if (warp == 0) {
        __syncwarp();   // lane 0 may come from the set-up above (and its bounded check wait)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tslot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tslot;
    const int Bact = nact ? *nact : B;   // right-hand sides in use (the first Bact slots)
    const int nbc = (Bact + RC - 1) / RC;
    const int64_t units = nitems * nbc;

    if (warp == kProdWarp) {
        // ---- work units
        if (lane == 0) {
            for (int uc = 0;; ++uc) {
                const int slot = uc % kUnitRing;
                if (uc >= kUnitRing &&
                    !bar_wait(smem_addr(&ring_empty[slot]), (uint32_t)((uc / kUnitRing) - 1) & 1u, &abort_s))
                    break;
                const int64_t u = abort_s ? units : (int64_t)atomicAdd(counter, 1);
                ring[slot] = u;
                bar_arrive(smem_addr(&ring_full[slot]));
                if (u >= units) break;
            }
        }
    } else if (warp == kMmaWarp) {
        // ---- MMA issue: one lane
        if (lane == 0) {
            int64_t seq = 0;
            int nu = 0;   // non-empty units so far (accumulator = nu & 1)
            for (int uc = 0;; ++uc) {
                const int slot = uc % kUnitRing;
                if (!bar_wait(smem_addr(&ring_full[slot]), (uint32_t)(uc / kUnitRing) & 1u, &abort_s)) break;
                const int64_t u = ring[slot];
                if (u >= units) break;
                const int4 item = __ldg(items + u / nbc);
                if (item.y < item.z) {
                    const int ab = nu & 1;
                    if (nu >= 2 && !bar_wait(smem_addr(&acc_empty[ab]), (uint32_t)((nu >> 1) - 1) & 1u, &abort_s))
                        break;
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t d = tmem + (uint32_t)(ab * kTcN);
                    bool ok = true, first = true;
                    for (int iv = item.y; iv < item.z && ok; ++iv) {
                        const int4 e = __ldg(ivl + iv);
                        for (int sb = e.x; sb < e.y; sb += kSrc, ++seq) {
                            const int s = (int)(seq % NS);
                            if (!bar_wait(smem_addr(&full_s[s]), (uint32_t)(seq / NS) & 1u, &abort_s)) {
                                ok = false;
                                break;
                            }
                            asm volatile("tcgen05.fence::after_thread_sync;");
                            const uint32_t st = sbase + (uint32_t)(s * S::STAGE);
#pragma unroll
                            for (int ks = 0; ks < kKC / 8; ++ks) {
                                const uint32_t off = ks * 256;   // two 16-byte column groups per K step of 8
                                const uint64_t dah = umma_desc(st + off, 128, kChunkSBO);
                                const uint64_t dal = umma_desc(st + S::A_CH + off, 128, kChunkSBO);
                                const uint64_t dbh = umma_desc(st + 2 * S::A_CH + off, 128, kChunkSBO);
                                const uint64_t dbl = umma_desc(st + 2 * S::A_CH + S::B_CH + off, 128, kChunkSBO);
                                tc_mma(d, dah, dbh, S::IDESC, first ? 0u : 1u);
                                first = false;
                                tc_mma(d, dah, dbl, S::IDESC, 1u);
                                if (!S::STACKED) tc_mma(d, dal, dbh, S::IDESC, 1u);
                            }
                            tc_commit(smem_addr(&empty_s[s]));
                        }
                    }
                    if (!ok) break;
                    tc_commit(smem_addr(&acc_full[ab]));
                    ++nu;
                }
                bar_arrive(smem_addr(&ring_empty[slot]));
            }
            // the MMAs in flight complete before the block frees the tensor memory
            tc_commit(smem_addr(&drain));
            drain_wait(smem_addr(&drain), 0u);
        }
    } else {
        // ---- generators: thread tid owns target tid of the group (row tid of the kernel tile)
        // and, for tid < 8 RC, the weight of source tid / RC and right-hand side tid % RC
        const int blk = tid / kTargetBlock;
        const int wsl = tid / RC, wj = tid % RC;
        int64_t seq = 0;
        int nu = 0;
        bool pend = false;
        int p_ab = 0, p_par = 0, p_b0 = 0, p_nb = 0;
        int64_t p_tbase = 0;
        auto drain_acc = [&]() -> bool {
            const int qd = warp & 3, half = warp >> 2;
            if (!warp_wait(smem_addr(&acc_full[p_ab]), (uint32_t)p_par, &abort_s)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;");
            if ((32 * qd) % S::ROWS < 4 * p_nb) {
                const int m = (32 * qd + lane) % S::ROWS, j = m >> 2, cpt = m & 3;
#pragma unroll 1
                for (int c0 = 0; c0 < kTcN / 2; c0 += 32) {
                    const int64_t tc = p_tbase + half * (kTcN / 2) + c0 + lane;   // this lane's column's target
                    const int pc = tc < ntgt ? panel_of(tgt[tc].w) : -1;
#pragma unroll
                    for (int h16 = 0; h16 < 32; h16 += 16) {
                        uint32_t v[16];
                        const uint32_t addr = tmem + ((uint32_t)(32 * qd) << 16) +
                                              (uint32_t)(p_ab * kTcN + half * (kTcN / 2) + c0 + h16);
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
                            "%14,%15}, [%16];"
                            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                              "=r"(v[14]), "=r"(v[15])
                            : "r"(addr));
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                        for (int x = 0; x < 16; ++x) {
                            const int p = __shfl_sync(0xffffffffu, pc, h16 + x);
                            if (j < p_nb && p >= 0)
                                atomicAdd(acc + 4 * ((int64_t)p * B + p_b0 + j) + cpt, (double)__uint_as_float(v[x]));
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) bar_arrive(smem_addr(&acc_empty[p_ab]));
            pend = false;
            return true;
        };
        bool ok = true;
        for (int uc = 0; ok; ++uc) {
            const int slot = uc % kUnitRing;
            if (!warp_wait(smem_addr(&ring_full[slot]), (uint32_t)(uc / kUnitRing) & 1u, &abort_s)) {
                ok = false;
                break;
            }
            const int64_t u = ring[slot];
            if (u >= units) break;
            const int64_t ii = u / nbc;
            const int b0 = (int)(u - ii * nbc) * RC, nb = min(RC, Bact - b0);
            const int4 item = __ldg(items + ii);
            const int64_t tbase = (int64_t)item.x * kTcN;   // first target of the group
            const int64_t ti = tbase + tid;
            const bool live = ti < ntgt;
            const float4 q = live ? tgt[ti] : tgt[0];
            const int tp = live ? panel_of(q.w) : -1;
            for (int iv = item.y; iv < item.z && ok; ++iv) {
                const int4 e = __ldg(ivl + iv);
                const bool on = live && ((e.z >> blk) & 1);   // uniform over the warp but for the tail
                for (int sb = e.x; sb < e.y && ok; sb += kSrc) {
                    // the kernel tile row of this target: G and dG/dn of the stage's sources
                    // the kernel tile row of this target: G and dG/dn of the stage's sources
                    float g[kSrc], h[kSrc];
#pragma unroll
                    for (int k = 0; k < kSrc; ++k) {
                        g[k] = 0.f;
                        h[k] = 0.f;
                        if (on && sb + k < e.y) {
                            const float4 p = __ldg(spos + sb + k), n = __ldg(snrm + sb + k);
                            const float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
                            float r = rsq(dx * dx + dy * dy + dz * dz);
                            r = panel_of(n.w) == tp ? 0.f : r;
                            g[k] = r;
                            h[k] = (dx * n.x + dy * n.y + dz * n.z) * (r * r) * r;
                        }
                    }
                    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (tid < kSrc * RC && sb + wsl < e.y && wj < nb) w = __ldg(sw + (int64_t)(sb + wsl) * B + b0 + wj);
                    const int s = (int)(seq % NS);
                    if (seq >= NS && !warp_wait(smem_addr(&empty_s[s]), (uint32_t)((seq / NS) - 1) & 1u, &abort_s)) {
                        ok = false;
                        break;
                    }
                    unsigned char *ah = tc_smem + s * S::STAGE, *al = ah + S::A_CH;
                    unsigned char *bh = ah + 2 * S::A_CH, *bl = bh + S::B_CH;
                    if (tid < kSrc * RC) {
                        // V channels (rows 4 j, 4 j + 1) in the G column of the source, K channels
                        // (rows 4 j + 2, 4 j + 3) in its dG/dn column
                        const float v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int off = core_off(4 * wj + c, (c < 2 ? 0 : kSrc) + wsl);
                            const float hi = tf32_hi(v[c]);
                            *(float *)(ah + off) = hi;
                            *(float *)(al + off) = v[c] - hi;
                        }
                    }
#pragma unroll
                    for (int k4 = 0; k4 < kSrc / 4; ++k4) {
                        const float4 gv = make_float4(g[4 * k4], g[4 * k4 + 1], g[4 * k4 + 2], g[4 * k4 + 3]);
                        const float4 hv = make_float4(h[4 * k4], h[4 * k4 + 1], h[4 * k4 + 2], h[4 * k4 + 3]);
                        const float4 gh = f4_hi(gv), hh = f4_hi(hv);
                        *(float4 *)(bh + core_off(tid, 4 * k4)) = gh;
                        *(float4 *)(bl + core_off(tid, 4 * k4)) = f4_sub(gv, gh);
                        *(float4 *)(bh + core_off(tid, kSrc + 4 * k4)) = hh;
                        *(float4 *)(bl + core_off(tid, kSrc + 4 * k4)) = f4_sub(hv, hh);
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    bar_arrive(smem_addr(&full_s[s]));
                    ++seq;
                    if (pend) ok = drain_acc();   // the previous unit, behind this unit's first stage
                }
            }
            if (ok && pend) ok = drain_acc();     // the previous unit, if this one had no source
            if (!ok) break;
            if (item.y < item.z) {
                pend = true;
                p_ab = nu & 1;
                p_par = (nu >> 1) & 1;
                p_tbase = tbase;
                p_b0 = b0;
                p_nb = nb;
                ++nu;
            }
            __syncwarp();
            if (lane == 0) bar_arrive(smem_addr(&ring_empty[slot]));
        }
        if (ok && pend) drain_acc();
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    if (tid == 0 && abort_s) atomicAdd(error, 1);
}

template <int RC>
int tc_p2p(lspr_ctx *ctx, double *acc, cudaStream_t st, int *counter, int B) {
    using S = P2PShape<RC>;
    static int smem_set[kSmemDevices] = {};
    Tree &tr = ctx->tree;
    if (tr.n_tcp_items == 0) return LSPR_OK;
    if (!ctx->dev_err.p) return LSPR_E_STATE;
    LSPR_TRY(ctx, allow_smem(p2p_tc_kernel<RC>, S::SMEM, ctx->device, smem_set));
    const int nrc = (B + RC - 1) / RC;
    const unsigned grid =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>(tr.n_tcp_items * nrc, std::max(1, ctx->num_sms)));
    p2p_tc_kernel<RC><<<grid, kTcThreads, S::SMEM, st>>>(tr.tcp_items.p, tr.n_tcp_items, tr.tcp_ivl.p, B,
                                                        Views<float>::tgt(ctx), ctx->mesh.N, Views<float>::spos(ctx),
                                                        Views<float>::snrm(ctx), Views<float>::w(ctx), acc, counter,
                                                        ctx->dev_err.p, ctx->rhs_nact);
    return LSPR_OK;
}

}  // namespace

// FP32 tree P2P of B >= 2 right-hand sides on the tensor cores
int p2p_tc_launch(lspr_ctx *ctx, double *acc, cudaStream_t st, int *counter, int B) {
    if (!ctx->tree.tcp_built) LSPR_TRY_ST(tree_tc_lists(ctx, true));
    return B <= 16 ? tc_p2p<16>(ctx, acc, st, counter, B) : tc_p2p<32>(ctx, acc, st, counter, B);
}

}  // namespace lspr
