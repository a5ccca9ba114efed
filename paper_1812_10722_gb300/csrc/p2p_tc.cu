// P2P of several right-hand sides on the fifth-generation tensor cores (tcgen05).
//
// The direct far-rule sums of Eq. summation for a target x over sources y_s,
//   V_j(x) = sum_s G(x, y_s) q_s[j],   K_j(x) = sum_s dG/dn(x, y_s) mu_s[j],
// (q, mu complex per right-hand side j) are two matrix products once the kernel values of a
// tile are laid out as operands:
//   D_V[channel][target] += W_V[channel][source] G[source][target]
//   D_K[channel][target] += W_K[channel][source] dG/dn[source][target]
// with the channels (re and im of each of up to 64 right-hand sides: 128 rows) as the MMA's M,
// the 256 targets of a group of four consecutive 64-target blocks as its N, and 8 sources per
// pipeline stage as its K.  W_V holds only single-layer weights and W_K only double-layer ones,
// so no operand carries structural zeros, and one kernel tile serves 64 right-hand sides.
// The group walks the union of its blocks' P2P source ranges; a target whose block does not sum
// a range gets zero kernel values there, and a target's own panel is skipped (its exact integral
// is in the near correction), as in p2p_kernel.  Both operands are split into TF32 high and low
// parts (each rounded to nearest) with FP32 accumulation in tensor memory: with more than 32
// right-hand sides in the unit, three MMAs per operand pair give W_hi G_hi + W_hi G_lo +
// W_lo G_hi (3xTF32); with at most 32,
// W_hi and W_lo are the two halves of one 128-row operand and two MMAs give all four products
// (the epilogue adds both halves).
//
// Roles (persistent, one CTA per SM, both accumulators in the SM's 512 tensor-memory columns):
//   warp 16 (one lane) fetches work units into a small ring and bulk-copies every stage's inputs
//     (the positions, normals and weights of its eight sources) into the stage;
//   warps 0-15 (two threads per target of the group, four of the stage's eight sources each)
//     generate G and dG/dn of every stage in registers from those inputs, split them and write
//     the B operands; warps 8-11 also write the split weights (the A operands); after the first
//     stage of the next unit they drain the finished unit's accumulators (tcgen05.ld) into the
//     FP64 accumulators;
//   warp 17 (one lane) issues the MMAs of each stage once it is written, commits to the stage's
//     "empty" barrier and, at the end of a unit, to the accumulator barrier.
// Every wait is bounded (about a second): one that runs out raises an abort flag that the
// other roles see, the block drains its bulk copies and MMAs in flight, frees its tensor memory
// and returns,
// and the context's device error count (error[0]) records it.  With error[1] set, thread 0
// first waits on a barrier that nothing arrives on, so that the wait runs out before any work
// is issued (the host's check of this failure path).
#include "farfield.cuh"
#include "tcgen05.cuh"

namespace lspr {

namespace {

using namespace tc;

constexpr int kSrc = 8;                        // sources per stage (the MMA's K)
constexpr int kRC = 64;                        // right-hand sides per work unit
constexpr int kTcN = kTcGroup * kTargetBlock;  // targets per work unit (the MMA's N)
constexpr int kSBO = (kSrc / 4) * 128;         // bytes per 8-row group of a stage operand
constexpr int kGenSplit = 2;                   // generating threads per target (4 of the 8 sources each)
constexpr int kGenThreads = kGenSplit * kTcN;
constexpr int kGenWarps = kGenThreads / 32;
constexpr int kProdWarp = kGenWarps, kMmaWarp = kGenWarps + 1;
constexpr int kTcThreads = 32 * (kGenWarps + 2);
constexpr int kUnitRing = 4;
constexpr int kRingConsumers = kGenWarps + 1;  // lane 0 of each consumer warp
constexpr uint32_t kTmemCols = 2 * kTcN;       // D_V in columns [0, 256), D_K in [256, 512)
constexpr int kAPart = (128 / 8) * kSBO;       // one split part of a weight operand (128 rows)
constexpr int kBPart = (kTcN / 8) * kSBO;      // one split part of a kernel operand (256 rows)
// stage: W_V hi | W_V lo | W_K hi | W_K lo | G hi | G lo | dG hi | dG lo | the stage's inputs as
// bulk-copied from global memory: source positions (8 float4), normals (8 float4), weights
// (8 sources x 64 right-hand sides float4)
constexpr int kOffWV = 0, kOffWK = 2 * kAPart, kOffG = 4 * kAPart, kOffD = 4 * kAPart + 2 * kBPart;
constexpr int kOffRaw = 4 * kAPart + 4 * kBPart;
constexpr int kRawPos = 0, kRawNrm = kSrc * 16, kRawW = 2 * kSrc * 16;
constexpr int kStage = kOffRaw + 2 * kSrc * 16 + kSrc * kRC * 16;
constexpr int kStages = 4;
constexpr int kSmem = kStages * kStage;
static_assert(kSmem + 1024 <= 232448, "the stages and the static shared memory fit one SM");
constexpr uint32_t kIdesc = idesc_tf32(128, kTcN);
static_assert(kTmemCols <= 512 && kTcN <= 256, "both accumulators fit the tensor memory");
static_assert(kStages >= 2, "at least two stages");
static_assert(kRC * 2 == 128, "re and im of the unit's right-hand sides fill the MMA's M");

// byte offset of (row r, column k) inside one split part of a stage operand (K-major 8 x 16-byte
// core matrices, no swizzle)
__device__ __forceinline__ int core_off(int r, int k) {
    return (r >> 3) * kSBO + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

__global__ void __launch_bounds__(kTcThreads, 1)
    p2p_tc_kernel(const int4 *__restrict__ items, int64_t nitems, const int4 *__restrict__ ivl, int B,
                  const float4 *__restrict__ tgt, int64_t ntgt, const float4 *__restrict__ spos,
                  const float4 *__restrict__ snrm, const float4 *__restrict__ sw, double *__restrict__ acc,
                  int *counter, int *error, const int *nact, int min_rhs) {
    // fewer right-hand sides in use than min_rhs: the FP32-pipe P2P takes this product
    if ((nact ? *nact : B) < min_rhs) return;
    extern __shared__ __align__(128) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t full_s[kStages], empty_s[kStages], raw_s[kStages];
    __shared__ __align__(8) uint64_t acc_full, acc_empty, ring_full[kUnitRing], ring_empty[kUnitRing], drain, gate;
    __shared__ int64_t ring[kUnitRing];
    __shared__ uint32_t tslot;
    __shared__ volatile int abort_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = smem_addr(tc_smem);
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            bar_init(smem_addr(&full_s[s]), kGenThreads);   // one arrival per generating thread
            bar_init(smem_addr(&empty_s[s]), 1);     // the MMAs' commit
            bar_init(smem_addr(&raw_s[s]), 1);       // the producer's expect_tx (+ the copies' bytes)
        }
        bar_init(smem_addr(&acc_full), 1);
        bar_init(smem_addr(&acc_empty), kGenWarps);
        for (int r = 0; r < kUnitRing; ++r) {
            bar_init(smem_addr(&ring_full[r]), 1);
            bar_init(smem_addr(&ring_empty[r]), kRingConsumers);
        }
        bar_init(smem_addr(&drain), 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // failure-path check (error[1] set by the host): a bounded wait on a barrier that nothing
        // arrives on runs out before any work is issued, and the block returns without work
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
    const int nbc = (Bact + kRC - 1) / kRC;
    const int64_t units = nitems * nbc;

    if (warp == kProdWarp) {
        // ---- work units, and the inputs of every stage by bulk copies: positions and normals
        // of the stage's sources, their weights for the unit's right-hand sides
        if (lane == 0) {
            int64_t seq = 0;   // stages armed so far
            for (int uc = 0;; ++uc) {
                const int slot = uc % kUnitRing;
                if (uc >= kUnitRing &&
                    !bar_wait(smem_addr(&ring_empty[slot]), (uint32_t)((uc / kUnitRing) - 1) & 1u, &abort_s))
                    break;
                const int64_t u = abort_s ? units : (int64_t)atomicAdd(counter, 1);
                ring[slot] = u;
                bar_arrive(smem_addr(&ring_full[slot]));
                if (u >= units) break;
                const int64_t ii = u / nbc;
                const int b0 = (int)(u - ii * nbc) * kRC, nb = min(kRC, Bact - b0);
                const int4 item = __ldg(items + ii);
                bool ok = true;
                for (int iv = item.y; iv < item.z && ok; ++iv) {
                    const int4 e = __ldg(ivl + iv);
                    for (int sb = e.x; sb < e.y; sb += kSrc, ++seq) {
                        const int s = (int)(seq % kStages);
                        if (seq >= kStages &&
                            !bar_wait(smem_addr(&empty_s[s]), (uint32_t)((seq / kStages) - 1) & 1u, &abort_s)) {
                            ok = false;
                            break;
                        }
                        const int n = min(kSrc, e.y - sb);
                        const uint32_t rb = smem_addr(&raw_s[s]);
                        const uint32_t dst = sbase + (uint32_t)(s * kStage + kOffRaw);
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(rb),
                                     "r"((uint32_t)(n * 32 + n * nb * 16))
                                     : "memory");
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                dst + kRawPos),
                            "l"(spos + sb), "r"(n * 16), "r"(rb)
                            : "memory");
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                dst + kRawNrm),
                            "l"(snrm + sb), "r"(n * 16), "r"(rb)
                            : "memory");
                        for (int k = 0; k < n; ++k)
                            asm volatile(
                                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                    dst + kRawW + (uint32_t)(k * kRC * 16)),
                                "l"(sw + (int64_t)(sb + k) * B + b0), "r"(nb * 16), "r"(rb)
                                : "memory");
                    }
                }
                if (!ok) break;
            }
            // the copies of the last armed stages may still be in flight
            for (int64_t k = seq > kStages ? seq - kStages : 0; k < seq; ++k)
                drain_wait(smem_addr(&raw_s[k % kStages]), (uint32_t)(k / kStages) & 1u);
        }
    } else if (warp == kMmaWarp) {
        // ---- MMA issue: one lane
        if (lane == 0) {
            int64_t seq = 0;
            int nu = 0;   // units with stages so far
            for (int uc = 0;; ++uc) {
                const int slot = uc % kUnitRing;
                if (!bar_wait(smem_addr(&ring_full[slot]), (uint32_t)(uc / kUnitRing) & 1u, &abort_s)) break;
                const int64_t u = ring[slot];
                if (u >= units) break;
                const int64_t ii = u / nbc;
                const int nb = min(kRC, Bact - (int)(u - ii * nbc) * kRC);
                const bool stacked = nb <= kRC / 2;
                const int4 item = __ldg(items + ii);
                if (item.y < item.z) {
                    // the accumulators are free once the previous unit is drained
                    if (nu >= 1 && !bar_wait(smem_addr(&acc_empty), (uint32_t)((nu - 1) & 1), &abort_s)) break;
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t dv = tmem, dk = tmem + (uint32_t)kTcN;
                    bool ok = true, first = true;
                    for (int iv = item.y; iv < item.z && ok; ++iv) {
                        const int4 e = __ldg(ivl + iv);
                        for (int sb = e.x; sb < e.y; sb += kSrc, ++seq) {
                            const int s = (int)(seq % kStages);
                            if (!bar_wait(smem_addr(&full_s[s]), (uint32_t)(seq / kStages) & 1u, &abort_s)) {
                                ok = false;
                                break;
                            }
                            asm volatile("tcgen05.fence::after_thread_sync;");
                            const uint32_t st = sbase + (uint32_t)(s * kStage);
                            const uint64_t wvh = umma_desc(st + kOffWV, 128, kSBO);
                            const uint64_t wvl = umma_desc(st + kOffWV + kAPart, 128, kSBO);
                            const uint64_t wkh = umma_desc(st + kOffWK, 128, kSBO);
                            const uint64_t wkl = umma_desc(st + kOffWK + kAPart, 128, kSBO);
                            const uint64_t gh = umma_desc(st + kOffG, 128, kSBO);
                            const uint64_t gl = umma_desc(st + kOffG + kBPart, 128, kSBO);
                            const uint64_t hh = umma_desc(st + kOffD, 128, kSBO);
                            const uint64_t hl = umma_desc(st + kOffD + kBPart, 128, kSBO);
                            const uint32_t on = first ? 0u : 1u;
                            first = false;
                            tc_mma(dv, wvh, gh, kIdesc, on);
                            tc_mma(dv, wvh, gl, kIdesc, 1u);
                            tc_mma(dk, wkh, hh, kIdesc, on);
                            tc_mma(dk, wkh, hl, kIdesc, 1u);
                            if (!stacked) {
                                tc_mma(dv, wvl, gh, kIdesc, 1u);
                                tc_mma(dk, wkl, hh, kIdesc, 1u);
                            }
                            tc_commit(smem_addr(&empty_s[s]));
                        }
                    }
                    if (!ok) break;
                    tc_commit(smem_addr(&acc_full));
                    ++nu;
                }
                bar_arrive(smem_addr(&ring_empty[slot]));
            }
            // the MMAs in flight complete before the block frees the tensor memory
            tc_commit(smem_addr(&drain));
            drain_wait(smem_addr(&drain), 0u);
        }
    } else {
        // ---- generators: thread tid owns target tt = tid mod 256 of the group (row tt of the
        // kernel operands) for the four sources 4 hf .. 4 hf + 3 of each stage, hf = tid / 256;
        // threads 256..383 also stage the weights of one right-hand side for four sources
        const int tt = tid & (kTcN - 1), hf = tid / kTcN, wt = tid - kTcN;
        const int blk = tt / kTargetBlock;
        int64_t seq = 0;
        int nu = 0;
        bool pend = false;
        int p_nb = 0, p_b0 = 0;
        bool p_stacked = false;
        int64_t p_tbase = 0;
        // epilogue: warp w reads tensor-memory lanes 32 (w % 4).. (channel rows) and the 64
        // targets from column 64 (w / 4) of both accumulators; false: a wait ran out
        auto drain_acc = [&]() -> bool {
            const int qd = warp & 3, part = warp >> 2;
            if (!warp_wait(smem_addr(&acc_full), (uint32_t)((nu - 1) & 1), &abort_s)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int m = 32 * qd + lane;
            // row m: without stacking re (m < 64) / im of right-hand side m % 64; stacked: re / im
            // of m % 32 in the high (m < 64) or the low half
            const int j = p_stacked ? (m & 31) : (m & 63);
            const int cpt = p_stacked ? ((m >> 5) & 1) : (m >> 6);
            const bool row_on = j < p_nb;
            if (__any_sync(0xffffffffu, row_on)) {
#pragma unroll 1
                for (int c0 = 0; c0 < kTcN / 4; c0 += 32) {
                    const int64_t tc = p_tbase + part * (kTcN / 4) + c0 + lane;   // this lane's column's target
                    const int pc = tc < ntgt ? panel_of(tgt[tc].w) : -1;
#pragma unroll 1
                    for (int op = 0; op < 2; ++op) {   // D_V, then D_K
#pragma unroll
                        for (int h16 = 0; h16 < 32; h16 += 16) {
                            uint32_t v[16];
                            const uint32_t addr = tmem + ((uint32_t)(32 * qd) << 16) +
                                                  (uint32_t)(op * kTcN + part * (kTcN / 4) + c0 + h16);
                            asm volatile(
                                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
                                "%14,%15}, [%16];"
                                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                                  "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                                : "r"(addr));
                            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                            for (int x = 0; x < 16; ++x) {
                                const int p = __shfl_sync(0xffffffffu, pc, h16 + x);
                                if (row_on && p >= 0)
                                    atomicAdd(acc + 4 * ((int64_t)p * B + p_b0 + j) + 2 * op + cpt,
                                              (double)__uint_as_float(v[x]));
                            }
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) bar_arrive(smem_addr(&acc_empty));
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
            const int b0 = (int)(u - ii * nbc) * kRC, nb = min(kRC, Bact - b0);
            const bool stacked = nb <= kRC / 2;
            const int4 item = __ldg(items + ii);
            const int64_t tbase = (int64_t)item.x * kTcN;   // first target of the group
            const int64_t ti = tbase + tt;
            const bool live = ti < ntgt;
            const float4 q = live ? tgt[ti] : tgt[0];
            const int tp = live ? panel_of(q.w) : -1;
            // weight staging (rows of the weight operands as documented at drain_acc): right-hand
            // side wj at the sources of columns wk..wk+3; stacked units need threads 0..63 only
            const bool wr = wt >= 0 && wt < 128 && (!stacked || wt < 64);
            const int wj = stacked ? (wt & 31) : (wt & 31) + 32 * (wt >> 6);
            const int wk = stacked ? 4 * (wt >> 5) : 4 * ((wt >> 5) & 1);
            for (int iv = item.y; iv < item.z && ok; ++iv) {
                const int4 e = __ldg(ivl + iv);
                const bool on = live && ((e.z >> blk) & 1);   // uniform over the warp but for the tail
                for (int sb = e.x; sb < e.y && ok; sb += kSrc) {
                    // the stage's inputs have landed (and its operands are free: the producer
                    // armed the copies after the stage's previous MMAs completed)
                    const int s = (int)(seq % kStages);
                    if (!warp_wait(smem_addr(&raw_s[s]), (uint32_t)(seq / kStages) & 1u, &abort_s)) {
                        ok = false;
                        break;
                    }
                    unsigned char *stg = tc_smem + s * kStage;
                    const float4 *rpos = (const float4 *)(stg + kOffRaw + kRawPos);
                    const float4 *rnrm = (const float4 *)(stg + kOffRaw + kRawNrm);
                    const float4 *rw = (const float4 *)(stg + kOffRaw + kRawW);
                    // this thread's part of the kernel operand row of its target: G and dG/dn of
                    // the stage's sources 4 hf .. 4 hf + 3
                    constexpr int kPart = kSrc / kGenSplit;
                    float g[kPart], h[kPart];
#pragma unroll
                    for (int kk = 0; kk < kPart; ++kk) {
                        const int k = kPart * hf + kk;
                        g[kk] = 0.f;
                        h[kk] = 0.f;
                        if (on && sb + k < e.y) {
                            const float4 p = rpos[k], n = rnrm[k];
                            const float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
                            float r = rsq(dx * dx + dy * dy + dz * dz);
                            r = panel_of(n.w) == tp ? 0.f : r;
                            g[kk] = r;
                            h[kk] = (dx * n.x + dy * n.y + dz * n.z) * (r * r) * r;
                        }
                    }
                    // the weights of right-hand side wj at the four sources from column wk
                    float4 w[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        w[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (wr && wj < nb && sb + wk + i < e.y) w[i] = rw[(wk + i) * kRC + wj];
                    }
                    if (wr) {
                        const float4 vre = make_float4(w[0].x, w[1].x, w[2].x, w[3].x);
                        const float4 vim = make_float4(w[0].y, w[1].y, w[2].y, w[3].y);
                        const float4 kre = make_float4(w[0].z, w[1].z, w[2].z, w[3].z);
                        const float4 kim = make_float4(w[0].w, w[1].w, w[2].w, w[3].w);
                        const TfPair svr = tf32_split(vre), svi = tf32_split(vim);
                        const TfPair skr = tf32_split(kre), ski = tf32_split(kim);
                        unsigned char *av = stg + kOffWV, *ak = stg + kOffWK;
                        if (stacked) {
                            // rows: re hi wj, im hi 32 + wj, re lo 64 + wj, im lo 96 + wj
                            *(float4 *)(av + core_off(wj, wk)) = svr.hi;
                            *(float4 *)(av + core_off(32 + wj, wk)) = svi.hi;
                            *(float4 *)(av + core_off(64 + wj, wk)) = svr.lo;
                            *(float4 *)(av + core_off(96 + wj, wk)) = svi.lo;
                            *(float4 *)(ak + core_off(wj, wk)) = skr.hi;
                            *(float4 *)(ak + core_off(32 + wj, wk)) = ski.hi;
                            *(float4 *)(ak + core_off(64 + wj, wk)) = skr.lo;
                            *(float4 *)(ak + core_off(96 + wj, wk)) = ski.lo;
                        } else {
                            // rows: re wj, im 64 + wj; the high part, then the low part
                            *(float4 *)(av + core_off(wj, wk)) = svr.hi;
                            *(float4 *)(av + core_off(64 + wj, wk)) = svi.hi;
                            *(float4 *)(av + kAPart + core_off(wj, wk)) = svr.lo;
                            *(float4 *)(av + kAPart + core_off(64 + wj, wk)) = svi.lo;
                            *(float4 *)(ak + core_off(wj, wk)) = skr.hi;
                            *(float4 *)(ak + core_off(64 + wj, wk)) = ski.hi;
                            *(float4 *)(ak + kAPart + core_off(wj, wk)) = skr.lo;
                            *(float4 *)(ak + kAPart + core_off(64 + wj, wk)) = ski.lo;
                        }
                    }
                    unsigned char *bg = stg + kOffG, *bd = stg + kOffD;
                    static_assert(kPart == 4, "a thread writes one 4-column slice of its row");
                    {
                        const float4 gv = make_float4(g[0], g[1], g[2], g[3]);
                        const float4 hv = make_float4(h[0], h[1], h[2], h[3]);
                        const TfPair sg = tf32_split(gv), sh = tf32_split(hv);
                        *(float4 *)(bg + core_off(tt, kPart * hf)) = sg.hi;
                        *(float4 *)(bg + kBPart + core_off(tt, kPart * hf)) = sg.lo;
                        *(float4 *)(bd + core_off(tt, kPart * hf)) = sh.hi;
                        *(float4 *)(bd + kBPart + core_off(tt, kPart * hf)) = sh.lo;
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
                p_tbase = tbase;
                p_b0 = b0;
                p_nb = nb;
                p_stacked = stacked;
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

}  // namespace

// FP32 tree P2P of B >= 2 right-hand sides on the tensor cores
int p2p_tc_launch(lspr_ctx *ctx, double *acc, cudaStream_t st, int *counter, int B, int min_rhs) {
    static int smem_set[kSmemDevices] = {};
    Tree &tr = ctx->tree;
    if (!tr.tcp_built) LSPR_TRY_ST(tree_tc_lists(ctx, true));
    if (tr.n_tcp_items == 0) return LSPR_OK;
    if (!ctx->dev_err.p) return LSPR_E_STATE;
    LSPR_TRY(ctx, allow_smem(p2p_tc_kernel, kSmem, ctx->device, smem_set));
    const int nrc = (B + kRC - 1) / kRC;
    const unsigned grid =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>(tr.n_tcp_items * nrc, std::max(1, ctx->num_sms)));
    p2p_tc_kernel<<<grid, kTcThreads, kSmem, st>>>(tr.tcp_items.p, tr.n_tcp_items, tr.tcp_ivl.p, B,
                                                  Views<float>::tgt(ctx), ctx->mesh.N, Views<float>::spos(ctx),
                                                  Views<float>::snrm(ctx), Views<float>::w(ctx), acc, counter,
                                                  ctx->dev_err.p, ctx->rhs_nact, min_rhs);
    return LSPR_OK;
}

}  // namespace lspr
