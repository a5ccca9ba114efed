// M2P of several right-hand sides on the fifth-generation tensor cores (tcgen05).
//
// The contraction over the Taylor terms is a matrix product per box b,
//   D[channel][target] += sum_k M_k(b)[channel] a_k(target - c_b),
// with the channels (4 per right-hand side: V re, V im, K re, K im) as the MMA's M dimension,
// the targets as its N and the terms as its K.  A tcgen05 MMA costs the same time whatever
// its shape, so N is made as wide as the instruction allows: a work unit is a group of four
// consecutive 64-target blocks (N = 256) and walks the sorted union of their M2P lists; the
// coefficients of a block that did not accept a box are zero, so every block still receives
// exactly the boxes its own acceptance test chose.  Both operands are split into TF32 high
// and low parts (FP32 accumulation in tensor memory): with 32 right-hand sides per unit
// (128 channels) the product is A_hi B_hi + A_hi B_lo + A_lo B_hi (3xTF32); with 16 (64
// channels) A_hi and A_lo are stacked into the 128 rows of one operand and two MMAs give all
// four products.
//
// Two kernels per product:
//   - tc_image_kernel writes, once per product, the split moments of every box in the
//     operand layout of one pipeline stage (K-major 8x16-byte core matrices, no swizzle),
//     so that staging A is a single bulk copy;
//   - m2p_tc_kernel is persistent and warp-specialised.  The terms of each (unit, box) are
//     cut into chunks of 16, one pipeline stage each (a ring of NS stages in shared memory):
//       warps 0-7 (one thread per target of the group) compute the coefficients a_k by the
//         recurrence of m2p_kernel and write the split B part of each stage; they drain each
//         unit's accumulator (tcgen05.ld) into the FP64 accumulators once the next unit's
//         first box is staged, so that the MMAs keep going meanwhile;
//       warp 8 (one lane) fetches work units, publishes them in a small ring, and streams
//         each stage's A part with cp.async.bulk;
//       warp 9 (one lane) issues the MMAs of each stage once both parts are in, commits to
//         the stage's "empty" barrier and, at the end of a unit, to an accumulator barrier
//         (two accumulators of 256 columns alternate between units).
// Every wait is bounded (about a second): one that runs out raises an abort flag that the
// other roles see, the block drains its bulk copies and MMAs in flight, frees its tensor
// memory and returns, and the context's device error count (error[0]) records it.  With
// error[1] set, thread 0 first waits on a barrier that nothing arrives on, so that the wait
// runs out before any work is issued (the host's check of this failure path).
#include "farfield.cuh"
#include "tcgen05.cuh"

namespace lspr {

namespace {

using namespace tc;

constexpr int kKC = 16;                        // terms per pipeline stage (two MMA K steps)
constexpr int kTcN = kTcGroup * kTargetBlock;  // targets per work unit (the MMA's N)
constexpr int kChunkSBO = (kKC / 4) * 128;     // bytes per 8-row group of a stage operand
constexpr int kGenWarps = kTcN / 32;           // one thread per target
constexpr int kProdWarp = kGenWarps, kMmaWarp = kGenWarps + 1;
constexpr int kTcThreads = 32 * (kGenWarps + 2);
constexpr int kUnitRing = 4;
constexpr int kRingConsumers = kGenWarps + 1;  // lane 0 of each consumer warp
constexpr uint32_t kTmemCols = 2 * kTcN;       // two accumulators
static_assert(kTmemCols <= 512 && kTcN <= 256, "one MMA spans the group");

// Stage geometry for order P and RC right-hand sides per unit (ROWS = 4 RC channels).
// RC = 32: A_hi B_hi, A_hi B_lo and A_lo B_hi are three M = 128 MMAs into one accumulator.
// RC = 16: A_hi and A_lo (adjacent in the stage) are the two halves of one M = 128 operand,
// so two MMAs, [A_hi; A_lo] B_hi and [A_hi; A_lo] B_lo, give A_hi B in accumulator rows 0..63
// and A_lo B in rows 64..127 (all four products); the epilogue adds both halves.  Row m of
// an M = 128 accumulator sits in TMEM lane m.
// RC = 64: two halves of 32 right-hand sides share each stage's coefficients (B): the stage
// holds both halves' A parts, each half takes the three MMAs of RC = 32 into its own accumulator
// (both 256-column accumulators belong to the unit), so the recurrence, the split coefficients
// and the stage hand-overs of a (group, box) serve 64 right-hand sides.
template <int P, int RC>
struct TcShape {
    static constexpr int NT = n_terms(P);
    static constexpr int NKC = (NT + kKC - 1) / kKC;
    static constexpr int HALVES = RC == 64 ? 2 : 1;       // A parts (accumulators) per unit
    static constexpr int HRC = RC / HALVES;               // right-hand sides per A part
    static constexpr int ROWS = 4 * HRC;
    static constexpr bool STACKED = ROWS == 64;           // hi and lo halves of one operand
    static constexpr uint32_t IDESC = idesc_tf32(128, kTcN);
    static constexpr int A_CH = (ROWS / 8) * kChunkSBO;   // one split part of one A per stage
    static constexpr int B_CH = (kTcN / 8) * kChunkSBO;   // one split part of B per stage
    static constexpr int OFF_B = HALVES * 2 * A_CH;       // [A_hi | A_lo] per half, then B_hi | B_lo
    static constexpr int STAGE = OFF_B + 2 * B_CH;
    static constexpr int NS = (200 * 1024) / STAGE;
    static constexpr int SMEM = NS * STAGE;
    static_assert(ROWS == 64 || ROWS == 128, "A parts of 16 or 32 right-hand sides");
    static_assert(HALVES == 1 || ROWS == 128, "pairs of 32-right-hand-side halves");
    static_assert(NS >= 2, "at least two stages");
};

// byte offset of (row r, term k) inside one split part of a stage operand
__device__ __forceinline__ int core_off(int r, int k) {
    return (r >> 3) * kChunkSBO + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

// The split moments of every box in stage layout: image[((box * nrc + rc) * NKC + kc)] holds
// A_hi then A_lo of right-hand sides rc*RC.. and terms kc*16..; rows of right-hand sides at
// or beyond the active count and terms beyond NT are zero.  One thread per 16 bytes of A_hi.
template <int P, int RC>
__global__ void tc_image_kernel(int64_t nbox, int B, int nrc, const float4 *__restrict__ mom,
                                unsigned char *__restrict__ img, const int *nact) {
    using S = TcShape<P, RC>;
    constexpr int per_chunk = S::A_CH / 16;
    const int Bact = nact ? *nact : B;
    const int64_t total = nbox * nrc * S::NKC * per_chunk;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / per_chunk;   // (box, rc, kc)
        const int e = (int)(i - c * per_chunk);
        const int kc = (int)(c % S::NKC);
        const int64_t brc = c / S::NKC;
        const int rc = (int)(brc % nrc);
        const int64_t box = brc / nrc;
        // e enumerates the part's 16-byte segments in address order
        const int r = ((e >> 3) / (kKC / 4)) * 8 + (e & 7), k4 = (e >> 3) % (kKC / 4);
        const int j = rc * RC + (r >> 2), cpt = r & 3;
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = kc * kKC + 4 * k4 + u;
            float x = 0.f;
            if (t < S::NT && j < Bact) x = __ldg((const float *)(mom + (box * S::NT + t) * B + j) + cpt);
            v[u] = x;
        }
        const TfPair sp = tf32_split(make_float4(v[0], v[1], v[2], v[3]));
        unsigned char *dst = img + c * (2 * S::A_CH) + 16 * e;
        *(float4 *)dst = sp.hi;
        *(float4 *)(dst + S::A_CH) = sp.lo;
    }
}

template <int P, int RC>
__global__ void __launch_bounds__(kTcThreads, 1)
    m2p_tc_kernel(const int4 *__restrict__ items, int64_t nitems, int B, int nrc, const float4 *__restrict__ tgt,
                  int64_t ntgt, const int2 *__restrict__ list, const float4 *__restrict__ box_c,
                  const unsigned char *__restrict__ img, double *__restrict__ acc, int *counter, int *error,
                  const int *nact) {
    using S = TcShape<P, RC>;
    constexpr int NT = S::NT, NKC = S::NKC, NS = S::NS;
    extern __shared__ __align__(128) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t full_a[NS], full_b[NS], empty_s[NS];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], ring_full[kUnitRing], ring_empty[kUnitRing], drain, gate;
    __shared__ int64_t ring[kUnitRing];
    __shared__ uint32_t tslot;
    __shared__ volatile int abort_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = smem_addr(tc_smem);
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            bar_init(smem_addr(&full_a[s]), 1);      // the producer's expect_tx (+ the copy's bytes)
            bar_init(smem_addr(&full_b[s]), kTcN);   // one arrival per generating thread
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
        // ---- producer: work units and the A part of every stage
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
                const int rc = (int)(u - ii * nbc);
                const int4 item = __ldg(items + ii);
                bool ok = true;
                int b_nx = item.y < item.z ? __ldg(&list[item.y].x) : 0;   // one box ahead
                // A parts present: the halves of the unit holding right-hand sides in use
                const int nh = min(S::HALVES, (Bact - rc * RC + S::HRC - 1) / S::HRC);
                for (int l = item.y; l < item.z && ok; ++l) {
                    const unsigned char *src = img + ((int64_t)b_nx * nrc + rc * S::HALVES) * NKC * (2 * S::A_CH);
                    if (l + 1 < item.z) b_nx = __ldg(&list[l + 1].x);
                    for (int kc = 0; kc < NKC; ++kc, ++seq) {
                        const int s = (int)(seq % NS);
                        if (seq >= NS &&
                            !bar_wait(smem_addr(&empty_s[s]), (uint32_t)((seq / NS) - 1) & 1u, &abort_s)) {
                            ok = false;
                            break;
                        }
                        const uint32_t fb = smem_addr(&full_a[s]);
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                     "r"((uint32_t)(nh * 2 * S::A_CH))
                                     : "memory");
                        for (int h = 0; h < nh; ++h)
                            asm volatile(
                                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                    sbase + (uint32_t)(s * S::STAGE + h * 2 * S::A_CH)),
                                "l"(src + ((int64_t)h * NKC + kc) * 2 * S::A_CH), "r"(2 * S::A_CH), "r"(fb)
                                : "memory");
                    }
                }
                if (!ok) break;
            }
            // the copies of the last NS armed stages may still be in flight
            for (int64_t k = seq > NS ? seq - NS : 0; k < seq; ++k)
                drain_wait(smem_addr(&full_a[k % NS]), (uint32_t)(k / NS) & 1u);
        }
    } else if (warp == kMmaWarp) {
        // ---- MMA issue: one lane
        if (lane == 0) {
            int64_t seq = 0;
            int nu = 0;   // non-empty units so far (accumulator = nu & 1; pairs: both, every unit)
            for (int uc = 0;; ++uc) {
                const int slot = uc % kUnitRing;
                if (!bar_wait(smem_addr(&ring_full[slot]), (uint32_t)(uc / kUnitRing) & 1u, &abort_s)) break;
                const int64_t u = ring[slot];
                if (u >= units) break;
                const int4 item = __ldg(items + u / nbc);
                if (item.y < item.z) {
                    const int ab = S::HALVES == 2 ? 0 : (nu & 1);
                    const bool wait = S::HALVES == 2 ? nu >= 1 : nu >= 2;
                    const uint32_t wpar = (uint32_t)(S::HALVES == 2 ? (nu - 1) : ((nu >> 1) - 1)) & 1u;
                    if (wait && !bar_wait(smem_addr(&acc_empty[ab]), wpar, &abort_s)) break;
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t d = tmem + (uint32_t)(ab * kTcN);
                    const int rc = (int)(u % nbc);
                    const int nh = min(S::HALVES, (Bact - rc * RC + S::HRC - 1) / S::HRC);
                    bool ok = true;
                    for (int l = item.y; l < item.z && ok; ++l) {
                        for (int kc = 0; kc < NKC; ++kc, ++seq) {
                            const int s = (int)(seq % NS);
                            const uint32_t par = (uint32_t)(seq / NS) & 1u;
                            if (!bar_wait(smem_addr(&full_a[s]), par, &abort_s) ||
                                !bar_wait(smem_addr(&full_b[s]), par, &abort_s)) {
                                ok = false;
                                break;
                            }
                            asm volatile("tcgen05.fence::after_thread_sync;");
                            const uint32_t st = sbase + (uint32_t)(s * S::STAGE);
                            const int ksteps = (min(kKC, NT - kc * kKC) + 7) / 8;
                            for (int ks = 0; ks < ksteps; ++ks) {
                                const uint32_t off = ks * 256;   // two 16-byte column groups per K step of 8
                                const uint64_t dbh = umma_desc(st + S::OFF_B + off, 128, kChunkSBO);
                                const uint64_t dbl = umma_desc(st + S::OFF_B + S::B_CH + off, 128, kChunkSBO);
                                const uint32_t on = (l == item.y && kc == 0 && ks == 0) ? 0u : 1u;
                                for (int h = 0; h < nh; ++h) {   // half h into accumulator d + h kTcN
                                    const uint32_t ah = st + (uint32_t)(h * 2 * S::A_CH);
                                    const uint64_t dah = umma_desc(ah + off, 128, kChunkSBO);
                                    const uint64_t dal = umma_desc(ah + S::A_CH + off, 128, kChunkSBO);
                                    const uint32_t dh = d + (uint32_t)(h * kTcN);
                                    tc_mma(dh, dah, dbh, S::IDESC, on);
                                    tc_mma(dh, dah, dbl, S::IDESC, 1u);
                                    if (!S::STACKED) tc_mma(dh, dal, dbh, S::IDESC, 1u);
                                }
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
        // ---- generators (one thread per target of the group); each unit's epilogue is
        // taken once the first box of the next unit is staged, so that the MMAs keep going
        const int blk = tid / kTargetBlock;   // block of the group this thread's target is in
        int64_t seq = 0;
        int nu = 0;
        // the unit whose accumulator is still to be drained
        bool pend = false;
        int p_ab = 0, p_par = 0, p_b0 = 0, p_nb = 0;
        int64_t p_tbase = 0;
        // epilogue: warp w reads lane quarter w % 4 (accumulator rows 32 (w % 4)..) and columns
        // 128 (w / 4)..; channel = row mod ROWS (both halves of a stacked accumulator are
        // added); false: a wait ran out
        auto drain_acc = [&]() -> bool {
            const int qd = warp & 3, half = warp >> 2;
            if (!warp_wait(smem_addr(&acc_full[p_ab]), (uint32_t)p_par, &abort_s)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
            for (int hh = 0; hh < S::HALVES; ++hh) {   // the unit's A parts (accumulators)
            const int hnb = p_nb - hh * S::HRC;          // right-hand sides of this half
            if ((32 * qd) % S::ROWS < 4 * hnb) {
                const int m = (32 * qd + lane) % S::ROWS, j = m >> 2, cpt = m & 3;
                const int jb = p_b0 + hh * S::HRC + j;   // the right-hand side of row m
#pragma unroll 1
                for (int c0 = 0; c0 < kTcN / 2; c0 += 32) {
                    const int64_t tc = p_tbase + half * (kTcN / 2) + c0 + lane;   // this lane's column's target
                    const int pc = tc < ntgt ? panel_of(tgt[tc].w) : -1;
#pragma unroll
                    for (int h16 = 0; h16 < 32; h16 += 16) {
                        uint32_t v[16];
                        const uint32_t addr = tmem + ((uint32_t)(32 * qd) << 16) +
                                              (uint32_t)((p_ab + hh) * kTcN + half * (kTcN / 2) + c0 + h16);
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
                            if (j < hnb && p >= 0)
                                atomicAdd(acc + 4 * ((int64_t)p * B + jb) + cpt, (double)__uint_as_float(v[x]));
                        }
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
            int ustage = 0;   // stages of this unit written so far
            const int64_t ti = tbase + tid;
            const bool live = ti < ntgt;
            const float4 q = live ? tgt[ti] : tgt[0];
            // the next box's list entry and centre are loaded one box ahead
            int2 e_nx = item.y < item.z ? __ldg(list + item.y) : make_int2(0, 0);
            float4 c_nx = item.y < item.z ? box_c[e_nx.x] : make_float4(0.f, 0.f, 0.f, 0.f);
            for (int l = item.y; l < item.z && ok; ++l) {
                const int2 e = e_nx;
                const float4 c = c_nx;
                if (l + 1 < item.z) {
                    e_nx = __ldg(list + l + 1);
                    c_nx = box_c[e_nx.x];
                }
                const bool on = live && ((e.y >> blk) & 1);   // uniform over the warp but for the tail
                float a[NT];
                if (on) {
                    constexpr MultiIndex<P> mi{};
                    const float R[3] = {q.x - c.x, q.y - c.y, q.z - c.z};
                    a[0] = rsq(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
                    const float ir2 = a[0] * a[0];
#pragma unroll
                    for (int t = 1; t < NT; ++t) {
                        const int n = mi.deg[t];
                        float s1 = 0.f, s2 = 0.f;
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            if (mi.m1[t][d] >= 0) s1 += R[d] * a[mi.m1[t][d]];
                            if (mi.m2[t][d] >= 0) s2 += a[mi.m2[t][d]];
                        }
                        const float c1 = (float)(-(2.0 * n - 1.0) / n), c2 = (float)(-(n - 1.0) / n);
                        a[t] = (c1 * s1 + c2 * s2) * ir2;
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < NT; ++t) a[t] = 0.f;
                }
#pragma unroll
                for (int kc = 0; kc < NKC; ++kc) {
                    // pairs hold both accumulators per unit: the previous unit is drained before
                    // this unit's stage NS, whose slot the MMAs of its first stage must free
                    if (S::HALVES == 2 && pend && ustage >= NS && !(ok = drain_acc())) break;
                    ++ustage;
                    const int s = (int)(seq % NS);
                    if (seq >= NS && !warp_wait(smem_addr(&empty_s[s]), (uint32_t)((seq / NS) - 1) & 1u, &abort_s)) {
                        ok = false;
                        break;
                    }
                    unsigned char *bh = tc_smem + s * S::STAGE + S::OFF_B, *bl = bh + S::B_CH;
                    // four terms per 16-byte store: the eight lanes of a quarter warp fill one
                    // core matrix, free of bank conflicts
#pragma unroll
                    for (int t4 = 0; t4 < kKC / 4; ++t4) {
                        float v[4];
#pragma unroll
                        for (int w = 0; w < 4; ++w) {
                            const int t = kc * kKC + 4 * t4 + w;
                            v[w] = t < NT ? a[t < NT ? t : 0] : 0.f;
                        }
                        const TfPair sp = tf32_split(make_float4(v[0], v[1], v[2], v[3]));
                        *(float4 *)(bh + core_off(tid, 4 * t4)) = sp.hi;
                        *(float4 *)(bl + core_off(tid, 4 * t4)) = sp.lo;
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    bar_arrive(smem_addr(&full_b[s]));
                    ++seq;
                }
                if (ok && pend) ok = drain_acc();   // the previous unit, behind this unit's first box
            }
            if (ok && pend) ok = drain_acc();       // the previous unit, if this one had no box
            if (!ok) break;
            if (item.y < item.z) {
                pend = true;
                p_ab = S::HALVES == 2 ? 0 : (nu & 1);
                p_par = (S::HALVES == 2 ? nu : (nu >> 1)) & 1;
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

template <int P, int RC>
int tc_launch(lspr_ctx *ctx, double *acc, int *counter, int B) {
    using S = TcShape<P, RC>;
    static int smem_set[kSmemDevices] = {};
    Tree &tr = ctx->tree;
    if (tr.n_tc_items == 0) return LSPR_OK;
    const int nrc = (B + S::HRC - 1) / S::HRC;   // A parts of 16 or 32 right-hand sides in the image
    const int nunit = (B + RC - 1) / RC;          // work units per group item
    const int64_t segs = tr.nboxes * nrc * S::NKC * (S::A_CH / 16);
    LSPR_TRY(ctx, ctx->tc_img.ensure((size_t)segs * 32));
    if (!ctx->dev_err.p) return LSPR_E_STATE;
    LSPR_TRY(ctx, allow_smem(m2p_tc_kernel<P, RC>, S::SMEM, ctx->device, smem_set));
    ++ctx->n_launches;   // the image; the caller counts the M2P launch
    const unsigned gi =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>((segs + 255) / 256, 8 * std::max(1, ctx->num_sms)));
    tc_image_kernel<P, S::HRC><<<gi, 256, 0, ctx->stream>>>(tr.nboxes, B, nrc, Views<float>::mom(ctx),
                                                              ctx->tc_img.p, ctx->rhs_nact);
    const unsigned grid =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>(tr.n_tc_items * nunit, std::max(1, ctx->num_sms)));
    m2p_tc_kernel<P, RC><<<grid, kTcThreads, S::SMEM, ctx->stream>>>(
        tr.tc_items.p, tr.n_tc_items, B, nrc, Views<float>::tgt(ctx), ctx->mesh.N, tr.tc_list.p,
        Views<float>::bc(ctx), ctx->tc_img.p, acc, counter, ctx->dev_err.p, ctx->rhs_nact);
    return LSPR_OK;
}

template <int P>
int tc_launch_p(lspr_ctx *ctx, double *acc, int *counter, int B) {
    return B <= 16 ? tc_launch<P, 16>(ctx, acc, counter, B)
                   : (B <= 32 ? tc_launch<P, 32>(ctx, acc, counter, B) : tc_launch<P, 64>(ctx, acc, counter, B));
}

}  // namespace

// FP32 M2P of B >= 2 right-hand sides on the tensor cores; LSPR_E_STATE: not applicable
int m2p_tc_launch(lspr_ctx *ctx, double *acc, int *counter, int B) {
    if (!ctx->tree.tc_built) LSPR_TRY_ST(tree_tc_lists(ctx, false));
    switch (ctx->tree.P) {
    case 1: return tc_launch_p<1>(ctx, acc, counter, B);
    case 2: return tc_launch_p<2>(ctx, acc, counter, B);
    case 3: return tc_launch_p<3>(ctx, acc, counter, B);
    case 4: return tc_launch_p<4>(ctx, acc, counter, B);
    case 5: return tc_launch_p<5>(ctx, acc, counter, B);
    case 6: return tc_launch_p<6>(ctx, acc, counter, B);
    case 7: return tc_launch_p<7>(ctx, acc, counter, B);
    case 8: return tc_launch_p<8>(ctx, acc, counter, B);
    default: return LSPR_E_STATE;
    }
}

}  // namespace lspr
