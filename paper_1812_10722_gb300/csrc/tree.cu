// Treecode structures (Sec. II.D): the octree over the Gauss-node sources with at
// most N_crit sources per leaf, and per block of 64 collocation targets the list of
// boxes accepted by the multipole-acceptance criterion r_b < theta * r (Taylor
// expansion, M2P) and of leaves summed directly (P2P).
//
// Device pipeline: bounding cube -> 30-bit Morton keys (10 bits per axis) ->
// LSD radix sort (4-bit digits, stable) of sources and targets -> permuted
// work-order arrays -> octree, level by level in one CTA (deterministic box
// numbering) -> box centres (centre of the sources' bounding box) and radii
// r_b = max |y - c| -> target-block bounding boxes -> interaction lists (count,
// scan, fill; one thread per target block walks the tree depth first).
#include <algorithm>
#include <cstdlib>
#include <cmath>

#include "lspr_internal.cuh"
#include "tc_lists.h"

namespace lspr {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kDigitBits = 4;
constexpr int kDigits = 1 << kDigitBits;
constexpr int kP2PChunk = 256;      // sources per P2P work item (upper bound)
constexpr int kM2PSeg = 16;         // boxes per M2P work item
constexpr int kP2MChunk = 512;      // sources per P2M work item
constexpr int kStack = 96;
constexpr int kGeomThreads = 256;

// ------------------------------------------------------------ bounding cube
// two stages: kBoxBlocks blocks reduce slices of the points into part[block][6], then one
// block reduces the partials into out = (lo[3], hi[3])
constexpr int kBoxBlocks = 128;
__global__ void bbox_partial_kernel(const dbl4 *__restrict__ a, int64_t na, const dbl4 *__restrict__ b, int64_t nb,
                                    double *part) {
    __shared__ double red[6][256];
    const int t = threadIdx.x;
    double l[3] = {1e300, 1e300, 1e300}, h[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + t; i < na + nb; i += (int64_t)gridDim.x * blockDim.x) {
        const dbl4 p = i < na ? a[i] : b[i - na];
        l[0] = fmin(l[0], p.x); l[1] = fmin(l[1], p.y); l[2] = fmin(l[2], p.z);
        h[0] = fmax(h[0], p.x); h[1] = fmax(h[1], p.y); h[2] = fmax(h[2], p.z);
    }
    for (int d = 0; d < 3; ++d) { red[d][t] = l[d]; red[3 + d][t] = h[d]; }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s)
            for (int d = 0; d < 3; ++d) {
                red[d][t] = fmin(red[d][t], red[d][t + s]);
                red[3 + d][t] = fmax(red[3 + d][t], red[3 + d][t + s]);
            }
        __syncthreads();
    }
    if (t == 0)
        for (int q = 0; q < 6; ++q) part[blockIdx.x * 6 + q] = red[q][0];
}

__global__ void bbox_final_kernel(const double *part, int nparts, double *out) {
    const int q = threadIdx.x;
    if (q >= 6) return;
    double v = q < 3 ? 1e300 : -1e300;
    for (int k = 0; k < nparts; ++k) v = q < 3 ? fmin(v, part[k * 6 + q]) : fmax(v, part[k * 6 + q]);
    out[q] = v;
}

// key bit 3l+2 / 3l+1 / 3l = x / y / z bit l, so the top triple selects the octant
__global__ void morton_kernel(const dbl4 *__restrict__ p, int64_t n, const double *cube /* lo[3], size */,
                              unsigned *keys, int *vals) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const dbl4 q = p[i];
    const double inv = 1024.0 / cube[3];
    unsigned ix = (unsigned)min(1023.0, fmax(0.0, floor((q.x - cube[0]) * inv)));
    unsigned iy = (unsigned)min(1023.0, fmax(0.0, floor((q.y - cube[1]) * inv)));
    unsigned iz = (unsigned)min(1023.0, fmax(0.0, floor((q.z - cube[2]) * inv)));
    keys[i] = (spread10(ix) << 2) | (spread10(iy) << 1) | spread10(iz);
    vals[i] = (int)i;
}

// ----------------------------------------------------------------- radix sort
__global__ void radix_hist_kernel(const unsigned *__restrict__ keys, int64_t n, int shift, int nblocks, int *hist) {
    __shared__ int cnt[kDigits];
    if (threadIdx.x < kDigits) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int k = threadIdx.x; k < kSortTile; k += blockDim.x) {
        const int64_t i = base + k;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & (kDigits - 1)], 1);
    }
    __syncthreads();
    if (threadIdx.x < kDigits) hist[threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// exclusive scan of an int array (single block, any length)
__global__ void scan_int_kernel(const int *in, int64_t n, int *out, int64_t *total) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t b = t * per, e = min(n, b + per);
    int64_t s = 0;
    for (int64_t k = b; k < e; ++k) s += in[k];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        int64_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = part[t] - s;
    for (int64_t k = b; k < e; ++k) {
        out[k] = (int)run;
        run += in[k];
    }
    if (t == blockDim.x - 1 && total) *total = part[t];
}

__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const unsigned *__restrict__ kin,
                                                                     const int *__restrict__ vin, int64_t n, int shift,
                                                                     int nblocks, const int *__restrict__ offs,
                                                                     unsigned *kout, int *vout) {
    __shared__ int cnt[kDigits * kSortThreads];
    __shared__ int tsum[kSortThreads];
    const int t = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)t * kSortItems;
    unsigned k[kSortItems];
    int v[kSortItems];
    for (int d = 0; d < kDigits; ++d) cnt[d * kSortThreads + t] = 0;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int64_t i = base + j;
        k[j] = i < n ? kin[i] : 0u;
        v[j] = i < n ? vin[i] : 0;
        if (i < n) cnt[((k[j] >> shift) & (kDigits - 1)) * kSortThreads + t] += 1;
    }
    __syncthreads();
    // exclusive scan over cnt in digit-major order (each thread owns kDigits consecutive entries)
    int own[kDigits];
    int s = 0;
#pragma unroll
    for (int j = 0; j < kDigits; ++j) {
        own[j] = cnt[t * kDigits + j];
        s += own[j];
    }
    tsum[t] = s;
    __syncthreads();
    for (int off = 1; off < kSortThreads; off <<= 1) {
        int x = t >= off ? tsum[t - off] : 0;
        __syncthreads();
        tsum[t] += x;
        __syncthreads();
    }
    int run = tsum[t] - s;
#pragma unroll
    for (int j = 0; j < kDigits; ++j) {
        cnt[t * kDigits + j] = run;
        run += own[j];
    }
    __syncthreads();
    int local[kDigits];
#pragma unroll
    for (int d = 0; d < kDigits; ++d) local[d] = 0;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int64_t i = base + j;
        if (i >= n) continue;
        const int d = (k[j] >> shift) & (kDigits - 1);
        int r = 0;
#pragma unroll
        for (int q = 0; q < kDigits; ++q)
            if (q == d) { r = local[q]; local[q] = r + 1; }
        const int pos = offs[d * nblocks + blockIdx.x] + (cnt[d * kSortThreads + t] - cnt[d * kSortThreads]) + r;
        kout[pos] = k[j];
        vout[pos] = v[j];
    }
}

// sorts (keys, vals) of length n in place using the given scratch
int64_t radix_sort_scratch_ints(int64_t n) { return kDigits * ((n + kSortTile - 1) / kSortTile); }

int radix_sort(lspr_ctx *ctx, unsigned *keys, int *vals, unsigned *ktmp, int *vtmp, int64_t n, int bits,
                      int *hist, int *offs) {
    const int nblocks = (int)((n + kSortTile - 1) / kSortTile);
    cudaStream_t st = ctx->stream;
    unsigned *ka = keys, *kb = ktmp;
    int *va = vals, *vb = vtmp;
    const int passes = (bits + kDigitBits - 1) / kDigitBits;
    for (int p = 0; p < passes; ++p) {
        const int shift = p * kDigitBits;
        ++ctx->n_launches;
        radix_hist_kernel<<<nblocks, kSortThreads, 0, st>>>(ka, n, shift, nblocks, hist);
        ++ctx->n_launches;
        scan_int_kernel<<<1, 1024, 0, st>>>(hist, (int64_t)kDigits * nblocks, offs, nullptr);
        ++ctx->n_launches;
        radix_scatter_kernel<<<nblocks, kSortThreads, 0, st>>>(ka, va, n, shift, nblocks, offs, kb, vb);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    LSPR_TRY(ctx, cudaGetLastError());
    if (ka != keys) {
        LSPR_TRY(ctx, cudaMemcpyAsync(keys, ka, sizeof(unsigned) * n, cudaMemcpyDeviceToDevice, st));
        LSPR_TRY(ctx, cudaMemcpyAsync(vals, va, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
    }
    return LSPR_OK;
}

__global__ void permute_sources_kernel(int64_t Ns, const int *__restrict__ perm, const dbl4 *__restrict__ pos,
                                       const dbl4 *__restrict__ nrm, dbl4 *spos64, dbl4 *snrm64,
                                       float4 *spos32, float4 *snrm32, int *src_panel) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= Ns) return;
    const int o = perm[s];
    const dbl4 p = pos[o], n = nrm[o];
    const int pid = (int)n.w;
    spos64[s] = p;
    snrm64[s] = n;
    spos32[s] = make_float4((float)p.x, (float)p.y, (float)p.z, (float)p.w);
    snrm32[s] = make_float4((float)n.x, (float)n.y, (float)n.z, __int_as_float(pid));
    src_panel[s] = pid;
}

__global__ void permute_targets_kernel(int64_t N, const int *__restrict__ perm, const dbl4 *__restrict__ tgt,
                                       dbl4 *tgt64, float4 *tgt32, int *tgt_panel, int *tgt_pos) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int o = perm[i];
    const dbl4 t = tgt[o];
    tgt64[i] = t;
    tgt32[i] = make_float4((float)t.x, (float)t.y, (float)t.z, __int_as_float(o));
    tgt_panel[i] = o;
    tgt_pos[o] = (int)i;
}

__global__ void src_tblock_kernel(int64_t Ns, const int *__restrict__ src_panel, const int *__restrict__ tgt_pos,
                                  int *src_tblock) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= Ns) return;
    src_tblock[s] = tgt_pos[src_panel[s]] / kTargetBlock;
}

// --------------------------------------------------------------------- octree
__device__ int lower_bound_key(const unsigned *keys, int lo, int hi, unsigned v) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (keys[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// block-wide exclusive scan of n ints in place (blockDim.x == 1024); returns the total
__device__ int block_scan_inplace(int *a, int n, int *sh) {
    int carry = 0;
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < n ? a[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < (int)blockDim.x; off <<= 1) {
            int x = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
            __syncthreads();
            sh[threadIdx.x] += x;
            __syncthreads();
        }
        if (i < n) a[i] = carry + sh[threadIdx.x] - v;
        const int tot = sh[blockDim.x - 1];
        __syncthreads();
        carry += tot;
    }
    return carry;
}

// One CTA, level by level.  Box b covers keys [beg, end) sharing the top 3*level
// bits; it is split into its non-empty octants while it holds more than ncrit
// sources and is above the maximum depth.  Children of a box are contiguous and
// ordered by octant; boxes are numbered level by level (deterministic).
__global__ void __launch_bounds__(1024) octree_kernel(const unsigned *__restrict__ keys, int Ns, int ncrit, int cap,
                                                      int *beg, int *end, int *child, int *nchild, int *level,
                                                      unsigned *bkey, int *scratch, int *out_nboxes) {
    __shared__ int sh[1024];
    __shared__ int s_lb, s_le, s_overflow;
    if (threadIdx.x == 0) {
        beg[0] = 0; end[0] = Ns; level[0] = 0; bkey[0] = 0u; child[0] = -1; nchild[0] = 0;
        s_lb = 0; s_le = 1; s_overflow = 0;
    }
    __syncthreads();
    for (int l = 0; l < kMaxDepth; ++l) {
        const int lb = s_lb, le = s_le;
        if (lb == le) break;
        const int shift = 3 * (kMaxDepth - 1 - l);
        // count non-empty children
        for (int b = lb + threadIdx.x; b < le; b += blockDim.x) {
            int c = 0;
            if (end[b] - beg[b] > ncrit) {
                for (int o = 0; o < 8; ++o) {
                    const unsigned p = (bkey[b] << 3) | o;
                    const int s0 = lower_bound_key(keys, beg[b], end[b], p << shift);
                    const int s1 = lower_bound_key(keys, s0, end[b], (p + 1) << shift);
                    c += s1 > s0;
                }
            }
            scratch[b - lb] = c;
        }
        __syncthreads();
        const int total = block_scan_inplace(scratch, le - lb, sh);
        if (le + total > cap) {
            if (threadIdx.x == 0) s_overflow = 1;
            __syncthreads();
            break;
        }
        for (int b = lb + threadIdx.x; b < le; b += blockDim.x) {
            int pos = le + scratch[b - lb];
            child[b] = -1;
            nchild[b] = 0;
            if (end[b] - beg[b] > ncrit) {
                int first = pos;
                for (int o = 0; o < 8; ++o) {
                    const unsigned p = (bkey[b] << 3) | o;
                    const int s0 = lower_bound_key(keys, beg[b], end[b], p << shift);
                    const int s1 = lower_bound_key(keys, s0, end[b], (p + 1) << shift);
                    if (s1 > s0) {
                        beg[pos] = s0; end[pos] = s1; level[pos] = l + 1; bkey[pos] = p;
                        child[pos] = -1; nchild[pos] = 0;
                        ++pos;
                    }
                }
                child[b] = first;
                nchild[b] = pos - first;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) { s_lb = le; s_le = le + total; }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out_nboxes = s_overflow ? -1 : s_le;
}

// Centre of the bounding box of the box's sources and r_b = max distance to it, from
// the FP32 source copies (FP64 min/max would run on the narrow FP64 pipe of a single
// block for the root).  The radius is enlarged to cover the FP32 rounding of the
// coordinates (<= 2^-24 |y| each) and of the distance itself, so it bounds the true one.
__global__ void box_geometry_kernel(int nboxes, const int *beg, const int *end, const float4 *__restrict__ spos,
                                    dbl4 *c64, float4 *c32) {
    __shared__ float red[6][kGeomThreads];
    __shared__ float cen[3];
    const int b = blockIdx.x;
    if (b >= nboxes) return;
    const int t = threadIdx.x;
    float l[3] = {3e38f, 3e38f, 3e38f}, h[3] = {-3e38f, -3e38f, -3e38f};
    for (int s = beg[b] + t; s < end[b]; s += blockDim.x) {
        const float4 p = spos[s];
        l[0] = fminf(l[0], p.x); l[1] = fminf(l[1], p.y); l[2] = fminf(l[2], p.z);
        h[0] = fmaxf(h[0], p.x); h[1] = fmaxf(h[1], p.y); h[2] = fmaxf(h[2], p.z);
    }
    for (int d = 0; d < 3; ++d) { red[d][t] = l[d]; red[3 + d][t] = h[d]; }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s)
            for (int d = 0; d < 3; ++d) {
                red[d][t] = fminf(red[d][t], red[d][t + s]);
                red[3 + d][t] = fmaxf(red[3 + d][t], red[3 + d][t + s]);
            }
        __syncthreads();
    }
    if (t == 0)
        for (int d = 0; d < 3; ++d) cen[d] = 0.5f * (red[d][0] + red[3 + d][0]);
    __syncthreads();
    float r2 = 0.f, ymax = 0.f;
    for (int s = beg[b] + t; s < end[b]; s += blockDim.x) {
        const float4 p = spos[s];
        const float dx = p.x - cen[0], dy = p.y - cen[1], dz = p.z - cen[2];
        r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
        ymax = fmaxf(ymax, fmaxf(fabsf(p.x), fmaxf(fabsf(p.y), fabsf(p.z))));
    }
    __syncthreads();
    red[0][t] = r2;
    red[1][t] = ymax;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s) {
            red[0][t] = fmaxf(red[0][t], red[0][t + s]);
            red[1][t] = fmaxf(red[1][t], red[1][t + s]);
        }
        __syncthreads();
    }
    if (t == 0) {
        const double rb = (double)sqrtf(red[0][0]) * (1.0 + 1e-6) + 4e-7 * (double)red[1][0];
        c64[b] = make_dbl4(cen[0], cen[1], cen[2], rb);
        c32[b] = make_float4(cen[0], cen[1], cen[2], (float)(rb * (1.0 + 1e-6)));
    }
}

__global__ void tblock_bbox_kernel(int64_t ntb, int64_t N, const dbl4 *__restrict__ tgt, dbl4 *lo, dbl4 *hi) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= ntb) return;
    double l[3] = {1e300, 1e300, 1e300}, h[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = b * kTargetBlock; i < min(N, (b + 1) * kTargetBlock); ++i) {
        const dbl4 p = tgt[i];
        l[0] = fmin(l[0], p.x); l[1] = fmin(l[1], p.y); l[2] = fmin(l[2], p.z);
        h[0] = fmax(h[0], p.x); h[1] = fmax(h[1], p.y); h[2] = fmax(h[2], p.z);
    }
    lo[b] = make_dbl4(l[0], l[1], l[2], 0);
    hi[b] = make_dbl4(h[0], h[1], h[2], 0);
}

// Multipole-acceptance test of box (c, r_b) against a target block's bounding box:
// r = distance from c to the nearest point of the block.  Accepted iff
// r_b < theta * r and the box keeps clear of every target's own panel and of its
// near-singular panels (r - r_b > clear), so that those stay in direct sums.
__device__ __forceinline__ bool mac_accept(const dbl4 &c, const dbl4 &lo, const dbl4 &hi, double theta,
                                           double clear) {
    const double dx = fmax(0.0, fmax(lo.x - c.x, c.x - hi.x));
    const double dy = fmax(0.0, fmax(lo.y - c.y, c.y - hi.y));
    const double dz = fmax(0.0, fmax(lo.z - c.z, c.z - hi.z));
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    return c.w < theta * r && r - c.w > clear;
}

// One warp per target block walks the tree depth first.  A popped box is known to be
// rejected by the MAC: a leaf becomes a direct (P2P) source range, merged with the
// previous range when contiguous; for an internal box the lanes test its children in
// parallel, accepted children join the block's M2P list and rejected ones are pushed in
// reverse octant order, so leaves come out in Morton order.
// FILL = false: count P2P items, M2P boxes and M2P items per target block.
// FILL = true: write them at the scanned offsets and mark accepted boxes as used.
constexpr int kListWarps = 4;
template <bool FILL>
__global__ void __launch_bounds__(kListWarps * 32) lists_kernel(
    int64_t ntb, int64_t N, const dbl4 *lo, const dbl4 *hi, const dbl4 *__restrict__ bc,
    const int *__restrict__ beg, const int *__restrict__ end, const int *__restrict__ child,
    const int *__restrict__ nchild, double theta, double clear, int *n_p2p, int *n_m2p, int *n_m2pi,
    const int *o_p2p, const int *o_m2p, const int *o_m2pi, int4 *p2p_items, int *m2p_list, int4 *m2p_items,
    int *used, unsigned long long *pairs, int *overflow) {
    __shared__ int stk[kListWarps][kStack];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t tb = (int64_t)blockIdx.x * kListWarps + warp;
    if (tb >= ntb) return;
    int *stack = stk[warp];
    const dbl4 l = lo[tb], h = hi[tb];
    const int ntgt = (int)min((int64_t)kTargetBlock, N - tb * kTargetBlock);
    if (lane == 0) stack[0] = 0;
    __syncwarp();
    int sp = 1;
    int np = 0, nm = 0;
    int cur_b = -1, cur_e = -1;   // pending merged P2P range
    int p_out = FILL ? o_p2p[tb] : 0, m_out = FILL ? o_m2p[tb] : 0;
    unsigned long long pp = 0;
    auto flush = [&](int b0, int e0) {
        const int n = e0 - b0;
        const int k = (n + kP2PChunk - 1) / kP2PChunk;
        for (int q = 0; q < k; ++q) {
            const int s0 = b0 + (int)((int64_t)n * q / k), s1 = b0 + (int)((int64_t)n * (q + 1) / k);
            if (FILL && lane == 0) p2p_items[p_out] = make_int4((int)tb, s0, s1, 0);
            ++p_out;
        }
        np += k;
        pp += (unsigned long long)n * ntgt;
    };
    bool ovf = false;
    while (sp > 0) {
        const int b = stack[--sp];
        __syncwarp();
        const int nc = nchild[b];
        if (nc == 0) {
            if (cur_e == beg[b]) {
                cur_e = end[b];
            } else {
                if (cur_b >= 0) flush(cur_b, cur_e);
                cur_b = beg[b];
                cur_e = end[b];
            }
            continue;
        }
        int ch = -1;
        bool acc = false, push = false;
        if (lane < nc) {
            ch = child[b] + lane;
            acc = mac_accept(bc[ch], l, h, theta, clear);
            push = !acc;
        }
        const unsigned am = __ballot_sync(0xffffffffu, acc), pm = __ballot_sync(0xffffffffu, push);
        const unsigned below = (1u << lane) - 1u;
        if (FILL && acc) {
            m2p_list[m_out + __popc(am & below)] = ch;
            used[ch] = 1;
        }
        m_out += __popc(am);
        nm += __popc(am);
        const int npush = __popc(pm);
        if (sp + npush > kStack) {
            ovf = true;
            break;
        }
        if (push) stack[sp + npush - 1 - __popc(pm & below)] = ch;
        __syncwarp();
        sp += npush;
    }
    if (ovf) {
        if (lane == 0) atomicOr(overflow, 1);
        return;
    }
    if (cur_b >= 0) flush(cur_b, cur_e);
    const int nmi = (nm + kM2PSeg - 1) / kM2PSeg;
    if (lane != 0) return;
    if (!FILL) {
        n_p2p[tb] = np;
        n_m2p[tb] = nm;
        n_m2pi[tb] = nmi;
        atomicAdd(pairs, pp);
    } else {
        const int base = o_m2p[tb];
        for (int q = 0; q < nmi; ++q) {
            const int s0 = base + q * kM2PSeg, s1 = min(base + nm, s0 + kM2PSeg);
            m2p_items[o_m2pi[tb] + q] = make_int4((int)tb, s0, s1, 0);
        }
    }
}

// --------------------------------------------------------------------- driver
int tree_build(lspr_ctx *ctx, double theta, int P, int Ncrit) {
    Mesh &m = ctx->mesh;
    Tree &tr = ctx->tree;
    WorkOrder &w = ctx->wo;
    cudaStream_t st = ctx->stream;
    tr.ready = false;
    tr.theta = theta;
    tr.P = P;
    tr.Ncrit = Ncrit;
    tr.NT = n_terms(P);
    const int64_t Ns = m.Ns, N = m.N;
    cudaEvent_t ev;
    timer_begin(ctx, T_TREE, &ev);

    Tmp<double> cube(ctx->scratch[0]);
    LSPR_TRY(ctx, cube.ensure(8 + 6 * kBoxBlocks));
    ++ctx->n_launches;
    bbox_partial_kernel<<<kBoxBlocks, 256, 0, st>>>(m.src_pos64.p, Ns, m.tgt64.p, N, cube.p + 8);
    ++ctx->n_launches;
    bbox_final_kernel<<<1, 32, 0, st>>>(cube.p + 8, kBoxBlocks, cube.p);
    double hb[6];
    LSPR_TRY(ctx, cudaMemcpyAsync(hb, cube.p, sizeof(hb), cudaMemcpyDeviceToHost, st));
    LSPR_TRY(ctx, cudaStreamSynchronize(st));
    double size = std::max(hb[3] - hb[0], std::max(hb[4] - hb[1], hb[5] - hb[2]));
    size = size * (1.0 + 1e-6) + 1e-12;
    double hc[4] = {hb[0] - 1e-7 * size, hb[1] - 1e-7 * size, hb[2] - 1e-7 * size, size * (1.0 + 2e-7)};
    LSPR_TRY(ctx, cudaMemcpyAsync(cube.p, hc, sizeof(hc), cudaMemcpyHostToDevice, st));

    // keys and sort
    Tmp<unsigned> keys(ctx->scratch[1]), ktmp(ctx->scratch[2]);
    Tmp<int> vals(ctx->scratch[3]), vtmp(ctx->scratch[4]), hist(ctx->scratch[5]), offs(ctx->scratch[6]);
    const int64_t nmax = std::max(Ns, N);
    LSPR_TRY(ctx, keys.ensure(nmax));
    LSPR_TRY(ctx, ktmp.ensure(nmax));
    LSPR_TRY(ctx, vals.ensure(nmax));
    LSPR_TRY(ctx, vtmp.ensure(nmax));
    const int64_t nblk = (nmax + kSortTile - 1) / kSortTile;
    LSPR_TRY(ctx, hist.ensure(kDigits * nblk));
    LSPR_TRY(ctx, offs.ensure(kDigits * nblk));
    LSPR_TRY(ctx, w.spos64.ensure(Ns));
    LSPR_TRY(ctx, w.snrm64.ensure(Ns));
    LSPR_TRY(ctx, w.spos32.ensure(Ns));
    LSPR_TRY(ctx, w.snrm32.ensure(Ns));
    LSPR_TRY(ctx, w.src_panel.ensure(Ns));
    LSPR_TRY(ctx, w.tgt64.ensure(N));
    LSPR_TRY(ctx, w.tgt32.ensure(N));
    LSPR_TRY(ctx, w.tgt_panel.ensure(N));
    LSPR_TRY(ctx, w.tgt_pos.ensure(N));
    LSPR_TRY(ctx, w.src_tblock.ensure(Ns));

    // targets first (their sorted keys are not kept)
    ++ctx->n_launches;
    morton_kernel<<<grid_for(N, 256), 256, 0, st>>>(m.tgt64.p, N, cube.p, keys.p, vals.p);
    LSPR_TRY_ST(radix_sort(ctx, keys.p, vals.p, ktmp.p, vtmp.p, N, 30, hist.p, offs.p));
    ++ctx->n_launches;
    permute_targets_kernel<<<grid_for(N, 256), 256, 0, st>>>(N, vals.p, m.tgt64.p, w.tgt64.p, w.tgt32.p, w.tgt_panel.p,
                                                              w.tgt_pos.p);
    // sources
    ++ctx->n_launches;
    morton_kernel<<<grid_for(Ns, 256), 256, 0, st>>>(m.src_pos64.p, Ns, cube.p, keys.p, vals.p);
    LSPR_TRY_ST(radix_sort(ctx, keys.p, vals.p, ktmp.p, vtmp.p, Ns, 30, hist.p, offs.p));
    ++ctx->n_launches;
    permute_sources_kernel<<<grid_for(Ns, 256), 256, 0, st>>>(Ns, vals.p, m.src_pos64.p, m.src_nrm64.p, w.spos64.p,
                                                              w.snrm64.p, w.spos32.p, w.snrm32.p, w.src_panel.p);
    ++ctx->n_launches;
    src_tblock_kernel<<<grid_for(Ns, 256), 256, 0, st>>>(Ns, w.src_panel.p, w.tgt_pos.p, w.src_tblock.p);
    LSPR_TRY(ctx, cudaGetLastError());
    // the direct-mode items now address the Morton work order: refresh their own-panel flags
    LSPR_TRY_ST(launch_item_flags(ctx, ctx->direct.items.p, ctx->direct.n));
    LSPR_TRY_ST(launch_ff_geometry(ctx));

    // octree
    const int64_t cap64 = 1 + 8LL * kMaxDepth * (Ns / (Ncrit + 1) + 1);
    const int cap = (int)std::min<int64_t>(cap64, 1 << 30);
    for (DArr<int> *a : {&tr.box_beg, &tr.box_end, &tr.box_child, &tr.box_nchild, &tr.box_level, &tr.box_used})
        LSPR_TRY(ctx, a->ensure(cap));
    LSPR_TRY(ctx, tr.box_key.ensure(cap));
    Tmp<int> scratch(ctx->scratch[7]), nbox_d(ctx->scratch[8]);
    LSPR_TRY(ctx, scratch.ensure(cap));
    LSPR_TRY(ctx, nbox_d.ensure(1));
    ++ctx->n_launches;
    octree_kernel<<<1, 1024, 0, st>>>(keys.p, (int)Ns, Ncrit, cap, tr.box_beg.p, tr.box_end.p, tr.box_child.p,
                                      tr.box_nchild.p, tr.box_level.p, tr.box_key.p, scratch.p, nbox_d.p);
    LSPR_TRY(ctx, cudaGetLastError());
    int nboxes = 0;
    LSPR_TRY(ctx, cudaMemcpyAsync(&nboxes, nbox_d.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    LSPR_TRY(ctx, cudaStreamSynchronize(st));
    if (nboxes <= 0) {
        ctx->last_error = "octree capacity exceeded";
        return LSPR_E_OOM;
    }
    tr.nboxes = nboxes;
    LSPR_TRY(ctx, tr.box_c64.ensure(nboxes));
    LSPR_TRY(ctx, tr.box_c32.ensure(nboxes));
    ++ctx->n_launches;
    box_geometry_kernel<<<nboxes, kGeomThreads, 0, st>>>(nboxes, tr.box_beg.p, tr.box_end.p, w.spos32.p, tr.box_c64.p,
                                                tr.box_c32.p);
    LSPR_TRY_ST(launch_ff_boxes(ctx));

    // target blocks
    const int64_t ntb = (N + kTargetBlock - 1) / kTargetBlock;
    tr.ntblocks = ntb;
    Tmp<dbl4> tlo(ctx->scratch[9]), thi(ctx->scratch[10]);
    LSPR_TRY(ctx, tlo.ensure(ntb));
    LSPR_TRY(ctx, thi.ensure(ntb));
    ++ctx->n_launches;
    tblock_bbox_kernel<<<grid_for(ntb, 128), 128, 0, st>>>(ntb, N, w.tgt64.p, tlo.p, thi.p);

    // lists: count
    const double clear = m.Lmax / m.thr + m.rho_max;
    Tmp<int> cnt3(ctx->scratch[11]), off3(ctx->scratch[12]);
    Tmp<int64_t> tot3(ctx->scratch[13]);
    Tmp<unsigned long long> pairs(ctx->scratch[14]);
    Tmp<int> ovf(ctx->scratch[15]);
    LSPR_TRY(ctx, cnt3.ensure(3 * ntb));
    LSPR_TRY(ctx, off3.ensure(3 * ntb));
    LSPR_TRY(ctx, tot3.ensure(3));
    LSPR_TRY(ctx, pairs.ensure(1));
    LSPR_TRY(ctx, ovf.ensure(1));
    LSPR_TRY(ctx, cudaMemsetAsync(pairs.p, 0, sizeof(unsigned long long), st));
    LSPR_TRY(ctx, cudaMemsetAsync(ovf.p, 0, sizeof(int), st));
    LSPR_TRY(ctx, cudaMemsetAsync(tr.box_used.p, 0, sizeof(int) * nboxes, st));
    ++ctx->n_launches;
    lists_kernel<false><<<grid_for(ntb, kListWarps), kListWarps * 32, 0, st>>>(
        ntb, N, tlo.p, thi.p, tr.box_c64.p, tr.box_beg.p, tr.box_end.p, tr.box_child.p, tr.box_nchild.p, theta, clear,
        cnt3.p, cnt3.p + ntb, cnt3.p + 2 * ntb, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
        pairs.p, ovf.p);
    for (int q = 0; q < 3; ++q) {
        ++ctx->n_launches;
        scan_int_kernel<<<1, 1024, 0, st>>>(cnt3.p + q * ntb, ntb, off3.p + q * ntb, tot3.p + q);
    }
    LSPR_TRY(ctx, cudaGetLastError());
    int64_t tot[3];
    unsigned long long hp = 0;
    int hovf = 0;
    LSPR_TRY(ctx, cudaMemcpyAsync(tot, tot3.p, sizeof(tot), cudaMemcpyDeviceToHost, st));
    LSPR_TRY(ctx, cudaMemcpyAsync(&hp, pairs.p, sizeof(hp), cudaMemcpyDeviceToHost, st));
    LSPR_TRY(ctx, cudaMemcpyAsync(&hovf, ovf.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    LSPR_TRY(ctx, cudaStreamSynchronize(st));
    if (hovf) {
        ctx->last_error = "tree traversal stack overflow";
        return LSPR_E_ARG;
    }
    tr.n_p2p_items = tot[0];
    tr.n_m2p_pairs = tot[1];
    tr.n_m2p_items = tot[2];
    tr.p2p_pairs = (int64_t)hp;
    LSPR_TRY(ctx, tr.p2p_items.ensure(std::max<int64_t>(1, tot[0])));
    LSPR_TRY(ctx, tr.m2p_list.ensure(std::max<int64_t>(1, tot[1])));
    LSPR_TRY(ctx, tr.m2p_items.ensure(std::max<int64_t>(1, tot[2])));
    ++ctx->n_launches;
    lists_kernel<true><<<grid_for(ntb, kListWarps), kListWarps * 32, 0, st>>>(
        ntb, N, tlo.p, thi.p, tr.box_c64.p, tr.box_beg.p, tr.box_end.p, tr.box_child.p, tr.box_nchild.p, theta, clear,
        nullptr, nullptr, nullptr, off3.p, off3.p + ntb, off3.p + 2 * ntb, tr.p2p_items.p, tr.m2p_list.p,
        tr.m2p_items.p, tr.box_used.p, pairs.p, ovf.p);
    LSPR_TRY(ctx, cudaGetLastError());
    LSPR_TRY_ST(launch_item_flags(ctx, tr.p2p_items.p, tr.n_p2p_items));

    // P2M work: the leaves with an accepted box among themselves or their ancestors; each
    // leaf chunk's moments are shifted into every accepted ancestor inside the P2M kernel
    // (host side: a few thousand boxes).
    std::vector<int> hbeg(nboxes), hend(nboxes), hused(nboxes), hch(nboxes), hnch(nboxes), hpar(nboxes, -1);
    LSPR_TRY(ctx, cudaMemcpyAsync(hbeg.data(), tr.box_beg.p, sizeof(int) * nboxes, cudaMemcpyDeviceToHost, st));
    LSPR_TRY(ctx, cudaMemcpyAsync(hend.data(), tr.box_end.p, sizeof(int) * nboxes, cudaMemcpyDeviceToHost, st));
    LSPR_TRY(ctx, cudaMemcpyAsync(hused.data(), tr.box_used.p, sizeof(int) * nboxes, cudaMemcpyDeviceToHost, st));
    LSPR_TRY(ctx, cudaMemcpyAsync(hch.data(), tr.box_child.p, sizeof(int) * nboxes, cudaMemcpyDeviceToHost, st));
    LSPR_TRY(ctx, cudaMemcpyAsync(hnch.data(), tr.box_nchild.p, sizeof(int) * nboxes, cudaMemcpyDeviceToHost, st));
    LSPR_TRY(ctx, cudaStreamSynchronize(st));
    std::vector<char> under(nboxes, 0);   // the box or an ancestor is accepted
    for (int b = 0; b < nboxes; ++b) {    // children are numbered after their parent
        under[b] = under[b] || hused[b];
        for (int c = 0; c < hnch[b]; ++c) {
            hpar[hch[b] + c] = b;
            under[hch[b] + c] = under[b];
        }
    }
    std::vector<int4> p2m;
    for (int b = 0; b < nboxes; ++b) {
        if (!under[b] || hnch[b] != 0) continue;
        for (int s0 = hbeg[b]; s0 < hend[b]; s0 += kP2MChunk)
            p2m.push_back(make_int4(b, s0, std::min(hend[b], s0 + kP2MChunk), 0));
    }
    tr.n_p2m_items = (int64_t)p2m.size();
    LSPR_TRY(ctx, tr.p2m_items.ensure(std::max<size_t>(1, p2m.size())));
    if (!p2m.empty())
        LSPR_TRY(ctx, cudaMemcpyAsync(tr.p2m_items.p, p2m.data(), sizeof(int4) * p2m.size(), cudaMemcpyHostToDevice, st));
    // the group lists of the tensor-core far field are formed on first use (tree_tc_lists)
    tr.tc_built = tr.tcp_built = false;
    tr.n_tc_items = tr.n_tc_pairs = tr.n_tcp_items = tr.n_tcp_ivl = tr.n_tcp_sources = tr.n_tcp_stages = 0;
    LSPR_TRY(ctx, tr.box_parent.ensure(nboxes));
    LSPR_TRY(ctx, cudaMemcpyAsync(tr.box_parent.p, hpar.data(), sizeof(int) * nboxes, cudaMemcpyHostToDevice, st));
    timer_end(ctx, T_TREE, ev);
    LSPR_TRY(ctx, cudaStreamSynchronize(st));
    tr.ready = true;
    return LSPR_OK;
}


// Group lists of the tensor-core far field (groups of kTcGroup consecutive target blocks), formed
// on the host from the tree's lists on first use after a tree build: the M2P lists always, the
// P2P source ranges when p2p is set.  Host copies and a synchronisation: not to be called while
// a stream is being captured (solves form them before their first product).
int tree_tc_lists(lspr_ctx *ctx, bool p2p) {
    Tree &tr = ctx->tree;
    cudaStream_t st = ctx->stream;
    const int64_t ntb = tr.ntblocks;
    if (!tr.ready) return LSPR_E_STATE;
    if (!tr.tc_built) {
        // M2P lists of the groups (tc_group_m2p)
        std::vector<int> hlist((size_t)tr.n_m2p_pairs);
        std::vector<int4> hitems((size_t)tr.n_m2p_items);
        if (tr.n_m2p_pairs > 0) {
            LSPR_TRY(ctx, cudaMemcpyAsync(hlist.data(), tr.m2p_list.p, sizeof(int) * tr.n_m2p_pairs, cudaMemcpyDeviceToHost, st));
            LSPR_TRY(ctx, cudaMemcpyAsync(hitems.data(), tr.m2p_items.p, sizeof(int4) * tr.n_m2p_items, cudaMemcpyDeviceToHost, st));
            LSPR_TRY(ctx, cudaStreamSynchronize(st));
        }
        std::vector<TcEntry> glist;
        std::vector<TcItem> gitems;
        tc_group_m2p(ntb, kTcGroup, kTcGroupSeg, hlist.data(), (const int *)hitems.data(), tr.n_m2p_items, glist,
                     gitems);
        tr.n_tc_pairs = (int64_t)glist.size();
        tr.n_tc_items = (int64_t)gitems.size();
        LSPR_TRY(ctx, tr.tc_list.ensure(std::max<size_t>(1, glist.size())));
        LSPR_TRY(ctx, tr.tc_items.ensure(std::max<size_t>(1, gitems.size())));
        if (!glist.empty()) {
            static_assert(sizeof(TcEntry) == sizeof(int2) && sizeof(TcItem) == sizeof(int4), "device layouts");
            LSPR_TRY(ctx, cudaMemcpyAsync(tr.tc_list.p, glist.data(), sizeof(int2) * glist.size(), cudaMemcpyHostToDevice, st));
            LSPR_TRY(ctx, cudaMemcpyAsync(tr.tc_items.p, gitems.data(), sizeof(int4) * gitems.size(), cudaMemcpyHostToDevice, st));
        }
        LSPR_TRY(ctx, cudaStreamSynchronize(st));
        tr.tc_built = true;
    }
    if (p2p && !tr.tcp_built) {
        // P2P source ranges of the same groups (tc_group_p2p)
        std::vector<int4> hp2p((size_t)tr.n_p2p_items);
        if (tr.n_p2p_items > 0) {
            LSPR_TRY(ctx, cudaMemcpyAsync(hp2p.data(), tr.p2p_items.p, sizeof(int4) * tr.n_p2p_items,
                                          cudaMemcpyDeviceToHost, st));
            LSPR_TRY(ctx, cudaStreamSynchronize(st));
        }
        std::vector<TcRange> pivl;
        std::vector<TcItem> pitems;
        static_assert(sizeof(TcRange) == sizeof(int4), "device layout");
        const int64_t psrc = tc_group_p2p(ntb, kTcGroup, kTcP2PSrc, (const int *)hp2p.data(), tr.n_p2p_items, pivl, pitems);
        tr.n_tcp_items = (int64_t)pitems.size();
        tr.n_tcp_ivl = (int64_t)pivl.size();
        tr.n_tcp_sources = psrc;
        tr.n_tcp_stages = 0;
        for (const TcRange &r : pivl) tr.n_tcp_stages += (r.s1 - r.s0 + 7) / 8;
        LSPR_TRY(ctx, tr.tcp_items.ensure(std::max<size_t>(1, pitems.size())));
        LSPR_TRY(ctx, tr.tcp_ivl.ensure(std::max<size_t>(1, pivl.size())));
        if (!pitems.empty()) {
            LSPR_TRY(ctx, cudaMemcpyAsync(tr.tcp_items.p, pitems.data(), sizeof(int4) * pitems.size(),
                                          cudaMemcpyHostToDevice, st));
            LSPR_TRY(ctx, cudaMemcpyAsync(tr.tcp_ivl.p, pivl.data(), sizeof(int4) * pivl.size(), cudaMemcpyHostToDevice, st));
        }
        LSPR_TRY(ctx, cudaStreamSynchronize(st));
        tr.tcp_built = true;
    }
    return LSPR_OK;
}

}  // namespace lspr
