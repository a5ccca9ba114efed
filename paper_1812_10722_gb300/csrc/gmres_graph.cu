// Restarted GMRES(m) (Sec. II.D-E: complex GMRES) for B systems in lockstep.
//
// One Arnoldi cycle:
//   init        v_0 = r / beta, g = beta e_1
//   loop        (the body is one Arnoldi step; its last kernel decides, on the device,
//               whether another step follows)
//                 z = M^-1 v_j                      (v_j = w / ||w|| formed here, j > 0)
//                 w = A z                           (the far field, near SpMV and block rows)
//                 classical Gram-Schmidt h = V^H w, w -= V h, repeated once for the systems
//                 whose w lost more than a factor 1/sqrt(2) of its norm in the first pass
//                 (the Daniel-Gragg-Kaufman-Stewart criterion: one repetition restores
//                 orthogonality to working precision, and a pass that removes little
//                 needs none)
//                 ||w||, Givens rotation of the new Hessenberg column, residual
//                 estimate |g_{j+1}|, per-system stop test
//   back substitution R y = g, x += M^-1 V y
// The cycle is recorded once as a CUDA graph whose loop is a conditional WHILE node, so the
// host only takes part once per cycle (explicit residual and stop decision).  Without graphs
// (or with per-kernel timing) the host launches the same kernels itself and reads the loop
// condition after every step.  Inner products reduce over blocks with a last-block ticket
// instead of a second launch.
//
// Precision.  The Krylov basis, the Gram-Schmidt coefficients and the vector being
// orthogonalised are float-float (hi + lo FP32 pairs, ~48 significant bits): on this GPU the
// FP64 pipe runs at 1/64 of the FP32 rate, and the Gram-Schmidt passes (8 FP64 multiply-adds
// per basis entry and pass) would be bound by it at ~3x the time of reading the basis from
// memory.  In float-float they are bound by the basis traffic.  A basis entry takes 16 bytes
// as in FP64.  The rotations, the small triangular solve, norms' final sums, the residual and
// the solution stay FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cplx.cuh"
#include "ffloat.cuh"
#include "lspr_internal.cuh"

namespace lspr {
namespace {

constexpr int kT = 256;                 // threads per block of the vector kernels
constexpr int kPer = 8;                 // entries per thread of an inner-product block's chunk
constexpr double kReorthEta = 0.70710678118654752;   // second pass when ||w_1|| < eta ||w_0||
constexpr int kDotChunk = kT * kPer;    // elements per inner-product block
constexpr int kMaxWarpsSmall = 16;      // warps of the per-system (rotation, back substitution) kernels

// one complex entry in float-float: re = rh + rl, im = ih + il
struct __align__(16) cff {
    float rh, ih, rl, il;
};
static_assert(sizeof(cff) == sizeof(float4), "a basis entry is one 16-byte word");

__device__ __forceinline__ cff to_cff(double2 v) {
    const float rh = (float)v.x, ih = (float)v.y;
    return {rh, ih, (float)(v.x - (double)rh), (float)(v.y - (double)ih)};
}
__device__ __forceinline__ double2 to_d2(const cff &v) {
    return make_double2((double)v.rh + (double)v.rl, (double)v.ih + (double)v.il);
}
__device__ __forceinline__ ffloat re_of(const cff &v) { return ffloat(v.rh, v.rl); }
__device__ __forceinline__ ffloat im_of(const cff &v) { return ffloat(v.ih, v.il); }

// hi + lo renormalised (|lo| <= ulp(hi)/2) after unnormalised accumulation
__device__ __forceinline__ ffloat ff_norm(const ffloat &x) {
    ffloat r;
    ff_two_sum(x.hi, x.lo, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ cff pack(const ffloat &re, const ffloat &im) {
    const ffloat r = ff_norm(re), i = ff_norm(im);
    return {r.hi, i.hi, r.lo, i.lo};
}

// (sr, si) += conj(v) w
__device__ __forceinline__ void cff_conj_mac(ffloat &sr, ffloat &si, const cff &v, const cff &w) {
    const ffloat vr = re_of(v), vi = im_of(v), wr = re_of(w), wi = im_of(w);
    ff_mac(sr, vr, wr);
    ff_mac(sr, vi, wi);
    ff_mac(si, vr, wi);
    ff_mac(si, -vi, wr);
}
// (ar, ai) += v h, or -= v h with SUB
template <bool SUB>
__device__ __forceinline__ void cff_mac(ffloat &ar, ffloat &ai, const cff &v, const cff &h) {
    const ffloat vr = SUB ? -re_of(v) : re_of(v), vi = SUB ? -im_of(v) : im_of(v);
    const ffloat hr = re_of(h), hi = im_of(h);
    ff_mac(ar, vr, hr);
    ff_mac(ar, -vi, hi);
    ff_mac(ai, vr, hi);
    ff_mac(ai, vi, hr);
}
// |v|^2 added to s
__device__ __forceinline__ void cff_abs2_mac(ffloat &s, const ffloat &re, const ffloat &im) {
    ff_mac(s, re, re);
    ff_mac(s, im, im);
}

struct Arn {
    int B, m, nch, nblk;
    int64_t N, n2, vstride;
    cff *V;              // [B][m+1][2N] Krylov basis
    double2 *w;          // [B][2N] A z (FP64 from the operator; float-float in place once the
                         // first Gram-Schmidt pass has read it)
    double2 *z, *x;
    const double2 *b, *s;
    const double *vinv;  // [N] 1 / V_ii (preconditioner)
    const double2 *pq;   // [B][S] 1 / (1 + s) (preconditioner)
    const int *surf;     // surface of each panel; s is [B][S]
    int S;
    double2 *h, *hcol, *part, *H, *sn, *g, *y;
    cff *hff, *yff;      // [B][m+1] Gram-Schmidt coefficients, [B][m] update coefficients
    ffloat *ninv;        // [B] 1 / ||w||
    double *npart, *nrm, *cs, *res, *npart0, *nrm0;
    int *reorth;
    const double *bn, *par;
    unsigned *tick;
    int *jdev, *active, *jb, *iters;
    int *rmap;   // [2B + 2]: slot -> system, system -> slot (-1: not running), running count,
                 // channel sets in use (running count x surfaces)
    int *go;     // host-driven cycles: the loop condition (nullptr inside a graph)
    unsigned long long *stats;   // [4] sum (j+1), system-steps, the same over second passes
    cudaGraphConditionalHandle cond;
};

__device__ __forceinline__ cff *wff(const Arn &a, int b) { return (cff *)(a.w + (int64_t)b * a.n2); }

// packs the running systems into the first slots (single thread)
__device__ __forceinline__ void pack_running(const Arn &a) {
    int n = 0;
    for (int b = 0; b < a.B; ++b) {
        if (a.active[b]) {
            a.rmap[n] = b;
            a.rmap[a.B + b] = n++;
        } else {
            a.rmap[a.B + b] = -1;
        }
    }
    for (int q = n; q < a.B; ++q) a.rmap[q] = 0;
    a.rmap[2 * a.B] = n;
    a.rmap[2 * a.B + 1] = n * a.S;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double2 warp_sum2(double2 v) { return make_double2(warp_sum(v.x), warp_sum(v.y)); }

__device__ __forceinline__ ffloat shfl_xor(const ffloat &v, int o) {
    return ffloat(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}
__device__ __forceinline__ ffloat ff_warp_sum(ffloat v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = v + shfl_xor(v, o);
    return v;
}

// sum over a block of kT threads, valid in warp 0
__device__ __forceinline__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) t = warp_sum(threadIdx.x < kT / 32 ? sh[threadIdx.x] : 0.0);
    return t;
}
// float-float partial sums of a block: warps reduce in float-float, warp 0 sums the kT/32
// warp results in FP64 (valid in thread 0)
__device__ __forceinline__ double block_sum_ff(const ffloat &v, double *sh) {
    const ffloat s = ff_warp_sum(ff_norm(v));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < kT / 32; ++q) t += sh[q];
    return t;
}

// true in every thread of the block that arrives last among `count` blocks on ticket *t
// (the partial results written before the call are visible to it)
__device__ __forceinline__ bool last_block(unsigned *t, unsigned count) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(t, 1u) == count - 1;
    __syncthreads();
    return last;
}

// final sum of the squared-norm partials of system b into nrm[b] and 1/nrm[b] (last block
// only); decide: the first Gram-Schmidt pass decides whether the second runs
__device__ __forceinline__ void norm_final(const Arn &a, int b, double *sh, bool decide = false) {
    double t = 0.0;
    for (int c = threadIdx.x; c < a.nblk; c += kT) t += __ldcg(a.npart + (int64_t)b * a.nblk + c);
    t = block_sum(t, sh);
    if (threadIdx.x == 0) {
        const double r = sqrt(t);
        a.nrm[b] = r;
        a.ninv[b] = ffloat(r > 0 ? 1.0 / r : 0.0);
        if (decide) a.reorth[b] = !(r >= kReorthEta * __ldcg(a.nrm0 + b));
        a.tick[a.B + b] = 0;
    }
}

// Right preconditioner of panel i (inverse of the diagonal 2x2 block of the operator,
// [[1/2 + K_ii, -V_ii], [1/2 - K_ii, s V_ii]] with K_ii = 0):
//   o0 = 2 (s u0 + u1) / (1 + s),  o1 = (u1 - u0) / (V_ii (1 + s))
// with pq = 1 / (1 + s) and vinv = 1 / V_ii formed once per solve (no division per entry)
__device__ __forceinline__ void precond(double vinv, double2 q, double2 s, double2 u0, double2 u1, double2 &o0,
                                        double2 &o1) {
    o0 = cscale(cmul(q, cadd(cmul(s, u0), u1)), 2.0);
    o1 = cscale(cmul(q, csub(u1, u0)), vinv);
}

// w = A x - b (w holds A x on entry; x_zero: x = 0 and w = -b), nrm[b] = ||w||
__global__ void __launch_bounds__(kT) arn_resid_kernel(Arn a, int x_zero) {
    __shared__ double sh[kT / 32];
    const int b = blockIdx.y;
    const int64_t k = blockIdx.x * (int64_t)kT + threadIdx.x;
    double q = 0.0;
    if (k < a.n2) {
        const int64_t o = (int64_t)b * a.n2 + k;
        const double2 bb = a.b[o];
        const double2 v = x_zero ? make_double2(-bb.x, -bb.y) : csub(a.w[o], bb);
        a.w[o] = v;
        q = cabs2(v);
    }
    q = block_sum(q, sh);
    if (threadIdx.x == 0) a.npart[(int64_t)b * a.nblk + blockIdx.x] = q;
    if (last_block(a.tick + a.B + b, a.nblk)) norm_final(a, b, sh);
}

// v_0 = -w / beta for the running systems (w = A x - b); cycle state reset
__global__ void __launch_bounds__(kT) arn_init_kernel(Arn a) {
    const int b = blockIdx.y;
    const int64_t k = blockIdx.x * (int64_t)kT + threadIdx.x;
    const bool act = a.active[b] != 0;
    if (act && k < a.n2) a.V[(int64_t)b * a.vstride + k] = to_cff(cscale(a.w[(int64_t)b * a.n2 + k], -1.0 / a.nrm[b]));
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i <= a.m; i += kT)
            a.g[(int64_t)b * (a.m + 1) + i] = make_double2(i == 0 && act ? a.nrm[b] : 0.0, 0.0);
        if (threadIdx.x == 0) {
            a.jb[b] = 0;
            a.tick[b] = 0;
            a.tick[a.B + b] = 0;
            if (b == 0) {
                *a.jdev = 0;
                pack_running(a);
            }
        }
    }
}

// v_j = w / ||w|| (j > 0, w float-float; v_0 comes from the init kernel), z = M^-1 v_j
__global__ void __launch_bounds__(kT) arn_precond_kernel(Arn a) {
    const int b = blockIdx.y;
    const int64_t t = blockIdx.x * (int64_t)kT + threadIdx.x;
    if (t >= a.N || !a.active[b]) return;
    const int j = *a.jdev;
    cff *Vj = a.V + (int64_t)b * a.vstride + (int64_t)j * a.n2;
    cff v0, v1;
    if (j == 0) {
        v0 = Vj[t];
        v1 = Vj[a.N + t];
    } else {
        const ffloat inv = a.ninv[b];
        const cff *wb = wff(a, b);
        const cff w0 = wb[t], w1 = wb[a.N + t];
        v0 = pack(re_of(w0) * inv, im_of(w0) * inv);
        v1 = pack(re_of(w1) * inv, im_of(w1) * inv);
        Vj[t] = v0;
        Vj[a.N + t] = v1;
    }
    double2 o0, o1;
    precond(a.vinv[t], a.pq[b * a.S + a.surf[t]], a.s[b * a.S + a.surf[t]], to_d2(v0), to_d2(v1), o0, o1);
    a.z[(int64_t)b * a.n2 + t] = o0;
    a.z[(int64_t)b * a.n2 + a.N + t] = o1;
}

// One classical Gram-Schmidt pass, first half: h_i = <v_i, w> for i <= j.  A block takes a
// chunk of kDotChunk entries of one system: its threads stage the chunk of w in shared memory
// (pass 0 converts w to float-float in place and forms ||w||^2 of the chunk), then warp q takes
// the basis vectors q, q + 8, ...: its lanes stride over the chunk (64 entries each, with four
// independent float-float accumulator pairs, so many loads are in flight) and one warp reduction
// per vector gives the chunk's partial product.  The last block of the system sums the chunks
// into h (FP64 and float-float) and into the Hessenberg column (hcol = h on pass 0, hcol += h on
// pass 1).
__global__ void __launch_bounds__(kT) arn_dot_kernel(Arn a, int pass) {
    __shared__ cff ws[kDotChunk];
    __shared__ double2 red[kMaxRestart + 1];
    __shared__ double shn[kT / 32];
    const int b = blockIdx.y, chunk = blockIdx.x;
    if (!a.active[b] || (pass && !a.reorth[b])) return;
    const int nv = *a.jdev + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c0 = (int64_t)chunk * kDotChunk;
    const int len = (int)min((int64_t)kDotChunk, a.n2 - c0);
    cff *wb = wff(a, b) + c0;
    ffloat w2(0.f, 0.f);
    for (int e = threadIdx.x; e < kDotChunk; e += kT) {
        cff v = {0.f, 0.f, 0.f, 0.f};
        if (e < len) {
            if (pass == 0) {
                v = to_cff(a.w[(int64_t)b * a.n2 + c0 + e]);
                wb[e] = v;
            } else {
                v = wb[e];
            }
        }
        ws[e] = v;
        if (pass == 0) cff_abs2_mac(w2, re_of(v), im_of(v));
    }
    if (pass == 0) {   // ||A z||^2 of this chunk, for the second-pass criterion
        const double t = block_sum_ff(w2, shn);
        if (threadIdx.x == 0) a.npart0[(int64_t)b * a.nch + chunk] = t;
    }
    __syncthreads();
    const cff *Vb = a.V + (int64_t)b * a.vstride + c0;
    for (int i = warp; i < nv; i += kT / 32) {
        const cff *v = Vb + (int64_t)i * a.n2;
        ffloat sr[4], si[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) sr[u] = si[u] = ffloat(0.f, 0.f);
        if (len == kDotChunk) {
            // eight entries per lane loaded together before they are used (more bytes in flight)
#pragma unroll 1
            for (int e0 = lane; e0 < kDotChunk; e0 += 256) {
                float4 vv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) vv[u] = __ldg((const float4 *)(v + e0 + 32 * u));
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const cff x = {vv[u].x, vv[u].y, vv[u].z, vv[u].w};
                    cff_conj_mac(sr[u & 3], si[u & 3], x, ws[e0 + 32 * u]);
                }
            }
        } else {   // the ragged last chunk
            for (int e = lane; e < len; e += 32) cff_conj_mac(sr[0], si[0], v[e], ws[e]);
        }
        ffloat tr = ff_norm(sr[0]) + ff_norm(sr[1]) + (ff_norm(sr[2]) + ff_norm(sr[3]));
        ffloat ti = ff_norm(si[0]) + ff_norm(si[1]) + (ff_norm(si[2]) + ff_norm(si[3]));
        tr = ff_warp_sum(tr);
        ti = ff_warp_sum(ti);
        if (lane == 0) red[i] = make_double2((double)tr, (double)ti);
    }
    __syncthreads();
    double2 *pb = a.part + (int64_t)b * (a.m + 1) * a.nch;
    for (int i = threadIdx.x; i < nv; i += kT) pb[(int64_t)i * a.nch + chunk] = red[i];
    if (!last_block(a.tick + b, a.nch)) return;
    if (pass == 0) {
        double t = 0.0;
        for (int c = threadIdx.x; c < a.nch; c += kT) t += __ldcg(a.npart0 + (int64_t)b * a.nch + c);
        t = block_sum(t, shn);
        if (threadIdx.x == 0) a.nrm0[b] = sqrt(t);
    }
    // rows i = warp + 8 u: lanes stride over the chunks
    for (int i0 = warp; i0 < nv; i0 += 4 * (kT / 32)) {
        double2 t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            t[u] = make_double2(0.0, 0.0);
            const int i = i0 + u * (kT / 32);
            if (i < nv)
                for (int c = lane; c < a.nch; c += 32) t[u] = cadd(t[u], __ldcg(pb + (int64_t)i * a.nch + c));
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * (kT / 32);
            const double2 sum = warp_sum2(t[u]);
            if (lane == 0 && i < nv) {
                a.h[(int64_t)b * (a.m + 1) + i] = sum;
                a.hff[(int64_t)b * (a.m + 1) + i] = to_cff(sum);
                double2 &e = a.hcol[(int64_t)b * (a.m + 1) + i];
                e = pass ? cadd(e, sum) : sum;
            }
        }
    }
    if (threadIdx.x == 0) a.tick[b] = 0;
}

// Second half of a pass: w -= sum_{i <= j} v_i h_i (float-float), then ||w|| into nrm[b]
// (partials per block, the last block sums them); after the first pass the last block also
// decides whether the second runs (reorth[b])
__global__ void __launch_bounds__(kT) arn_axpy_kernel(Arn a, int pass) {
    __shared__ double sh[kT / 32];
    __shared__ cff hs[kMaxRestart + 1];
    const int b = blockIdx.y;
    if (!a.active[b] || (pass && !a.reorth[b])) return;
    const int nv = *a.jdev + 1;
    for (int i = threadIdx.x; i < nv; i += kT) hs[i] = a.hff[(int64_t)b * (a.m + 1) + i];
    __syncthreads();
    const int64_t k = blockIdx.x * (int64_t)kT + threadIdx.x;
    ffloat q(0.f, 0.f);
    if (k < a.n2) {
        const cff *Vb = a.V + (int64_t)b * a.vstride + k;
        cff *wk = wff(a, b) + k;
        const cff w0 = *wk;
        ffloat ar = re_of(w0), ai = im_of(w0);
#pragma unroll 4
        for (int i = 0; i < nv; ++i) cff_mac<true>(ar, ai, Vb[(int64_t)i * a.n2], hs[i]);
        const cff w1 = pack(ar, ai);
        *wk = w1;
        cff_abs2_mac(q, re_of(w1), im_of(w1));
    }
    const double t = block_sum_ff(q, sh);
    if (threadIdx.x == 0) a.npart[(int64_t)b * a.nblk + blockIdx.x] = t;
    if (last_block(a.tick + a.B + b, a.nblk)) norm_final(a, b, sh, pass == 0);
}

// shared memory of the rotation kernel per warp: column (m+1), sines (m), cosines (m)
inline size_t tail_smem_per_warp(int m) { return (size_t)(3 * m + 1) * sizeof(double2); }

// End of an Arnoldi step, one warp per system: the new Hessenberg column (hcol, ||w||)
// is rotated by the previous Givens rotations, a new rotation zeroes its subdiagonal,
// g is rotated, |g_{j+1}| is the residual estimate and decides whether the system keeps
// running.  The block then advances j and sets the loop condition (the graph's, or the flag
// the host reads): another step runs while a system is running and j < m.
__global__ void arn_tail_kernel(Arn a) {
    extern __shared__ double2 dsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int m = a.m, j = *a.jdev;
    double2 *col = dsm + (size_t)warp * (3 * m + 1);
    double2 *snw = col + m + 1;
    double2 *csw = snw + m;
    const double tol = a.par[0];
    const int maxit = (int)a.par[1];
    int any = 0;
    for (int b = warp; b < a.B; b += nw) {
        if (!a.active[b]) continue;   // warp-uniform
        const double2 *hc = a.hcol + (int64_t)b * (m + 1);
        for (int i = lane; i <= j; i += 32) col[i] = hc[i];
        for (int i = lane; i < j; i += 32) {
            snw[i] = a.sn[(int64_t)b * m + i];
            csw[i] = make_double2(a.cs[(int64_t)b * m + i], 0.0);
        }
        __syncwarp();
        int act = 0;
        if (lane == 0) {
            double2 *Hb = a.H + (int64_t)b * (m + 1) * m;
            double2 a0 = col[0];
            for (int i = 0; i < j; ++i) {   // previous rotations, carrying row i+1
                const double c = csw[i].x;
                const double2 sg = snw[i], d0 = col[i + 1];
                Hb[(int64_t)i * m + j] = cadd(cscale(a0, c), cmul(sg, d0));
                a0 = csub(cscale(d0, c), cmul(cconj(sg), a0));
            }
            const double hn = a.nrm[b];   // subdiagonal entry ||w||, real
            const double aa = sqrt(cabs2(a0)), t = sqrt(aa * aa + hn * hn);
            double c;
            double2 sg;
            if (aa == 0.0) {
                c = 0.0;
                sg = make_double2(1.0, 0.0);
            } else {
                c = aa / t;
                sg = cscale(a0, hn / (aa * t));
            }
            Hb[(int64_t)j * m + j] = cadd(cscale(a0, c), cscale(sg, hn));
            a.cs[(int64_t)b * m + j] = c;
            a.sn[(int64_t)b * m + j] = sg;
            double2 *gb = a.g + (int64_t)b * (m + 1);
            const double2 gj = gb[j];
            gb[j + 1] = cmul(make_double2(-sg.x, sg.y), gj);   // -conj(s) g_j
            gb[j] = cscale(gj, c);
            const double r = sqrt(cabs2(gb[j + 1]));
            a.res[b] = r;
            a.jb[b] = j + 1;
            atomicAdd(a.stats + 0, (unsigned long long)(j + 1));
            atomicAdd(a.stats + 1, 1ull);
            if (a.reorth[b]) {
                atomicAdd(a.stats + 2, (unsigned long long)(j + 1));
                atomicAdd(a.stats + 3, 1ull);
            }
            const int it = ++a.iters[b];
            act = (r / a.bn[b] > tol) && it < maxit && isfinite(r);
            a.active[b] = act;
        }
        any |= __shfl_sync(0xffffffffu, act, 0);
        __syncwarp();
    }
    const int go = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        pack_running(a);
        *a.jdev = j + 1;
        const unsigned more = (go && j + 1 < m) ? 1u : 0u;
        if (a.go)
            *a.go = (int)more;
        else
            cudaGraphSetConditional(a.cond, more);
    }
}

// R y = g by back substitution (one warp per system), y into a.y (FP64) and a.yff
__global__ void arn_backsub_kernel(Arn a) {
    extern __shared__ double2 ysm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int m = a.m;
    double2 *ys = ysm + (size_t)warp * m;
    for (int b = warp; b < a.B; b += nw) {
        const int n = a.jb[b];
        const double2 *Hb = a.H + (int64_t)b * (m + 1) * m, *gb = a.g + (int64_t)b * (m + 1);
        for (int i = n - 1; i >= 0; --i) {
            double2 s = make_double2(0.0, 0.0);
            for (int k = i + 1 + lane; k < n; k += 32) s = cadd(s, cmul(Hb[(int64_t)i * m + k], ys[k]));
            s = warp_sum2(s);
            if (lane == 0) ys[i] = cdiv(csub(gb[i], s), Hb[(int64_t)i * m + i]);
            __syncwarp();
        }
        for (int i = lane; i < n; i += 32) {
            a.y[(int64_t)b * m + i] = ys[i];
            a.yff[(int64_t)b * m + i] = to_cff(ys[i]);
        }
        __syncwarp();
    }
}

// x += M^-1 sum_{i < jb} v_i y_i (the sum in float-float)
__global__ void __launch_bounds__(kT) arn_update_kernel(Arn a) {
    const int b = blockIdx.y;
    const int64_t t = blockIdx.x * (int64_t)kT + threadIdx.x;
    const int n = a.jb[b];
    if (t >= a.N || n == 0) return;
    const cff *Vb = a.V + (int64_t)b * a.vstride;
    const cff *yb = a.yff + (int64_t)b * a.m;
    ffloat r0(0.f, 0.f), i0(0.f, 0.f), r1(0.f, 0.f), i1(0.f, 0.f);
    for (int i = 0; i < n; ++i) {
        const cff yi = yb[i];
        cff_mac<false>(r0, i0, Vb[(int64_t)i * a.n2 + t], yi);
        cff_mac<false>(r1, i1, Vb[(int64_t)i * a.n2 + a.N + t], yi);
    }
    const double2 u0 = make_double2((double)r0, (double)i0), u1 = make_double2((double)r1, (double)i1);
    double2 o0, o1;
    const int q = b * a.S + a.surf[t];
    precond(a.vinv[t], a.pq[q], a.s[q], u0, u1, o0, o1);
    double2 *xb = a.x + (int64_t)b * a.n2;
    xb[t] = cadd(xb[t], o0);
    xb[a.N + t] = cadd(xb[a.N + t], o1);
}

// preconditioner constants of a solve: vinv = 1 / V_ii, pq = 1 / (1 + s)
__global__ void arn_precond_setup_kernel(int64_t N, int BS, const double *Vself, const double2 *s, double *vinv,
                                         double2 *pq) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < N) vinv[t] = 1.0 / Vself[t];
    if (t < BS) pq[t] = cdiv(make_double2(1.0, 0.0), make_double2(1.0 + s[t].x, s[t].y));
}

int small_kernel_warps(int B, int m) {
    const int by_smem = (int)(45000 / tail_smem_per_warp(m));
    return std::max(1, std::min({B, kMaxWarpsSmall, by_smem}));
}

// Records one Arnoldi cycle into gc: [init] -> while{step} -> [back substitution, update].
// Launches go to ctx->gstream (ctx->stream is redirected there while recording so that
// the operator's launchers record into the graph too).  Kernel counts of the recording
// are kept in gc and removed from the context's counters.
int capture_cycle(lspr_ctx *ctx, int mode, const Arn &a0, GraphCache &gc) {
    gc.reset();
    cudaStream_t cs = ctx->gstream, saved = ctx->stream;
    const int64_t l0 = ctx->n_launches, mv0 = ctx->matvec_count;
    const int nw = small_kernel_warps(a0.B, a0.m);
    const dim3 gv(grid_for(a0.n2, kT), a0.B), gN(grid_for(a0.N, kT), a0.B);
    cudaGraph_t g = nullptr;
    bool capturing = false;
    auto fail = [&](int code) {
        if (capturing) {
            cudaGraph_t tmp = nullptr;
            cudaStreamEndCapture(cs, &tmp);
        }
        cudaGetLastError();
        ctx->stream = saved;
        ctx->n_launches = l0;
        ctx->matvec_count = mv0;
        if (g) cudaGraphDestroy(g);
        return code;
    };
#define CAP_TRY(expr)                                                      \
    do {                                                                   \
        cudaError_t e__ = (expr);                                          \
        if (e__ != cudaSuccess) return fail(cuda_status(ctx, e__, #expr)); \
    } while (0)
    CAP_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    CAP_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    Arn a = a0;
    a.cond = h;
    a.go = nullptr;
    ctx->stream = cs;
    // head: v_0 and the cycle state
    CAP_TRY(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    capturing = true;
    arn_init_kernel<<<gv, kT, 0, cs>>>(a);
    CAP_TRY(cudaGetLastError());
    CAP_TRY(cudaStreamEndCapture(cs, &g));
    capturing = false;
    cudaGraphNode_t head = nullptr;
    size_t nn = 1;
    CAP_TRY(cudaGraphGetNodes(g, &head, &nn));
    // the loop over Arnoldi steps
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t loop = nullptr;
    CAP_TRY(cudaGraphAddNode(&loop, g, &head, nullptr, 1, &p));
    cudaGraph_t body = p.conditional.phGraph_out[0];
    const int64_t l1 = ctx->n_launches;
    CAP_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    capturing = true;
    arn_precond_kernel<<<gN, kT, 0, cs>>>(a);
    ++ctx->n_launches;
    // the product works on the running systems only, packed into the first slots (with
    // several surfaces, the S channel sets of a system follow each other)
    ctx->rhs_map = a.rmap;
    ctx->rhs_inv = a.rmap + a.B;
    ctx->rhs_nact = a.rmap + 2 * a.B + 1;
    const int rc = apply_operator(ctx, mode, a.z, a.w, a.s, a.B);
    ctx->rhs_map = ctx->rhs_inv = ctx->rhs_nact = nullptr;
    if (rc != LSPR_OK) return fail(rc);
    for (int pass = 0; pass < 2; ++pass) {
        arn_dot_kernel<<<dim3(a.nch, a.B), kT, 0, cs>>>(a, pass);
        arn_axpy_kernel<<<gv, kT, 0, cs>>>(a, pass);
        ctx->n_launches += 2;
    }
    arn_tail_kernel<<<1, 32 * nw, nw * tail_smem_per_warp(a.m), cs>>>(a);
    ++ctx->n_launches;
    CAP_TRY(cudaGetLastError());
    CAP_TRY(cudaStreamEndCapture(cs, &body));
    capturing = false;
    const int64_t l2 = ctx->n_launches;
    // tail: x += M^-1 V y
    CAP_TRY(cudaStreamBeginCaptureToGraph(cs, g, &loop, nullptr, 1, cudaStreamCaptureModeRelaxed));
    capturing = true;
    arn_backsub_kernel<<<1, 32 * nw, nw * a.m * sizeof(double2), cs>>>(a);
    arn_update_kernel<<<gN, kT, 0, cs>>>(a);
    CAP_TRY(cudaGetLastError());
    CAP_TRY(cudaStreamEndCapture(cs, &g));
    capturing = false;
    cudaGraphExec_t exec = nullptr;
    CAP_TRY(cudaGraphInstantiate(&exec, g, 0));
#undef CAP_TRY
    ctx->stream = saved;
    ctx->n_launches = l0;
    ctx->matvec_count = mv0;
    gc.graph = g;
    gc.exec = exec;
    gc.per_step = l2 - l1;
    gc.outer = 3;   // init, back substitution, update
    return LSPR_OK;
}

// One Arnoldi cycle launched from the host, without a graph: the kernels of the recorded
// cycle in the same order, the loop condition read back after every step.  With per-kernel
// timing the vector kernels are timed under T_GMRES (the operator's under their own slots).
// Launches are counted as they happen; products are counted by the caller per running
// system, as for a recorded cycle.
int host_cycle(lspr_ctx *ctx, int mode, const Arn &a0, int *go_d) {
    cudaStream_t st = ctx->stream;
    Arn a = a0;
    a.go = go_d;
    a.cond = 0;
    const int64_t mv0 = ctx->matvec_count;
    const int nw = small_kernel_warps(a.B, a.m);
    const dim3 gv(grid_for(a.n2, kT), a.B), gN(grid_for(a.N, kT), a.B);
    cudaEvent_t ev;
    timer_begin(ctx, T_GMRES, &ev);
    arn_init_kernel<<<gv, kT, 0, st>>>(a);
    ++ctx->n_launches;
    timer_end(ctx, T_GMRES, ev);
    int more = 1, sets = a.B * a.S;
    const bool count = ctx->timing.enabled;   // channel sets of each product, for the timing counts
    if (count) {
        LSPR_TRY(ctx, cudaMemcpyAsync(&sets, a.rmap + 2 * a.B + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        LSPR_TRY(ctx, cudaStreamSynchronize(st));
    }
    while (more) {
        timer_begin(ctx, T_GMRES, &ev);
        arn_precond_kernel<<<gN, kT, 0, st>>>(a);
        ++ctx->n_launches;
        timer_end(ctx, T_GMRES, ev);
        ctx->rhs_map = a.rmap;
        ctx->rhs_inv = a.rmap + a.B;
        ctx->rhs_nact = a.rmap + 2 * a.B + 1;
        ctx->timing_sets = count ? sets : -1;
        const int rc = apply_operator(ctx, mode, a.z, a.w, a.s, a.B);
        ctx->rhs_map = ctx->rhs_inv = ctx->rhs_nact = nullptr;
        ctx->timing_sets = -1;
        LSPR_TRY_ST(rc);
        timer_begin(ctx, T_GMRES, &ev);
        for (int pass = 0; pass < 2; ++pass) {
            arn_dot_kernel<<<dim3(a.nch, a.B), kT, 0, st>>>(a, pass);
            arn_axpy_kernel<<<gv, kT, 0, st>>>(a, pass);
            ctx->n_launches += 2;
        }
        arn_tail_kernel<<<1, 32 * nw, nw * tail_smem_per_warp(a.m), st>>>(a);
        ++ctx->n_launches;
        timer_end(ctx, T_GMRES, ev);
        LSPR_TRY(ctx, cudaGetLastError());
        LSPR_TRY(ctx, cudaMemcpyAsync(&more, go_d, sizeof(int), cudaMemcpyDeviceToHost, st));
        if (count)
            LSPR_TRY(ctx, cudaMemcpyAsync(&sets, a.rmap + 2 * a.B + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        LSPR_TRY(ctx, cudaStreamSynchronize(st));
    }
    timer_begin(ctx, T_GMRES, &ev);
    arn_backsub_kernel<<<1, 32 * nw, nw * a.m * sizeof(double2), st>>>(a);
    arn_update_kernel<<<gN, kT, 0, st>>>(a);
    ctx->n_launches += 2;
    timer_end(ctx, T_GMRES, ev);
    LSPR_TRY(ctx, cudaGetLastError());
    ctx->matvec_count = mv0;
    return LSPR_OK;
}

}  // namespace

int gmres_graph_solve(lspr_ctx *ctx, int mode, int B, int m, int maxiter, double tol, const double2 *s_d,
                      const double2 *b_d, double2 *x_d, bool x_zero, bool trust_estimate, std::vector<int> &iters,
                      std::vector<double> &relres, const std::vector<double> &bnorm) {
    if (B < 1 || m < 1 || m > kMaxRestart) return LSPR_E_ARG;
    const Mesh &me = ctx->mesh;
    const int64_t N = me.N, n2 = 2 * N;
    cudaStream_t st = ctx->stream;
    if (ctx->use_graphs && !ctx->timing.enabled && !ctx->gstream) {
        LSPR_TRY(ctx, cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
        LSPR_TRY(ctx, cudaEventCreateWithFlags(&ctx->ev_g0, cudaEventDisableTiming));
        LSPR_TRY(ctx, cudaEventCreateWithFlags(&ctx->ev_g1, cudaEventDisableTiming));
    }
    ArnoldiBufs &ab = ctx->arn;
    const int nch = (int)((n2 + kDotChunk - 1) / kDotChunk), nblk = (int)grid_for(n2, kT);
    const int64_t vstride = (int64_t)(m + 1) * n2;
    LSPR_TRY(ctx, ctx->gm_V.ensure((size_t)B * vstride));
    LSPR_TRY(ctx, ctx->gm_w.ensure((size_t)B * n2));
    LSPR_TRY(ctx, ctx->gm_z.ensure((size_t)B * n2));
    LSPR_TRY(ctx, ab.h.ensure((size_t)B * (m + 1)));
    LSPR_TRY(ctx, ab.hcol.ensure((size_t)B * (m + 1)));
    LSPR_TRY(ctx, ab.part.ensure((size_t)B * (m + 1) * nch));
    LSPR_TRY(ctx, ab.npart.ensure((size_t)B * nblk));
    LSPR_TRY(ctx, ab.nrm.ensure(B));
    LSPR_TRY(ctx, ab.npart0.ensure((size_t)B * nch));
    LSPR_TRY(ctx, ab.nrm0.ensure(B));
    LSPR_TRY(ctx, ab.reorth.ensure(B));
    LSPR_TRY(ctx, ab.H.ensure((size_t)B * (m + 1) * m));
    LSPR_TRY(ctx, ab.cs.ensure((size_t)B * m));
    LSPR_TRY(ctx, ab.sn.ensure((size_t)B * m));
    LSPR_TRY(ctx, ab.g.ensure((size_t)B * (m + 1)));
    LSPR_TRY(ctx, ab.y.ensure((size_t)B * m));
    LSPR_TRY(ctx, ab.res.ensure(B));
    LSPR_TRY(ctx, ab.bn.ensure(B));
    LSPR_TRY(ctx, ab.par.ensure(2));
    LSPR_TRY(ctx, ab.tick.ensure(2 * (size_t)B));
    LSPR_TRY(ctx, ab.ctl.ensure(1 + 3 * (size_t)B));
    LSPR_TRY(ctx, ab.rmap.ensure(2 * (size_t)B + 2));
    LSPR_TRY(ctx, ab.hff.ensure((size_t)B * (m + 1)));
    LSPR_TRY(ctx, ab.yff.ensure((size_t)B * m));
    LSPR_TRY(ctx, ab.ninv.ensure(B));
    LSPR_TRY(ctx, ab.vinv.ensure(N));
    LSPR_TRY(ctx, ab.pq.ensure((size_t)B * me.S));
    LSPR_TRY(ctx, ab.go.ensure(1));
    if (!ab.stats.p) {
        LSPR_TRY(ctx, ab.stats.ensure(4));
        LSPR_TRY(ctx, cudaMemsetAsync(ab.stats.p, 0, 4 * sizeof(unsigned long long), st));
    }
    Arn a;
    a.B = B;
    a.m = m;
    a.nch = nch;
    a.nblk = nblk;
    a.N = N;
    a.n2 = n2;
    a.vstride = vstride;
    a.V = (cff *)ctx->gm_V.p;
    a.w = ctx->gm_w.p;
    a.z = ctx->gm_z.p;
    a.x = x_d;
    a.b = b_d;
    a.s = s_d;
    a.vinv = ab.vinv.p;
    a.pq = ab.pq.p;
    a.surf = me.surf.p;
    a.S = me.S;
    a.h = ab.h.p;
    a.hcol = ab.hcol.p;
    a.part = ab.part.p;
    a.H = ab.H.p;
    a.sn = ab.sn.p;
    a.g = ab.g.p;
    a.y = ab.y.p;
    a.npart = ab.npart.p;
    a.nrm = ab.nrm.p;
    a.npart0 = ab.npart0.p;
    a.nrm0 = ab.nrm0.p;
    a.reorth = ab.reorth.p;
    a.cs = ab.cs.p;
    a.res = ab.res.p;
    a.bn = ab.bn.p;
    a.par = ab.par.p;
    a.tick = ab.tick.p;
    a.jdev = ab.ctl.p;
    a.active = ab.ctl.p + 1;
    a.jb = ab.ctl.p + 1 + B;
    a.iters = ab.ctl.p + 1 + 2 * B;
    a.rmap = ab.rmap.p;
    a.hff = (cff *)ab.hff.p;
    a.yff = (cff *)ab.yff.p;
    a.ninv = (ffloat *)ab.ninv.p;
    a.go = nullptr;
    a.stats = ab.stats.p;
    a.cond = 0;
    // per-call parameters live in device memory, so one recorded graph serves every call
    const double par[2] = {tol, (double)std::max(1, maxiter)};
    LSPR_TRY(ctx, cudaMemcpyAsync(ab.bn.p, bnorm.data(), sizeof(double) * B, cudaMemcpyHostToDevice, st));
    LSPR_TRY(ctx, cudaMemcpyAsync(ab.par.p, par, sizeof(par), cudaMemcpyHostToDevice, st));
    LSPR_TRY(ctx, cudaMemsetAsync(ab.ctl.p, 0, sizeof(int) * (1 + 3 * (size_t)B), st));
    LSPR_TRY(ctx, cudaMemsetAsync(ab.tick.p, 0, sizeof(unsigned) * 2 * (size_t)B, st));
    ++ctx->n_launches;
    arn_precond_setup_kernel<<<grid_for(std::max<int64_t>(N, (int64_t)B * me.S), kT), kT, 0, st>>>(
        N, B * me.S, me.Vself.p, s_d, ab.vinv.p, ab.pq.p);
    for (int b = 0; b < B; ++b) {
        iters[b] = 0;
        relres[b] = 1.0;
    }
    std::vector<int> act(B), ctl(1 + 3 * (size_t)B);
    std::vector<double> est(B), beta(B);
    const dim3 gv(grid_for(n2, kT), B);
    static uint64_t clock = 0;
    bool first = true;
    while (true) {
        // explicit residual w = A x - b and beta = ||w|| (x = 0 on entry: w = -b)
        const bool skip_mv = first && x_zero;
        if (!skip_mv) LSPR_TRY_ST(apply_operator(ctx, mode, x_d, a.w, s_d, B));
        ++ctx->n_launches;
        arn_resid_kernel<<<gv, kT, 0, st>>>(a, skip_mv ? 1 : 0);
        LSPR_TRY(ctx, cudaGetLastError());
        LSPR_TRY(ctx, cudaMemcpyAsync(beta.data(), a.nrm, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
        LSPR_TRY(ctx, cudaStreamSynchronize(st));
        first = false;
        bool any = false;
        for (int b = 0; b < B; ++b) {
            relres[b] = beta[b] / bnorm[b];
            act[b] = relres[b] > tol && iters[b] < maxiter && std::isfinite(relres[b]);
            any = any || act[b];
        }
        if (!any) break;
        LSPR_TRY(ctx, cudaMemcpyAsync(a.active, act.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
        // The graph recorded for this configuration.  Recorded launches hold buffer
        // addresses (unchanged while no buffer is reallocated: the allocation count) and
        // sizes that set grids and loop bounds (the counts below); a geometry or tree
        // rebuilt with the same sizes reuses the graph, since the kernels read the new
        // contents from the same buffers.
        const Tree &tr = ctx->tree;
        uint64_t key[24] = {g_alloc_generation.load(), (uint64_t)mode, (uint64_t)B, (uint64_t)m,
                            (uint64_t)(uintptr_t)x_d, (uint64_t)(uintptr_t)b_d, (uint64_t)(uintptr_t)s_d,
                            (uint64_t)N, (uint64_t)me.Ns, (uint64_t)me.nnz, (uint64_t)tr.ready, (uint64_t)tr.P,
                            (uint64_t)tr.NT, (uint64_t)tr.nboxes, (uint64_t)tr.n_p2p_items,
                            (uint64_t)tr.n_m2p_items, (uint64_t)tr.n_p2m_items, (uint64_t)ctx->direct.n,
                            (uint64_t)(uintptr_t)ctx->gm_V.p, (uint64_t)ctx->num_sms, (uint64_t)me.S,
                            (uint64_t)ctx->tensor_cores, (uint64_t)tr.n_tc_items, (uint64_t)tr.n_tcp_items};
        GraphCache *gc = nullptr;
        const bool graphs = ctx->use_graphs && !ctx->timing.enabled;
        for (GraphCache &c : ctx->gcache)
            if (graphs && c.exec && std::equal(key, key + 24, c.key)) gc = &c;
        if (graphs && !gc) {
            gc = &ctx->gcache[0];
            for (GraphCache &c : ctx->gcache)
                if (c.use < gc->use) gc = &c;
            // the operator's buffers must exist before recording (no allocation inside a graph)
            if (skip_mv) LSPR_TRY_ST(apply_operator(ctx, mode, b_d, a.z, s_d, B));
            LSPR_TRY(ctx, cudaStreamSynchronize(st));
            if (capture_cycle(ctx, mode, a, *gc) != LSPR_OK) {
                ctx->use_graphs = false;   // host-driven cycles from now on
                gc = nullptr;
            }
            if (gc) {
                ++ctx->graph_recordings;
                key[0] = g_alloc_generation.load();   // buffers the recording itself sized
                std::copy(key, key + 24, gc->key);
            }
        }
        if (gc) {
            gc->use = ++clock;
            LSPR_TRY(ctx, cudaEventRecord(ctx->ev_g0, st));
            LSPR_TRY(ctx, cudaStreamWaitEvent(ctx->gstream, ctx->ev_g0, 0));
            LSPR_TRY(ctx, cudaGraphLaunch(gc->exec, ctx->gstream));
            LSPR_TRY(ctx, cudaEventRecord(ctx->ev_g1, ctx->gstream));
            LSPR_TRY(ctx, cudaStreamWaitEvent(st, ctx->ev_g1, 0));
        }
        if (!gc) LSPR_TRY_ST(host_cycle(ctx, mode, a, ab.go.p));
        LSPR_TRY(ctx, cudaMemcpyAsync(ctl.data(), ab.ctl.p, sizeof(int) * ctl.size(), cudaMemcpyDeviceToHost, st));
        LSPR_TRY(ctx, cudaMemcpyAsync(est.data(), a.res, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
        LSPR_TRY(ctx, cudaStreamSynchronize(st));
        const int steps = ctl[0];
        if (gc) {
            ++ctx->graph_cycles;
            ctx->n_launches += gc->outer + gc->per_step * steps;
        }
        bool all_met = true;
        for (int b = 0; b < B; ++b) {
            ctx->matvec_count += ctl[1 + 2 * B + b] - iters[b];   // products of the running systems only
            iters[b] = ctl[1 + 2 * B + b];
            if (act[b]) {
                const double r = est[b] / bnorm[b];
                if (!(r <= tol) && iters[b] < maxiter) all_met = false;
                relres[b] = r;
            }
        }
        if (trust_estimate && all_met) break;
    }
    return LSPR_OK;
}

}  // namespace lspr
