// Far-field kernel templates shared by the far-field translation units (the
// per-precision instantiations of the Taylor-order dispatch are compiled separately to
// keep each unit's build short).  The operations are described in farfield.cu.
#pragma once

#include <algorithm>
#include <type_traits>

#include "ffloat.cuh"
#include "lspr_internal.cuh"

namespace lspr {

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = dbl4; };
template <> struct Vec4<ffloat> { using type = ff4; };

// moments accumulate with atomics: FP32/FP64 in place, float-float through an FP64 buffer
template <typename T> struct MomAcc { using type = typename Vec4<T>::type; using scalar = T; };
template <> struct MomAcc<ffloat> { using type = dbl4; using scalar = double; };
static __device__ __forceinline__ void acc_add(float *g, float v) { atomicAdd(g, v); }
static __device__ __forceinline__ void acc_add(double *g, double v) { atomicAdd(g, v); }
static __device__ __forceinline__ void acc_add(double *g, const ffloat &v) { atomicAdd(g, (double)v); }
// four channels added to a 16-byte-aligned float4 of moments: one vector reduction (one L2
// request instead of four)
static __device__ __forceinline__ void acc_add4(float *g, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(g), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}
template <typename S>
static __device__ __forceinline__ void acc_add4(S *g, S a, S b, S c, S d) {
    acc_add(g + 0, a);
    acc_add(g + 1, b);
    acc_add(g + 2, c);
    acc_add(g + 3, d);
}

static __device__ __forceinline__ int panel_of(float w) { return __float_as_int(w); }
static __device__ __forceinline__ int panel_of(double w) { return (int)w; }
static __device__ __forceinline__ int panel_of(const ffloat &w) { return __float_as_int(w.hi); }
// FP32 1/sqrt(x): the hardware approximation with denormal inputs flushed (squared
// distances here are far above the denormal range), which spares the denormal fix-up
// instructions that rsqrtf carries without -ftz
static __device__ __forceinline__ float rsq(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// FP64 1/sqrt(x): the FP32 reciprocal square root as the seed and one Newton-Raphson
// step y <- y + y (1 - x y^2) / 2; a seed error e leaves ~1.5 e^2 (~2e-14 relative).
// Used for squared distances, which stay far inside the FP32 range.
static __device__ __forceinline__ double rsq(double x) {
    const double y = (double)rsqrtf((float)x);
    const double h = fma(-x * y, y, 1.0);
    return fma(0.5 * y, h, y);
}

template <typename T4>
__device__ __forceinline__ T4 zero4() {
    T4 z;
    z.x = 0;
    z.y = 0;
    z.z = 0;
    z.w = 0;
    return z;
}

static __device__ __forceinline__ void atomic_add4(double *o, double a, double b, double c, double d) {
    atomicAdd(o + 0, a);
    atomicAdd(o + 1, b);
    atomicAdd(o + 2, c);
    atomicAdd(o + 3, d);
}

// right-hand sides per chunk: 1 for a single wavelength, else 8 (FP32) or 4 (FP64)
template <typename T>
constexpr int batch_chunk(int B) { return B <= 1 ? 1 : (sizeof(T) == 4 ? 8 : 4); }   // float-float: 8 bytes

// --------------------------------------------------------------------- P2P
constexpr int p2p_warps(int NB) { return NB > 1 ? 4 : 8; }

// Sources [beg, end) against the lane's two targets for right-hand sides [b0, b0 + nb):
// the warp stages 32 sources (position, normal, NB weights) in its shared slice and every
// lane reads them by broadcast; G and dG/dn are formed once per pair.
// CHECK: the range may hold sources of a target's own panel, whose far-rule terms are
// skipped (the exact singular integral replaces them).
template <typename T, typename T4, int NB, bool CHECK>
__device__ __forceinline__ void p2p_range(int beg, int end, int lane, int B, int b0, int nb, T4 (*sh)[32],
                                          T4 (*shw)[NB], const T4 *__restrict__ spos, const T4 *__restrict__ snrm,
                                          const T4 *__restrict__ sw, const T4 &q0, const T4 &q1, int tp0, int tp1,
                                          T (&a0)[NB][4], T (&a1)[NB][4]) {
    for (int base = beg; base < end; base += 32) {
        const int s = base + lane;
        if (s < end) {
            sh[0][lane] = spos[s];
            sh[1][lane] = snrm[s];
#pragma unroll
            for (int k = 0; k < NB; ++k) shw[lane][k] = k < nb ? sw[(int64_t)s * B + b0 + k] : zero4<T4>();
        }
        __syncwarp();
        const int cnt = min(32, end - base);
#pragma unroll 4
        for (int kk = 0; kk < cnt; ++kk) {
            const T4 p = sh[0][kk], n = sh[1][kk];
            const int pid = panel_of(n.w);
            const T dx0 = q0.x - p.x, dy0 = q0.y - p.y, dz0 = q0.z - p.z;
            const T dx1 = q1.x - p.x, dy1 = q1.y - p.y, dz1 = q1.z - p.z;
            T r0 = rsq(dx0 * dx0 + dy0 * dy0 + dz0 * dz0);
            T r1 = rsq(dx1 * dx1 + dy1 * dy1 + dz1 * dz1);
            if (CHECK) {
                r0 = (pid == tp0) ? T(0) : r0;
                r1 = (pid == tp1) ? T(0) : r1;
            }
            const T t0 = (dx0 * n.x + dy0 * n.y + dz0 * n.z) * (r0 * r0) * r0;
            const T t1 = (dx1 * n.x + dy1 * n.y + dz1 * n.z) * (r1 * r1) * r1;
            if constexpr (std::is_same<T, float>::value) {
                // packed FP32 (FFMA2): the (re, im) channel pairs of a weight share the factor,
                // the same fused multiply-adds in half the instructions
                const float2 rr0 = make_float2(r0, r0), rr1 = make_float2(r1, r1);
                const float2 tt0 = make_float2(t0, t0), tt1 = make_float2(t1, t1);
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    const T4 w = shw[kk][k];
                    const float2 wv = make_float2(w.x, w.y), wk = make_float2(w.z, w.w);
                    float2 v0 = __ffma2_rn(rr0, wv, make_float2(a0[k][0], a0[k][1]));
                    float2 k0 = __ffma2_rn(tt0, wk, make_float2(a0[k][2], a0[k][3]));
                    float2 v1 = __ffma2_rn(rr1, wv, make_float2(a1[k][0], a1[k][1]));
                    float2 k1 = __ffma2_rn(tt1, wk, make_float2(a1[k][2], a1[k][3]));
                    a0[k][0] = v0.x; a0[k][1] = v0.y; a0[k][2] = k0.x; a0[k][3] = k0.y;
                    a1[k][0] = v1.x; a1[k][1] = v1.y; a1[k][2] = k1.x; a1[k][3] = k1.y;
                }
            } else if constexpr (std::is_same<T, ffloat>::value) {
                // float-float: products accumulated without per-step renormalisation (ff_mac)
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    const T4 w = shw[kk][k];
                    ff_mac(a0[k][0], r0, w.x);
                    ff_mac(a0[k][1], r0, w.y);
                    ff_mac(a0[k][2], t0, w.z);
                    ff_mac(a0[k][3], t0, w.w);
                    ff_mac(a1[k][0], r1, w.x);
                    ff_mac(a1[k][1], r1, w.y);
                    ff_mac(a1[k][2], t1, w.z);
                    ff_mac(a1[k][3], t1, w.w);
                }
            } else {
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    const T4 w = shw[kk][k];
                    a0[k][0] += r0 * w.x;
                    a0[k][1] += r0 * w.y;
                    a0[k][2] += t0 * w.z;
                    a0[k][3] += t0 * w.w;
                    a1[k][0] += r1 * w.x;
                    a1[k][1] += r1 * w.y;
                    a1[k][2] += t1 * w.z;
                    a1[k][3] += t1 * w.w;
                }
            }
        }
        __syncwarp();
    }
}

// Work units: (item, right-hand-side chunk), item = (target block, source begin, source
// end, own-panel flag); one per warp.  DYNAMIC: a persistent grid whose warps take units
// from an atomic counter.  acc is [panel][B][4].  The kernel does nothing when at least
// skip_from right-hand sides are in use (the tensor-core P2P then takes the product).
template <typename T, int NB, bool DYNAMIC>
__global__ void __launch_bounds__(p2p_warps(NB) * 32)
    p2p_kernel(const int4 *__restrict__ items, int64_t nitems, int nbc, int B,
               const typename Vec4<T>::type *__restrict__ tgt, int64_t ntgt,
               const typename Vec4<T>::type *__restrict__ spos, const typename Vec4<T>::type *__restrict__ snrm,
               const typename Vec4<T>::type *__restrict__ sw, double *__restrict__ acc, int *counter,
               const int *nact, int skip_from) {
    using T4 = typename Vec4<T>::type;
    constexpr int W = p2p_warps(NB);
    __shared__ T4 sh[W][2][32];
    __shared__ T4 shw[W][32][NB];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Bact = nact ? *nact : B;   // right-hand sides in use (the first Bact slots)
    if (Bact >= skip_from) return;       // the tensor-core P2P takes this product
    nbc = (Bact + NB - 1) / NB;
    const int64_t units = nitems * nbc;
    int64_t it = (int64_t)blockIdx.x * W + warp;
    while (true) {
        if (DYNAMIC) {
            int v = 0;
            if (lane == 0) v = atomicAdd(counter, 1);
            it = __shfl_sync(0xffffffffu, v, 0);
        }
        if (it >= units) return;
        const int64_t ii = it / nbc;
        const int b0 = (int)(it - ii * nbc) * NB, nb = min(NB, Bact - b0);
        const int4 item = __ldg(items + ii);
        const int64_t t0 = (int64_t)item.x * kTargetBlock + lane, t1 = t0 + 32;
        const T4 q0 = t0 < ntgt ? tgt[t0] : tgt[0];
        const T4 q1 = t1 < ntgt ? tgt[t1] : tgt[0];
        const int tp0 = panel_of(q0.w), tp1 = panel_of(q1.w);
        T a0[NB][4], a1[NB][4];
#pragma unroll
        for (int k = 0; k < NB; ++k)
#pragma unroll
            for (int c = 0; c < 4; ++c) a0[k][c] = a1[k][c] = T(0);
        if (item.w)
            p2p_range<T, T4, NB, true>(item.y, item.z, lane, B, b0, nb, sh[warp], shw[warp], spos, snrm, sw, q0, q1,
                                       tp0, tp1, a0, a1);
        else
            p2p_range<T, T4, NB, false>(item.y, item.z, lane, B, b0, nb, sh[warp], shw[warp], spos, snrm, sw, q0,
                                        q1, tp0, tp1, a0, a1);
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            if (k >= nb) break;
            if (t0 < ntgt) atomic_add4(acc + 4 * ((int64_t)tp0 * B + b0 + k), a0[k][0], a0[k][1], a0[k][2], a0[k][3]);
            if (t1 < ntgt) atomic_add4(acc + 4 * ((int64_t)tp1 * B + b0 + k), a1[k][0], a1[k][1], a1[k][2], a1[k][3]);
        }
        if (!DYNAMIC) return;
    }
}

// ------------------------------------------------------- P2P, one right-hand side
// FP32 direct sums of one right-hand side with the arithmetic packed two targets at a time
// (f32x2: FADD2 / FMUL2 / FFMA2 on target pairs).  A warp takes one work item (a 64-target block
// and a source range); lane l of half h (h = lane / 16) holds the four targets l, l + 16, l + 32,
// l + 48 of the block as two pairs, and the two halves take alternate sources of each staged
// chunk of 32, so every source operand read from shared memory feeds four targets.  A source is
// staged once per chunk with each component duplicated into both halves of a register pair
// (position, normal, the four weight channels) and its panel id beside; at the end the halves'
// partial sums are added with one exchange and each lane adds two targets into the FP64
// accumulators.  The sums and the own-panel rule are those of p2p_kernel.
constexpr int kP1Warps = 8;
struct P1Src {   // one staged source, 96 bytes: duplicated pairs (the position negated)
    float4 pxy;   // (-px, -px, -py, -py)
    float4 pzn;   // (-pz, -pz, nx, nx)
    float4 nyz;   // (ny, ny, nz, nz)
    float4 wv;    // (w.x, w.x, w.y, w.y): single-layer weight, re and im
    float4 wk;    // (w.z, w.z, w.w, w.w): double-layer weight, re and im
    int pid, pad0, pad1, pad2;
};

template <bool CHECK>
__device__ __forceinline__ void p1_range(int beg, int end, int lane, P1Src *sh, const float4 *__restrict__ spos,
                                         const float4 *__restrict__ snrm, const float4 *__restrict__ sw,
                                         const float2 (&qx)[2], const float2 (&qy)[2], const float2 (&qz)[2],
                                         const int (&tp)[4], float2 (&av)[2][2], float2 (&ak)[2][2]) {
    const int h = lane >> 4;
    for (int base = beg; base < end; base += 32) {
        const int s = base + lane;
        if (s < end) {
            const float4 p = spos[s], n = snrm[s], w = sw[s];
            P1Src e;
            e.pxy = make_float4(-p.x, -p.x, -p.y, -p.y);
            e.pzn = make_float4(-p.z, -p.z, n.x, n.x);
            e.nyz = make_float4(n.y, n.y, n.z, n.z);
            e.wv = make_float4(w.x, w.x, w.y, w.y);
            e.wk = make_float4(w.z, w.z, w.w, w.w);
            e.pid = panel_of(n.w);
            sh[lane] = e;
        }
        __syncwarp();
        const int cnt = min(32, end - base);
#pragma unroll 2
        for (int kk = h; kk < cnt; kk += 2) {
            const float4 a = sh[kk].pxy, b = sh[kk].pzn, c = sh[kk].nyz, wv = sh[kk].wv, wk = sh[kk].wk;
            const float2 px = make_float2(a.x, a.y), py = make_float2(a.z, a.w), pz = make_float2(b.x, b.y);
            const float2 nx = make_float2(b.z, b.w), ny = make_float2(c.x, c.y), nz = make_float2(c.z, c.w);
            const float2 wvr = make_float2(wv.x, wv.y), wvi = make_float2(wv.z, wv.w);
            const float2 wkr = make_float2(wk.x, wk.y), wki = make_float2(wk.z, wk.w);
            const int pid = sh[kk].pid;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float2 dx = __fadd2_rn(qx[u], px), dy = __fadd2_rn(qy[u], py), dz = __fadd2_rn(qz[u], pz);
                const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                float r0 = rsq(r2.x), r1 = rsq(r2.y);
                if (CHECK) {
                    r0 = pid == tp[2 * u] ? 0.f : r0;
                    r1 = pid == tp[2 * u + 1] ? 0.f : r1;
                }
                const float2 r = make_float2(r0, r1);
                const float2 dn = __ffma2_rn(dz, nz, __ffma2_rn(dy, ny, __fmul2_rn(dx, nx)));
                const float2 t = __fmul2_rn(__fmul2_rn(dn, __fmul2_rn(r, r)), r);
                av[u][0] = __ffma2_rn(r, wvr, av[u][0]);
                av[u][1] = __ffma2_rn(r, wvi, av[u][1]);
                ak[u][0] = __ffma2_rn(t, wkr, ak[u][0]);
                ak[u][1] = __ffma2_rn(t, wki, ak[u][1]);
            }
        }
        __syncwarp();
    }
}

template <bool DYNAMIC>
__global__ void __launch_bounds__(kP1Warps * 32)
    p2p1_kernel(const int4 *__restrict__ items, int64_t nitems, const float4 *__restrict__ tgt, int64_t ntgt,
                const float4 *__restrict__ spos, const float4 *__restrict__ snrm, const float4 *__restrict__ sw,
                double *__restrict__ acc, int *counter, const int *nact) {
    __shared__ P1Src sh[kP1Warps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, l = lane & 15, h = lane >> 4;
    if (nact && *nact < 1) return;   // no right-hand side in use
    int64_t it = (int64_t)blockIdx.x * kP1Warps + warp;
    while (true) {
        if (DYNAMIC) {
            int v = 0;
            if (lane == 0) v = atomicAdd(counter, 1);
            it = __shfl_sync(0xffffffffu, v, 0);
        }
        if (it >= nitems) return;
        const int4 item = __ldg(items + it);
        const int64_t t0 = (int64_t)item.x * kTargetBlock + l;
        float4 q[4];
        int tp[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t ti = t0 + 16 * i;
            q[i] = ti < ntgt ? tgt[ti] : tgt[0];
            tp[i] = panel_of(q[i].w);
        }
        const float2 qx[2] = {make_float2(q[0].x, q[1].x), make_float2(q[2].x, q[3].x)};
        const float2 qy[2] = {make_float2(q[0].y, q[1].y), make_float2(q[2].y, q[3].y)};
        const float2 qz[2] = {make_float2(q[0].z, q[1].z), make_float2(q[2].z, q[3].z)};
        float2 av[2][2], ak[2][2];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int c = 0; c < 2; ++c) av[u][c] = ak[u][c] = make_float2(0.f, 0.f);
        if (item.w)
            p1_range<true>(item.y, item.z, lane, sh[warp], spos, snrm, sw, qx, qy, qz, tp, av, ak);
        else
            p1_range<false>(item.y, item.z, lane, sh[warp], spos, snrm, sw, qx, qy, qz, tp, av, ak);
        // add the two halves; lanes of half h keep the pair u = h (targets l + 32 h, l + 16 + 32 h)
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                av[u][c].x += __shfl_xor_sync(0xffffffffu, av[u][c].x, 16);
                av[u][c].y += __shfl_xor_sync(0xffffffffu, av[u][c].y, 16);
                ak[u][c].x += __shfl_xor_sync(0xffffffffu, ak[u][c].x, 16);
                ak[u][c].y += __shfl_xor_sync(0xffffffffu, ak[u][c].y, 16);
            }
        const float2 v0 = h ? av[1][0] : av[0][0], v1 = h ? av[1][1] : av[0][1];
        const float2 k0 = h ? ak[1][0] : ak[0][0], k1 = h ? ak[1][1] : ak[0][1];
        const int64_t ta = t0 + 32 * h, tb = ta + 16;
        const int pa = h ? tp[2] : tp[0], pb = h ? tp[3] : tp[1];
        if (ta < ntgt) atomic_add4(acc + 4 * (int64_t)pa, v0.x, v1.x, k0.x, k1.x);
        if (tb < ntgt) atomic_add4(acc + 4 * (int64_t)pb, v0.y, v1.y, k0.y, k1.y);
        if (!DYNAMIC) return;
    }
}

// ------------------------------------------------------------ multi-indices
// Terms ordered by degree n = k1+k2+k3; within a degree k1 descending, then k2.
__host__ __device__ constexpr int mi_index(int a, int b, int c) {
    const int n = a + b + c;
    return n_terms(n - 1) + (n - a) * (n - a + 1) / 2 + (n - a - b);
}

template <int P>
struct MultiIndex {
    static constexpr int NT = n_terms(P);
    int k[NT][3];
    int deg[NT];
    int m1[NT][3];   // index of k - e_d, or -1
    int m2[NT][3];   // index of k - 2 e_d, or -1
    constexpr MultiIndex() : k(), deg(), m1(), m2() {
        int t = 0;
        for (int n = 0; n <= P; ++n)
            for (int a = n; a >= 0; --a)
                for (int b = n - a; b >= 0; --b) {
                    k[t][0] = a;
                    k[t][1] = b;
                    k[t][2] = n - a - b;
                    deg[t] = n;
                    ++t;
                }
        for (int u = 0; u < NT; ++u)
            for (int d = 0; d < 3; ++d) {
                int e1[3] = {k[u][0], k[u][1], k[u][2]};
                int e2[3] = {k[u][0], k[u][1], k[u][2]};
                e1[d] -= 1;
                e2[d] -= 2;
                m1[u][d] = e1[d] >= 0 ? mi_index(e1[0], e1[1], e1[2]) : -1;
                m2[u][d] = e2[d] >= 0 ? mi_index(e2[0], e2[1], e2[2]) : -1;
            }
    }
};

// decode the multi-index of term t
static __device__ __forceinline__ void mi_decode(int t, int &k1, int &k2, int &k3) {
    int n = 0;
    while (n_terms(n) <= t) ++n;
    int r = t - n_terms(n - 1), a = n;
    while (r > n - a) {
        r -= n - a + 1;
        --a;
    }
    k1 = a;
    k2 = n - a - r;
    k3 = n - k1 - k2;
}

// --------------------------------------------------------------------- M2P
// One target against one box: the coefficients a_k(R) are generated by the recurrence
// and contracted with the box's moments of NB right-hand sides, mom[k * NB + j].
template <typename T, int P, int NB>
__device__ __forceinline__ void m2p_one(T Rx, T Ry, T Rz, const typename Vec4<T>::type *__restrict__ mom,
                                        T (&acc)[NB][4]) {
    constexpr MultiIndex<P> mi{};
    constexpr int NT = MultiIndex<P>::NT;
    const T R[3] = {Rx, Ry, Rz};
    const T r2 = Rx * Rx + Ry * Ry + Rz * Rz;
    T a[NT];
    a[0] = rsq(r2);
    const T ir2 = a[0] * a[0];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const auto m = mom[j];
        acc[j][0] += a[0] * m.x;
        acc[j][1] += a[0] * m.y;
        acc[j][2] += a[0] * m.z;
        acc[j][3] += a[0] * m.w;
    }
#pragma unroll
    for (int t = 1; t < NT; ++t) {
        const int n = mi.deg[t];
        T s1 = T(0), s2 = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (mi.m1[t][d] >= 0) s1 += R[d] * a[mi.m1[t][d]];
            if (mi.m2[t][d] >= 0) s2 += a[mi.m2[t][d]];
        }
        const T c1 = T(-(2.0 * n - 1.0) / n), c2 = T(-(n - 1.0) / n);
        a[t] = (c1 * s1 + c2 * s2) * ir2;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const auto m = mom[t * NB + j];
            acc[j][0] += a[t] * m.x;
            acc[j][1] += a[t] * m.y;
            acc[j][2] += a[t] * m.z;
            acc[j][3] += a[t] * m.w;
        }
    }
}

// warps per block such that the staged moments of every warp fit in 46 KB
template <typename T, int P, int NB>
constexpr int m2p_warps() {
    constexpr int per = n_terms(P) * NB * (int)sizeof(typename Vec4<T>::type);
    constexpr int w = 46000 / per;
    return w < 1 ? 1 : (w > 4 ? 4 : w);
}

// Work units: (item, right-hand-side chunk), item = (target block, list begin, list end):
// each lane evaluates the listed boxes' expansions at its two targets; a box's moments
// for the chunk are staged in the warp's shared slice.
template <typename T, int P, int NB, bool DYNAMIC>
__global__ void __launch_bounds__(m2p_warps<T, P, NB>() * 32)
    m2p_kernel(const int4 *__restrict__ items, int64_t nitems, int nbc, int B,
               const typename Vec4<T>::type *__restrict__ tgt, int64_t ntgt, const int *__restrict__ list,
               const typename Vec4<T>::type *__restrict__ box_c, const typename Vec4<T>::type *__restrict__ mom,
               double *__restrict__ acc, int *counter, const int *nact) {
    using T4 = typename Vec4<T>::type;
    constexpr int NT = n_terms(P);
    constexpr int W = m2p_warps<T, P, NB>();
    __shared__ T4 sm[W][NT * NB];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Bact = nact ? *nact : B;   // right-hand sides in use (the first Bact slots)
    nbc = (Bact + NB - 1) / NB;
    const int64_t units = nitems * nbc;
    int64_t it = (int64_t)blockIdx.x * W + warp;
    while (true) {
        if (DYNAMIC) {
            int v = 0;
            if (lane == 0) v = atomicAdd(counter, 1);
            it = __shfl_sync(0xffffffffu, v, 0);
        }
        if (it >= units) return;
        const int64_t ii = it / nbc;
        const int b0 = (int)(it - ii * nbc) * NB, nb = min(NB, Bact - b0);
        const int4 item = __ldg(items + ii);
        const int64_t t0 = (int64_t)item.x * kTargetBlock + lane, t1 = t0 + 32;
        const T4 q0 = t0 < ntgt ? tgt[t0] : tgt[0];
        const T4 q1 = t1 < ntgt ? tgt[t1] : tgt[0];
        if constexpr (NB == 1) {
            // both targets per staged box; the non-unrolled loop over the two targets keeps
            // the compiler from interleaving their recurrences (register pressure)
            T a0[1][4] = {{0, 0, 0, 0}}, a1[1][4] = {{0, 0, 0, 0}};
#pragma unroll 1
            for (int l = item.y; l < item.z; ++l) {
                const int b = __ldg(list + l);
                const T4 c = box_c[b];
                __syncwarp();
                for (int t = lane; t < NT; t += 32) sm[warp][t] = mom[((int64_t)b * NT + t) * B + b0];
                __syncwarp();
#pragma unroll 1
                for (int h = 0; h < 2; ++h) {
                    if (h == 0) m2p_one<T, P, 1>(q0.x - c.x, q0.y - c.y, q0.z - c.z, sm[warp], a0);
                    else m2p_one<T, P, 1>(q1.x - c.x, q1.y - c.y, q1.z - c.z, sm[warp], a1);
                }
            }
            if (t0 < ntgt)
                atomic_add4(acc + 4 * ((int64_t)panel_of(q0.w) * B + b0), a0[0][0], a0[0][1], a0[0][2], a0[0][3]);
            if (t1 < ntgt)
                atomic_add4(acc + 4 * ((int64_t)panel_of(q1.w) * B + b0), a1[0][0], a1[0][1], a1[0][2], a1[0][3]);
        } else {
            // one target at a time keeps one accumulator set (NB x 4) and one recurrence live
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                const T4 q = h ? q1 : q0;
                T a[NB][4];
#pragma unroll
                for (int j = 0; j < NB; ++j)
#pragma unroll
                    for (int c = 0; c < 4; ++c) a[j][c] = T(0);
#pragma unroll 1
                for (int l = item.y; l < item.z; ++l) {
                    const int b = __ldg(list + l);
                    const T4 c = box_c[b];
                    __syncwarp();
                    for (int q2 = lane; q2 < NT * NB; q2 += 32) {
                        const int t = q2 / NB, j = q2 - t * NB;
                        sm[warp][q2] = j < nb ? mom[((int64_t)b * NT + t) * B + b0 + j] : zero4<T4>();
                    }
                    __syncwarp();
                    m2p_one<T, P, NB>(q.x - c.x, q.y - c.y, q.z - c.z, sm[warp], a);
                }
                const int64_t ti = h ? t1 : t0;
                if (ti < ntgt) {
                    const int64_t tp = panel_of(q.w);
#pragma unroll
                    for (int j = 0; j < NB; ++j)
                        if (j < nb) atomic_add4(acc + 4 * (tp * B + b0 + j), a[j][0], a[j][1], a[j][2], a[j][3]);
                }
            }
        }
        if (!DYNAMIC) return;
    }
}

// ------------------------------------------------------- M2P, several right-hand sides
// With NB right-hand sides the contraction (4 NB channels per coefficient) outweighs the
// recurrence, so a (target block, box) pair is handled as a small matrix product:
//   phase 1  each of 64 threads generates the coefficients a_k of one target into shared
//            memory, coef[k][target];
//   phase 2  C[target][channel] += sum_k coef[k][target] M[k][channel], each thread owning a
//            4-target x (CH/4)-channel tile of C in registers (CH = 4 NB channels).
// The tile stays in registers over all boxes of the work unit; one block of 64 threads
// works on one unit at a time.
constexpr int kM2PGemmThreads = 64;

template <typename T, int P>
__device__ __forceinline__ void m2p_coeffs(T Rx, T Ry, T Rz, T *__restrict__ out) {   // out[k * 64]
    constexpr MultiIndex<P> mi{};
    constexpr int NT = MultiIndex<P>::NT;
    const T R[3] = {Rx, Ry, Rz};
    T a[NT];
    a[0] = rsq(Rx * Rx + Ry * Ry + Rz * Rz);
    const T ir2 = a[0] * a[0];
    out[0] = a[0];
#pragma unroll
    for (int t = 1; t < NT; ++t) {
        const int n = mi.deg[t];
        T s1 = T(0), s2 = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (mi.m1[t][d] >= 0) s1 += R[d] * a[mi.m1[t][d]];
            if (mi.m2[t][d] >= 0) s2 += a[mi.m2[t][d]];
        }
        const T c1 = T(-(2.0 * n - 1.0) / n), c2 = T(-(n - 1.0) / n);
        a[t] = (c1 * s1 + c2 * s2) * ir2;
        out[t * kM2PGemmThreads] = a[t];
    }
}

template <typename T, int P, int NB>
__host__ __device__ constexpr size_t m2p_gemm_smem() {
    return (size_t)n_terms(P) * (kM2PGemmThreads + 4 * NB) * sizeof(T);
}

template <typename T, int P, int NB>
__global__ void __launch_bounds__(kM2PGemmThreads)
    m2p_gemm_kernel(const int4 *__restrict__ items, int64_t nitems, int B,
                    const typename Vec4<T>::type *__restrict__ tgt, int64_t ntgt, const int *__restrict__ list,
                    const typename Vec4<T>::type *__restrict__ box_c, const typename Vec4<T>::type *__restrict__ mom,
                    double *__restrict__ acc, int *counter, const int *nact) {
    using T4 = typename Vec4<T>::type;
    constexpr int NT = n_terms(P);
    constexpr int CH = 4 * NB;           // channels of a right-hand-side chunk
    constexpr int CPT = CH / 4;          // channels per thread (4 channel groups)
    extern __shared__ __align__(16) unsigned char gemm_smem[];
    T *coef = (T *)gemm_smem;            // [NT][64]
    T *ms = coef + NT * kM2PGemmThreads; // [NT][CH]
    __shared__ int64_t unit_s;
    const int tid = threadIdx.x;
    const int tg = tid & 15, cg = tid >> 4;   // targets 4 tg .. 4 tg + 3, channels CPT cg ..
    const int Bact = nact ? *nact : B;
    const int nbc = (Bact + NB - 1) / NB;
    const int64_t units = nitems * nbc;
    while (true) {
        __syncthreads();   // the previous unit's readers are done with unit_s and the buffers
        if (tid == 0) unit_s = atomicAdd(counter, 1);
        __syncthreads();
        const int64_t it = unit_s;
        if (it >= units) return;
        const int64_t ii = it / nbc;
        const int b0 = (int)(it - ii * nbc) * NB, nb = min(NB, Bact - b0);
        const int4 item = __ldg(items + ii);
        const int64_t tb = (int64_t)item.x * kTargetBlock;
        const int64_t ti = tb + tid;
        const T4 q = ti < ntgt ? tgt[ti] : tgt[0];
        T c[4][CPT];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < CPT; ++j) c[i][j] = T(0);
#pragma unroll 1
        for (int l = item.y; l < item.z; ++l) {
            const int b = __ldg(list + l);
            const T4 bc = box_c[b];
            __syncthreads();   // phase 2 of the previous box is done with coef and ms
            for (int q2 = tid; q2 < NT * NB; q2 += kM2PGemmThreads) {
                const int t = q2 / NB, j = q2 - t * NB;
                const T4 m = j < nb ? mom[((int64_t)b * NT + t) * B + b0 + j] : zero4<T4>();
                T *d = ms + t * CH + 4 * j;
                d[0] = m.x;
                d[1] = m.y;
                d[2] = m.z;
                d[3] = m.w;
            }
            m2p_coeffs<T, P>(q.x - bc.x, q.y - bc.y, q.z - bc.z, coef + tid);
            __syncthreads();
#pragma unroll 2
            for (int k = 0; k < NT; ++k) {
                T a4[4], m8[CPT];
#pragma unroll
                for (int i = 0; i < 4; ++i) a4[i] = coef[k * kM2PGemmThreads + 4 * tg + i];
#pragma unroll
                for (int j = 0; j < CPT; ++j) m8[j] = ms[k * CH + CPT * cg + j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < CPT; ++j) c[i][j] += a4[i] * m8[j];
            }
        }
        // channel CPT cg + j = component (CPT cg + j) % 4 of right-hand side b0 + (CPT cg + j) / 4
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t t = tb + 4 * tg + i;
            if (t >= ntgt) continue;
            const int64_t tp = panel_of(tgt[t].w);
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                const int ch = CPT * cg + j, r = ch >> 2;
                if (r < nb) atomicAdd(acc + 4 * (tp * B + b0 + r) + (ch & 3), (double)c[i][j]);
            }
        }
    }
}

// --------------------------------------------------------------------- P2M
constexpr int kP2MTile = 32;

// binomial coefficients C(n, r), n, r <= kMaxP
static __constant__ float c_binom[kMaxP + 1][kMaxP + 1] = {
    {1, 0, 0, 0, 0, 0, 0, 0, 0},     {1, 1, 0, 0, 0, 0, 0, 0, 0},     {1, 2, 1, 0, 0, 0, 0, 0, 0},
    {1, 3, 3, 1, 0, 0, 0, 0, 0},     {1, 4, 6, 4, 1, 0, 0, 0, 0},     {1, 5, 10, 10, 5, 1, 0, 0, 0},
    {1, 6, 15, 20, 15, 6, 1, 0, 0},  {1, 7, 21, 35, 35, 21, 7, 1, 0}, {1, 8, 28, 56, 70, 56, 28, 8, 1}};

// One block per work unit (leaf chunk, right-hand-side chunk), one thread per term k.
// The chunk's moments about the leaf centre c are added to the leaf if some target block
// accepted it, and shifted into every accepted ancestor a (upward pass folded in):
//   M_k(a) = sum_{l <= k} C(k, l) (a - c)^(k - l) M_l(c),  C(k, l) = prod_d binom(k_d, l_d),
// valid for both moment kinds since (a - y)^k = ((a - c) + (c - y))^k.
template <typename T, int P, int NB>
__global__ void p2m_kernel(const int4 *__restrict__ items, int64_t nitems, int nbc, int B,
                           const typename Vec4<T>::type *__restrict__ spos,
                           const typename Vec4<T>::type *__restrict__ snrm, const typename Vec4<T>::type *__restrict__ sw,
                           const typename Vec4<T>::type *__restrict__ box_c, const int *__restrict__ parent,
                           const int *__restrict__ used, typename MomAcc<T>::type *__restrict__ mom,
                           const int *nact) {
    using S = typename MomAcc<T>::scalar;
    using T4 = typename Vec4<T>::type;
    constexpr int NT = n_terms(P);
    __shared__ T pw[kP2MTile][3][P + 1];
    __shared__ T4 shn[kP2MTile];
    __shared__ T4 shw[kP2MTile][NB];
    __shared__ T4 lm[NT][NB];
    __shared__ T dpw[3][P + 1];
    const int64_t u = blockIdx.x;
    if (u >= nitems * nbc) return;
    const int64_t ii = u / nbc;
    const int b0 = (int)(u - ii * nbc) * NB;
    const int Bact = nact ? *nact : B;   // right-hand sides in use (the first Bact slots)
    if (b0 >= Bact) return;
    const int nb = min(NB, Bact - b0);
    const int4 item = items[ii];
    const T4 c = box_c[item.x];
    const int t = threadIdx.x;
    int k1 = 0, k2 = 0, k3 = 0;
    if (t < NT) mi_decode(t, k1, k2, k3);
    T acc[NB][4];
#pragma unroll
    for (int j = 0; j < NB; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][q] = T(0);
    for (int base = item.y; base < item.z; base += kP2MTile) {
        __syncthreads();
        const int cnt = min(kP2MTile, item.z - base);
        if (t < cnt) {
            const T4 y = spos[base + t];
            const T d[3] = {c.x - y.x, c.y - y.y, c.z - y.z};
            for (int q = 0; q < 3; ++q) {
                T v = 1;
                for (int e = 0; e <= P; ++e) {
                    pw[t][q][e] = v;
                    v *= d[q];
                }
            }
            shn[t] = snrm[base + t];
#pragma unroll
            for (int j = 0; j < NB; ++j) shw[t][j] = j < nb ? sw[(int64_t)(base + t) * B + b0 + j] : zero4<T4>();
        }
        __syncthreads();
        if (t < NT) {
            for (int s = 0; s < cnt; ++s) {
                const T px = pw[s][0][k1], py = pw[s][1][k2], pz = pw[s][2][k3];
                const T mono = px * py * pz;
                const T4 n = shn[s];
                T dm = 0;
                if (k1) dm += n.x * T(k1) * pw[s][0][k1 - 1] * py * pz;
                if (k2) dm += n.y * T(k2) * px * pw[s][1][k2 - 1] * pz;
                if (k3) dm += n.z * T(k3) * px * py * pw[s][2][k3 - 1];
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    const T4 w = shw[s][j];
                    acc[j][0] += w.x * mono;
                    acc[j][1] += w.y * mono;
                    acc[j][2] -= w.z * dm;
                    acc[j][3] -= w.w * dm;
                }
            }
        }
    }
    if (t < NT) {
        const bool own = used[item.x] != 0;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            T4 o;
            o.x = acc[j][0]; o.y = acc[j][1]; o.z = acc[j][2]; o.w = acc[j][3];
            lm[t][j] = o;
            if (own && j < nb) {
                S *g = (S *)(mom + ((int64_t)item.x * NT + t) * B + b0 + j);
                acc_add4(g, (S)acc[j][0], (S)acc[j][1], (S)acc[j][2], (S)acc[j][3]);
            }
        }
    }
    for (int A = parent[item.x]; A >= 0; A = parent[A]) {
        if (!used[A]) continue;
        __syncthreads();
        if (t < 3) {
            const T4 ca = box_c[A];
            const T delta = t == 0 ? ca.x - c.x : (t == 1 ? ca.y - c.y : ca.z - c.z);
            T v = 1;
            for (int e = 0; e <= P; ++e) {
                dpw[t][e] = v;
                v *= delta;
            }
        }
        __syncthreads();
        if (t < NT) {
#pragma unroll
            for (int j = 0; j < NB; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[j][q] = T(0);
            for (int l1 = 0; l1 <= k1; ++l1)
                for (int l2 = 0; l2 <= k2; ++l2)
                    for (int l3 = 0; l3 <= k3; ++l3) {
                        const T coef = T(c_binom[k1][l1] * c_binom[k2][l2] * c_binom[k3][l3]) * dpw[0][k1 - l1] *
                                       dpw[1][k2 - l2] * dpw[2][k3 - l3];
                        const int li = mi_index(l1, l2, l3);
#pragma unroll
                        for (int j = 0; j < NB; ++j) {
                            const T4 m = lm[li][j];
                            acc[j][0] += coef * m.x;
                            acc[j][1] += coef * m.y;
                            acc[j][2] += coef * m.z;
                            acc[j][3] += coef * m.w;
                        }
                    }
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                if (j >= nb) break;
                S *g = (S *)(mom + ((int64_t)A * NT + t) * B + b0 + j);
                acc_add4(g, (S)acc[j][0], (S)acc[j][1], (S)acc[j][2], (S)acc[j][3]);
            }
        }
    }
}

// persistent-grid size: resident blocks per SM x SMs (queried once per kernel instance)
template <class K>
static unsigned persistent_grid(lspr_ctx *ctx, K kernel, int threads, int *cache) {
    if (*cache <= 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        *cache = per_sm;
    }
    return (unsigned)(*cache * std::max(1, ctx->num_sms));
}

// per-precision views of the context's geometry and scratch
template <typename T> struct Views;
template <> struct Views<float> {
    static const float4 *tgt(lspr_ctx *c) { return c->wo.tgt32.p; }
    static const float4 *spos(lspr_ctx *c) { return c->wo.spos32.p; }
    static const float4 *snrm(lspr_ctx *c) { return c->wo.snrm32.p; }
    static const float4 *w(lspr_ctx *c) { return c->w32.p; }
    static const float4 *bc(lspr_ctx *c) { return c->tree.box_c32.p; }
    static const float4 *mom(lspr_ctx *c) { return c->tree.mom32.p; }
    static float4 *mom_acc(lspr_ctx *c) { return c->tree.mom32.p; }
};
template <> struct Views<double> {
    static const dbl4 *tgt(lspr_ctx *c) { return c->wo.tgt64.p; }
    static const dbl4 *spos(lspr_ctx *c) { return c->wo.spos64.p; }
    static const dbl4 *snrm(lspr_ctx *c) { return c->wo.snrm64.p; }
    static const dbl4 *w(lspr_ctx *c) { return c->w64.p; }
    static const dbl4 *bc(lspr_ctx *c) { return c->tree.box_c64.p; }
    static const dbl4 *mom(lspr_ctx *c) { return c->tree.mom64.p; }
    static dbl4 *mom_acc(lspr_ctx *c) { return c->tree.mom64.p; }
};
template <> struct Views<ffloat> {
    static const ff4 *tgt(lspr_ctx *c) { return c->wo.tgt_ff.p; }
    static const ff4 *spos(lspr_ctx *c) { return c->wo.spos_ff.p; }
    static const ff4 *snrm(lspr_ctx *c) { return c->wo.snrm_ff.p; }
    static const ff4 *w(lspr_ctx *c) { return c->w_ff.p; }
    static const ff4 *bc(lspr_ctx *c) { return c->tree.box_c_ff.p; }
    static const ff4 *mom(lspr_ctx *c) { return c->tree.mom_ff.p; }
    static dbl4 *mom_acc(lspr_ctx *c) { return c->tree.mom64.p; }
};

template <typename T, int NB>
static void p2p_launch(lspr_ctx *ctx, const int4 *items, int64_t nitems, int B, double *acc, cudaStream_t st,
                       int *counter, int skip_from = 1 << 30) {
    static int occ = 0;
    constexpr int W = p2p_warps(NB);
    const int nbc = (B + NB - 1) / NB;
    const unsigned grid = std::min<unsigned>(grid_for(nitems * nbc, W),
                                             persistent_grid(ctx, p2p_kernel<T, NB, true>, W * 32, &occ));
    p2p_kernel<T, NB, true><<<grid, W * 32, 0, st>>>(items, nitems, nbc, B, Views<T>::tgt(ctx), ctx->mesh.N,
                                                      Views<T>::spos(ctx), Views<T>::snrm(ctx), Views<T>::w(ctx),
                                                      acc, counter, ctx->rhs_nact, skip_from);
}

// the packed single-right-hand-side P2P (FP32)
static void p2p1_launch(lspr_ctx *ctx, const int4 *items, int64_t nitems, double *acc, cudaStream_t st,
                        int *counter) {
    static int occ = 0;
    const unsigned grid = std::min<unsigned>(grid_for(nitems, kP1Warps),
                                             persistent_grid(ctx, p2p1_kernel<true>, kP1Warps * 32, &occ));
    p2p1_kernel<true><<<grid, kP1Warps * 32, 0, st>>>(items, nitems, Views<float>::tgt(ctx), ctx->mesh.N,
                                                       Views<float>::spos(ctx), Views<float>::snrm(ctx),
                                                       Views<float>::w(ctx), acc, counter, ctx->rhs_nact);
}

template <typename T, int P, int NB>
static void p2m_launch(lspr_ctx *ctx, int B) {
    Tree &tr = ctx->tree;
    const int threads = ((n_terms(P) + 31) / 32) * 32;
    const int nbc = (B + NB - 1) / NB;
    p2m_kernel<T, P, NB><<<(unsigned)(tr.n_p2m_items * nbc), threads, 0, ctx->stream>>>(
        tr.p2m_items.p, tr.n_p2m_items, nbc, B, Views<T>::spos(ctx), Views<T>::snrm(ctx), Views<T>::w(ctx),
        Views<T>::bc(ctx), tr.box_parent.p, tr.box_used.p, Views<T>::mom_acc(ctx), ctx->rhs_nact);
}

template <typename T, int P, int NB>
static void m2p_launch(lspr_ctx *ctx, double *acc, int *counter, int B) {
    static int occ = 0;
    static int smem_set[kSmemDevices] = {};
    Tree &tr = ctx->tree;
    if constexpr (NB > 1) {
        constexpr size_t smem = m2p_gemm_smem<T, P, NB>();
        // a failure here shows as the launch's error, which the caller checks
        (void)allow_smem(m2p_gemm_kernel<T, P, NB>, (int)smem, ctx->device, smem_set);
        if (occ <= 0) {
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, m2p_gemm_kernel<T, P, NB>, kM2PGemmThreads,
                                                              smem) != cudaSuccess ||
                per_sm < 1)
                per_sm = 1;
            occ = per_sm;
        }
        const int nbc = (B + NB - 1) / NB;
        const unsigned grid = (unsigned)std::min<int64_t>(tr.n_m2p_items * nbc, (int64_t)occ * std::max(1, ctx->num_sms));
        m2p_gemm_kernel<T, P, NB><<<grid, kM2PGemmThreads, smem, ctx->stream>>>(
            tr.m2p_items.p, tr.n_m2p_items, B, Views<T>::tgt(ctx), ctx->mesh.N, tr.m2p_list.p, Views<T>::bc(ctx),
            Views<T>::mom(ctx), acc, counter, ctx->rhs_nact);
        return;
    }
    constexpr int W = m2p_warps<T, P, NB>();
    const int nbc = (B + NB - 1) / NB;
    const unsigned grid = std::min<unsigned>(grid_for(tr.n_m2p_items * nbc, W),
                                             persistent_grid(ctx, m2p_kernel<T, P, NB, true>, W * 32, &occ));
    m2p_kernel<T, P, NB, true><<<grid, W * 32, 0, ctx->stream>>>(tr.m2p_items.p, tr.n_m2p_items, nbc, B,
                                                                  Views<T>::tgt(ctx), ctx->mesh.N, tr.m2p_list.p,
                                                                  Views<T>::bc(ctx), Views<T>::mom(ctx), acc, counter,
                                                                  ctx->rhs_nact);
}

// dispatch over the compiled Taylor orders and over single / chunked right-hand sides
#define LSPR_DISPATCH_P(FN, T, B, ...)                                                      \
    do {                                                                                    \
        constexpr int NBB = batch_chunk<T>(2);                                              \
        switch (ctx->tree.P) {                                                              \
        case 1: if ((B) == 1) FN<T, 1, 1>(__VA_ARGS__); else FN<T, 1, NBB>(__VA_ARGS__); break; \
        case 2: if ((B) == 1) FN<T, 2, 1>(__VA_ARGS__); else FN<T, 2, NBB>(__VA_ARGS__); break; \
        case 3: if ((B) == 1) FN<T, 3, 1>(__VA_ARGS__); else FN<T, 3, NBB>(__VA_ARGS__); break; \
        case 4: if ((B) == 1) FN<T, 4, 1>(__VA_ARGS__); else FN<T, 4, NBB>(__VA_ARGS__); break; \
        case 5: if ((B) == 1) FN<T, 5, 1>(__VA_ARGS__); else FN<T, 5, NBB>(__VA_ARGS__); break; \
        case 6: if ((B) == 1) FN<T, 6, 1>(__VA_ARGS__); else FN<T, 6, NBB>(__VA_ARGS__); break; \
        case 7: if ((B) == 1) FN<T, 7, 1>(__VA_ARGS__); else FN<T, 7, NBB>(__VA_ARGS__); break; \
        case 8: if ((B) == 1) FN<T, 8, 1>(__VA_ARGS__); else FN<T, 8, NBB>(__VA_ARGS__); break; \
        default: return LSPR_E_ARG;                                                         \
        }                                                                                   \
    } while (0)

// per-precision Taylor-order dispatch (farfield_f32.cu, farfield_f64.cu, farfield_ff.cu)
int p2m_orders_f32(lspr_ctx *ctx, int B);
int p2m_orders_f64(lspr_ctx *ctx, int B);
int p2m_orders_ff(lspr_ctx *ctx, int B);
int m2p_orders_f32(lspr_ctx *ctx, double *acc, int *counter, int B);
// tensor-core M2P (m2p_tc.cu): FP32 operands as 3xTF32, B >= 2; LSPR_E_STATE otherwise
int m2p_tc_launch(lspr_ctx *ctx, double *acc, int *counter, int B);
// tensor-core P2P of the tree mode (p2p_tc.cu): FP32 weights as TF32 high/low parts, B >= 2
// min_rhs: the kernel does nothing when fewer right-hand sides are in use (the FP32-pipe P2P
// then takes the product)
int p2p_tc_launch(lspr_ctx *ctx, double *acc, cudaStream_t st, int *counter, int B, int min_rhs);
int m2p_orders_f64(lspr_ctx *ctx, double *acc, int *counter, int B);
int m2p_orders_ff(lspr_ctx *ctx, double *acc, int *counter, int B);
// float-float P2P of B >= 2 right-hand sides (farfield_ff.cu), one target per lane
int p2p_ff_multi(lspr_ctx *ctx, const int4 *items, int64_t nitems, int B, double *acc, cudaStream_t st, int *counter);

}  // namespace lspr
