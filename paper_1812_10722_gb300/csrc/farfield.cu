// Far-field kernels of the matrix-vector product (Sec. II.D, Eq. summation):
// sources are the far-rule Gauss nodes y_j with weights q_j = w_j A_j dphi_j / (4 pi)
// (single layer) and mu_j = w_j A_j phi_j / (4 pi) (double layer); targets are the
// panel centroids x_i.  For every target
//     Vd_i = sum_j q_j / |x_i - y_j|,   Kp_i = sum_j mu_j (x_i - y_j).n_j / |x_i - y_j|^3
// over all sources except those of panel i itself (its singular integral is
// added exactly by the near-field correction).  Complex weights are carried as
// two real channels (the paper's real/imaginary split of the treecode work).
//
//   p2p_kernel  direct sums of a 64-target block against a contiguous source range
//   p2m_kernel  Cartesian Taylor moments of a leaf about its centre c, shifted into
//               every accepted ancestor box:
//                 M^V_k = sum_j q_j (c - y_j)^k
//                 M^K_k = sum_j mu_j * (-sum_d n_{j,d} k_d (c - y_j)^(k - e_d))
//   m2p_kernel  Vd_i += sum_{|k|<=P} a_k(x_i - c) M^V_k (same for K), with
//               a_k(R) = D^k (1/|R|) / k! from the recurrence
//               n |R|^2 a_k + (2n-1) sum_d R_d a_(k-e_d) + (n-1) sum_d a_(k-2e_d) = 0,
//               n = |k|, a_0 = 1/|R|.
// Partial sums are formed in the kernel's precision (FP32 or FP64) per work
// item and accumulated in FP64 with atomics.
#include <algorithm>

#include "lspr_internal.cuh"

namespace lspr {

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = dbl4; };

__device__ __forceinline__ int panel_of(float w) { return __float_as_int(w); }
__device__ __forceinline__ int panel_of(double w) { return (int)w; }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
// FP64 1/sqrt(x): the FP32 reciprocal square root as the seed and one Newton-Raphson
// step y <- y + y (1 - x y^2) / 2; a seed error e leaves ~1.5 e^2 (~2e-14 relative).
// Used for squared distances, which stay far inside the FP32 range.
__device__ __forceinline__ double rsq(double x) {
    const double y = (double)rsqrtf((float)x);
    const double h = fma(-x * y, y, 1.0);
    return fma(0.5 * y, h, y);
}

// ----------------------------------------------------------------- weights
template <typename T4>
__global__ void weights_kernel(int64_t Ns, int64_t N, const dbl4 *__restrict__ spos64,
                               const int *__restrict__ src_panel, const double2 *__restrict__ x, T4 *__restrict__ w) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= Ns) return;
    const int p = src_panel[s];
    const double wa = spos64[s].w * kInv4Pi;
    const double2 phi = x[p], dphi = x[N + p];
    T4 o;
    o.x = wa * dphi.x;
    o.y = wa * dphi.y;
    o.z = wa * phi.x;
    o.w = wa * phi.y;
    w[s] = o;
}

// --------------------------------------------------------------------- P2P
template <typename T>
struct P2PAcc {
    T vr, vi, kr, ki;
};

// One (target, source) pair.  CHECK: the item may hold sources of the target's own
// panel, whose far-rule terms are skipped (the exact singular integral replaces them).
template <typename T, typename T4, bool CHECK>
__device__ __forceinline__ void p2p_pair(const T4 &p, const T4 &n, const T4 &w, int pid, T tx, T ty, T tz, int tp,
                                         P2PAcc<T> &a) {
    const T dx = tx - p.x, dy = ty - p.y, dz = tz - p.z;
    const T r2 = dx * dx + dy * dy + dz * dz;
    T ri = rsq(r2);
    if (CHECK) ri = (pid == tp) ? T(0) : ri;
    const T dn = dx * n.x + dy * n.y + dz * n.z;
    const T t3 = dn * (ri * ri) * ri;
    a.vr += ri * w.x;
    a.vi += ri * w.y;
    a.kr += t3 * w.z;
    a.ki += t3 * w.w;
}

constexpr int kP2PWarps = 8;

// Sources [beg, end) against the lane's two targets; the warp stages 32 sources at a
// time in its shared-memory slice and every lane reads them by broadcast.
template <typename T, typename T4, bool CHECK>
__device__ __forceinline__ void p2p_range(int beg, int end, int lane, T4 (*sh)[32], const T4 *__restrict__ spos,
                                          const T4 *__restrict__ snrm, const T4 *__restrict__ sw, const T4 &q0,
                                          const T4 &q1, int tp0, int tp1, P2PAcc<T> &a0, P2PAcc<T> &a1) {
    for (int base = beg; base < end; base += 32) {
        const int s = base + lane;
        if (s < end) {
            sh[0][lane] = spos[s];
            sh[1][lane] = snrm[s];
            sh[2][lane] = sw[s];
        }
        __syncwarp();
        const int cnt = min(32, end - base);
        if (cnt == 32) {
#pragma unroll 8
            for (int k = 0; k < 32; ++k) {
                const T4 p = sh[0][k], n = sh[1][k], w = sh[2][k];
                const int pid = panel_of(n.w);
                p2p_pair<T, T4, CHECK>(p, n, w, pid, q0.x, q0.y, q0.z, tp0, a0);
                p2p_pair<T, T4, CHECK>(p, n, w, pid, q1.x, q1.y, q1.z, tp1, a1);
            }
        } else {
            for (int k = 0; k < cnt; ++k) {
                const T4 p = sh[0][k], n = sh[1][k], w = sh[2][k];
                const int pid = panel_of(n.w);
                p2p_pair<T, T4, CHECK>(p, n, w, pid, q0.x, q0.y, q0.z, tp0, a0);
                p2p_pair<T, T4, CHECK>(p, n, w, pid, q1.x, q1.y, q1.z, tp1, a1);
            }
        }
        __syncwarp();
    }
}

__device__ __forceinline__ void atomic_add4(double *o, double a, double b, double c, double d) {
    atomicAdd(o + 0, a);
    atomicAdd(o + 1, b);
    atomicAdd(o + 2, c);
    atomicAdd(o + 3, d);
}

// Work items (target block, source begin, source end, own-panel flag), one per warp.
// DYNAMIC: a persistent grid whose warps take items from an atomic counter.
template <typename T, bool DYNAMIC>
__global__ void __launch_bounds__(kP2PWarps * 32) p2p_kernel(const int4 *__restrict__ items, int64_t nitems,
                                                             const typename Vec4<T>::type *__restrict__ tgt, int64_t ntgt,
                                                             const typename Vec4<T>::type *__restrict__ spos,
                                                             const typename Vec4<T>::type *__restrict__ snrm,
                                                             const typename Vec4<T>::type *__restrict__ sw,
                                                             double *__restrict__ acc, int *counter) {
    using T4 = typename Vec4<T>::type;
    __shared__ T4 sh[kP2PWarps][3][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t it = (int64_t)blockIdx.x * kP2PWarps + warp;
    while (true) {
        if (DYNAMIC) {
            int v = 0;
            if (lane == 0) v = atomicAdd(counter, 1);
            it = __shfl_sync(0xffffffffu, v, 0);
        }
        if (it >= nitems) return;
        const int4 item = __ldg(items + it);
        const int64_t t0 = (int64_t)item.x * kTargetBlock + lane, t1 = t0 + 32;
        const T4 q0 = t0 < ntgt ? tgt[t0] : tgt[0];
        const T4 q1 = t1 < ntgt ? tgt[t1] : tgt[0];
        const int tp0 = panel_of(q0.w), tp1 = panel_of(q1.w);
        P2PAcc<T> a0 = {0, 0, 0, 0}, a1 = {0, 0, 0, 0};
        if (item.w)
            p2p_range<T, T4, true>(item.y, item.z, lane, sh[warp], spos, snrm, sw, q0, q1, tp0, tp1, a0, a1);
        else
            p2p_range<T, T4, false>(item.y, item.z, lane, sh[warp], spos, snrm, sw, q0, q1, tp0, tp1, a0, a1);
        if (t0 < ntgt) atomic_add4(acc + 4 * (int64_t)tp0, a0.vr, a0.vi, a0.kr, a0.ki);
        if (t1 < ntgt) atomic_add4(acc + 4 * (int64_t)tp1, a1.vr, a1.vi, a1.kr, a1.ki);
        if (!DYNAMIC) return;
    }
}

// item.w = 1 iff some source of [item.y, item.z) belongs to a panel of the item's target block
__global__ void item_flags_kernel(int4 *items, int64_t nitems, const int *__restrict__ src_tblock) {
    const int64_t it = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (it >= nitems) return;
    int4 item = items[it];
    int hit = 0;
    for (int s = item.y + lane; s < item.z; s += 32) hit |= src_tblock[s] == item.x;
    hit = __any_sync(0xffffffffu, hit);
    if (lane == 0) items[it].w = hit;
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

// --------------------------------------------------------------------- M2P
template <typename T, int P>
__device__ __forceinline__ void m2p_one(T Rx, T Ry, T Rz, const typename Vec4<T>::type *__restrict__ mom,
                                        P2PAcc<T> &acc) {
    constexpr MultiIndex<P> mi{};
    constexpr int NT = MultiIndex<P>::NT;
    const T R[3] = {Rx, Ry, Rz};
    const T r2 = Rx * Rx + Ry * Ry + Rz * Rz;
    T a[NT];
    a[0] = rsq(r2);
    const T ir2 = a[0] * a[0];
    {
        const auto m = mom[0];
        acc.vr += a[0] * m.x;
        acc.vi += a[0] * m.y;
        acc.kr += a[0] * m.z;
        acc.ki += a[0] * m.w;
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
        const auto m = mom[t];
        acc.vr += a[t] * m.x;
        acc.vi += a[t] * m.y;
        acc.kr += a[t] * m.z;
        acc.ki += a[t] * m.w;
    }
}

constexpr int kM2PWarps = 4;

// Work items (target block, list begin, list end): each lane evaluates the boxes'
// expansions at its two targets; a box's moments are staged in the warp's shared slice.
template <typename T, int P, bool DYNAMIC>
__global__ void __launch_bounds__(kM2PWarps * 32) m2p_kernel(const int4 *__restrict__ items, int64_t nitems,
                                                             const typename Vec4<T>::type *__restrict__ tgt, int64_t ntgt,
                                                             const int *__restrict__ list,
                                                             const typename Vec4<T>::type *__restrict__ box_c,
                                                             const typename Vec4<T>::type *__restrict__ mom,
                                                             double *__restrict__ acc, int *counter) {
    using T4 = typename Vec4<T>::type;
    constexpr int NT = n_terms(P);
    __shared__ T4 sm[kM2PWarps][NT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t it = (int64_t)blockIdx.x * kM2PWarps + warp;
    while (true) {
        if (DYNAMIC) {
            int v = 0;
            if (lane == 0) v = atomicAdd(counter, 1);
            it = __shfl_sync(0xffffffffu, v, 0);
        }
        if (it >= nitems) return;
        const int4 item = __ldg(items + it);
        const int64_t t0 = (int64_t)item.x * kTargetBlock + lane, t1 = t0 + 32;
        const T4 q0 = t0 < ntgt ? tgt[t0] : tgt[0];
        const T4 q1 = t1 < ntgt ? tgt[t1] : tgt[0];
        P2PAcc<T> a0 = {0, 0, 0, 0}, a1 = {0, 0, 0, 0};
#pragma unroll 1
        for (int l = item.y; l < item.z; ++l) {
            const int b = __ldg(list + l);
            const T4 c = box_c[b];
            __syncwarp();
            for (int t = lane; t < NT; t += 32) sm[warp][t] = mom[(int64_t)b * NT + t];
            __syncwarp();
            m2p_one<T, P>(q0.x - c.x, q0.y - c.y, q0.z - c.z, sm[warp], a0);
            m2p_one<T, P>(q1.x - c.x, q1.y - c.y, q1.z - c.z, sm[warp], a1);
        }
        if (t0 < ntgt) atomic_add4(acc + 4 * (int64_t)panel_of(q0.w), a0.vr, a0.vi, a0.kr, a0.ki);
        if (t1 < ntgt) atomic_add4(acc + 4 * (int64_t)panel_of(q1.w), a1.vr, a1.vi, a1.kr, a1.ki);
        if (!DYNAMIC) return;
    }
}

// --------------------------------------------------------------------- P2M
constexpr int kP2MTile = 32;

// binomial coefficients C(n, r), n, r <= kMaxP
__constant__ float c_binom[kMaxP + 1][kMaxP + 1] = {
    {1, 0, 0, 0, 0, 0, 0, 0, 0},     {1, 1, 0, 0, 0, 0, 0, 0, 0},     {1, 2, 1, 0, 0, 0, 0, 0, 0},
    {1, 3, 3, 1, 0, 0, 0, 0, 0},     {1, 4, 6, 4, 1, 0, 0, 0, 0},     {1, 5, 10, 10, 5, 1, 0, 0, 0},
    {1, 6, 15, 20, 15, 6, 1, 0, 0},  {1, 7, 21, 35, 35, 21, 7, 1, 0}, {1, 8, 28, 56, 70, 56, 28, 8, 1}};

template <typename T, int P>
__global__ void p2m_kernel(const int4 *__restrict__ items, int64_t nitems, const typename Vec4<T>::type *__restrict__ spos,
                           const typename Vec4<T>::type *__restrict__ snrm, const typename Vec4<T>::type *__restrict__ sw,
                           const typename Vec4<T>::type *__restrict__ box_c, const int *__restrict__ parent,
                           const int *__restrict__ used, typename Vec4<T>::type *__restrict__ mom) {
    using T4 = typename Vec4<T>::type;
    constexpr int NT = n_terms(P);
    __shared__ T pw[kP2MTile][3][P + 1];
    __shared__ T4 lm[NT];
    __shared__ T dpw[3][P + 1];
    __shared__ T4 shn[kP2MTile], shw[kP2MTile];
    const int64_t it = blockIdx.x;
    if (it >= nitems) return;
    const int4 item = items[it];
    const T4 c = box_c[item.x];
    const int t = threadIdx.x;
    int k1 = 0, k2 = 0, k3 = 0;
    if (t < NT) {   // decode the multi-index of this thread
        int n = 0;
        while (n_terms(n) <= t) ++n;
        int r = t - n_terms(n - 1);
        int a = n;
        while (r > n - a) {
            r -= n - a + 1;
            --a;
        }
        k1 = a;
        k2 = n - a - r;
        k3 = n - k1 - k2;
    }
    T vr = 0, vi = 0, kr = 0, ki = 0;
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
            shw[t] = sw[base + t];
        }
        __syncthreads();
        if (t < NT) {
            for (int s = 0; s < cnt; ++s) {
                const T px = pw[s][0][k1], py = pw[s][1][k2], pz = pw[s][2][k3];
                const T mono = px * py * pz;
                const T4 n = shn[s], w = shw[s];
                T dm = 0;
                if (k1) dm += n.x * T(k1) * pw[s][0][k1 - 1] * py * pz;
                if (k2) dm += n.y * T(k2) * px * pw[s][1][k2 - 1] * pz;
                if (k3) dm += n.z * T(k3) * px * py * pw[s][2][k3 - 1];
                vr += w.x * mono;
                vi += w.y * mono;
                kr -= w.z * dm;
                ki -= w.w * dm;
            }
        }
    }
    // the chunk's moments about its leaf centre: added to the leaf if it is accepted by some
    // target block, and shifted into every accepted ancestor (upward pass folded in):
    //   M_k(a) = sum_{l <= k} C(k, l) (a - c)^(k - l) M_l(c),  C(k, l) = prod_d binom(k_d, l_d),
    // valid for both moment kinds since (a - y)^k = ((a - c) + (c - y))^k.
    if (t < NT) {
        T4 o;
        o.x = vr; o.y = vi; o.z = kr; o.w = ki;
        lm[t] = o;
        if (used[item.x]) {
            T *g = (T *)(mom + (int64_t)item.x * NT + t);
            atomicAdd(g + 0, vr);
            atomicAdd(g + 1, vi);
            atomicAdd(g + 2, kr);
            atomicAdd(g + 3, ki);
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
            T sr = 0, si = 0, skr = 0, ski = 0;
            for (int l1 = 0; l1 <= k1; ++l1)
                for (int l2 = 0; l2 <= k2; ++l2)
                    for (int l3 = 0; l3 <= k3; ++l3) {
                        const T coef = T(c_binom[k1][l1] * c_binom[k2][l2] * c_binom[k3][l3]) * dpw[0][k1 - l1] *
                                       dpw[1][k2 - l2] * dpw[2][k3 - l3];
                        const T4 m = lm[mi_index(l1, l2, l3)];
                        sr += coef * m.x;
                        si += coef * m.y;
                        skr += coef * m.z;
                        ski += coef * m.w;
                    }
            T *g = (T *)(mom + (int64_t)A * NT + t);
            atomicAdd(g + 0, sr);
            atomicAdd(g + 1, si);
            atomicAdd(g + 2, skr);
            atomicAdd(g + 3, ski);
        }
    }
}

// --------------------------------------------------------------- launchers
int launch_weights(lspr_ctx *ctx, bool fp64, const double2 *x, int64_t N) {
    const int64_t Ns = ctx->mesh.Ns;
    cudaEvent_t ev;
    timer_begin(ctx, T_WEIGHTS, &ev);
    if (fp64) {
        LSPR_TRY(ctx, ctx->w64.ensure(Ns));
        ++ctx->n_launches;
        weights_kernel<dbl4><<<grid_for(Ns, 256), 256, 0, ctx->stream>>>(Ns, N, ctx->wo.spos64.p,
                                                                            ctx->wo.src_panel.p, x, ctx->w64.p);
    } else {
        LSPR_TRY(ctx, ctx->w32.ensure(Ns));
        ++ctx->n_launches;
        weights_kernel<float4><<<grid_for(Ns, 256), 256, 0, ctx->stream>>>(Ns, N, ctx->wo.spos64.p,
                                                                           ctx->wo.src_panel.p, x, ctx->w32.p);
    }
    timer_end(ctx, T_WEIGHTS, ev);
    LSPR_TRY(ctx, cudaGetLastError());
    return LSPR_OK;
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

int launch_p2p(lspr_ctx *ctx, bool fp64, const int4 *items, int64_t nitems, double *acc, cudaStream_t st,
               int *counter) {
    if (nitems == 0) return LSPR_OK;
    static int occ32 = 0, occ64 = 0;
    cudaEvent_t ev;
    const int slot = fp64 ? T_P2P64 : T_P2P;
    timer_begin_on(ctx, slot, &ev, st);
    ++ctx->n_launches;
    if (fp64) {
        const unsigned grid = std::min<unsigned>(grid_for(nitems, kP2PWarps),
                                                 persistent_grid(ctx, p2p_kernel<double, true>, kP2PWarps * 32, &occ64));
        p2p_kernel<double, true><<<grid, kP2PWarps * 32, 0, st>>>(items, nitems, ctx->wo.tgt64.p, ctx->mesh.N,
                                                                  ctx->wo.spos64.p, ctx->wo.snrm64.p, ctx->w64.p, acc,
                                                                  counter);
    } else {
        const unsigned grid = std::min<unsigned>(grid_for(nitems, kP2PWarps),
                                                 persistent_grid(ctx, p2p_kernel<float, true>, kP2PWarps * 32, &occ32));
        p2p_kernel<float, true><<<grid, kP2PWarps * 32, 0, st>>>(items, nitems, ctx->wo.tgt32.p, ctx->mesh.N,
                                                                 ctx->wo.spos32.p, ctx->wo.snrm32.p, ctx->w32.p, acc,
                                                                 counter);
    }
    timer_end_on(ctx, slot, ev, st);
    LSPR_TRY(ctx, cudaGetLastError());
    return LSPR_OK;
}

int launch_item_flags(lspr_ctx *ctx, int4 *items, int64_t nitems) {
    if (nitems == 0) return LSPR_OK;
    ++ctx->n_launches;
    item_flags_kernel<<<grid_for(nitems * 32, 256), 256, 0, ctx->stream>>>(items, nitems, ctx->wo.src_tblock.p);
    LSPR_TRY(ctx, cudaGetLastError());
    return LSPR_OK;
}

template <typename T, int P>
static void p2m_launch(lspr_ctx *ctx) {
    using T4 = typename Vec4<T>::type;
    Tree &tr = ctx->tree;
    const int threads = ((n_terms(P) + 31) / 32) * 32;
    const T4 *spos, *snrm, *w, *bc;
    T4 *mom;
    if constexpr (sizeof(T) == 8) {
        spos = ctx->wo.spos64.p; snrm = ctx->wo.snrm64.p; w = ctx->w64.p; bc = tr.box_c64.p; mom = tr.mom64.p;
    } else {
        spos = ctx->wo.spos32.p; snrm = ctx->wo.snrm32.p; w = ctx->w32.p; bc = tr.box_c32.p; mom = tr.mom32.p;
    }
    ++ctx->n_launches;
    p2m_kernel<T, P><<<(unsigned)tr.n_p2m_items, threads, 0, ctx->stream>>>(tr.p2m_items.p, tr.n_p2m_items, spos, snrm,
                                                                           w, bc, tr.box_parent.p, tr.box_used.p, mom);
}

template <typename T, int P>
static void m2p_launch(lspr_ctx *ctx, double *acc, int *counter) {
    using T4 = typename Vec4<T>::type;
    static int occ = 0;
    Tree &tr = ctx->tree;
    const T4 *tgt, *bc, *mom;
    if constexpr (sizeof(T) == 8) {
        tgt = ctx->wo.tgt64.p; bc = tr.box_c64.p; mom = tr.mom64.p;
    } else {
        tgt = ctx->wo.tgt32.p; bc = tr.box_c32.p; mom = tr.mom32.p;
    }
    const unsigned grid = std::min<unsigned>(grid_for(tr.n_m2p_items, kM2PWarps),
                                             persistent_grid(ctx, m2p_kernel<T, P, true>, kM2PWarps * 32, &occ));
    m2p_kernel<T, P, true><<<grid, kM2PWarps * 32, 0, ctx->stream>>>(tr.m2p_items.p, tr.n_m2p_items, tgt, ctx->mesh.N,
                                                                    tr.m2p_list.p, bc, mom, acc, counter);
}

#define LSPR_DISPATCH_P(FN, T, ...)           \
    switch (ctx->tree.P) {                    \
    case 1: FN<T, 1>(__VA_ARGS__); break;     \
    case 2: FN<T, 2>(__VA_ARGS__); break;     \
    case 3: FN<T, 3>(__VA_ARGS__); break;     \
    case 4: FN<T, 4>(__VA_ARGS__); break;     \
    case 5: FN<T, 5>(__VA_ARGS__); break;     \
    case 6: FN<T, 6>(__VA_ARGS__); break;     \
    case 7: FN<T, 7>(__VA_ARGS__); break;     \
    case 8: FN<T, 8>(__VA_ARGS__); break;     \
    default: return LSPR_E_ARG;               \
    }

int launch_p2m(lspr_ctx *ctx, bool fp64) {
    Tree &tr = ctx->tree;
    if (tr.n_p2m_items == 0) return LSPR_OK;
    cudaEvent_t ev;
    const int slot = fp64 ? T_P2M64 : T_P2M;
    timer_begin(ctx, slot, &ev);
    if (fp64) {
        LSPR_TRY(ctx, tr.mom64.ensure(tr.nboxes * tr.NT));
        LSPR_TRY(ctx, cudaMemsetAsync(tr.mom64.p, 0, sizeof(dbl4) * tr.nboxes * tr.NT, ctx->stream));
        LSPR_DISPATCH_P(p2m_launch, double, ctx);
    } else {
        LSPR_TRY(ctx, tr.mom32.ensure(tr.nboxes * tr.NT));
        LSPR_TRY(ctx, cudaMemsetAsync(tr.mom32.p, 0, sizeof(float4) * tr.nboxes * tr.NT, ctx->stream));
        LSPR_DISPATCH_P(p2m_launch, float, ctx);
    }
    timer_end(ctx, slot, ev);
    LSPR_TRY(ctx, cudaGetLastError());
    return LSPR_OK;
}

int launch_m2p(lspr_ctx *ctx, bool fp64, double *acc, int *counter) {
    Tree &tr = ctx->tree;
    if (tr.n_m2p_items == 0) return LSPR_OK;
    cudaEvent_t ev;
    const int slot = fp64 ? T_M2P64 : T_M2P;
    timer_begin(ctx, slot, &ev);
    if (fp64) {
        LSPR_DISPATCH_P(m2p_launch, double, ctx, acc, counter);
    } else {
        LSPR_DISPATCH_P(m2p_launch, float, ctx, acc, counter);
    }
    timer_end(ctx, slot, ev);
    LSPR_TRY(ctx, cudaGetLastError());
    return LSPR_OK;
}

}  // namespace lspr

namespace lspr {

// Launchers on explicit buffers (no context-owned scratch): used by the
// allocation-free matvec entry point.
int launch_weights_fp32_raw(cudaStream_t st, int64_t Ns, int64_t N, const dbl4 *spos64, const int *src_panel,
                            const double2 *x, float4 *w) {
    weights_kernel<float4><<<grid_for(Ns, 256), 256, 0, st>>>(Ns, N, spos64, src_panel, x, w);
    return cudaGetLastError() == cudaSuccess ? LSPR_OK : LSPR_E_CUDA;
}

int launch_p2p_fp32_raw(cudaStream_t st, const int4 *items, int64_t nitems, const float4 *tgt, int64_t ntgt,
                        const float4 *spos, const float4 *snrm, const float4 *w, double *acc) {
    if (nitems == 0) return LSPR_OK;
    p2p_kernel<float, false><<<grid_for(nitems, kP2PWarps), kP2PWarps * 32, 0, st>>>(items, nitems, tgt, ntgt, spos,
                                                                                    snrm, w, acc, nullptr);
    return cudaGetLastError() == cudaSuccess ? LSPR_OK : LSPR_E_CUDA;
}

}  // namespace lspr
