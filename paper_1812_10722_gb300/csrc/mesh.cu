// Geometry and quadrature precompute (Sec. II.C of the paper):
//   panel centroids / normals / areas / L = sqrt(2A), Gauss-node sources of the
//   far rule, semi-analytical self integrals, the near-singular pair list and
//   its FP64 corrections.  Everything here depends only on the mesh and the
//   quadrature options, so it runs once per geometry.
#include <algorithm>
#include <cmath>

#include "lspr_internal.cuh"

namespace lspr {

// ----------------------------------------------------------------------------
// Dunavant's symmetric triangle rules (Dunavant 1985), barycentric points and
// weights normalised to sum 1.  Orbit form: type 0 centroid, type 1 (a,b,b)
// with b = (1-a)/2, type 2 all permutations of (a, b, 1-a-b).
// ----------------------------------------------------------------------------
struct Orbit {
    int type;
    double a, b, w;
};
static const Orbit kR1[] = {{0, 0., 0., 1.0}};
static const Orbit kR3[] = {{1, 0.666666666666667, 0., 0.333333333333333}};
static const Orbit kR4[] = {{0, 0., 0., -0.5625}, {1, 0.6, 0., 0.520833333333333}};
static const Orbit kR19[] = {{0, 0., 0., 0.097135796282799},
                             {1, 0.020634961602525, 0., 0.031334700227139},
                             {1, 0.125820817014127, 0., 0.077827541004774},
                             {1, 0.623592928761935, 0., 0.079647738927210},
                             {1, 0.910540973211095, 0., 0.025577675658698},
                             {2, 0.036838412054736, 0.221962989160766, 0.043283539377289}};
static const Orbit kR25[] = {{0, 0., 0., 0.090817990382754},
                             {1, 0.028844733232685, 0., 0.036725957756467},
                             {1, 0.781036849029926, 0., 0.045321059435528},
                             {2, 0.141707219414880, 0.307939838764121, 0.072757916845420},
                             {2, 0.025003534762686, 0.246672560639903, 0.028327242531057},
                             {2, 0.009540815400299, 0.066803251012200, 0.009421666963733}};
static const Orbit kR37[] = {{0, 0., 0., 0.052520923400802},
                             {1, 0.009903630120591, 0., 0.011280145209330},
                             {1, 0.062566729780852, 0., 0.031423518362454},
                             {1, 0.170957326397447, 0., 0.047072502504194},
                             {1, 0.541200855914337, 0., 0.047363586536355},
                             {1, 0.771151009607340, 0., 0.031167529045794},
                             {1, 0.950377217273082, 0., 0.007975771465074},
                             {2, 0.094853828379579, 0.268794997058761, 0.036848402728732},
                             {2, 0.018100773278807, 0.291730066734288, 0.017401463303822},
                             {2, 0.022233076674090, 0.126357385491669, 0.015521786839045}};

// fills bary[3*K], w[K]; returns the point count or -1
static int expand_rule(int K, double *bary, double *w) {
    const Orbit *o = nullptr;
    int no = 0;
    if (K == 1) { o = kR1; no = 1; }
    else if (K == 3) { o = kR3; no = 1; }
    else if (K == 4) { o = kR4; no = 2; }
    else if (K == 19) { o = kR19; no = 6; }
    else if (K == 25) { o = kR25; no = 6; }
    else if (K == 37) { o = kR37; no = 10; }
    else return -1;
    int k = 0;
    for (int r = 0; r < no; ++r) {
        const double a = o[r].a;
        if (o[r].type == 0) {
            bary[3 * k] = bary[3 * k + 1] = bary[3 * k + 2] = 1.0 / 3.0;
            w[k++] = o[r].w;
        } else if (o[r].type == 1) {
            const double b = 0.5 * (1.0 - a);
            const double pts[3][3] = {{a, b, b}, {b, a, b}, {b, b, a}};
            for (auto &p : pts) {
                bary[3 * k] = p[0]; bary[3 * k + 1] = p[1]; bary[3 * k + 2] = p[2];
                w[k++] = o[r].w;
            }
        } else {
            const double b = o[r].b, c = 1.0 - a - b;
            const double pts[6][3] = {{a, b, c}, {a, c, b}, {b, a, c}, {b, c, a}, {c, a, b}, {c, b, a}};
            for (auto &p : pts) {
                bary[3 * k] = p[0]; bary[3 * k + 1] = p[1]; bary[3 * k + 2] = p[2];
                w[k++] = o[r].w;
            }
        }
    }
    return k;
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
static void gauss_legendre(int n, double *x, double *w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double pp = 0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

__constant__ double c_far_bary[37 * 3];
__constant__ double c_far_w[37];
__constant__ double c_fine_bary[37 * 3];
__constant__ double c_fine_w[37];
__constant__ double c_gl_x[kMaxNk];
__constant__ double c_gl_w[kMaxNk];

// ----------------------------------------------------------------------------
// Panel geometry with every FP64 operation rounded on its own (no contraction),
// so centroids, areas and L are reproducible bit for bit on any IEEE machine;
// the near-singular classification depends on them.
// ----------------------------------------------------------------------------
__global__ void panel_kernel(const double *__restrict__ verts, const int *__restrict__ tris, int64_t N, int64_t nv,
                             double *cx, double *cy, double *cz, double *nx, double *ny, double *nz, double *area,
                             double *L, int *bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int i0 = tris[3 * i], i1 = tris[3 * i + 1], i2 = tris[3 * i + 2];
    if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nv || i1 >= nv || i2 >= nv) {
        atomicOr(bad, 1);
        return;
    }
    double v[3][3];
    for (int d = 0; d < 3; ++d) {
        v[0][d] = verts[3 * (int64_t)i0 + d];
        v[1][d] = verts[3 * (int64_t)i1 + d];
        v[2][d] = verts[3 * (int64_t)i2 + d];
    }
    double e1[3], e2[3];
    for (int d = 0; d < 3; ++d) {
        e1[d] = __dsub_rn(v[1][d], v[0][d]);
        e2[d] = __dsub_rn(v[2][d], v[0][d]);
    }
    double c0 = __dsub_rn(__dmul_rn(e1[1], e2[2]), __dmul_rn(e1[2], e2[1]));
    double c1 = __dsub_rn(__dmul_rn(e1[2], e2[0]), __dmul_rn(e1[0], e2[2]));
    double c2 = __dsub_rn(__dmul_rn(e1[0], e2[1]), __dmul_rn(e1[1], e2[0]));
    double nc = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(c0, c0), __dmul_rn(c1, c1)), __dmul_rn(c2, c2)));
    if (!(nc > 0.0) || !isfinite(nc)) {
        atomicOr(bad, 2);
        nc = 1.0;
    }
    nx[i] = __ddiv_rn(c0, nc);
    ny[i] = __ddiv_rn(c1, nc);
    nz[i] = __ddiv_rn(c2, nc);
    cx[i] = __ddiv_rn(__dadd_rn(__dadd_rn(v[0][0], v[1][0]), v[2][0]), 3.0);
    cy[i] = __ddiv_rn(__dadd_rn(__dadd_rn(v[0][1], v[1][1]), v[2][1]), 3.0);
    cz[i] = __ddiv_rn(__dadd_rn(__dadd_rn(v[0][2], v[1][2]), v[2][2]), 3.0);
    double A = __dmul_rn(0.5, nc);
    area[i] = A;
    L[i] = __dsqrt_rn(__dmul_rn(2.0, A));
}

__device__ __forceinline__ void atomic_max_pos(double *addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

// Far-rule Gauss nodes in natural order s = K*i + g: position, w_g*A_i, normal, panel id.
__global__ void sources_kernel(const double *__restrict__ verts, const int *__restrict__ tris, int64_t N, int K,
                               const double *area, const double *nx, const double *ny, const double *nz,
                               const double *cx, const double *cy, const double *cz, dbl4 *pos, dbl4 *nrm,
                               dbl4 *tgt, double *rho_max, double *L_max, const double *L) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N * K) return;
    int64_t i = s / K;
    int g = (int)(s - i * K);
    double y[3];
    const int *t = tris + 3 * i;
    for (int d = 0; d < 3; ++d)
        y[d] = c_far_bary[3 * g] * verts[3 * (int64_t)t[0] + d] + c_far_bary[3 * g + 1] * verts[3 * (int64_t)t[1] + d] +
               c_far_bary[3 * g + 2] * verts[3 * (int64_t)t[2] + d];
    pos[s] = make_dbl4(y[0], y[1], y[2], c_far_w[g] * area[i]);
    nrm[s] = make_dbl4(nx[i], ny[i], nz[i], (double)i);
    double dx = y[0] - cx[i], dy = y[1] - cy[i], dz = y[2] - cz[i];
    atomic_max_pos(rho_max, sqrt(dx * dx + dy * dy + dz * dz));
    if (g == 0) {
        tgt[i] = make_dbl4(cx[i], cy[i], cz[i], (double)i);
        atomic_max_pos(L_max, L[i]);
        atomic_max_pos(L_max + 1, fmax(fabs(cx[i]), fmax(fabs(cy[i]), fabs(cz[i]))));
    }
}

// Semi-analytical singular integral: for x = centroid of panel i, the panel
// is split at x into three triangles over its edges.  In polar coordinates about
// x the radial integral of 1/rho * rho is exact (the distance to the edge,
// h / cos(phi)); the angle from phi_a to phi_b is integrated by N_k-point
// Gauss-Legendre, i.e. N_k nodes on each edge.
__global__ void self_kernel(const double *__restrict__ verts, const int *__restrict__ tris, int64_t N, int Nk,
                            const double *cx, const double *cy, const double *cz, double *Vself) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double x[3] = {cx[i], cy[i], cz[i]};
    double v[3][3];
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) v[k][d] = verts[3 * (int64_t)tris[3 * i + k] + d];
    double sum = 0.0;
    for (int e = 0; e < 3; ++e) {
        const double *a = v[e], *b = v[(e + 1) % 3];
        double t[3], ax[3];
        double len = 0;
        for (int d = 0; d < 3; ++d) {
            t[d] = b[d] - a[d];
            len += t[d] * t[d];
        }
        len = sqrt(len);
        double sa = 0, sb = 0;
        for (int d = 0; d < 3; ++d) {
            t[d] /= len;
            ax[d] = a[d] - x[d];
            sa += ax[d] * t[d];
            sb += (b[d] - x[d]) * t[d];
        }
        double h2 = 0;
        for (int d = 0; d < 3; ++d) {
            double p = ax[d] - sa * t[d];
            h2 += p * p;
        }
        double h = sqrt(h2);
        if (!(h > 0)) continue;
        double pa = atan2(sa, h), pb = atan2(sb, h);
        double mid = 0.5 * (pa + pb), half = 0.5 * (pb - pa);
        double q = 0;
        for (int k = 0; k < Nk; ++k) q += c_gl_w[k] / cos(mid + half * c_gl_x[k]);
        sum += h * half * q;
    }
    Vself[i] = sum * kInv4Pi;
}

// ----------------------------------------------------------------------------
// Near-singular decision: the FP64 test L_j / |c_i - c_j| >= threshold with every
// operation rounded separately (reproducible on any IEEE machine).
// ----------------------------------------------------------------------------
__device__ __forceinline__ bool near_exact(double xi, double yi, double zi, double xj, double yj, double zj,
                                           double Lj, double thr) {
    double dx = __dsub_rn(xi, xj), dy = __dsub_rn(yi, yj), dz = __dsub_rn(zi, zj);
    double dist = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    return __ddiv_rn(Lj, dist) >= thr;
}

// ----------------------------------------------------------------------------
// Cell list for the near-singular search: cubic cells of edge h >= L_max/threshold,
// panels sorted by the Morton key of the cell holding their centroid.  Every panel
// j with L_j/|c_i - c_j| >= threshold lies within L_max/threshold of c_i, hence in
// one of the 27 cells around c_i's cell.  Cell coordinates come from the same FP64
// expression for keys and queries.
// ----------------------------------------------------------------------------
__device__ __forceinline__ int cell_coord(double c, double lo, double inv_h) {
    const double u = floor((c - lo) * inv_h);
    return (int)fmin(1023.0, fmax(0.0, u));
}

__device__ __forceinline__ unsigned cell_key(int ix, int iy, int iz) {
    return (spread10((unsigned)ix) << 2) | (spread10((unsigned)iy) << 1) | spread10((unsigned)iz);
}

__global__ void cell_key_kernel(int64_t N, const double *__restrict__ cx, const double *__restrict__ cy,
                                const double *__restrict__ cz, const double *__restrict__ L, double thr,
                                const double *grid /* lo[3], 1/h */, unsigned *keys, int *vals, float4 *cf) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    cf[i] = make_float4((float)cx[i], (float)cy[i], (float)cz[i], (float)(L[i] / thr));
    keys[i] = cell_key(cell_coord(cx[i], grid[0], grid[3]), cell_coord(cy[i], grid[1], grid[3]),
                       cell_coord(cz[i], grid[2], grid[3]));
    vals[i] = (int)i;
}

__device__ __forceinline__ int lower_bound_u(const unsigned *a, int n, unsigned v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Near decision from FP32 copies when the FP32 distance is clearly inside or outside
// L_j/threshold, else the exact FP64 test.  band bounds |d32 - d| + |r32 - r|: FP32
// rounding of the coordinates (2^-24 |c| each) and of the arithmetic.
__device__ __forceinline__ bool near_decide(const float4 &fi, const float4 &fj, float band, double xi, double yi,
                                            double zi, int j, const double *__restrict__ cx,
                                            const double *__restrict__ cy, const double *__restrict__ cz,
                                            const double *__restrict__ L, double thr) {
    const float dx = fi.x - fj.x, dy = fi.y - fj.y, dz = fi.z - fj.z;
    const float d2 = dx * dx + dy * dy + dz * dz;
    const float r = fj.w, lo = fmaxf(r - band, 0.f), hi = r + band;
    if (d2 < lo * lo) return true;
    if (d2 > hi * hi) return false;
    return near_exact(xi, yi, zi, cx[j], cy[j], cz[j], L[j], thr);
}

// One warp per target: lane c < 27 searches neighbour cell c and tests its panels; the
// row is laid out as the self entry, then the hits of cell 0, 1, ... in sorted order.
template <bool FILL>
__global__ void near_cells_kernel(int64_t N, const double *__restrict__ cx, const double *__restrict__ cy,
                                  const double *__restrict__ cz, const double *__restrict__ L, double thr,
                                  const double *grid, const unsigned *__restrict__ skeys, const int *__restrict__ sidx,
                                  const float4 *__restrict__ cf, int64_t *count, const int64_t *ptr, int *col,
                                  int *row) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    const double xi = cx[i], yi = cy[i], zi = cz[i];
    const float4 fi = cf[i];
    const float cmax = (float)grid[4];
    const int ix = cell_coord(xi, grid[0], grid[3]), iy = cell_coord(yi, grid[1], grid[3]),
              iz = cell_coord(zi, grid[2], grid[3]);
    int k0 = 0, k1 = 0;
    if (lane < 27) {
        const int qx = ix + lane % 3 - 1, qy = iy + (lane / 3) % 3 - 1, qz = iz + lane / 9 - 1;
        if (qx >= 0 && qy >= 0 && qz >= 0 && qx <= 1023 && qy <= 1023 && qz <= 1023) {
            const unsigned key = cell_key(qx, qy, qz);
            k0 = lower_bound_u(skeys, (int)N, key);
            k1 = k0;
            while (k1 < N && skeys[k1] == key) ++k1;
        }
    }
    int c = 0;
    for (int k = k0; k < k1; ++k) {
        const int j = sidx[k];
        if (j == i) continue;
        const float4 fj = cf[j];
        c += near_decide(fi, fj, 1e-6f * fj.w + 5e-7f * cmax, xi, yi, zi, j, cx, cy, cz, L, thr);
    }
    // inclusive warp scan of the per-lane hit counts
    int inc = c;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    const int total = __shfl_sync(0xffffffffu, inc, 31);
    if (!FILL) {
        if (lane == 0) count[i] = total + 1;
        return;
    }
    int64_t out = ptr[i];
    if (lane == 0) {
        col[out] = (int)i;   // self entry first
        row[out] = (int)i;
    }
    out += 1 + (inc - c);
    for (int k = k0; k < k1; ++k) {
        const int j = sidx[k];
        if (j == i) continue;
        const float4 fj = cf[j];
        if (near_decide(fi, fj, 1e-6f * fj.w + 5e-7f * cmax, xi, yi, zi, j, cx, cy, cz, L, thr)) {
            col[out] = j;
            row[out] = (int)i;
            ++out;
        }
    }
}

// exclusive scan of n int64 counts into ptr[0..n], single block
__global__ void scan_kernel(const int64_t *in, int64_t n, int64_t *out) {
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
        out[k] = run;
        run += in[k];
    }
    if (t == blockDim.x - 1) out[n] = part[t];
}

// FP32 copies (dV, dK) of the near-field corrections, read by the FP32 products of several
// right-hand sides
__global__ void near_f32_kernel(int64_t nnz, const double *__restrict__ dV, const double *__restrict__ dK,
                                float2 *__restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < nnz) out[e] = make_float2((float)dV[e], (float)dK[e]);
}

// Per near pair: dV, dK = (K_fine rule - far rule) over panel j seen from c_i,
// and for the self entry V_ii (the far-field kernels skip a panel's own nodes).
__global__ void near_values_kernel(int64_t nnz, const int *row, const int *col, const double *__restrict__ verts,
                                   const int *__restrict__ tris, const double *cx, const double *cy, const double *cz,
                                   const double *nx, const double *ny, const double *nz, const double *area,
                                   const double *Vself, int K, int Kf, double *dV, double *dK) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const int i = row[e], j = col[e];
    if (i == j) {
        dV[e] = Vself[i];
        dK[e] = 0.0;
        return;
    }
    const double x[3] = {cx[i], cy[i], cz[i]};
    const double n[3] = {nx[j], ny[j], nz[j]};
    double v[3][3];
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) v[k][d] = verts[3 * (int64_t)tris[3 * (int64_t)j + k] + d];
    double fv = 0, fk = 0, cv = 0, ck = 0;
    for (int g = 0; g < Kf; ++g) {
        double d[3];
        for (int q = 0; q < 3; ++q)
            d[q] = x[q] - (c_fine_bary[3 * g] * v[0][q] + c_fine_bary[3 * g + 1] * v[1][q] + c_fine_bary[3 * g + 2] * v[2][q]);
        double ri = rsqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
        fv += c_fine_w[g] * ri;
        fk += c_fine_w[g] * dn * ri * ri * ri;
    }
    for (int g = 0; g < K; ++g) {
        double d[3];
        for (int q = 0; q < 3; ++q)
            d[q] = x[q] - (c_far_bary[3 * g] * v[0][q] + c_far_bary[3 * g + 1] * v[1][q] + c_far_bary[3 * g + 2] * v[2][q]);
        double ri = rsqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
        cv += c_far_w[g] * ri;
        ck += c_far_w[g] * dn * ri * ri * ri;
    }
    const double A = area[j] * kInv4Pi;
    dV[e] = (fv - cv) * A;
    dK[e] = (fk - ck) * A;
}

__global__ void natural_order_kernel(int64_t N, int K, const dbl4 *pos, const dbl4 *nrm, const dbl4 *tgt,
                                     dbl4 *spos64, dbl4 *snrm64, float4 *spos32, float4 *snrm32,
                                     dbl4 *tgt64, float4 *tgt32, int *src_panel, int *tgt_panel, int *tgt_pos,
                                     int *src_tblock) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N * K) return;
    dbl4 p = pos[s], n = nrm[s];
    int pid = (int)(s / K);
    spos64[s] = p;
    snrm64[s] = n;
    spos32[s] = make_float4((float)p.x, (float)p.y, (float)p.z, (float)p.w);
    snrm32[s] = make_float4((float)n.x, (float)n.y, (float)n.z, __int_as_float(pid));
    src_panel[s] = pid;
    src_tblock[s] = pid / kTargetBlock;
    if (s % K == 0) {
        dbl4 t = tgt[pid];
        tgt64[pid] = t;
        tgt32[pid] = make_float4((float)t.x, (float)t.y, (float)t.z, __int_as_float(pid));
        tgt_panel[pid] = pid;
        tgt_pos[pid] = pid;
    }
}

// ----------------------------------------------------------------------------
int cuda_status(lspr_ctx *ctx, cudaError_t e, const char *what) {
    ctx->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return LSPR_E_OOM;
    }
    return LSPR_E_CUDA;
}

// flags[0] |= 1 for a surface index outside [0, S)
__global__ void surf_check_kernel(int64_t N, int S, const int *__restrict__ surf, int *flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N && (surf[i] < 0 || surf[i] >= S)) atomicOr(flag, 1);
}

int mesh_build(lspr_ctx *ctx, const double *verts, int64_t nv, const int *tris, int64_t N, const int *surf,
               int nsurf, int on_device, const lspr_quad_opts &q) {
    Mesh &m = ctx->mesh;
    cudaStream_t st = ctx->stream;
    m.ready = false;
    ctx->tree.ready = false;
    double fb[37 * 3], fw[37], gb[37 * 3], gw[37], glx[kMaxNk], glw[kMaxNk];
    if (expand_rule(q.K, fb, fw) != q.K || (q.K != 1 && q.K != 3 && q.K != 4)) return LSPR_E_ARG;
    if (expand_rule(q.K_fine, gb, gw) != q.K_fine || q.K_fine < 19) return LSPR_E_ARG;
    if (q.N_k < 1 || q.N_k > kMaxNk || !(q.threshold > 0)) return LSPR_E_ARG;
    gauss_legendre(q.N_k, glx, glw);
    LSPR_TRY(ctx, cudaMemcpyToSymbolAsync(c_far_bary, fb, sizeof(double) * 3 * q.K, 0, cudaMemcpyHostToDevice, st));
    LSPR_TRY(ctx, cudaMemcpyToSymbolAsync(c_far_w, fw, sizeof(double) * q.K, 0, cudaMemcpyHostToDevice, st));
    LSPR_TRY(ctx, cudaMemcpyToSymbolAsync(c_fine_bary, gb, sizeof(double) * 3 * q.K_fine, 0, cudaMemcpyHostToDevice, st));
    LSPR_TRY(ctx, cudaMemcpyToSymbolAsync(c_fine_w, gw, sizeof(double) * q.K_fine, 0, cudaMemcpyHostToDevice, st));
    LSPR_TRY(ctx, cudaMemcpyToSymbolAsync(c_gl_x, glx, sizeof(double) * q.N_k, 0, cudaMemcpyHostToDevice, st));
    LSPR_TRY(ctx, cudaMemcpyToSymbolAsync(c_gl_w, glw, sizeof(double) * q.N_k, 0, cudaMemcpyHostToDevice, st));

    m.N = N;
    m.nv = nv;
    m.K = q.K;
    m.Kf = q.K_fine;
    m.Nk = q.N_k;
    m.thr = q.threshold;
    m.Ns = N * q.K;
    LSPR_TRY(ctx, m.verts.ensure(3 * nv));
    LSPR_TRY(ctx, m.tris.ensure(3 * N));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    LSPR_TRY(ctx, cudaMemcpyAsync(m.verts.p, verts, sizeof(double) * 3 * nv, kind, st));
    LSPR_TRY(ctx, cudaMemcpyAsync(m.tris.p, tris, sizeof(int) * 3 * N, kind, st));
    for (DArr<double> *a : {&m.cx, &m.cy, &m.cz, &m.nx, &m.ny, &m.nz, &m.area, &m.L, &m.Vself})
        LSPR_TRY(ctx, a->ensure(N));
    LSPR_TRY(ctx, m.src_pos64.ensure(m.Ns));
    LSPR_TRY(ctx, m.src_nrm64.ensure(m.Ns));
    LSPR_TRY(ctx, m.tgt64.ensure(N));

    // scratch: [0] bad flag (int), [1] rho_max, [2] L_max, [3] largest |coordinate| of a centroid
    Tmp<double> flags(ctx->scratch[0]);
    LSPR_TRY(ctx, flags.ensure(4));
    LSPR_TRY(ctx, cudaMemsetAsync(flags.p, 0, 4 * sizeof(double), st));
    m.S = nsurf;
    LSPR_TRY(ctx, m.surf.ensure(N));
    if (surf) {
        LSPR_TRY(ctx, cudaMemcpyAsync(m.surf.p, surf, sizeof(int) * N, kind, st));
        ++ctx->n_launches;
        surf_check_kernel<<<grid_for(N, 256), 256, 0, st>>>(N, nsurf, m.surf.p, (int *)flags.p);
    } else {
        LSPR_TRY(ctx, cudaMemsetAsync(m.surf.p, 0, sizeof(int) * N, st));
    }
    cudaEvent_t ev;
    timer_begin(ctx, T_MESH, &ev);
    ++ctx->n_launches;
    panel_kernel<<<grid_for(N, 256), 256, 0, st>>>(m.verts.p, m.tris.p, N, nv, m.cx.p, m.cy.p, m.cz.p, m.nx.p, m.ny.p,
                                                   m.nz.p, m.area.p, m.L.p, (int *)flags.p);
    ++ctx->n_launches;
    sources_kernel<<<grid_for(m.Ns, 256), 256, 0, st>>>(m.verts.p, m.tris.p, N, m.K, m.area.p, m.nx.p, m.ny.p,
                                                        m.nz.p, m.cx.p, m.cy.p, m.cz.p, m.src_pos64.p,
                                                        m.src_nrm64.p, m.tgt64.p, flags.p + 1, flags.p + 2, m.L.p);
    ++ctx->n_launches;
    self_kernel<<<grid_for(N, 128), 128, 0, st>>>(m.verts.p, m.tris.p, N, m.Nk, m.cx.p, m.cy.p, m.cz.p, m.Vself.p);
    LSPR_TRY(ctx, cudaGetLastError());
    double hflags[4];
    LSPR_TRY(ctx, cudaMemcpyAsync(hflags, flags.p, sizeof(hflags), cudaMemcpyDeviceToHost, st));
    LSPR_TRY(ctx, cudaStreamSynchronize(st));
    int bad;
    std::memcpy(&bad, &hflags[0], sizeof(int));
    m.rho_max = hflags[1];
    m.Lmax = hflags[2];
    if (bad & 1) return LSPR_E_ARG;
    if (bad & 2) return LSPR_E_MESH;

    // near-singular list from a cell list (cell edge >= L_max / threshold)
    Tmp<int64_t> cnt(ctx->scratch[1]);
    LSPR_TRY(ctx, cnt.ensure(N));
    LSPR_TRY(ctx, m.near_ptr.ensure(N + 1));
    double hgrid[5];
    {
        std::vector<double> hc(3 * N);
        // bounding box of the centroids (host copy of three N-vectors, once per geometry)
        LSPR_TRY(ctx, cudaMemcpyAsync(hc.data(), m.cx.p, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
        LSPR_TRY(ctx, cudaMemcpyAsync(hc.data() + N, m.cy.p, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
        LSPR_TRY(ctx, cudaMemcpyAsync(hc.data() + 2 * N, m.cz.p, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
        LSPR_TRY(ctx, cudaStreamSynchronize(st));
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int d = 0; d < 3; ++d)
            for (int64_t i = 0; i < N; ++i) {
                lo[d] = std::min(lo[d], hc[d * N + i]);
                hi[d] = std::max(hi[d], hc[d * N + i]);
            }
        const double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
        const double h = std::max(m.Lmax / m.thr * (1.0 + 1e-9), ext / 1023.0) * (1.0 + 1e-12) + 1e-300;
        hgrid[0] = lo[0];
        hgrid[1] = lo[1];
        hgrid[2] = lo[2];
        hgrid[3] = 1.0 / h;
        hgrid[4] = std::max(std::max(std::fabs(lo[0]), std::fabs(hi[0])),
                            std::max(std::max(std::fabs(lo[1]), std::fabs(hi[1])),
                                     std::max(std::fabs(lo[2]), std::fabs(hi[2]))));
    }
    Tmp<double> grid(ctx->scratch[2]);
    Tmp<unsigned> keys(ctx->scratch[3]), ktmp(ctx->scratch[4]);
    Tmp<int> vals(ctx->scratch[5]), vtmp(ctx->scratch[6]), hist(ctx->scratch[7]), offs(ctx->scratch[8]);
    LSPR_TRY(ctx, grid.ensure(5));
    Tmp<float4> cf(ctx->scratch[9]);
    LSPR_TRY(ctx, cf.ensure(N));
    LSPR_TRY(ctx, keys.ensure(N));
    LSPR_TRY(ctx, ktmp.ensure(N));
    LSPR_TRY(ctx, vals.ensure(N));
    LSPR_TRY(ctx, vtmp.ensure(N));
    LSPR_TRY(ctx, hist.ensure(radix_sort_scratch_ints(N)));
    LSPR_TRY(ctx, offs.ensure(radix_sort_scratch_ints(N)));
    LSPR_TRY(ctx, cudaMemcpyAsync(grid.p, hgrid, sizeof(hgrid), cudaMemcpyHostToDevice, st));
    ++ctx->n_launches;
    cell_key_kernel<<<grid_for(N, 256), 256, 0, st>>>(N, m.cx.p, m.cy.p, m.cz.p, m.L.p, m.thr, grid.p, keys.p,
                                                      vals.p, cf.p);
    LSPR_TRY_ST(radix_sort(ctx, keys.p, vals.p, ktmp.p, vtmp.p, N, 30, hist.p, offs.p));
    ++ctx->n_launches;
    near_cells_kernel<false><<<grid_for(N * 32, 128), 128, 0, st>>>(N, m.cx.p, m.cy.p, m.cz.p, m.L.p, m.thr, grid.p,
                                                               keys.p, vals.p, cf.p, cnt.p, nullptr, nullptr, nullptr);
    ++ctx->n_launches;
    scan_kernel<<<1, 1024, 0, st>>>(cnt.p, N, m.near_ptr.p);
    LSPR_TRY(ctx, cudaGetLastError());
    LSPR_TRY(ctx, cudaMemcpyAsync(&m.nnz, m.near_ptr.p + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LSPR_TRY(ctx, cudaStreamSynchronize(st));
    LSPR_TRY(ctx, m.near_col.ensure(m.nnz));
    LSPR_TRY(ctx, m.near_dV.ensure(m.nnz));
    LSPR_TRY(ctx, m.near_dK.ensure(m.nnz));
    Tmp<int> rowidx(ctx->scratch[10]);
    LSPR_TRY(ctx, rowidx.ensure(m.nnz));
    ++ctx->n_launches;
    near_cells_kernel<true><<<grid_for(N * 32, 128), 128, 0, st>>>(N, m.cx.p, m.cy.p, m.cz.p, m.L.p, m.thr, grid.p,
                                                              keys.p, vals.p, cf.p, nullptr, m.near_ptr.p, m.near_col.p,
                                                              rowidx.p);
    ++ctx->n_launches;
    near_values_kernel<<<grid_for(m.nnz, 128), 128, 0, st>>>(m.nnz, rowidx.p, m.near_col.p, m.verts.p, m.tris.p,
                                                             m.cx.p, m.cy.p, m.cz.p, m.nx.p, m.ny.p, m.nz.p, m.area.p,
                                                             m.Vself.p, m.K, m.Kf, m.near_dV.p, m.near_dK.p);
    LSPR_TRY(ctx, m.near_f32.ensure(m.nnz));
    ++ctx->n_launches;
    near_f32_kernel<<<grid_for(m.nnz, 256), 256, 0, st>>>(m.nnz, m.near_dV.p, m.near_dK.p, m.near_f32.p);
    LSPR_TRY(ctx, cudaGetLastError());
    timer_end(ctx, T_MESH, ev);
    LSPR_TRY(ctx, cudaStreamSynchronize(st));
    m.ready = true;
    return workorder_natural(ctx);
}

// item i = (target block i mod ntb, source chunk i / ntb): consecutive warps share a chunk
__global__ void direct_items_kernel(int4 *items, int64_t ntb, int64_t nch, int64_t chunk, int64_t Ns) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ntb * nch) return;
    const int64_t c = i / ntb, tb = i - c * ntb;
    items[i] = make_int4((int)tb, (int)(c * chunk), (int)min(Ns, (c + 1) * chunk), 0);
}

int workorder_natural(lspr_ctx *ctx) {
    Mesh &m = ctx->mesh;
    WorkOrder &w = ctx->wo;
    cudaStream_t st = ctx->stream;
    LSPR_TRY(ctx, w.spos64.ensure(m.Ns));
    LSPR_TRY(ctx, w.snrm64.ensure(m.Ns));
    LSPR_TRY(ctx, w.spos32.ensure(m.Ns));
    LSPR_TRY(ctx, w.snrm32.ensure(m.Ns));
    LSPR_TRY(ctx, w.tgt64.ensure(m.N));
    LSPR_TRY(ctx, w.tgt32.ensure(m.N));
    LSPR_TRY(ctx, w.src_panel.ensure(m.Ns));
    LSPR_TRY(ctx, w.tgt_panel.ensure(m.N));
    LSPR_TRY(ctx, w.tgt_pos.ensure(m.N));
    LSPR_TRY(ctx, w.src_tblock.ensure(m.Ns));
    ++ctx->n_launches;
    natural_order_kernel<<<grid_for(m.Ns, 256), 256, 0, st>>>(m.N, m.K, m.src_pos64.p, m.src_nrm64.p, m.tgt64.p,
                                                              w.spos64.p, w.snrm64.p, w.spos32.p, w.snrm32.p,
                                                              w.tgt64.p, w.tgt32.p, w.src_panel.p, w.tgt_panel.p,
                                                              w.tgt_pos.p, w.src_tblock.p);
    LSPR_TRY(ctx, cudaGetLastError());
    // direct-mode work items: every target block against source chunks
    const int64_t ntb = (m.N + kTargetBlock - 1) / kTargetBlock;
    const int64_t chunk = 512;
    const int64_t nch = (m.Ns + chunk - 1) / chunk;
    ctx->direct.n = ntb * nch;
    LSPR_TRY(ctx, ctx->direct.items.ensure(ctx->direct.n));
    ++ctx->n_launches;
    direct_items_kernel<<<grid_for(ctx->direct.n, 256), 256, 0, st>>>(ctx->direct.items.p, ntb, nch, chunk, m.Ns);
    LSPR_TRY_ST(launch_item_flags(ctx, ctx->direct.items.p, ctx->direct.n));
    LSPR_TRY_ST(launch_ff_geometry(ctx));
    LSPR_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return LSPR_OK;
}

}  // namespace lspr
