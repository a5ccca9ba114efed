/*
 * lspr_oracle.c -- plain, slow, FP64 CPU oracle of the quasistatic LSPR
 * boundary-element method (Clementi, Cooper & Barba, arXiv:1812.10722).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header, table or helper with the CUDA
 * library: the quadrature tables below are this file's own transcription.
 *
 * What it computes (section / equation of the paper in brackets):
 *   - flat-triangle panel geometry, centroid collocation        [Sec. II.C "Discretization"]
 *   - matrix entries V_ij, K_ij of the single/double layer      [Eq. layers_element]
 *       * singular (j == i): V_ii as the exact integral of 1/(4 pi |x-y|)
 *         over the flat panel (closed form, the quantity the paper's
 *         semi-analytical rule approximates), K_ii = 0 because
 *         (x - y).n_j vanishes on a flat panel              [Sec. II.C "Integral evaluation"]
 *       * near-singular (L_j/|c_i - c_j| >= threshold): K_fine-point rule
 *       * far: K-point rule
 *   - the 2x2 block operator of one interface                  [Eq. matrix_lspr]
 *   - its right-hand side V((eps2-eps1)/eps2 dphi_inc/dn)       [Eq. matrix_lspr]
 *   - the operator of several closed interfaces in one host (a particle
 *     and analyte surfaces), its right-hand side and the dipole of one
 *     surface                                                    [Eqs. integral_eq_lspr_system, matrix_multi]
 *   - the Coulomb term of point charges inside a surface on its interior
 *     row                                                        [Eqs. integral_eq_lspr_system, matrix_multi]
 *   - complex GMRES (restarted, right block-Jacobi preconditioner) and a
 *     dense complex LU with partial pivoting for small systems  [Sec. II.D]
 *   - the dipole moment from boundary data                      [Eq. dipole_def_gauss_i_final]
 *   - the extinction cross-section via the optical theorem     [Eqs. scat_efield_long_range, cext_fwa]
 *   - the closed-form sphere cross-section                      [Eq. an_sol]
 *
 * Readings of points the paper leaves open or prints inconsistently:
 *   - normals point outward (particle -> host); the double-layer kernel is
 *     dG/dn_y = (x - y).n_y / (4 pi |x - y|^3).
 *   - with outward normals the dipole is p = -eps2 * oint (x dphi2s/dn - phi2s n);
 *     the printed sign of Eq. dipole_def_gauss_i_final gives -p for a sphere.
 *   - dphi2s/dn = (eps1/eps2) dphi1s/dn - ((eps2-eps1)/eps2) dphi_inc/dn (interface
 *     condition of Eq. electrostatic_scatter), phi2s = phi1s on the interface.
 *   - incident potential phi_inc = -E0.r, so dphi_inc/dn = -E0.n.
 *   - forward direction perpendicular to e_i, so e_i.((k x p) x k) = e_i.p and
 *     sigma_ext = Im(k^2 e_i.p / (eps2 |E0|)) / Re(k), k = 2 pi sqrt(eps2) / lambda.
 *   - K and K_fine are Dunavant's symmetric triangle rules with 1/3/4 and
 *     19/25/37 points (degrees 1/2/3 and 9/10/13).
 *   - near-singular test: centroid-to-centroid distance, near iff
 *     L_j / dist >= threshold, L_j = sqrt(2 A_j); evaluated with every
 *     operation rounded separately (build with -ffp-contract=off) so that the
 *     classification is reproducible bit for bit.
 *
 *   - several surfaces t = 0..S-1 with permittivities eps_t in one host eps_out:
 *     on every surface the unknowns are phi (= phi_s on both sides) and the
 *     interior normal derivative dphi/dn of the scattered potential; the
 *     interior row of a panel on surface s holds that surface's layer
 *     potentials only, the exterior row those of every surface, each
 *     surface's single layer weighted by s_t = eps_t/eps_out:
 *       top_i = phi_i/2 + (K phi)_{s} - (V dphi)_{s}
 *       bot_i = phi_i/2 - sum_t (K phi)_t + sum_t s_t (V dphi)_t
 *     with right-hand side bot_i = sum_t ((eps_out - eps_t)/eps_out)(V dphi_inc/dn)_t
 *     (one surface: Eq. matrix_lspr).  The cross-section is that of surface 0,
 *     the particle, whose dipole uses eps_0.
 *
 * Complex arrays cross the C ABI as interleaved (re, im) doubles.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------------- */
/* Dunavant (1985) symmetric quadrature rules on a triangle, barycentric      */
/* coordinates, weights summing to one.  Orbits: S3 = centroid, S21 = (a,b,b) */
/* and permutations, S111 = all six permutations of (a,b,1-a-b).              */
/* ------------------------------------------------------------------------- */
typedef struct { int kind; double a, b, w; } orbit_t;   /* kind: 0 S3, 1 S21, 2 S111 */

static const orbit_t RULE1[] = {{0, 0, 0, 1.0}};
static const orbit_t RULE3[] = {{1, 2.0 / 3.0, 0, 1.0 / 3.0}};
static const orbit_t RULE4[] = {{0, 0, 0, -0.5625}, {1, 0.6, 0, 25.0 / 48.0}};
static const orbit_t RULE19[] = {
    {0, 0, 0, 0.097135796282799},
    {1, 0.020634961602525, 0, 0.031334700227139},
    {1, 0.125820817014127, 0, 0.077827541004774},
    {1, 0.623592928761935, 0, 0.079647738927210},
    {1, 0.910540973211095, 0, 0.025577675658698},
    {2, 0.036838412054736, 0.221962989160766, 0.043283539377289}};
static const orbit_t RULE25[] = {
    {0, 0, 0, 0.090817990382754},
    {1, 0.028844733232685, 0, 0.036725957756467},
    {1, 0.781036849029926, 0, 0.045321059435528},
    {2, 0.141707219414880, 0.307939838764121, 0.072757916845420},
    {2, 0.025003534762686, 0.246672560639903, 0.028327242531057},
    {2, 0.009540815400299, 0.066803251012200, 0.009421666963733}};
static const orbit_t RULE37[] = {
    {0, 0, 0, 0.052520923400802},
    {1, 0.009903630120591, 0, 0.011280145209330},
    {1, 0.062566729780852, 0, 0.031423518362454},
    {1, 0.170957326397447, 0, 0.047072502504194},
    {1, 0.541200855914337, 0, 0.047363586536355},
    {1, 0.771151009607340, 0, 0.031167529045794},
    {1, 0.950377217273082, 0, 0.007975771465074},
    {2, 0.094853828379579, 0.268794997058761, 0.036848402728732},
    {2, 0.018100773278807, 0.291730066734288, 0.017401463303822},
    {2, 0.022233076674090, 0.126357385491669, 0.015521786839045}};

/* Expand rule with K points into bary[K][3], w[K]; returns K or -1. */
int oracle_quad_rule(int K, double *bary, double *w)
{
    const orbit_t *o;
    int no;
    switch (K) {
    case 1: o = RULE1; no = 1; break;
    case 3: o = RULE3; no = 1; break;
    case 4: o = RULE4; no = 2; break;
    case 19: o = RULE19; no = 6; break;
    case 25: o = RULE25; no = 6; break;
    case 37: o = RULE37; no = 10; break;
    default: return -1;
    }
    int k = 0;
    for (int r = 0; r < no; ++r) {
        double a = o[r].a, b, c;
        if (o[r].kind == 0) {
            bary[3 * k] = bary[3 * k + 1] = bary[3 * k + 2] = 1.0 / 3.0;
            w[k++] = o[r].w;
        } else if (o[r].kind == 1) {
            b = 0.5 * (1.0 - a);
            double p[3][3] = {{a, b, b}, {b, a, b}, {b, b, a}};
            for (int q = 0; q < 3; ++q) {
                memcpy(&bary[3 * k], p[q], sizeof p[q]);
                w[k++] = o[r].w;
            }
        } else {
            b = o[r].b;
            c = 1.0 - a - b;
            double p[6][3] = {{a, b, c}, {a, c, b}, {b, a, c}, {b, c, a}, {c, a, b}, {c, b, a}};
            for (int q = 0; q < 6; ++q) {
                memcpy(&bary[3 * k], p[q], sizeof p[q]);
                w[k++] = o[r].w;
            }
        }
    }
    return k;
}

/* ------------------------------------------------------------------------- */
/* Panel geometry                                                            */
/* ------------------------------------------------------------------------- */
typedef struct {
    double v[3][3];   /* vertices */
    double c[3];      /* centroid (collocation point) */
    double n[3];      /* unit outward normal */
    double area;
    double L;         /* representative length sqrt(2 A) */
} panel_t;

static void make_panel(const double *verts, const int32_t *tris, int64_t i, panel_t *p)
{
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d)
            p->v[k][d] = verts[3 * (int64_t)tris[3 * i + k] + d];
    double e1[3], e2[3], cr[3];
    for (int d = 0; d < 3; ++d) {
        e1[d] = p->v[1][d] - p->v[0][d];
        e2[d] = p->v[2][d] - p->v[0][d];
    }
    cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double nc = sqrt((cr[0] * cr[0] + cr[1] * cr[1]) + cr[2] * cr[2]);
    for (int d = 0; d < 3; ++d) {
        p->n[d] = cr[d] / nc;
        p->c[d] = ((p->v[0][d] + p->v[1][d]) + p->v[2][d]) / 3.0;
    }
    p->area = 0.5 * nc;
    p->L = sqrt(2.0 * p->area);
}

void oracle_panels(const double *verts, const int32_t *tris, int64_t n,
                   double *c, double *nrm, double *area, double *L)
{
    for (int64_t i = 0; i < n; ++i) {
        panel_t p;
        make_panel(verts, tris, i, &p);
        for (int d = 0; d < 3; ++d) {
            c[3 * i + d] = p.c[d];
            nrm[3 * i + d] = p.n[d];
        }
        area[i] = p.area;
        L[i] = p.L;
    }
}

/* (1/4pi) * integral over the flat triangle (v0,v1,v2) of 1/|x - y| dA(y), x in
 * the plane of the triangle and inside it.  Exact: split at x into three
 * sub-triangles; in polar coordinates about x the sub-triangle over edge (a,b)
 * contributes h * [asinh(s_b/h) - asinh(s_a/h)], h the distance from x to the
 * edge line and s the tangential coordinates of the edge ends. */
double oracle_self_V(const double *v0, const double *v1, const double *v2, const double *x)
{
    const double *vv[3] = {v0, v1, v2};
    double sum = 0.0;
    for (int e = 0; e < 3; ++e) {
        const double *a = vv[e], *b = vv[(e + 1) % 3];
        double t[3], ax[3], bx[3];
        double len = 0.0;
        for (int d = 0; d < 3; ++d) {
            t[d] = b[d] - a[d];
            len += t[d] * t[d];
        }
        len = sqrt(len);
        double sa = 0.0, sb = 0.0;
        for (int d = 0; d < 3; ++d) {
            t[d] /= len;
            ax[d] = a[d] - x[d];
            bx[d] = b[d] - x[d];
            sa += ax[d] * t[d];
            sb += bx[d] * t[d];
        }
        double h2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            double perp = ax[d] - sa * t[d];
            h2 += perp * perp;
        }
        double h = sqrt(h2);
        if (h > 0.0)
            sum += h * (asinh(sb / h) - asinh(sa / h));
    }
    return sum / (4.0 * M_PI);
}

/* ------------------------------------------------------------------------- */
/* Matrix entries                                                            */
/* ------------------------------------------------------------------------- */
typedef struct {
    const double *verts;
    const int32_t *tris;
    int64_t n;
    panel_t *pan;
    int K, Kf;
    double bary[37 * 3], w[37];       /* far rule */
    double baryf[37 * 3], wf[37];     /* near-singular rule */
    double threshold;
    const int32_t *surf;              /* surface of each panel (NULL: all surface 0) */
    int S;                            /* number of surfaces */
} mesh_t;

static int surf_of(const mesh_t *m, int64_t i) { return m->surf ? m->surf[i] : 0; }

static int mesh_init(mesh_t *m, const double *verts, const int32_t *tris, int64_t n,
                     int K, int Kf, double threshold)
{
    m->verts = verts;
    m->tris = tris;
    m->n = n;
    m->K = K;
    m->Kf = Kf;
    m->threshold = threshold;
    m->surf = NULL;
    m->S = 1;
    if (oracle_quad_rule(K, m->bary, m->w) != K) return -1;
    if (oracle_quad_rule(Kf, m->baryf, m->wf) != Kf) return -1;
    m->pan = (panel_t *)malloc(sizeof(panel_t) * (size_t)(n > 0 ? n : 1));
    if (!m->pan) return -2;
    for (int64_t i = 0; i < n; ++i) make_panel(verts, tris, i, &m->pan[i]);
    return 0;
}

static void mesh_free(mesh_t *m) { free(m->pan); }

/* Near-singular classification (all operations separately rounded). */
static int is_near(const panel_t *ti, const panel_t *pj, double threshold)
{
    double dx = ti->c[0] - pj->c[0], dy = ti->c[1] - pj->c[1], dz = ti->c[2] - pj->c[2];
    double dist = sqrt((dx * dx + dy * dy) + dz * dz);
    return (pj->L / dist) >= threshold;
}

/* Rule applied to panel j seen from point x: V = sum_g w_g A G, K = sum_g w_g A dG/dn_j. */
static void rule_entry(const double *x, const panel_t *pj, int nq, const double *bary,
                       const double *w, double *V, double *Kd)
{
    double sv = 0.0, sk = 0.0;
    for (int g = 0; g < nq; ++g) {
        double y[3], d[3];
        for (int k = 0; k < 3; ++k)
            y[k] = bary[3 * g] * pj->v[0][k] + bary[3 * g + 1] * pj->v[1][k] + bary[3 * g + 2] * pj->v[2][k];
        for (int k = 0; k < 3; ++k) d[k] = x[k] - y[k];
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double dn = d[0] * pj->n[0] + d[1] * pj->n[1] + d[2] * pj->n[2];
        sv += w[g] / r;
        sk += w[g] * dn / (r * r * r);
    }
    *V = sv * pj->area / (4.0 * M_PI);
    *Kd = sk * pj->area / (4.0 * M_PI);
}

/* Entries V_ij, K_ij of Eq. layers_element with the three-regime rule. */
static void entry(const mesh_t *m, int64_t i, int64_t j, double *V, double *Kd)
{
    const panel_t *ti = &m->pan[i], *pj = &m->pan[j];
    if (i == j) {
        *V = oracle_self_V(pj->v[0], pj->v[1], pj->v[2], ti->c);
        *Kd = 0.0;
    } else if (is_near(ti, pj, m->threshold)) {
        rule_entry(ti->c, pj, m->Kf, m->baryf, m->wf, V, Kd);
    } else {
        rule_entry(ti->c, pj, m->K, m->bary, m->w, V, Kd);
    }
}

/* Rows [i0, i1) of V and K (row-major, n columns). */
int oracle_entries(const double *verts, const int32_t *tris, int64_t n, int K, int Kf,
                   double threshold, int64_t i0, int64_t i1, double *Vout, double *Kout)
{
    mesh_t m;
    int rc = mesh_init(&m, verts, tris, n, K, Kf, threshold);
    if (rc) return rc;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = i0; i < i1; ++i)
        for (int64_t j = 0; j < n; ++j)
            entry(&m, i, j, &Vout[(i - i0) * n + j], &Kout[(i - i0) * n + j]);
    mesh_free(&m);
    return 0;
}

/* Near-singular pairs per row (j != i), for checking the classification. */
int64_t oracle_near_pairs(const double *verts, const int32_t *tris, int64_t n, double threshold,
                          int64_t *count_per_row)
{
    mesh_t m;
    if (mesh_init(&m, verts, tris, n, 1, 19, threshold)) return -1;
    int64_t tot = 0;
#pragma omp parallel for reduction(+ : tot) schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        for (int64_t j = 0; j < n; ++j)
            if (j != i && is_near(&m.pan[i], &m.pan[j], threshold)) ++c;
        count_per_row[i] = c;
        tot += c;
    }
    mesh_free(&m);
    return tot;
}

/* ------------------------------------------------------------------------- */
/* Operator of the interfaces, Eqs. matrix_lspr / matrix_multi, matrix-free. */
/*   x = [phi (n) ; dphi/dn (n)], s[b][t] = eps_t/eps_out of wavelength b     */
/*   y_top = phi/2 + (K phi)_self - (V dphi)_self                             */
/*   y_bot = phi/2 - sum_t (K phi)_t + sum_t s_t (V dphi)_t                    */
/* (one surface: y_bot = phi/2 - K phi + s V dphi).                           */
/* ------------------------------------------------------------------------- */
/* Rows [i0, i1) of the product (the whole product: [0, n)). */
static void apply_operator_rows(const mesh_t *m, int B, const cplx *s, const cplx *x, cplx *y, int64_t i0,
                                int64_t i1)
{
    const int64_t n = m->n;
    const int S = m->S;
#pragma omp parallel
    {
        /* per wavelength and source surface: kp[b][t] = (K phi)_t, vd[b][t] = (V dphi)_t */
        cplx *kp = (cplx *)malloc(sizeof(cplx) * (size_t)B * S);
        cplx *vd = (cplx *)malloc(sizeof(cplx) * (size_t)B * S);
#pragma omp for schedule(dynamic, 8)
        for (int64_t i = i0; i < i1; ++i) {
            for (int q = 0; q < B * S; ++q) kp[q] = vd[q] = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                double V, Kd;
                entry(m, i, j, &V, &Kd);
                const int t = surf_of(m, j);
                for (int b = 0; b < B; ++b) {
                    const cplx *xb = x + (size_t)b * 2 * n;
                    kp[b * S + t] += Kd * xb[j];
                    vd[b * S + t] += V * xb[n + j];
                }
            }
            const int si = surf_of(m, i);
            for (int b = 0; b < B; ++b) {
                const cplx *xb = x + (size_t)b * 2 * n;
                cplx *yb = y + (size_t)b * 2 * n;
                cplx kall = 0.0, vall = 0.0;
                for (int t = 0; t < S; ++t) {
                    kall += kp[b * S + t];
                    vall += s[b * S + t] * vd[b * S + t];
                }
                yb[i] = 0.5 * xb[i] + kp[b * S + si] - vd[b * S + si];
                yb[n + i] = 0.5 * xb[i] - kall + vall;
            }
        }
        free(kp);
        free(vd);
    }
}

static void apply_operator(const mesh_t *m, int B, const cplx *s, const cplx *x, cplx *y)
{
    apply_operator_rows(m, B, s, x, y, 0, m->n);
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* y[b] = A(s_b) x[b] for B right-hand sides; x, y: [B][2n] complex; s: [B] complex. */
int oracle_matvec(const double *verts, const int32_t *tris, int64_t n, int K, int Kf,
                  double threshold, int B, const double *s, const double *x, double *y, int nthreads)
{
    mesh_t m;
    set_threads(nthreads);
    int rc = mesh_init(&m, verts, tris, n, K, Kf, threshold);
    if (rc) return rc;
    apply_operator(&m, B, (const cplx *)s, (const cplx *)x, (cplx *)y);
    mesh_free(&m);
    return 0;
}

/* Rows [i0, i1) of y[b] = A(s_b) x[b] (top and bottom rows of those panels; the other rows of y
 * are left as they are): the product of oracle_matvec restricted to a block of panels, for
 * timing a bounded share of it.  x, y: [B][2n]. */
int oracle_matvec_rows(const double *verts, const int32_t *tris, int64_t n, int K, int Kf, double threshold,
                       int B, const double *s, const double *x, double *y, int64_t i0, int64_t i1, int nthreads)
{
    mesh_t m;
    if (i0 < 0 || i1 > n || i0 > i1) return -3;
    set_threads(nthreads);
    int rc = mesh_init(&m, verts, tris, n, K, Kf, threshold);
    if (rc) return rc;
    apply_operator_rows(&m, B, (const cplx *)s, (const cplx *)x, (cplx *)y, i0, i1);
    mesh_free(&m);
    return 0;
}

/* Several surfaces: surf [n] surface of each panel (0..S-1); s: [B][S] complex. */
int oracle_matvec_multi(const double *verts, const int32_t *tris, const int32_t *surf, int64_t n, int S,
                        int K, int Kf, double threshold, int B, const double *s, const double *x, double *y,
                        int nthreads)
{
    mesh_t m;
    set_threads(nthreads);
    int rc = mesh_init(&m, verts, tris, n, K, Kf, threshold);
    if (rc) return rc;
    m.surf = surf;
    m.S = S;
    apply_operator(&m, B, (const cplx *)s, (const cplx *)x, (cplx *)y);
    mesh_free(&m);
    return 0;
}

/* Right-hand side: top 0, bottom sum_t ((eps_out - eps_t)/eps_out) (V dphi_inc/dn)_t,
 * dphi_inc/dn = -E0.n (one surface: Eq. matrix_lspr).  e1: [B][S] complex. */
static void rhs_impl(const mesh_t *m, int B, const cplx *e1, cplx e2, const double *E0, cplx *b)
{
    const int64_t n = m->n;
    const int S = m->S;
    double *vinc = (double *)malloc(sizeof(double) * (size_t)n * S);   /* [i][t] */
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < n; ++i) {
        for (int t = 0; t < S; ++t) vinc[i * S + t] = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double V, Kd;
            entry(m, i, j, &V, &Kd);
            double dphi_inc = -(E0[0] * m->pan[j].n[0] + E0[1] * m->pan[j].n[1] + E0[2] * m->pan[j].n[2]);
            vinc[i * S + surf_of(m, j)] += V * dphi_inc;
        }
    }
    for (int bb = 0; bb < B; ++bb)
        for (int64_t i = 0; i < n; ++i) {
            cplx acc = 0.0;
            for (int t = 0; t < S; ++t) acc += ((e2 - e1[bb * S + t]) / e2) * vinc[i * S + t];
            b[(size_t)bb * 2 * n + i] = 0.0;
            b[(size_t)bb * 2 * n + n + i] = acc;
        }
    free(vinc);
}

/* Right-hand side of Eq. matrix_lspr: top 0, bottom V((eps2-eps1)/eps2 dphi_inc/dn),
 * dphi_inc/dn = -E0.n.  b: [B][2n]; eps_in: [B] complex; eps_out complex (re, im). */
int oracle_rhs(const double *verts, const int32_t *tris, int64_t n, int K, int Kf, double threshold,
               int B, const double *eps_in, double eps_out_re, double eps_out_im, const double *E0,
               double *bout, int nthreads)
{
    mesh_t m;
    set_threads(nthreads);
    int rc = mesh_init(&m, verts, tris, n, K, Kf, threshold);
    if (rc) return rc;
    rhs_impl(&m, B, (const cplx *)eps_in, eps_out_re + I * eps_out_im, E0, (cplx *)bout);
    mesh_free(&m);
    return 0;
}

/* The same for several surfaces: eps_in [B][S] complex. */
int oracle_rhs_multi(const double *verts, const int32_t *tris, const int32_t *surf, int64_t n, int S, int K,
                     int Kf, double threshold, int B, const double *eps_in, double eps_out_re,
                     double eps_out_im, const double *E0, double *bout, int nthreads)
{
    mesh_t m;
    set_threads(nthreads);
    int rc = mesh_init(&m, verts, tris, n, K, Kf, threshold);
    if (rc) return rc;
    m.surf = surf;
    m.S = S;
    rhs_impl(&m, B, (const cplx *)eps_in, eps_out_re + I * eps_out_im, E0, (cplx *)bout);
    mesh_free(&m);
    return 0;
}

/* Point charges inside the surfaces [Eqs. integral_eq_lspr_system, matrix_multi: the interior
 * row of an analyte surface Gamma_2 carries (1 / (4 pi eps_3)) sum_k q_k / |r - r_k|]: charge k
 * (q_k at r_k, inside surface t_k) adds q_k / (4 pi eps_t |c_i - r_k|) to the interior (top) row
 * of every panel i of surface t_k, eps_t that surface's permittivity of the wavelength.
 * charges: [nq][4] (x, y, z, q); surf_q: [nq]; eps_in: [B][S] complex; b: [B][2n], added to. */
int oracle_rhs_charges(const double *verts, const int32_t *tris, const int32_t *surf, int64_t n, int S, int B,
                       const double *eps_in, int64_t nq, const double *charges, const int32_t *surf_q,
                       double *bout)
{
    cplx *b = (cplx *)bout;
    const cplx *e1 = (const cplx *)eps_in;
    for (int64_t k = 0; k < nq; ++k)
        if (surf_q[k] < 0 || surf_q[k] >= S) return 2;
    for (int64_t i = 0; i < n; ++i) {
        panel_t p;
        make_panel(verts, tris, i, &p);
        const int t = surf ? surf[i] : 0;
        double phi = 0.0;
        for (int64_t k = 0; k < nq; ++k) {
            if (surf_q[k] != t) continue;
            const double dx = p.c[0] - charges[4 * k], dy = p.c[1] - charges[4 * k + 1],
                         dz = p.c[2] - charges[4 * k + 2];
            phi += charges[4 * k + 3] / sqrt(dx * dx + dy * dy + dz * dz);
        }
        for (int bb = 0; bb < B; ++bb) b[(size_t)bb * 2 * n + i] += phi / (4.0 * M_PI * e1[(size_t)bb * S + t]);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Dense complex LU with partial pivoting (row-major A[n][n], solves in place) */
/* ------------------------------------------------------------------------- */
int oracle_lu_solve(int64_t n, double *Ain, double *bin)
{
    cplx *A = (cplx *)Ain, *b = (cplx *)bin;
    for (int64_t k = 0; k < n; ++k) {
        int64_t piv = k;
        double best = cabs(A[k * n + k]);
        for (int64_t r = k + 1; r < n; ++r)
            if (cabs(A[r * n + k]) > best) {
                best = cabs(A[r * n + k]);
                piv = r;
            }
        if (best == 0.0) return -1;
        if (piv != k) {
            for (int64_t c = 0; c < n; ++c) {
                cplx t = A[k * n + c];
                A[k * n + c] = A[piv * n + c];
                A[piv * n + c] = t;
            }
            cplx t = b[k];
            b[k] = b[piv];
            b[piv] = t;
        }
#pragma omp parallel for
        for (int64_t r = k + 1; r < n; ++r) {
            cplx f = A[r * n + k] / A[k * n + k];
            A[r * n + k] = f;
            for (int64_t c = k + 1; c < n; ++c) A[r * n + c] -= f * A[k * n + c];
            b[r] -= f * b[k];
        }
    }
    for (int64_t k = n - 1; k >= 0; --k) {
        cplx acc = b[k];
        for (int64_t c = k + 1; c < n; ++c) acc -= A[k * n + c] * b[c];
        b[k] = acc / A[k * n + k];
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Complex restarted GMRES(m) with a right block-Jacobi preconditioner: the   */
/* per-panel 2x2 diagonal block [[1/2 + K_ii, -V_ii], [1/2 - K_ii, s V_ii]].  */
/* x0 = 0; stops when the relative residual ||b - A x|| / ||b|| <= tol.       */
/* ------------------------------------------------------------------------- */
static double vnorm(const cplx *v, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
    return sqrt(s);
}

static void precond(const mesh_t *m, const double *Vii, const cplx *s, const cplx *u, cplx *x)
{
    const int64_t n = m->n;
    for (int64_t i = 0; i < n; ++i) {
        /* [[a, b], [c, d]] = [[1/2, -V], [1/2, s V]] (K_ii = 0 on flat panels), s of the
         * panel's surface */
        cplx a = 0.5, bq = -Vii[i], c = 0.5, d = s[surf_of(m, i)] * Vii[i];
        cplx det = a * d - bq * c;
        cplx u0 = u[i], u1 = u[n + i];
        x[i] = (d * u0 - bq * u1) / det;
        x[n + i] = (-c * u0 + a * u1) / det;
    }
}

/* GMRES(restart) for one wavelength, s[t] = eps_t/eps_out per surface */
static int gmres_impl(mesh_t *mp, const cplx *s, const double *bin, double *xout, double tol, int restart,
                      int maxiter, int *iters_out, double *relres_out)
{
    mesh_t m = *mp;
    const int64_t n = m.n;
    const int64_t N2 = 2 * n;
    const cplx *b = (const cplx *)bin;
    cplx *x = (cplx *)xout;
    double *Vii = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const panel_t *p = &m.pan[i];
        Vii[i] = oracle_self_V(p->v[0], p->v[1], p->v[2], p->c);
    }
    const int mr = restart;
    cplx *Vb = (cplx *)malloc(sizeof(cplx) * (size_t)N2 * (mr + 1));
    cplx *H = (cplx *)calloc((size_t)(mr + 1) * mr, sizeof(cplx));
    cplx *cs = (cplx *)malloc(sizeof(cplx) * mr), *sn = (cplx *)malloc(sizeof(cplx) * mr);
    cplx *g = (cplx *)malloc(sizeof(cplx) * (mr + 1)), *yv = (cplx *)malloc(sizeof(cplx) * mr);
    cplx *w = (cplx *)malloc(sizeof(cplx) * N2), *z = (cplx *)malloc(sizeof(cplx) * N2);
    for (int64_t i = 0; i < N2; ++i) x[i] = 0.0;
    double bnorm = vnorm(b, N2);
    if (bnorm == 0.0) bnorm = 1.0;
    int it = 0;
    double relres = 1.0;
    int status = 1;
    while (1) {
        /* explicit residual r = b - A x */
        apply_operator(&m, 1, s, x, w);
        for (int64_t i = 0; i < N2; ++i) w[i] = b[i] - w[i];
        double beta = vnorm(w, N2);
        relres = beta / bnorm;
        if (relres <= tol) { status = 0; break; }
        if (it >= maxiter) break;
        for (int64_t i = 0; i < N2; ++i) Vb[i] = w[i] / beta;
        for (int k = 0; k <= mr; ++k) g[k] = 0.0;
        g[0] = beta;
        int j = 0;
        for (; j < mr && it < maxiter; ++j) {
            cplx *vj = Vb + (size_t)j * N2, *vn = Vb + (size_t)(j + 1) * N2;
            precond(&m, Vii, s, vj, z);
            apply_operator(&m, 1, s, z, w);
            /* modified Gram-Schmidt, applied twice */
            for (int pass = 0; pass < 2; ++pass)
                for (int i = 0; i <= j; ++i) {
                    cplx *vi = Vb + (size_t)i * N2;
                    cplx h = 0.0;
                    for (int64_t k = 0; k < N2; ++k) h += conj(vi[k]) * w[k];
                    for (int64_t k = 0; k < N2; ++k) w[k] -= h * vi[k];
                    H[i * mr + j] += h;
                }
            double hn = vnorm(w, N2);
            H[(j + 1) * mr + j] = hn;
            for (int64_t k = 0; k < N2; ++k) vn[k] = hn > 0 ? w[k] / hn : 0.0;
            /* previous rotations on column j */
            for (int i = 0; i < j; ++i) {
                cplx a = H[i * mr + j], c2 = H[(i + 1) * mr + j];
                H[i * mr + j] = cs[i] * a + sn[i] * c2;
                H[(i + 1) * mr + j] = -conj(sn[i]) * a + cs[i] * c2;
            }
            /* new rotation zeroing H[j+1][j] */
            cplx a = H[j * mr + j];
            double bb = cabs(H[(j + 1) * mr + j]);
            double t = sqrt(cabs(a) * cabs(a) + bb * bb);
            if (cabs(a) == 0.0) {
                cs[j] = 0.0;
                sn[j] = 1.0;
            } else {
                cs[j] = cabs(a) / t;
                sn[j] = (a / cabs(a)) * conj(H[(j + 1) * mr + j]) / t;
            }
            H[j * mr + j] = cs[j] * a + sn[j] * H[(j + 1) * mr + j];
            H[(j + 1) * mr + j] = 0.0;
            g[j + 1] = -conj(sn[j]) * g[j];
            g[j] = cs[j] * g[j];
            ++it;
            if (cabs(g[j + 1]) / bnorm <= tol) { ++j; break; }
        }
        /* solve H y = g (upper triangular, size j), x += M^-1 V y */
        for (int i = j - 1; i >= 0; --i) {
            cplx acc = g[i];
            for (int k = i + 1; k < j; ++k) acc -= H[i * mr + k] * yv[k];
            yv[i] = acc / H[i * mr + i];
        }
        for (int64_t k = 0; k < N2; ++k) {
            cplx acc = 0.0;
            for (int i = 0; i < j; ++i) acc += Vb[(size_t)i * N2 + k] * yv[i];
            w[k] = acc;
        }
        precond(&m, Vii, s, w, z);
        for (int64_t k = 0; k < N2; ++k) x[k] += z[k];
        memset(H, 0, sizeof(cplx) * (size_t)(mr + 1) * mr);
    }
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = relres;
    free(Vb); free(H); free(cs); free(sn); free(g); free(yv); free(w); free(z); free(Vii);
    return status;
}

int oracle_gmres(const double *verts, const int32_t *tris, int64_t n, int K, int Kf, double threshold,
                 double s_re, double s_im, const double *bin, double *xout, double tol, int restart,
                 int maxiter, int *iters_out, double *relres_out, int nthreads)
{
    mesh_t m;
    set_threads(nthreads);
    int rc = mesh_init(&m, verts, tris, n, K, Kf, threshold);
    if (rc) return rc;
    const cplx s = s_re + I * s_im;
    int st = gmres_impl(&m, &s, bin, xout, tol, restart, maxiter, iters_out, relres_out);
    mesh_free(&m);
    return st;
}

/* Several surfaces: s [S] complex (eps_t/eps_out of one wavelength). */
int oracle_gmres_multi(const double *verts, const int32_t *tris, const int32_t *surf, int64_t n, int S, int K,
                       int Kf, double threshold, const double *s, const double *bin, double *xout, double tol,
                       int restart, int maxiter, int *iters_out, double *relres_out, int nthreads)
{
    mesh_t m;
    set_threads(nthreads);
    int rc = mesh_init(&m, verts, tris, n, K, Kf, threshold);
    if (rc) return rc;
    m.surf = surf;
    m.S = S;
    int st = gmres_impl(&m, (const cplx *)s, bin, xout, tol, restart, maxiter, iters_out, relres_out);
    mesh_free(&m);
    return st;
}

/* The same GMRES for B wavelengths in lockstep, one Krylov basis per wavelength, every
 * operator application shared by the wavelengths still iterating (apply_operator with B
 * right-hand sides: the matrix entries are evaluated once per row for all of them).  Each
 * wavelength takes exactly the steps of gmres_impl, in the same order, with the same
 * per-row accumulation order of the operator, so its iterate is the one gmres_impl would
 * produce bit for bit; only the cost is shared.  s: [B][S]; b, x: [B][2n]. */
static int gmres_batch_impl(mesh_t *mp, int B, const cplx *s, const cplx *b, cplx *x, double tol, int restart,
                            int maxiter, int *iters_out, double *relres_out)
{
    mesh_t m = *mp;
    const int64_t n = m.n;
    const int64_t N2 = 2 * n;
    const int S = m.S;
    const int mr = restart;
    double *Vii = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const panel_t *p = &m.pan[i];
        Vii[i] = oracle_self_V(p->v[0], p->v[1], p->v[2], p->c);
    }
    cplx *Vb = (cplx *)malloc(sizeof(cplx) * (size_t)N2 * (mr + 1) * B);
    cplx *H = (cplx *)calloc((size_t)(mr + 1) * mr * B, sizeof(cplx));
    cplx *cs = (cplx *)malloc(sizeof(cplx) * (size_t)mr * B), *sn = (cplx *)malloc(sizeof(cplx) * (size_t)mr * B);
    cplx *g = (cplx *)malloc(sizeof(cplx) * (size_t)(mr + 1) * B), *yv = (cplx *)malloc(sizeof(cplx) * mr);
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)N2 * B), *z = (cplx *)malloc(sizeof(cplx) * (size_t)N2 * B);
    cplx *sp = (cplx *)malloc(sizeof(cplx) * (size_t)B * S);     /* packed eps ratios of the active set */
    double *bnorm = (double *)malloc(sizeof(double) * B), *relres = (double *)malloc(sizeof(double) * B);
    int *it = (int *)calloc(B, sizeof(int)), *state = (int *)malloc(sizeof(int) * B);   /* -1 running, 0 ok, 1 not */
    int *jn = (int *)malloc(sizeof(int) * B), *live = (int *)malloc(sizeof(int) * B), *act = (int *)malloc(sizeof(int) * B);
    for (int q = 0; q < B; ++q) {
        for (int64_t i = 0; i < N2; ++i) x[(size_t)q * N2 + i] = 0.0;
        bnorm[q] = vnorm(b + (size_t)q * N2, N2);
        if (bnorm[q] == 0.0) bnorm[q] = 1.0;
        relres[q] = 1.0;
        state[q] = -1;
    }
    while (1) {
        /* explicit residuals r = b - A x of the running wavelengths, one shared product */
        int na = 0;
        for (int q = 0; q < B; ++q)
            if (state[q] < 0) act[na++] = q;
        if (na == 0) break;
        for (int a = 0; a < na; ++a) {
            memcpy(z + (size_t)a * N2, x + (size_t)act[a] * N2, sizeof(cplx) * (size_t)N2);
            memcpy(sp + (size_t)a * S, s + (size_t)act[a] * S, sizeof(cplx) * (size_t)S);
        }
        apply_operator(&m, na, sp, z, w);
        int nl = 0;
        for (int a = 0; a < na; ++a) {
            const int q = act[a];
            cplx *wq = w + (size_t)a * N2;
            const cplx *bq = b + (size_t)q * N2;
            for (int64_t i = 0; i < N2; ++i) wq[i] = bq[i] - wq[i];
            const double beta = vnorm(wq, N2);
            relres[q] = beta / bnorm[q];
            if (relres[q] <= tol) { state[q] = 0; continue; }
            if (it[q] >= maxiter) { state[q] = 1; continue; }
            cplx *v0 = Vb + (size_t)q * N2 * (mr + 1);
            for (int64_t i = 0; i < N2; ++i) v0[i] = wq[i] / beta;
            cplx *gq = g + (size_t)q * (mr + 1);
            for (int k = 0; k <= mr; ++k) gq[k] = 0.0;
            gq[0] = beta;
            jn[q] = 0;
            live[nl++] = q;
        }
        if (nl == 0) continue;
        /* Arnoldi steps; a wavelength leaves the cycle when its estimate meets tol or its
         * step budget runs out (jn = the steps it took in this cycle) */
        int *inner = (int *)malloc(sizeof(int) * nl);
        for (int a = 0; a < nl; ++a) inner[a] = 1;
        for (int j = 0; j < mr; ++j) {
            int ns = 0;
            for (int a = 0; a < nl; ++a) {
                const int q = live[a];
                if (inner[a] && it[q] < maxiter) act[ns++] = a;
                else inner[a] = 0;
            }
            if (ns == 0) break;
            for (int c = 0; c < ns; ++c) {
                const int q = live[act[c]];
                const cplx *vj = Vb + (size_t)q * N2 * (mr + 1) + (size_t)j * N2;
                precond(&m, Vii, s + (size_t)q * S, vj, z + (size_t)c * N2);
                memcpy(sp + (size_t)c * S, s + (size_t)q * S, sizeof(cplx) * (size_t)S);
            }
            apply_operator(&m, ns, sp, z, w);
            for (int c = 0; c < ns; ++c) {
                const int a = act[c], q = live[a];
                cplx *Vq = Vb + (size_t)q * N2 * (mr + 1);
                cplx *Hq = H + (size_t)q * (mr + 1) * mr, *csq = cs + (size_t)q * mr, *snq = sn + (size_t)q * mr;
                cplx *gq = g + (size_t)q * (mr + 1);
                cplx *wq = w + (size_t)c * N2, *vn = Vq + (size_t)(j + 1) * N2;
                for (int pass = 0; pass < 2; ++pass)
                    for (int i = 0; i <= j; ++i) {
                        cplx *vi = Vq + (size_t)i * N2;
                        cplx h = 0.0;
                        for (int64_t k = 0; k < N2; ++k) h += conj(vi[k]) * wq[k];
                        for (int64_t k = 0; k < N2; ++k) wq[k] -= h * vi[k];
                        Hq[i * mr + j] += h;
                    }
                double hn = vnorm(wq, N2);
                Hq[(j + 1) * mr + j] = hn;
                for (int64_t k = 0; k < N2; ++k) vn[k] = hn > 0 ? wq[k] / hn : 0.0;
                for (int i = 0; i < j; ++i) {
                    cplx aa = Hq[i * mr + j], c2 = Hq[(i + 1) * mr + j];
                    Hq[i * mr + j] = csq[i] * aa + snq[i] * c2;
                    Hq[(i + 1) * mr + j] = -conj(snq[i]) * aa + csq[i] * c2;
                }
                cplx aa = Hq[j * mr + j];
                double bb = cabs(Hq[(j + 1) * mr + j]);
                double t = sqrt(cabs(aa) * cabs(aa) + bb * bb);
                if (cabs(aa) == 0.0) {
                    csq[j] = 0.0;
                    snq[j] = 1.0;
                } else {
                    csq[j] = cabs(aa) / t;
                    snq[j] = (aa / cabs(aa)) * conj(Hq[(j + 1) * mr + j]) / t;
                }
                Hq[j * mr + j] = csq[j] * aa + snq[j] * Hq[(j + 1) * mr + j];
                Hq[(j + 1) * mr + j] = 0.0;
                gq[j + 1] = -conj(snq[j]) * gq[j];
                gq[j] = csq[j] * gq[j];
                ++it[q];
                jn[q] = j + 1;
                if (cabs(gq[j + 1]) / bnorm[q] <= tol) inner[a] = 0;
            }
        }
        free(inner);
        /* per wavelength: solve H y = g (upper triangular, size jn), x += M^-1 V y */
        for (int a = 0; a < nl; ++a) {
            const int q = live[a], jq = jn[q];
            cplx *Vq = Vb + (size_t)q * N2 * (mr + 1);
            cplx *Hq = H + (size_t)q * (mr + 1) * mr, *gq = g + (size_t)q * (mr + 1);
            for (int i = jq - 1; i >= 0; --i) {
                cplx acc = gq[i];
                for (int k = i + 1; k < jq; ++k) acc -= Hq[i * mr + k] * yv[k];
                yv[i] = acc / Hq[i * mr + i];
            }
            for (int64_t k = 0; k < N2; ++k) {
                cplx acc = 0.0;
                for (int i = 0; i < jq; ++i) acc += Vq[(size_t)i * N2 + k] * yv[i];
                w[k] = acc;
            }
            precond(&m, Vii, s + (size_t)q * S, w, z);
            cplx *xq = x + (size_t)q * N2;
            for (int64_t k = 0; k < N2; ++k) xq[k] += z[k];
            memset(Hq, 0, sizeof(cplx) * (size_t)(mr + 1) * mr);
        }
    }
    int bad = 0;
    for (int q = 0; q < B; ++q) {
        if (state[q] != 0) ++bad;
        if (iters_out) iters_out[q] = it[q];
        if (relres_out) relres_out[q] = relres[q];
    }
    free(Vb); free(H); free(cs); free(sn); free(g); free(yv); free(w); free(z); free(sp);
    free(bnorm); free(relres); free(it); free(state); free(jn); free(live); free(act); free(Vii);
    return bad;
}

/* ------------------------------------------------------------------------- */
/* Observables                                                               */
/* ------------------------------------------------------------------------- */
/* Dipole moment of the surface whose panels are [p0, p1):
 *   p = -eps2 * sum_j A_j (c_j dphi2s/dn_j - phi_j n_j),
 *   dphi2s/dn = (eps1/eps2) dphi1s/dn - ((eps2-eps1)/eps2) dphi_inc/dn.
 * phi and dphi1s/dn are constant per panel and x is linear, so the one-point
 * centroid rule integrates each panel exactly. */
void oracle_dipole(const double *verts, const int32_t *tris, int64_t n, int64_t p0, int64_t p1,
                   const double *xin, double eps_in_re, double eps_in_im, double eps_out_re,
                   double eps_out_im, const double *E0, double *pout)
{
    const cplx *x = (const cplx *)xin;
    cplx e1 = eps_in_re + I * eps_in_im, e2 = eps_out_re + I * eps_out_im;
    cplx p[3] = {0, 0, 0};
    for (int64_t j = p0; j < p1; ++j) {
        panel_t pj;
        make_panel(verts, tris, j, &pj);
        double dinc = -(E0[0] * pj.n[0] + E0[1] * pj.n[1] + E0[2] * pj.n[2]);
        cplx d2 = (e1 / e2) * x[n + j] - ((e2 - e1) / e2) * dinc;
        for (int d = 0; d < 3; ++d) p[d] += pj.area * (pj.c[d] * d2 - x[j] * pj.n[d]);
    }
    for (int d = 0; d < 3; ++d) {
        cplx v = -e2 * p[d];
        pout[2 * d] = creal(v);
        pout[2 * d + 1] = cimag(v);
    }
}

/* Dipole moment of the panels of surface `surface` (the formula of oracle_dipole with
 * that surface's eps). */
void oracle_dipole_surface(const double *verts, const int32_t *tris, const int32_t *surf, int64_t n,
                           int surface, const double *xin, double eps_in_re, double eps_in_im,
                           double eps_out_re, double eps_out_im, const double *E0, double *pout)
{
    const cplx *x = (const cplx *)xin;
    cplx e1 = eps_in_re + I * eps_in_im, e2 = eps_out_re + I * eps_out_im;
    cplx p[3] = {0, 0, 0};
    for (int64_t j = 0; j < n; ++j) {
        if (surf[j] != surface) continue;
        panel_t pj;
        make_panel(verts, tris, j, &pj);
        double dinc = -(E0[0] * pj.n[0] + E0[1] * pj.n[1] + E0[2] * pj.n[2]);
        cplx d2 = (e1 / e2) * x[n + j] - ((e2 - e1) / e2) * dinc;
        for (int d = 0; d < 3; ++d) p[d] += pj.area * (pj.c[d] * d2 - x[j] * pj.n[d]);
    }
    for (int d = 0; d < 3; ++d) {
        cplx v = -e2 * p[d];
        pout[2 * d] = creal(v);
        pout[2 * d + 1] = cimag(v);
    }
}

/* sigma_ext = Im(k^2 e.p / (eps2 |E0|)) / Re k, k = 2 pi sqrt(eps2) / lambda. */
double oracle_sigma_ext(const double *pin, double eps_out_re, double eps_out_im, const double *E0,
                        double lambda_nm)
{
    const cplx *p = (const cplx *)pin;
    cplx e2 = eps_out_re + I * eps_out_im;
    double E = sqrt(E0[0] * E0[0] + E0[1] * E0[1] + E0[2] * E0[2]);
    cplx ep = (E0[0] * p[0] + E0[1] * p[1] + E0[2] * p[2]) / E;
    cplx k = 2.0 * M_PI * csqrt(e2) / lambda_nm;
    return cimag(k * k * ep / (e2 * E)) / creal(k);
}

/* Eq. an_sol: C_ext = (4 pi a^3 / k') Im(k^2 (ep/em - 1)/(ep/em + 2)). */
double oracle_sigma_closed_form(double R, double ep_re, double ep_im, double em_re, double em_im,
                                double lambda_nm)
{
    cplx ep = ep_re + I * ep_im, em = em_re + I * em_im;
    cplx k = 2.0 * M_PI * csqrt(em) / lambda_nm;
    cplx r = ep / em;
    return 4.0 * M_PI * R * R * R / creal(k) * cimag(k * k * (r - 1.0) / (r + 2.0));
}

/* Full single-interface solve for B wavelengths, one after another:
 * RHS, GMRES, dipole of panels [0, n), sigma_ext.  Returns the number of
 * wavelengths that did not converge.  dip_out: [B][3] complex, sigma: [B]. */
int oracle_solve(const double *verts, const int32_t *tris, int64_t n, int K, int Kf, double threshold,
                 int B, const double *eps_in, double eps_out_re, double eps_out_im, const double *E0,
                 const double *lambda_nm, double tol, int restart, int maxiter, double *dip_out,
                 double *sigma_out, int *iters_out, int nthreads)
{
    const int64_t N2 = 2 * n;
    double *b = (double *)malloc(sizeof(double) * 2 * (size_t)N2);
    double *x = (double *)malloc(sizeof(double) * 2 * (size_t)N2);
    int bad = 0;
    for (int bb = 0; bb < B; ++bb) {
        oracle_rhs(verts, tris, n, K, Kf, threshold, 1, eps_in + 2 * bb, eps_out_re, eps_out_im, E0, b,
                   nthreads);
        cplx e1 = eps_in[2 * bb] + I * eps_in[2 * bb + 1];
        cplx s = e1 / (eps_out_re + I * eps_out_im);
        int it = 0;
        double rr = 0;
        int st = oracle_gmres(verts, tris, n, K, Kf, threshold, creal(s), cimag(s), b, x, tol, restart,
                              maxiter, &it, &rr, nthreads);
        if (st) ++bad;
        if (iters_out) iters_out[bb] = it;
        oracle_dipole(verts, tris, n, 0, n, x, eps_in[2 * bb], eps_in[2 * bb + 1], eps_out_re, eps_out_im,
                      E0, dip_out + 6 * bb);
        sigma_out[bb] = oracle_sigma_ext(dip_out + 6 * bb, eps_out_re, eps_out_im, E0, lambda_nm[bb]);
    }
    free(b);
    free(x);
    return bad;
}

/* Several surfaces, one wavelength after another: RHS, GMRES, dipole of surface 0
 * (the particle) and its sigma_ext.  eps_in: [B][S] complex.  Returns the number of
 * wavelengths that did not converge. */
int oracle_solve_multi(const double *verts, const int32_t *tris, const int32_t *surf, int64_t n, int S, int K,
                       int Kf, double threshold, int B, const double *eps_in, double eps_out_re,
                       double eps_out_im, const double *E0, const double *lambda_nm, double tol, int restart,
                       int maxiter, double *dip_out, double *sigma_out, int *iters_out, int nthreads,
                       int64_t nq, const double *charges, const int32_t *surf_q)
{
    const int64_t N2 = 2 * n;
    double *b = (double *)malloc(sizeof(double) * 2 * (size_t)N2);
    double *x = (double *)malloc(sizeof(double) * 2 * (size_t)N2);
    double *s = (double *)malloc(sizeof(double) * 2 * (size_t)S);
    int bad = 0;
    const cplx e2 = eps_out_re + I * eps_out_im;
    for (int bb = 0; bb < B; ++bb) {
        const double *e1 = eps_in + 2 * (size_t)S * bb;
        oracle_rhs_multi(verts, tris, surf, n, S, K, Kf, threshold, 1, e1, eps_out_re, eps_out_im, E0, b,
                         nthreads);
        if (nq > 0 && oracle_rhs_charges(verts, tris, surf, n, S, 1, e1, nq, charges, surf_q, b)) {
            bad = B;
            break;
        }
        for (int t = 0; t < S; ++t) {
            cplx st = (e1[2 * t] + I * e1[2 * t + 1]) / e2;
            s[2 * t] = creal(st);
            s[2 * t + 1] = cimag(st);
        }
        int it = 0;
        double rr = 0;
        int st = oracle_gmres_multi(verts, tris, surf, n, S, K, Kf, threshold, s, b, x, tol, restart, maxiter,
                                    &it, &rr, nthreads);
        if (st) ++bad;
        if (iters_out) iters_out[bb] = it;
        oracle_dipole_surface(verts, tris, surf, n, 0, x, e1[0], e1[1], eps_out_re, eps_out_im, E0,
                              dip_out + 6 * bb);
        sigma_out[bb] = oracle_sigma_ext(dip_out + 6 * bb, eps_out_re, eps_out_im, E0, lambda_nm[bb]);
    }
    free(b);
    free(x);
    free(s);
    return bad;
}

/* The solve of oracle_solve_multi (surf may be NULL for one surface) for B wavelengths with
 * every operator application shared across them: the right-hand sides of all wavelengths
 * from one pass over V, then gmres_batch_impl, then each wavelength's dipole of surface 0 and
 * sigma_ext.  Results equal oracle_solve / oracle_solve_multi wavelength by wavelength bit for
 * bit; only the matrix-entry evaluations are shared.  eps_in: [B][S] complex.  Returns the
 * number of wavelengths that did not converge. */
int oracle_solve_batch(const double *verts, const int32_t *tris, const int32_t *surf, int64_t n, int S, int K,
                       int Kf, double threshold, int B, const double *eps_in, double eps_out_re,
                       double eps_out_im, const double *E0, const double *lambda_nm, double tol, int restart,
                       int maxiter, double *dip_out, double *sigma_out, int *iters_out, double *relres_out,
                       int nthreads)
{
    mesh_t m;
    set_threads(nthreads);
    int rc = mesh_init(&m, verts, tris, n, K, Kf, threshold);
    if (rc) return -1;
    m.surf = surf;
    m.S = surf ? S : 1;
    const int64_t N2 = 2 * n;
    const cplx e2 = eps_out_re + I * eps_out_im;
    cplx *b = (cplx *)malloc(sizeof(cplx) * (size_t)N2 * B);
    cplx *x = (cplx *)malloc(sizeof(cplx) * (size_t)N2 * B);
    cplx *s = (cplx *)malloc(sizeof(cplx) * (size_t)B * m.S);
    rhs_impl(&m, B, (const cplx *)eps_in, e2, E0, b);
    for (int q = 0; q < B * m.S; ++q) s[q] = (eps_in[2 * q] + I * eps_in[2 * q + 1]) / e2;
    int bad = gmres_batch_impl(&m, B, s, b, x, tol, restart, maxiter, iters_out, relres_out);
    for (int q = 0; q < B; ++q) {
        const double *e1 = eps_in + 2 * (size_t)m.S * q;
        const double *xq = (const double *)(x + (size_t)q * N2);
        if (surf)
            oracle_dipole_surface(verts, tris, surf, n, 0, xq, e1[0], e1[1], eps_out_re, eps_out_im, E0,
                                  dip_out + 6 * q);
        else
            oracle_dipole(verts, tris, n, 0, n, xq, e1[0], e1[1], eps_out_re, eps_out_im, E0, dip_out + 6 * q);
        sigma_out[q] = oracle_sigma_ext(dip_out + 6 * q, eps_out_re, eps_out_im, E0, lambda_nm[q]);
    }
    free(b);
    free(x);
    free(s);
    mesh_free(&m);
    return bad;
}
