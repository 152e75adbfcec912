/*
 * Plain FP64 CPU oracle for the FMM-accelerated Helmholtz single-layer matvec.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code with the CUDA path.
 *
 * What it computes (paper: "Extreme Scale FMM-Accelerated Boundary Integral
 * Equation Solver for Wave Scattering", arXiv:1803.09948):
 *
 *   Green's function            G(x,y) = exp(i k R) / (4 pi R)        (Eq. 6)
 *   sound-soft single layer     int_S G q dS = p_inc                  (Eq. 7)
 *   Nystrom discretisation      Z I = V_inc, Z from Eq. 10 (Sec. 2.2), here on flat
 *                               triangles with three interior points each
 *   singular / near-singular    exact integrals over the own triangle and
 *   treatment                   the near triangles (Sec. 2.2, Listing 1)
 *   FMM                         P2M, M2M, M2L, L2L, L2P, P2P on an octree
 *                               with spherical-harmonic expansions (Eq. 11-14,
 *                               Sec. 2.3)
 *
 * Discrete operator (the definition every path is checked against):
 *   point (n,a), a = 0,1,2, sits at barycentric (2/3,1/6,1/6) (and
 *   permutations) of triangle n, weight w = area/3, basis L_(n,a) = 2 lambda_a - 1/3
 *   (the linear Lagrange function equal to 1 at point a and 0 at the other two).
 *   S(i) = own triangle of i, plus every triangle with a point within r_near of x_i.
 *   (Z s)_i = sum_{n not in S(i)} sum_a w_(n,a) G(x_i, x_(n,a)) s_(n,a)
 *           + sum_{n in S(i)}     sum_a s_(n,a) int_{T_n} G(x_i,y) L_(n,a)(y) dS_y
 *
 * The singular integrals use singularity subtraction (a method the paper cites
 * beside Duffy's, Sec. 2.2): the 1/R part in closed form (flat-triangle
 * potential formulas), the bounded remainder (exp(ikR)-1)/R by nested
 * adaptive Gauss-Legendre in polar coordinates about the foot point of x.
 * The CUDA path integrates the whole kernel with a Duffy-type
 * transformation instead; the two are independent routes to the same integral.
 *
 * Only real wavenumbers k are supported.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
static inline void v_sub(const double* a, const double* b, double* c) {
    c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2];
}
static inline double v_dot(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static inline void v_cross(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double v_norm(const double* a) { return sqrt(v_dot(a, a)); }

/* Green's function, Eq. 6 (real k). */
static inline cplx green(double k, double R) {
    return cexp(I * k * R) / (4.0 * OR_PI * R);
}

/* ------------------------------------------------------------------------ */
/* Mesh -> quadrature points (Sec. 2.2 with flat triangles)                  */
/* ------------------------------------------------------------------------ */
void or_points(const double* V, const int32_t* F, int64_t nt,
               double* X, double* W, int32_t* T) {
    for (int64_t n = 0; n < nt; ++n) {
        const double* v[3] = {V + 3 * (int64_t)F[3 * n], V + 3 * (int64_t)F[3 * n + 1],
                              V + 3 * (int64_t)F[3 * n + 2]};
        double e1[3], e2[3], c[3];
        v_sub(v[1], v[0], e1);
        v_sub(v[2], v[0], e2);
        v_cross(e1, e2, c);
        double area = 0.5 * v_norm(c);
        for (int a = 0; a < 3; ++a) {
            int64_t i = 3 * n + a;
            for (int d = 0; d < 3; ++d)
                X[3 * i + d] = (2.0 / 3.0) * v[a][d] + (1.0 / 6.0) * v[(a + 1) % 3][d] +
                               (1.0 / 6.0) * v[(a + 2) % 3][d];
            W[i] = area / 3.0;
            T[i] = (int32_t)n;
        }
    }
}

/* Mean edge length over all triangles (each triangle's three edges). */
double or_mean_edge(const double* V, const int32_t* F, int64_t nt) {
    double s = 0.0;
    for (int64_t n = 0; n < nt; ++n) {
        for (int a = 0; a < 3; ++a) {
            double e[3];
            v_sub(V + 3 * (int64_t)F[3 * n + (a + 1) % 3], V + 3 * (int64_t)F[3 * n + a], e);
            s += v_norm(e);
        }
    }
    return nt > 0 ? s / (3.0 * (double)nt) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Closed-form flat-triangle potentials of 1/R                               */
/*   I0 = int_T 1/R dS,  I1 = int_T (y - x_p)/R dS  (x_p: projection of x)   */
/* Derived edge by edge in polar coordinates about x_p; I1 from the surface  */
/* divergence theorem (grad_y R = (y - x_p)/R in the plane).                 */
/* ------------------------------------------------------------------------ */
static double log_l_plus_R(double l, double R, double R0sq) {
    /* log(l + R) with R = sqrt(l^2 + R0^2), stable for l << 0 */
    if (l >= 0.0) return log(l + R);
    return log(R0sq / (R - l));
}

void or_tri_potential_1overR(const double* x, const double* v, double* I0, double* I1) {
    const double* p[3] = {v, v + 3, v + 6};
    double e1[3], e2[3], nrm[3];
    v_sub(p[1], p[0], e1);
    v_sub(p[2], p[0], e2);
    v_cross(e1, e2, nrm);
    double nn = v_norm(nrm);
    for (int d = 0; d < 3; ++d) nrm[d] /= nn;
    double xv0[3];
    v_sub(x, p[0], xv0);
    double w = v_dot(xv0, nrm);
    double aw = fabs(w);
    double xp[3] = {x[0] - w * nrm[0], x[1] - w * nrm[1], x[2] - w * nrm[2]};
    double i0 = 0.0, i1[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 3; ++i) {
        const double* a = p[i];
        const double* b = p[(i + 1) % 3];
        double ed[3];
        v_sub(b, a, ed);
        double len = v_norm(ed);
        double lhat[3] = {ed[0] / len, ed[1] / len, ed[2] / len};
        double uhat[3];
        v_cross(lhat, nrm, uhat); /* outward in-plane edge normal */
        double am[3], bm[3];
        v_sub(a, xp, am);
        v_sub(b, xp, bm);
        double lm = v_dot(am, lhat), lp = v_dot(bm, lhat);
        double P0 = v_dot(am, uhat); /* >0 when x_p is on the inner side */
        double R0sq = P0 * P0 + w * w;
        double xa[3], xb[3];
        v_sub(x, a, xa);
        v_sub(x, b, xb);
        double Rm = v_norm(xa), Rp = v_norm(xb);
        double lg = 0.0;
        if (R0sq > 0.0) lg = log_l_plus_R(lp, Rp, R0sq) - log_l_plus_R(lm, Rm, R0sq);
        if (fabs(P0) > 0.0) {
            i0 += P0 * lg;
            if (aw > 0.0)
                i0 -= aw * (atan(P0 * lp / (R0sq + aw * Rp)) - atan(P0 * lm / (R0sq + aw * Rm)));
        }
        double edge_int = 0.5 * (R0sq * lg + lp * Rp - lm * Rm); /* int sqrt(l^2+R0^2) dl */
        for (int d = 0; d < 3; ++d) i1[d] += uhat[d] * edge_int;
    }
    *I0 = i0;
    I1[0] = i1[0]; I1[1] = i1[1]; I1[2] = i1[2];
}

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre nodes on [0,1] (Newton on P_n)                             */
/* ------------------------------------------------------------------------ */
static void gauss_legendre01(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double pp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            pp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * pp * pp);
    }
}

/* ------------------------------------------------------------------------ */
/* Bounded remainder (exp(ikR)-1)/R * L_a(y) in polar coordinates about x_p  */
/*                                                                          */
/* For each edge i the signed sub-triangle (x_p, v_i, v_i+1) is covered by   */
/* y(t,l) = x_p + t (f_i + l lhat_i - x_p), t in [0,1], l in [l-, l+], where */
/* f_i is the foot of the perpendicular from x_p to the edge line and P0 the */
/* signed distance to it; dS = P0 t dt dl.  R^2 = t^2 (P0^2 + l^2) + w^2.    */
/* Both 1-D integrals use adaptive Gauss-Legendre (10 points vs. the two    */
/* halves).                                                                  */
/* ------------------------------------------------------------------------ */
#define GLN 10
static double g_gl_x[GLN], g_gl_w[GLN];
static int g_gl_init = 0;

static void gl_init(void) {
    if (!g_gl_init) {
        gauss_legendre01(GLN, g_gl_x, g_gl_w);
        g_gl_init = 1;
    }
}

typedef struct {
    double x[3];
    double k;
    double v0[3];
    double gl[3][3]; /* gradients of barycentric coordinates */
    double l0[3];    /* barycentric values at v0 */
    double xp[3], w;
    /* current edge */
    double foot[3], lhat[3], P0;
} remainder_ctx;

static inline cplx expm1_over_R(double k, double R) {
    double z = k * R;
    if (fabs(z) < 1e-3) {
        cplx iz = I * z;
        return I * k * (1.0 + iz / 2.0 + iz * iz / 6.0 + iz * iz * iz / 24.0 + iz * iz * iz * iz / 120.0);
    }
    return (cexp(I * z) - 1.0) / R;
}

/* P0 * t * g(R) * L_a(y(t,l)) on GLN nodes of [t0,t1] */
static void rem_t_rule(const remainder_ctx* c, double l, double t0, double t1, cplx out[3]) {
    double E[3];
    for (int q = 0; q < 3; ++q) E[q] = c->foot[q] + l * c->lhat[q] - c->xp[q];
    double rho2 = v_dot(E, E);
    out[0] = out[1] = out[2] = 0.0;
    for (int i = 0; i < GLN; ++i) {
        double t = t0 + (t1 - t0) * g_gl_x[i];
        double wt = (t1 - t0) * g_gl_w[i];
        double R = sqrt(t * t * rho2 + c->w * c->w);
        cplx g = expm1_over_R(c->k, R);
        double yv[3];
        for (int q = 0; q < 3; ++q) yv[q] = c->xp[q] + t * E[q] - c->v0[q];
        for (int a = 0; a < 3; ++a) {
            double lam = c->l0[a] + v_dot(c->gl[a], yv);
            out[a] += wt * c->P0 * t * g * (2.0 * lam - 1.0 / 3.0);
        }
    }
}

static void rem_t_adapt(const remainder_ctx* c, double l, double t0, double t1, const cplx whole[3],
                        double tol, int depth, cplx acc[3]) {
    double tm = 0.5 * (t0 + t1);
    cplx a[3], b[3];
    rem_t_rule(c, l, t0, tm, a);
    rem_t_rule(c, l, tm, t1, b);
    double err = 0.0;
    for (int q = 0; q < 3; ++q) err = fmax(err, cabs(a[q] + b[q] - whole[q]));
    if (err <= tol || depth >= 50) {
        for (int q = 0; q < 3; ++q) acc[q] += a[q] + b[q];
        return;
    }
    rem_t_adapt(c, l, t0, tm, a, 0.5 * tol, depth + 1, acc);
    rem_t_adapt(c, l, tm, t1, b, 0.5 * tol, depth + 1, acc);
}

static void rem_inner(const remainder_ctx* c, double l, double tol, cplx out[3]) {
    cplx whole[3];
    rem_t_rule(c, l, 0.0, 1.0, whole);
    out[0] = out[1] = out[2] = 0.0;
    rem_t_adapt(c, l, 0.0, 1.0, whole, tol, 0, out);
}

static void rem_l_rule(const remainder_ctx* c, double l0, double l1, double tol, cplx out[3]) {
    out[0] = out[1] = out[2] = 0.0;
    for (int i = 0; i < GLN; ++i) {
        double l = l0 + (l1 - l0) * g_gl_x[i];
        double wt = (l1 - l0) * g_gl_w[i];
        cplx f[3];
        rem_inner(c, l, tol, f);
        for (int a = 0; a < 3; ++a) out[a] += wt * f[a];
    }
}

static void rem_l_adapt(const remainder_ctx* c, double l0, double l1, const cplx whole[3],
                        double tol, double itol, int depth, cplx acc[3]) {
    double lm = 0.5 * (l0 + l1);
    cplx a[3], b[3];
    rem_l_rule(c, l0, lm, itol, a);
    rem_l_rule(c, lm, l1, itol, b);
    double err = 0.0;
    for (int q = 0; q < 3; ++q) err = fmax(err, cabs(a[q] + b[q] - whole[q]));
    if (err <= tol || depth >= 50) {
        for (int q = 0; q < 3; ++q) acc[q] += a[q] + b[q];
        return;
    }
    rem_l_adapt(c, l0, lm, a, 0.5 * tol, itol, depth + 1, acc);
    rem_l_adapt(c, lm, l1, b, 0.5 * tol, itol, depth + 1, acc);
}

/*
 * out[a] = int_T G(x,y) L_a(y) dS_y, a = 0,1,2, with L_a = 2 lambda_a - 1/3 and
 * v the triangle's vertices (9 doubles, counter-clockwise).  Exact up to the
 * adaptive tolerance (absolute 1e-13 * |k| * area on the remainder).
 */
void or_tri_integrals(const double* x, const double* v, double k, double* out_ri) {
    gl_init();
    const double* p[3] = {v, v + 3, v + 6};
    double e1[3], e2[3], cr[3];
    v_sub(p[1], p[0], e1);
    v_sub(p[2], p[0], e2);
    v_cross(e1, e2, cr);
    double twoA = v_norm(cr);
    double nrm[3] = {cr[0] / twoA, cr[1] / twoA, cr[2] / twoA};
    remainder_ctx c;
    memcpy(c.x, x, sizeof(c.x));
    c.k = k;
    memcpy(c.v0, p[0], sizeof(c.v0));
    for (int a = 0; a < 3; ++a) {
        double opp[3];
        v_sub(p[(a + 2) % 3], p[(a + 1) % 3], opp);
        double g[3];
        v_cross(nrm, opp, g);
        for (int q = 0; q < 3; ++q) c.gl[a][q] = g[q] / twoA;
        c.l0[a] = (a == 0) ? 1.0 : 0.0;
    }
    /* singular part: (1/R) L_a, closed form */
    double I0, I1[3];
    or_tri_potential_1overR(x, v, &I0, I1);
    double xv0[3];
    v_sub(x, p[0], xv0);
    double wn = v_dot(xv0, nrm);
    double xp[3] = {x[0] - wn * nrm[0], x[1] - wn * nrm[1], x[2] - wn * nrm[2]};
    double xpv0[3];
    v_sub(xp, p[0], xpv0);
    cplx res[3];
    for (int a = 0; a < 3; ++a) {
        double lam_xp = c.l0[a] + v_dot(c.gl[a], xpv0);
        double La_xp = 2.0 * lam_xp - 1.0 / 3.0;
        res[a] = La_xp * I0 + 2.0 * v_dot(c.gl[a], I1);
    }
    /* bounded remainder, polar coordinates about x_p, edge by edge */
    double area = 0.5 * twoA;
    cplx rem[3] = {0, 0, 0};
    memcpy(c.xp, xp, sizeof(c.xp));
    c.w = wn;
    if (k != 0.0) {
        for (int e = 0; e < 3; ++e) {
            const double* a = p[e];
            const double* b = p[(e + 1) % 3];
            double ed[3];
            v_sub(b, a, ed);
            double len = v_norm(ed);
            double uhat[3];
            for (int q = 0; q < 3; ++q) c.lhat[q] = ed[q] / len;
            v_cross(c.lhat, nrm, uhat);
            double am[3], bm[3];
            v_sub(a, xp, am);
            v_sub(b, xp, bm);
            c.P0 = v_dot(am, uhat);
            if (fabs(c.P0) <= 1e-15 * len) continue;
            for (int q = 0; q < 3; ++q) c.foot[q] = xp[q] + c.P0 * uhat[q];
            double lm = v_dot(am, c.lhat), lp = v_dot(bm, c.lhat);
            double scale = fabs(k) * area + 1e-300;
            double tol = 1e-13 * scale, itol = 1e-14 * fabs(k) * fabs(c.P0) + 1e-300;
            cplx whole[3];
            rem_l_rule(&c, lm, lp, itol, whole);
            rem_l_adapt(&c, lm, lp, whole, tol, itol, 0, rem);
        }
    }
    for (int a = 0; a < 3; ++a) {
        cplx r = (res[a] + rem[a]) / (4.0 * OR_PI);
        out_ri[2 * a] = creal(r);
        out_ri[2 * a + 1] = cimag(r);
    }
}

/* ------------------------------------------------------------------------ */
/* Near sets: S(i) = {own triangle} u {n : min_a |x_i - x_(n,a)| <= r_near}   */
/* found with a uniform hash grid of cell size >= r_near.                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    double lo[3];
    double cell;
    int64_t dims[3];
    int64_t* start; /* cell -> first sorted point, size ncell + 1 */
    int64_t* order; /* sorted point ids */
} grid_t;

static int64_t grid_cell_of(const grid_t* g, const double* x, int64_t* c3) {
    for (int d = 0; d < 3; ++d) {
        int64_t c = (int64_t)floor((x[d] - g->lo[d]) / g->cell);
        if (c < 0) c = 0;
        if (c >= g->dims[d]) c = g->dims[d] - 1;
        c3[d] = c;
    }
    return (c3[2] * g->dims[1] + c3[1]) * g->dims[0] + c3[0];
}

static void grid_build(grid_t* g, const double* X, int64_t N, double r) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], X[3 * i + d]);
            hi[d] = fmax(hi[d], X[3 * i + d]);
        }
    double ext = fmax(hi[0] - lo[0], fmax(hi[1] - lo[1], hi[2] - lo[2]));
    double cell = fmax(r, ext / 256.0);
    if (cell <= 0.0) cell = 1.0;
    g->cell = cell;
    int64_t ncell = 1;
    for (int d = 0; d < 3; ++d) {
        g->lo[d] = lo[d];
        g->dims[d] = (int64_t)floor((hi[d] - lo[d]) / cell) + 1;
        ncell *= g->dims[d];
    }
    g->start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    g->order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    int64_t* cid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    int64_t c3[3];
    for (int64_t i = 0; i < N; ++i) {
        cid[i] = grid_cell_of(g, X + 3 * i, c3);
        g->start[cid[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) g->start[c + 1] += g->start[c];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    memcpy(fill, g->start, sizeof(int64_t) * (size_t)ncell);
    for (int64_t i = 0; i < N; ++i) g->order[fill[cid[i]]++] = i;
    free(fill);
    free(cid);
}

static void grid_free(grid_t* g) {
    free(g->start);
    free(g->order);
}

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/*
 * Collects the sorted, unique triangles of S(i) (own triangle, plus every
 * triangle with a point within r_near of x_i) into out.  Returns their number,
 * or -1 when the candidate list would exceed cap entries: the set is then
 * refused, never truncated.
 */
static int near_tris_of(const grid_t* g, const double* X, const int32_t* T, int64_t i,
                        double r_near, int32_t* out, int cap) {
    int cnt = 0;
    out[cnt++] = T[i];
    int64_t c3[3];
    grid_cell_of(g, X + 3 * i, c3);
    double r2 = r_near * r_near;
    for (int64_t dz = -1; dz <= 1; ++dz)
        for (int64_t dy = -1; dy <= 1; ++dy)
            for (int64_t dx = -1; dx <= 1; ++dx) {
                int64_t cx = c3[0] + dx, cy = c3[1] + dy, cz = c3[2] + dz;
                if (cx < 0 || cy < 0 || cz < 0 || cx >= g->dims[0] || cy >= g->dims[1] ||
                    cz >= g->dims[2])
                    continue;
                int64_t c = (cz * g->dims[1] + cy) * g->dims[0] + cx;
                for (int64_t s = g->start[c]; s < g->start[c + 1]; ++s) {
                    int64_t j = g->order[s];
                    double d[3];
                    v_sub(X + 3 * i, X + 3 * j, d);
                    if (v_dot(d, d) <= r2) {
                        if (cnt >= cap) return -1;
                        out[cnt++] = T[j];
                    }
                }
            }
    qsort(out, (size_t)cnt, sizeof(int32_t), cmp_i32);
    int u = 0;
    for (int q = 0; q < cnt; ++q)
        if (u == 0 || out[q] != out[u - 1]) out[u++] = out[q];
    return u;
}

#define NEAR_CAP 4096

/*
 * Correction matrix C = Z - Z_point restricted to the near sets, in CSR form
 * (rows and columns are point indices 3n+a; Z_point_ij = w_j G(x_i,x_j), 0 on
 * the diagonal).  Call once with col == NULL to get row counts in rowptr[1..N]
 * (rowptr[0] = 0 and the prefix sum are filled in), then again with storage.
 * Returns the number of nonzeros, or -1 if some near set exceeds NEAR_CAP
 * candidate entries (the matrix is then incomplete and must not be used).
 */
int64_t or_correction_csr(const double* V, const int32_t* F, int64_t nt, double k, double r_near,
                          int64_t* rowptr, int64_t* col, double* val_ri) {
    int64_t N = 3 * nt;
    double* X = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* W = (double*)malloc(sizeof(double) * (size_t)N);
    int32_t* T = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    or_points(V, F, nt, X, W, T);
    grid_t g;
    grid_build(&g, X, N, r_near);
    int overflow = 0;
    if (col == NULL) {
        rowptr[0] = 0;
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = 0; i < N; ++i) {
            int32_t buf[NEAR_CAP];
            int c = near_tris_of(&g, X, T, i, r_near, buf, NEAR_CAP);
            if (c < 0) {
#pragma omp atomic write
                overflow = 1;
                c = 0;
            }
            rowptr[i + 1] = 3 * (int64_t)c;
        }
        for (int64_t i = 0; i < N; ++i) rowptr[i + 1] += rowptr[i];
    } else {
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t i = 0; i < N; ++i) {
            int32_t buf[NEAR_CAP];
            int c = near_tris_of(&g, X, T, i, r_near, buf, NEAR_CAP);
            if (c < 0) {
#pragma omp atomic write
                overflow = 1;
                continue;
            }
            int64_t o = rowptr[i];
            for (int q = 0; q < c; ++q) {
                int64_t n = buf[q];
                double v[9];
                for (int a = 0; a < 3; ++a)
                    for (int d = 0; d < 3; ++d) v[3 * a + d] = V[3 * (int64_t)F[3 * n + a] + d];
                double ri[6];
                or_tri_integrals(X + 3 * i, v, k, ri);
                for (int a = 0; a < 3; ++a) {
                    int64_t j = 3 * n + a;
                    cplx z = ri[2 * a] + I * ri[2 * a + 1];
                    if (j != i) {
                        double d[3];
                        v_sub(X + 3 * i, X + 3 * j, d);
                        z -= W[j] * green(k, v_norm(d));
                    }
                    col[o] = j;
                    val_ri[2 * o] = creal(z);
                    val_ri[2 * o + 1] = cimag(z);
                    ++o;
                }
            }
        }
    }
    grid_free(&g);
    free(X);
    free(W);
    free(T);
    return overflow ? -1 : rowptr[N];
}

/*
 * Rows of Z s by the definition above (direct O(N) per row).
 * rows: nrows point indices; sigma: N complex (interleaved); out: nrows complex.
 * mode bit 0: include the point part; bit 1: include the near/self integrals.
 */
int or_direct_rows(const double* V, const int32_t* F, int64_t nt, double k, double r_near,
                   const int64_t* rows, int64_t nrows, const double* sigma_ri, double* out_ri,
                   int mode) {
    int overflow = 0;
    int64_t N = 3 * nt;
    double* X = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* W = (double*)malloc(sizeof(double) * (size_t)N);
    int32_t* T = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    or_points(V, F, nt, X, W, T);
    grid_t g;
    grid_build(&g, X, N, r_near);
#pragma omp parallel
    {
        unsigned char* mark = (unsigned char*)calloc((size_t)(nt > 0 ? nt : 1), 1);
#pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t i = rows[r];
            int32_t buf[NEAR_CAP];
            int c = near_tris_of(&g, X, T, i, r_near, buf, NEAR_CAP);
            if (c < 0) {
#pragma omp atomic write
                overflow = 1;
                out_ri[2 * r] = out_ri[2 * r + 1] = NAN;
                continue;
            }
            for (int q = 0; q < c; ++q) mark[buf[q]] = 1;
            cplx acc = 0.0;
            if (mode & 1) {
                for (int64_t j = 0; j < N; ++j) {
                    if (mark[T[j]]) continue;
                    double d[3];
                    v_sub(X + 3 * i, X + 3 * j, d);
                    cplx s = sigma_ri[2 * j] + I * sigma_ri[2 * j + 1];
                    acc += W[j] * green(k, v_norm(d)) * s;
                }
            }
            if (mode & 2) {
                for (int q = 0; q < c; ++q) {
                    int64_t n = buf[q];
                    double v[9];
                    for (int a = 0; a < 3; ++a)
                        for (int d = 0; d < 3; ++d) v[3 * a + d] = V[3 * (int64_t)F[3 * n + a] + d];
                    double ri[6];
                    or_tri_integrals(X + 3 * i, v, k, ri);
                    for (int a = 0; a < 3; ++a) {
                        int64_t j = 3 * n + a;
                        cplx s = sigma_ri[2 * j] + I * sigma_ri[2 * j + 1];
                        acc += (ri[2 * a] + I * ri[2 * a + 1]) * s;
                    }
                }
            }
            for (int q = 0; q < c; ++q) mark[buf[q]] = 0;
            out_ri[2 * r] = creal(acc);
            out_ri[2 * r + 1] = cimag(acc);
        }
        free(mark);
    }
    grid_free(&g);
    free(X);
    free(W);
    free(T);
    return overflow ? -1 : 0;
}

/* Dense Z (row-major, N x N complex interleaved) by the same definition.
   Returns 0, or -1 if some near set exceeds NEAR_CAP candidate entries. */
int or_dense_Z(const double* V, const int32_t* F, int64_t nt, double k, double r_near,
               double* Z_ri) {
    int overflow = 0;
    int64_t N = 3 * nt;
    double* X = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* W = (double*)malloc(sizeof(double) * (size_t)N);
    int32_t* T = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    or_points(V, F, nt, X, W, T);
    grid_t g;
    grid_build(&g, X, N, r_near);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < N; ++i) {
        int32_t buf[NEAR_CAP];
        int c = near_tris_of(&g, X, T, i, r_near, buf, NEAR_CAP);
        if (c < 0) {
#pragma omp atomic write
            overflow = 1;
            c = 0;
        }
        double* row = Z_ri + 2 * N * i;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) { row[2 * j] = row[2 * j + 1] = 0.0; continue; }
            double d[3];
            v_sub(X + 3 * i, X + 3 * j, d);
            cplx z = W[j] * green(k, v_norm(d));
            row[2 * j] = creal(z);
            row[2 * j + 1] = cimag(z);
        }
        for (int q = 0; q < c; ++q) {
            int64_t n = buf[q];
            double v[9];
            for (int a = 0; a < 3; ++a)
                for (int d = 0; d < 3; ++d) v[3 * a + d] = V[3 * (int64_t)F[3 * n + a] + d];
            double ri[6];
            or_tri_integrals(X + 3 * i, v, k, ri);
            for (int a = 0; a < 3; ++a) {
                row[2 * (3 * n + a)] = ri[2 * a];
                row[2 * (3 * n + a) + 1] = ri[2 * a + 1];
            }
        }
    }
    grid_free(&g);
    free(X);
    free(W);
    free(T);
    return overflow ? -1 : 0;
}

/*
 * The near sets S(i) themselves, in CSR form: ptr[0..N] and idx[ptr[i]..ptr[i+1])
 * = the sorted triangle ids of S(i) (Sec. 2.2: the own patch and the patches
 * within the near distance, which Listing 1 integrates apart).  Call with
 * idx == NULL for the counts (ptr gets the prefix sum), then with storage.
 * Returns the total number of entries, or -1 if some set exceeds NEAR_CAP
 * candidate entries.
 */
int64_t or_near_sets(const double* V, const int32_t* F, int64_t nt, double r_near, int64_t* ptr,
                     int32_t* idx) {
    int64_t N = 3 * nt;
    double* X = (double*)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    double* W = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    int32_t* T = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    or_points(V, F, nt, X, W, T);
    grid_t g;
    grid_build(&g, X, N, r_near);
    int overflow = 0;
    if (idx == NULL) ptr[0] = 0;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < N; ++i) {
        int32_t buf[NEAR_CAP];
        int c = near_tris_of(&g, X, T, i, r_near, buf, NEAR_CAP);
        if (c < 0) {
#pragma omp atomic write
            overflow = 1;
            c = 0;
        }
        if (idx == NULL) ptr[i + 1] = c;
        else memcpy(idx + ptr[i], buf, sizeof(int32_t) * (size_t)c);
    }
    if (idx == NULL)
        for (int64_t i = 0; i < N; ++i) ptr[i + 1] += ptr[i];
    grid_free(&g);
    free(X);
    free(W);
    free(T);
    return overflow ? -1 : ptr[N];
}

/* Raw kernel sum  out_i = sum_{j != i, R_ij > 0} w_j G(x_i, x_j) s_j  (no corrections). */
void or_point_sum(const double* X, const double* W, int64_t N, double k, const double* sigma_ri,
                  double* out_ri) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < N; ++i) {
        cplx acc = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double d[3];
            v_sub(X + 3 * i, X + 3 * j, d);
            double R = v_norm(d);
            if (j == i || R == 0.0) continue;
            acc += W[j] * green(k, R) * (sigma_ri[2 * j] + I * sigma_ri[2 * j + 1]);
        }
        out_ri[2 * i] = creal(acc);
        out_ri[2 * i + 1] = cimag(acc);
    }
}

/* Rows of the raw kernel sum: out_r = sum_{j != i, R_ij > 0} w_j G(x_i, x_j) s_j for i = rows[r]. */
void or_point_sum_rows(const double* X, const double* W, int64_t N, double k, const int64_t* rows,
                       int64_t nrows, const double* sigma_ri, double* out_ri) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        cplx acc = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double d[3];
            v_sub(X + 3 * i, X + 3 * j, d);
            double R = v_norm(d);
            if (j == i || R == 0.0) continue;
            acc += W[j] * green(k, R) * (sigma_ri[2 * j] + I * sigma_ri[2 * j + 1]);
        }
        out_ri[2 * r] = creal(acc);
        out_ri[2 * r + 1] = cimag(acc);
    }
}
