/*
 * Plain FP64 reference FMM for the point part of the discrete Helmholtz
 * single-layer operator:  out_i = sum_{j != i} w_j G(x_i, x_j) s_j,
 * G = exp(ikR)/(4 pi R) (Eq. 6).
 *
 * TEST INFRASTRUCTURE ONLY (see hfmm_oracle.c).  Shares no code with the
 * CUDA path.
 *
 * Steps in the paper's order (Sec. 2.3): octree on Morton-sorted points,
 * upward sweep (P2M at the leaves, M2M to the parents), traversal (M2L for
 * well-separated boxes, P2P for the rest), downward pass (L2L, then L2P).
 *
 * Expansions (Eq. 11-14, read as the local/multipole forms of the addition
 * theorem  G(x,y) = i k sum_{n,m} h_n(k r_x) Y_n^m(x^) j_n(k r_y) conj(Y_n^m(y^)),
 * r_y < r_x, orthonormal Y, truncated at degree n <= p, i.e. (p+1)^2 terms):
 *   multipole about c:  M_nm = sum_j w_j s_j  jt_n(k r_j) conj(Y_nm(y_j^))
 *                       phi(x) = (i k / s) sum M_nm ht_n(k r_x) Y_nm(x^)
 *   local about c:      phi(x) = sum L_nm jt_n(k r_x) Y_nm(x^)
 * with level scale s = min(1, k a) (a = box circumradius), jt_n = j_n / s^n and
 * ht_n = h_n s^(n+1) so coefficients stay in range at low frequency.
 *
 * A translation operator is the matrix of expansion coefficients of one
 * family of basis functions in another; each entry is defined as the
 * inner product of the function with the orthonormal Y on a sphere about the
 * new centre, divided by jt_n(k rho).  Here that inner product is evaluated
 * with a product rule (Gauss-Legendre in cos(theta), uniform in phi) exact
 * for every degree that matters.
 *
 * Octree: bounding cube centred on the point bounding box, side D = smallest
 * power of two >= the largest extent; depth L = smallest with at most
 * leaf_max points per level-L box (or a fixed depth).  Neighbours: the 27
 * boxes with index distance <= 1.  Interaction list of box b at level l >= 2:
 * the children of its parent's neighbours that are not neighbours of b.
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
#define MAXLEV 21

/* ------------------------------------------------------------------------ */
/* special functions                                                         */
/* ------------------------------------------------------------------------ */

/* out[n] = j_n(z) / s^n, n = 0..nmax, z >= 0 (power series below 2,
   Miller's backward recurrence above). */
static void sph_jn_scaled(int nmax, double z, double s, double* out) {
    if (z == 0.0) {
        out[0] = 1.0;
        for (int n = 1; n <= nmax; ++n) out[n] = 0.0;
        return;
    }
    if (z < 2.0) {
        double t = 1.0;
        for (int n = 0; n <= nmax; ++n) {
            if (n > 0) t *= (z / s) / (2.0 * n + 1.0);
            double sum = 1.0, term = 1.0;
            for (int k = 1; k < 80; ++k) {
                term *= -0.5 * z * z / (k * (2.0 * n + 2.0 * k + 1.0));
                sum += term;
                if (fabs(term) < 1e-18 * fabs(sum)) break;
            }
            out[n] = t * sum;
        }
        return;
    }
    int top = nmax + 40 + (int)z;
    double* f = (double*)malloc(sizeof(double) * (size_t)(top + 2));
    f[top + 1] = 0.0;
    f[top] = 1e-30;
    for (int n = top; n >= 1; --n) {
        f[n - 1] = (2.0 * n + 1.0) / z * f[n] - f[n + 1];
        if (fabs(f[n - 1]) > 1e250)
            for (int m = n - 1; m <= top + 1; ++m) f[m] *= 1e-250;
    }
    double j0 = sin(z) / z, j1 = sin(z) / (z * z) - cos(z) / z;
    double scale = (fabs(j0) >= fabs(j1)) ? j0 / f[0] : j1 / f[1];
    double sp = 1.0;
    for (int n = 0; n <= nmax; ++n) {
        out[n] = f[n] * scale / sp;
        sp *= s;
    }
    free(f);
}

/* out[n] = h^(1)_n(z) s^(n+1), n = 0..nmax, z > 0 */
static void sph_hn_scaled(int nmax, double z, double s, cplx* out) {
    double* jt = (double*)malloc(sizeof(double) * (size_t)(nmax + 1));
    sph_jn_scaled(nmax, z, s, jt);
    double y0 = -cos(z) / z * s;
    double y1 = (-cos(z) / (z * z) - sin(z) / z) * s * s;
    double yprev = y0, ycur = y1;
    double s2n1 = s; /* s^(2n+1) */
    for (int n = 0; n <= nmax; ++n) {
        double yn;
        if (n == 0) yn = y0;
        else if (n == 1) yn = y1;
        else {
            yn = (2.0 * (n - 1) + 1.0) * (s / z) * ycur - s * s * yprev;
            yprev = ycur;
            ycur = yn;
        }
        out[n] = jt[n] * s2n1 + I * yn;
        s2n1 *= s * s;
    }
    free(jt);
}

/* Y[n*n+n+m] = orthonormal Y_n^m of the direction of d (|m| <= n <= nmax),
   Y_n^m = Q_n^|m|(cos t) e^{i m phi}, Q with the Condon-Shortley phase. */
static void ylm_dir(int nmax, const double* d, cplx* Y) {
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double ct = 1.0, st = 0.0;
    cplx eph = 1.0;
    if (r > 0.0) {
        ct = d[2] / r;
        double rxy = sqrt(d[0] * d[0] + d[1] * d[1]);
        st = rxy / r;
        if (rxy > 0.0) eph = (d[0] + I * d[1]) / rxy;
    }
    double qmm = sqrt(1.0 / (4.0 * OR_PI));
    cplx em = 1.0;
    for (int m = 0; m <= nmax; ++m) {
        if (m > 0) {
            qmm *= -sqrt((2.0 * m + 1.0) / (2.0 * m)) * st;
            em *= eph;
        }
        double q2 = 0.0, q1 = qmm;
        for (int n = m; n <= nmax; ++n) {
            double q;
            if (n == m) q = qmm;
            else if (n == m + 1) q = sqrt(2.0 * m + 3.0) * ct * qmm;
            else {
                double a = sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
                double b = sqrt((((double)(n - 1) * (n - 1)) - (double)m * m) / (4.0 * (n - 1) * (n - 1) - 1.0));
                q = a * (ct * q1 - b * q2);
            }
            if (n > m) { q2 = q1; q1 = q; }
            Y[n * n + n + m] = q * em;
            if (m > 0) Y[n * n + n - m] = q * conj(em);
        }
    }
}

/* exported for the tests (pinned against library special functions) */
void or_sph_jn(int nmax, double z, double* out) { sph_jn_scaled(nmax, z, 1.0, out); }
void or_sph_yn(int nmax, double z, double* out) {
    cplx* h = (cplx*)malloc(sizeof(cplx) * (size_t)(nmax + 1));
    sph_hn_scaled(nmax, z, 1.0, h);
    for (int n = 0; n <= nmax; ++n) out[n] = cimag(h[n]);
    free(h);
}
void or_ylm(int nmax, double theta, double phi, double* out_ri) {
    double d[3] = {sin(theta) * cos(phi), sin(theta) * sin(phi), cos(theta)};
    int P = (nmax + 1) * (nmax + 1);
    cplx* Y = (cplx*)malloc(sizeof(cplx) * (size_t)P);
    ylm_dir(nmax, d, Y);
    for (int i = 0; i < P; ++i) {
        out_ri[2 * i] = creal(Y[i]);
        out_ri[2 * i + 1] = cimag(Y[i]);
    }
    free(Y);
}

static void gauss_legendre_pm1(int n, double* x, double* w) {
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
            pp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

/* ------------------------------------------------------------------------ */
/* translation operators by projection                                       */
/* ------------------------------------------------------------------------ */

/* radius in [0.5 a, a] keeping every j_n(k rho), n <= p, away from its zeros */
static double choose_rho(double k, double a, int p) {
    double best = a, best_score = -1.0;
    double* jn = (double*)malloc(sizeof(double) * (size_t)(p + 1));
    cplx* hn = (cplx*)malloc(sizeof(cplx) * (size_t)(p + 1));
    for (int t = 0; t <= 40; ++t) {
        double rho = a * (1.0 - 0.5 * t / 40.0);
        double z = k * rho;
        sph_jn_scaled(p, z, 1.0, jn);
        sph_hn_scaled(p, z, 1.0, hn);
        double score = 1e300;
        for (int n = 0; n <= p; ++n) score = fmin(score, fabs(jn[n]) / cabs(hn[n]));
        if (score > best_score * 1.0000001) {
            best_score = score;
            best = rho;
        }
    }
    free(jn);
    free(hn);
    return best;
}

/*
 * T (pb+1)^2 x (pf+1)^2, row-major:  f_j(x) = sum_i T[i][j] jt_{n_i}(k|x-cb|; sb) Y_i(x-cb)
 * for |x - cb| small, where the functions are
 *   type 0: f_j(x) = jt_{n_j}(k|x-cf|; sf) Y_j(x-cf)
 *   type 1: f_j(x) = (i k / sf) ht_{n_j}(k|x-cf|; sf) Y_j(x-cf)
 * and d0 = cf - cb.
 */
static void project(int type, double k, const double* d0, int pf, double sf, int pb, double sb,
                    double a_b, cplx* T) {
    int Pf = (pf + 1) * (pf + 1), Pb = (pb + 1) * (pb + 1);
    int nth = pb + pf / 2 + 24, nph = 2 * nth;
    double rho = choose_rho(k, a_b, pb);
    double* gx = (double*)malloc(sizeof(double) * (size_t)nth);
    double* gw = (double*)malloc(sizeof(double) * (size_t)nth);
    gauss_legendre_pm1(nth, gx, gw);
    memset(T, 0, sizeof(cplx) * (size_t)Pf * (size_t)Pb);
    cplx* Yb = (cplx*)malloc(sizeof(cplx) * (size_t)Pb);
    cplx* Yf = (cplx*)malloc(sizeof(cplx) * (size_t)Pf);
    cplx* f = (cplx*)malloc(sizeof(cplx) * (size_t)Pf);
    double* rj = (double*)malloc(sizeof(double) * (size_t)(pf + 1));
    cplx* rh = (cplx*)malloc(sizeof(cplx) * (size_t)(pf + 1));
    for (int it = 0; it < nth; ++it) {
        double ct = gx[it], st = sqrt(fmax(0.0, 1.0 - ct * ct));
        for (int ip = 0; ip < nph; ++ip) {
            double ph = 2.0 * OR_PI * ip / nph;
            double sh[3] = {st * cos(ph), st * sin(ph), ct};
            double wq = gw[it] * 2.0 * OR_PI / nph;
            ylm_dir(pb, sh, Yb);
            double y[3] = {rho * sh[0] - d0[0], rho * sh[1] - d0[1], rho * sh[2] - d0[2]};
            double ry = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
            ylm_dir(pf, y, Yf);
            if (type == 0) {
                sph_jn_scaled(pf, k * ry, sf, rj);
                for (int n = 0; n <= pf; ++n)
                    for (int m = -n; m <= n; ++m) f[n * n + n + m] = rj[n] * Yf[n * n + n + m];
            } else {
                sph_hn_scaled(pf, k * ry, sf, rh);
                for (int n = 0; n <= pf; ++n)
                    for (int m = -n; m <= n; ++m)
                        f[n * n + n + m] = (I * k / sf) * rh[n] * Yf[n * n + n + m];
            }
            for (int i = 0; i < Pb; ++i) {
                cplx c = wq * conj(Yb[i]);
                cplx* row = T + (size_t)i * Pf;
                for (int j = 0; j < Pf; ++j) row[j] += c * f[j];
            }
        }
    }
    double* jb = (double*)malloc(sizeof(double) * (size_t)(pb + 1));
    sph_jn_scaled(pb, k * rho, sb, jb);
    for (int n = 0; n <= pb; ++n)
        for (int m = -n; m <= n; ++m) {
            cplx* row = T + (size_t)(n * n + n + m) * Pf;
            for (int j = 0; j < Pf; ++j) row[j] /= jb[n];
        }
    free(jb);
    free(gx);
    free(gw);
    free(Yb);
    free(Yf);
    free(f);
    free(rj);
    free(rh);
}

/* ------------------------------------------------------------------------ */
/* octree                                                                    */
/* ------------------------------------------------------------------------ */
static uint64_t morton3(uint64_t ix, uint64_t iy, uint64_t iz) {
    uint64_t k = 0;
    for (int b = 0; b < 21; ++b) {
        k |= ((ix >> b) & 1ull) << (3 * b + 2);
        k |= ((iy >> b) & 1ull) << (3 * b + 1);
        k |= ((iz >> b) & 1ull) << (3 * b);
    }
    return k;
}
static void demorton3(uint64_t k, int64_t* i3) {
    i3[0] = i3[1] = i3[2] = 0;
    for (int b = 0; b < 21; ++b) {
        i3[0] |= (int64_t)((k >> (3 * b + 2)) & 1ull) << b;
        i3[1] |= (int64_t)((k >> (3 * b + 1)) & 1ull) << b;
        i3[2] |= (int64_t)((k >> (3 * b)) & 1ull) << b;
    }
}

typedef struct {
    uint64_t key;
    int64_t idx;
} kv_t;
static int cmp_kv(const void* a, const void* b) {
    const kv_t* x = (const kv_t*)a;
    const kv_t* y = (const kv_t*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

typedef struct {
    int L;
    double D, lo[3];
    int64_t N;
    int64_t* perm; /* sorted -> original */
    int64_t nbox[MAXLEV + 1];
    uint64_t* key[MAXLEV + 1];
    int64_t* pstart[MAXLEV + 1]; /* nbox+1 */
    int p[MAXLEV + 1];
    double s[MAXLEV + 1], side[MAXLEV + 1];
} otree;

static void leaf_coords(const otree* t, const double* x, int L, uint64_t* i3) {
    double scale = ldexp(1.0, L) / t->D;
    int64_t n = (int64_t)1 << L;
    for (int d = 0; d < 3; ++d) {
        int64_t c = (int64_t)floor((x[d] - t->lo[d]) * scale);
        if (c < 0) c = 0;
        if (c > n - 1) c = n - 1;
        i3[d] = (uint64_t)c;
    }
}

static int64_t find_box(const otree* t, int l, uint64_t key) {
    int64_t lo = 0, hi = t->nbox[l] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (t->key[l][mid] == key) return mid;
        if (t->key[l][mid] < key) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

static void tree_build(otree* t, const double* X, int64_t N, int depth, int leaf_max) {
    memset(t, 0, sizeof(*t));
    t->N = N;
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d) {
            mn[d] = fmin(mn[d], X[3 * i + d]);
            mx[d] = fmax(mx[d], X[3 * i + d]);
        }
    double ext = fmax(mx[0] - mn[0], fmax(mx[1] - mn[1], mx[2] - mn[2]));
    double D = 1.0;
    if (ext > 0.0) {
        while (D < ext) D *= 2.0;
        while (D * 0.5 >= ext) D *= 0.5;
    }
    t->D = D;
    for (int d = 0; d < 3; ++d) t->lo[d] = 0.5 * (mn[d] + mx[d]) - 0.5 * D;
    kv_t* kv = (kv_t*)malloc(sizeof(kv_t) * (size_t)(N > 0 ? N : 1));
    int L = depth > 0 ? depth : 0;
    for (;;) {
        for (int64_t i = 0; i < N; ++i) {
            uint64_t c[3];
            leaf_coords(t, X + 3 * i, L, c);
            kv[i].key = morton3(c[0], c[1], c[2]);
            kv[i].idx = i;
        }
        qsort(kv, (size_t)N, sizeof(kv_t), cmp_kv);
        if (depth > 0 || L >= 20) break;
        int64_t run = 0, best = 0;
        for (int64_t i = 0; i < N; ++i) {
            run = (i > 0 && kv[i].key == kv[i - 1].key) ? run + 1 : 1;
            if (run > best) best = run;
        }
        if (best <= leaf_max) break;
        ++L;
    }
    t->L = L;
    t->perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    uint64_t* lk = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) {
        t->perm[i] = kv[i].idx;
        lk[i] = kv[i].key;
    }
    for (int l = 0; l <= L; ++l) {
        int sh = 3 * (L - l);
        int64_t nb = 0;
        for (int64_t i = 0; i < N; ++i)
            if (i == 0 || (lk[i] >> sh) != (lk[i - 1] >> sh)) ++nb;
        t->nbox[l] = nb;
        t->key[l] = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nb > 0 ? nb : 1));
        t->pstart[l] = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nb + 1));
        int64_t b = 0;
        for (int64_t i = 0; i < N; ++i)
            if (i == 0 || (lk[i] >> sh) != (lk[i - 1] >> sh)) {
                t->key[l][b] = lk[i] >> sh;
                t->pstart[l][b] = i;
                ++b;
            }
        t->pstart[l][nb] = N;
        t->side[l] = D / ldexp(1.0, l);
    }
    free(lk);
    free(kv);
}

static void tree_free(otree* t) {
    free(t->perm);
    for (int l = 0; l <= t->L; ++l) {
        free(t->key[l]);
        free(t->pstart[l]);
    }
}

static void box_center(const otree* t, int l, uint64_t key, double* c) {
    int64_t i3[3];
    demorton3(key, i3);
    for (int d = 0; d < 3; ++d) c[d] = t->lo[d] + ((double)i3[d] + 0.5) * t->side[l];
}

/* expansion order of a level: fixed, or the per-level formula with a floor */
static int level_order(double k, double side, int p_fixed, int p_min) {
    if (p_fixed > 0) return p_fixed;
    double ka = k * 0.5 * sqrt(3.0) * side;
    int p = (int)ceil(ka + 6.0 * log10(ka + OR_PI));
    return p > p_min ? p : p_min;
}

/* ------------------------------------------------------------------------ */
/* FMM                                                                       */
/* ------------------------------------------------------------------------ */
/*
 * out_i (original order) = sum_{j != i} W_j G(x_i, x_j) s_j, approximated by
 * the FMM.  parts bit 0: near field (P2P), bit 1: far field (expansions).
 * info[0] = depth L, info[1..L] = order per level (0 for levels 0,1).
 */
int or_fmm(const double* X, const double* W, int64_t N, double k, int depth, int leaf_max,
           int p_fixed, int p_min, const double* sigma_ri, double* out_ri, int parts, int* info) {
    otree t;
    tree_build(&t, X, N, depth, leaf_max);
    int L = t.L;
    info[0] = L;
    for (int l = 0; l <= L; ++l) {
        t.p[l] = (l >= 2) ? level_order(k, t.side[l], p_fixed, p_min) : 0;
        t.s[l] = fmin(1.0, k * 0.5 * sqrt(3.0) * t.side[l]);
        if (l >= 1) info[l] = t.p[l];
    }
    cplx* q = (cplx*)malloc(sizeof(cplx) * (size_t)(N > 0 ? N : 1));
    cplx* res = (cplx*)calloc((size_t)(N > 0 ? N : 1), sizeof(cplx));
    double* xs = (double*)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) {
        int64_t o = t.perm[i];
        q[i] = W[o] * (sigma_ri[2 * o] + I * sigma_ri[2 * o + 1]);
        memcpy(xs + 3 * i, X + 3 * o, sizeof(double) * 3);
    }

    if ((parts & 2) && L >= 2) {
        cplx* M[MAXLEV + 1];
        cplx* Lc[MAXLEV + 1];
        for (int l = 2; l <= L; ++l) {
            int P = (t.p[l] + 1) * (t.p[l] + 1);
            M[l] = (cplx*)calloc((size_t)t.nbox[l] * P, sizeof(cplx));
            Lc[l] = (cplx*)calloc((size_t)t.nbox[l] * P, sizeof(cplx));
        }
        /* P2M at the leaves */
        {
            int p = t.p[L], P = (p + 1) * (p + 1);
#pragma omp parallel
            {
                double* jn = (double*)malloc(sizeof(double) * (size_t)(p + 1));
                cplx* Y = (cplx*)malloc(sizeof(cplx) * (size_t)P);
#pragma omp for schedule(dynamic, 16)
                for (int64_t b = 0; b < t.nbox[L]; ++b) {
                    double c[3];
                    box_center(&t, L, t.key[L][b], c);
                    cplx* Mb = M[L] + (size_t)b * P;
                    for (int64_t i = t.pstart[L][b]; i < t.pstart[L][b + 1]; ++i) {
                        double d[3] = {xs[3 * i] - c[0], xs[3 * i + 1] - c[1], xs[3 * i + 2] - c[2]};
                        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                        sph_jn_scaled(p, k * r, t.s[L], jn);
                        ylm_dir(p, d, Y);
                        for (int n = 0; n <= p; ++n)
                            for (int m = -n; m <= n; ++m)
                                Mb[n * n + n + m] += q[i] * jn[n] * conj(Y[n * n + n + m]);
                    }
                }
                free(jn);
                free(Y);
            }
        }
        /* translation matrices per level: 8 parent/child, 343 M2L offsets */
        cplx* TPC[MAXLEV + 1][8];   /* child basis (rows) <- parent regular functions */
        cplx* TM2L[MAXLEV + 1][343];
        memset(TPC, 0, sizeof(TPC));
        memset(TM2L, 0, sizeof(TM2L));
        for (int l = 3; l <= L; ++l) {
            int pc = t.p[l], pp = t.p[l - 1];
            int Pc = (pc + 1) * (pc + 1), Pp = (pp + 1) * (pp + 1);
#pragma omp parallel for schedule(dynamic, 1)
            for (int o = 0; o < 8; ++o) {
                double d0[3];
                for (int d = 0; d < 3; ++d) {
                    int bit = (o >> (2 - d)) & 1;
                    d0[d] = -0.25 * t.side[l - 1] * (2.0 * bit - 1.0); /* c_parent - c_child */
                }
                TPC[l][o] = (cplx*)malloc(sizeof(cplx) * (size_t)Pc * Pp);
                project(0, k, d0, pp, t.s[l - 1], pc, t.s[l], 0.5 * sqrt(3.0) * t.side[l], TPC[l][o]);
            }
        }
        for (int l = 2; l <= L; ++l) {
            int p = t.p[l], P = (p + 1) * (p + 1);
#pragma omp parallel for schedule(dynamic, 1)
            for (int o = 0; o < 343; ++o) {
                int dx = o / 49 - 3, dy = (o / 7) % 7 - 3, dz = o % 7 - 3;
                if (abs(dx) <= 1 && abs(dy) <= 1 && abs(dz) <= 1) continue;
                double d0[3] = {dx * t.side[l], dy * t.side[l], dz * t.side[l]}; /* c_s - c_t */
                TM2L[l][o] = (cplx*)malloc(sizeof(cplx) * (size_t)P * P);
                project(1, k, d0, p, t.s[l], p, t.s[l], 0.5 * sqrt(3.0) * t.side[l], TM2L[l][o]);
            }
        }
        /* M2M: children -> parent, A = (TPC)^H */
        for (int l = L - 1; l >= 2; --l) {
            int pc = t.p[l + 1], pp = t.p[l];
            int Pc = (pc + 1) * (pc + 1), Pp = (pp + 1) * (pp + 1);
#pragma omp parallel for schedule(dynamic, 16)
            for (int64_t b = 0; b < t.nbox[l]; ++b) {
                cplx* Mp = M[l] + (size_t)b * Pp;
                for (int o = 0; o < 8; ++o) {
                    int64_t cb = find_box(&t, l + 1, (t.key[l][b] << 3) | (uint64_t)o);
                    if (cb < 0) continue;
                    int64_t i3[3];
                    demorton3((uint64_t)o, i3);
                    int oc = (int)(i3[0] * 4 + i3[1] * 2 + i3[2]);
                    const cplx* A = TPC[l + 1][oc];
                    const cplx* Mc = M[l + 1] + (size_t)cb * Pc;
                    for (int jp = 0; jp < Pp; ++jp) {
                        cplx acc = 0.0;
                        for (int ic = 0; ic < Pc; ++ic) acc += conj(A[(size_t)ic * Pp + jp]) * Mc[ic];
                        Mp[jp] += acc;
                    }
                }
            }
        }
        /* M2L */
        for (int l = 2; l <= L; ++l) {
            int p = t.p[l], P = (p + 1) * (p + 1);
#pragma omp parallel for schedule(dynamic, 8)
            for (int64_t b = 0; b < t.nbox[l]; ++b) {
                int64_t it[3];
                demorton3(t.key[l][b], it);
                int64_t ip[3] = {it[0] >> 1, it[1] >> 1, it[2] >> 1};
                int64_t nl = (int64_t)1 << (l - 1);
                cplx* Lb = Lc[l] + (size_t)b * P;
                for (int64_t ex = -1; ex <= 1; ++ex)
                    for (int64_t ey = -1; ey <= 1; ++ey)
                        for (int64_t ez = -1; ez <= 1; ++ez) {
                            int64_t qx = ip[0] + ex, qy = ip[1] + ey, qz = ip[2] + ez;
                            if (qx < 0 || qy < 0 || qz < 0 || qx >= nl || qy >= nl || qz >= nl) continue;
                            if (find_box(&t, l - 1, morton3(qx, qy, qz)) < 0) continue;
                            for (int o = 0; o < 8; ++o) {
                                int64_t sx = 2 * qx + ((o >> 2) & 1), sy = 2 * qy + ((o >> 1) & 1),
                                        sz = 2 * qz + (o & 1);
                                int64_t dx = sx - it[0], dy = sy - it[1], dz = sz - it[2];
                                if (llabs(dx) <= 1 && llabs(dy) <= 1 && llabs(dz) <= 1) continue;
                                int64_t sb = find_box(&t, l, morton3(sx, sy, sz));
                                if (sb < 0) continue;
                                const cplx* T = TM2L[l][(dx + 3) * 49 + (dy + 3) * 7 + (dz + 3)];
                                const cplx* Ms = M[l] + (size_t)sb * P;
                                for (int i = 0; i < P; ++i) {
                                    cplx acc = 0.0;
                                    const cplx* row = T + (size_t)i * P;
                                    for (int j = 0; j < P; ++j) acc += row[j] * Ms[j];
                                    Lb[i] += acc;
                                }
                            }
                        }
            }
        }
        /* L2L: parent -> children */
        for (int l = 3; l <= L; ++l) {
            int pc = t.p[l], pp = t.p[l - 1];
            int Pc = (pc + 1) * (pc + 1), Pp = (pp + 1) * (pp + 1);
#pragma omp parallel for schedule(dynamic, 16)
            for (int64_t b = 0; b < t.nbox[l]; ++b) {
                int64_t pb = find_box(&t, l - 1, t.key[l][b] >> 3);
                int64_t i3[3];
                demorton3(t.key[l][b] & 7ull, i3);
                int oc = (int)(i3[0] * 4 + i3[1] * 2 + i3[2]);
                const cplx* C = TPC[l][oc];
                const cplx* Lp = Lc[l - 1] + (size_t)pb * Pp;
                cplx* Lb = Lc[l] + (size_t)b * Pc;
                for (int i = 0; i < Pc; ++i) {
                    cplx acc = 0.0;
                    for (int j = 0; j < Pp; ++j) acc += C[(size_t)i * Pp + j] * Lp[j];
                    Lb[i] += acc;
                }
            }
        }
        /* L2P */
        {
            int p = t.p[L], P = (p + 1) * (p + 1);
#pragma omp parallel
            {
                double* jn = (double*)malloc(sizeof(double) * (size_t)(p + 1));
                cplx* Y = (cplx*)malloc(sizeof(cplx) * (size_t)P);
#pragma omp for schedule(dynamic, 16)
                for (int64_t b = 0; b < t.nbox[L]; ++b) {
                    double c[3];
                    box_center(&t, L, t.key[L][b], c);
                    const cplx* Lb = Lc[L] + (size_t)b * P;
                    for (int64_t i = t.pstart[L][b]; i < t.pstart[L][b + 1]; ++i) {
                        double d[3] = {xs[3 * i] - c[0], xs[3 * i + 1] - c[1], xs[3 * i + 2] - c[2]};
                        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                        sph_jn_scaled(p, k * r, t.s[L], jn);
                        ylm_dir(p, d, Y);
                        cplx acc = 0.0;
                        for (int n = 0; n <= p; ++n)
                            for (int m = -n; m <= n; ++m) acc += Lb[n * n + n + m] * jn[n] * Y[n * n + n + m];
                        res[i] += acc;
                    }
                }
                free(jn);
                free(Y);
            }
        }
        for (int l = 2; l <= L; ++l) {
            free(M[l]);
            free(Lc[l]);
            for (int o = 0; o < 343; ++o) free(TM2L[l][o]);
            for (int o = 0; o < 8; ++o) free(TPC[l][o]);
        }
    }

    if (parts & 1) {
        /* P2P over the 27 neighbour leaves (self included, j != i) */
        int64_t nl = (int64_t)1 << L;
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t b = 0; b < t.nbox[L]; ++b) {
            int64_t it[3];
            demorton3(t.key[L][b], it);
            for (int64_t ex = -1; ex <= 1; ++ex)
                for (int64_t ey = -1; ey <= 1; ++ey)
                    for (int64_t ez = -1; ez <= 1; ++ez) {
                        int64_t sx = it[0] + ex, sy = it[1] + ey, sz = it[2] + ez;
                        if (sx < 0 || sy < 0 || sz < 0 || sx >= nl || sy >= nl || sz >= nl) continue;
                        int64_t sb = find_box(&t, L, morton3(sx, sy, sz));
                        if (sb < 0) continue;
                        for (int64_t i = t.pstart[L][b]; i < t.pstart[L][b + 1]; ++i) {
                            cplx acc = 0.0;
                            for (int64_t j = t.pstart[L][sb]; j < t.pstart[L][sb + 1]; ++j) {
                                if (j == i) continue;
                                double d[3] = {xs[3 * i] - xs[3 * j], xs[3 * i + 1] - xs[3 * j + 1],
                                               xs[3 * i + 2] - xs[3 * j + 2]};
                                double R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                                if (R == 0.0) continue;
                                acc += cexp(I * k * R) / (4.0 * OR_PI * R) * q[j];
                            }
                            res[i] += acc;
                        }
                    }
        }
    }
    for (int64_t i = 0; i < N; ++i) {
        int64_t o = t.perm[i];
        out_ri[2 * o] = creal(res[i]);
        out_ri[2 * o + 1] = cimag(res[i]);
    }
    free(q);
    free(res);
    free(xs);
    tree_free(&t);
    return 0;
}
