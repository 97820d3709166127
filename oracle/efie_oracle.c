/*
 * FP64 CPU oracle for the Galerkin EFIE impedance matrix with RWG basis
 * functions.  TEST INFRASTRUCTURE ONLY: the tests, the benchmark's CPU
 * baseline leg and the package's smoke check call it; the GPU library never
 * does, and this file shares no code with it.
 *
 * What it computes (Section II, Eqs. (1)-(5)):
 *
 *   Z_ij = i k eta < f_i, G, f_j >,   G = [I - grad grad' / k^2] g,
 *   g(R) = exp(i k R) / R              (Eq. (3): no 1/(4 pi), exp(-i w t)).
 *
 * After the usual integration by parts (RWG functions have continuous
 * normal components across their common edge, so boundary terms cancel):
 *
 *   Z_ij = i k eta sum_{T in f_i} sum_{T' in f_j} int_T int_T'
 *          [ f_i(r) . f_j(r') - (div f_i)(div' f_j) / k^2 ] g(R) dS' dS.
 *
 * RWG function on its two triangles (the paper names the basis without
 * printing it; this is the standard form):
 *   T+ : f(r) = +l/(2A+) (r - v+),  div f = +l/A+
 *   T- : f(r) = -l/(2A-) (r - v-),  div f = -l/A-
 * with l the common edge's length and v+- the free vertices.
 *
 * Quadrature: the seven-point degree-5 rule on each triangle for the outer
 * integral and, for well separated triangle pairs, for the inner one.
 *
 * Singularity extraction (the paper is silent; reading used here): for
 * triangle pairs that coincide, share a vertex, or whose centroids are closer
 * than twice the larger of their longest edges, g = 1/R + (exp(ikR)-1)/R.
 * The 1/R and r'/R inner integrals are done in closed form over the source
 * triangle (the potential integrals of a uniform and a linear density on a
 * flat triangle), the bounded remainder with the seven-point rule.  The
 * outer integral always uses seven points.  Because analytic-inner /
 * numeric-outer is not symmetric, the matrix is symmetrised,
 * Z = (Zraw + Zraw^T) / 2, where Zraw_ij takes f_i outer and f_j inner.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

/* ---------------------------------------------------------------- rule --- */
/* barycentric (l1, l2, l3) and weight (relative to area, sum 1) */
static double Q7[7][4];
static int q7_ready = 0;

static void q7_init(void)
{
    if (q7_ready) return;
    const double s15 = sqrt(15.0);
    const double a = (6.0 - s15) / 21.0, b = (6.0 + s15) / 21.0;
    const double wa = (155.0 - s15) / 1200.0, wb = (155.0 + s15) / 1200.0;
    const double pts[7][4] = {
        {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, 9.0 / 40.0},
        {a, a, 1.0 - 2.0 * a, wa}, {a, 1.0 - 2.0 * a, a, wa}, {1.0 - 2.0 * a, a, a, wa},
        {b, b, 1.0 - 2.0 * b, wb}, {b, 1.0 - 2.0 * b, b, wb}, {1.0 - 2.0 * b, b, b, wb},
    };
    memcpy(Q7, pts, sizeof(pts));
    q7_ready = 1;
}

int oracle_rule7(double *out /* [7][4] */)
{
    q7_init();
    memcpy(out, Q7, sizeof(Q7));
    return 0;
}

/* ---------------------------------------------------------- vectors --- */
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static void sub3(const double *a, const double *b, double *c) { c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2]; }
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* ------------------------------------------------------------- mesh --- */
typedef struct {
    int nt;
    const double *V;     /* [nv][3] */
    const int32_t *T;    /* [nt][3] */
    double *qp;          /* [nt][7][3] quadrature points */
    double *area;        /* [nt] */
    double *cen;         /* [nt][3] */
    double *hmax;        /* [nt] longest edge */
} mesh_t;

static int mesh_init(mesh_t *M, int nt, const double *V, const int32_t *T)
{
    q7_init();
    M->nt = nt; M->V = V; M->T = T;
    M->qp = (double *)malloc(sizeof(double) * 21 * (size_t)nt);
    M->area = (double *)malloc(sizeof(double) * (size_t)nt);
    M->cen = (double *)malloc(sizeof(double) * 3 * (size_t)nt);
    M->hmax = (double *)malloc(sizeof(double) * (size_t)nt);
    if (!M->qp || !M->area || !M->cen || !M->hmax) return -1;
    for (int t = 0; t < nt; ++t) {
        const double *p1 = V + 3 * T[3 * t], *p2 = V + 3 * T[3 * t + 1], *p3 = V + 3 * T[3 * t + 2];
        double e1[3], e2[3], e3[3], n[3];
        sub3(p2, p1, e1); sub3(p3, p1, e2); sub3(p3, p2, e3);
        cross3(e1, e2, n);
        M->area[t] = 0.5 * norm3(n);
        double h = norm3(e1), h2 = norm3(e2), h3 = norm3(e3);
        if (h2 > h) h = h2;
        if (h3 > h) h = h3;
        M->hmax[t] = h;
        for (int d = 0; d < 3; ++d) M->cen[3 * t + d] = (p1[d] + p2[d] + p3[d]) / 3.0;
        for (int q = 0; q < 7; ++q)
            for (int d = 0; d < 3; ++d)
                M->qp[21 * t + 3 * q + d] = Q7[q][0] * p1[d] + Q7[q][1] * p2[d] + Q7[q][2] * p3[d];
    }
    return 0;
}

static void mesh_free(mesh_t *M)
{
    free(M->qp); free(M->area); free(M->cen); free(M->hmax);
}

/* Triangle pairs whose inner integral gets singularity extraction. */
static int pair_is_singular(const mesh_t *M, int t, int s)
{
    if (t == s) return 1;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (M->T[3 * t + a] == M->T[3 * s + b]) return 1;
    double d[3];
    sub3(M->cen + 3 * t, M->cen + 3 * s, d);
    double h = M->hmax[t] > M->hmax[s] ? M->hmax[t] : M->hmax[s];
    return norm3(d) < 2.0 * h;
}

/* ------------------------------------------------ closed-form 1/R terms --- */
/* log((R+ + l+)/(R- + l-)) written so that no difference of close numbers
 * is formed; (R+l)(R-l) = R0^2 along a straight edge. */
static double edge_log(double lp, double lm, double Rp, double Rm, double R0sq)
{
    if (lm >= 0.0) return log((Rp + lp) / (Rm + lm));
    if (lp <= 0.0) return log((Rm - lm) / (Rp - lp));
    return log((Rp + lp) * (Rm - lm) / R0sq);
}

/*
 * For an observation point r and a flat triangle (p1, p2, p3):
 *   I0    = int_T dS' / |r - r'|
 *   I1    = int_T (rho' - rho) dS' / |r - r'|      (in-plane vector)
 *   rho   = projection of r onto the triangle's plane.
 * Sum over the three edges of the edge-line integrals that the surface
 * integrals reduce to by the divergence theorem in the plane.
 */
static void static_potential(const double *r, const double *p1, const double *p2, const double *p3,
                             double *I0, double *I1, double *rho)
{
    double e1[3], e2[3], n[3];
    sub3(p2, p1, e1); sub3(p3, p1, e2);
    cross3(e1, e2, n);
    double nn = norm3(n);
    for (int d = 0; d < 3; ++d) n[d] /= nn;
    double rp1[3];
    sub3(r, p1, rp1);
    const double h = dot3(n, rp1);
    const double ah = fabs(h);
    for (int d = 0; d < 3; ++d) rho[d] = r[d] - h * n[d];
    const double *va[3] = {p1, p2, p3};
    const double *vb[3] = {p2, p3, p1};
    *I0 = 0.0;
    I1[0] = I1[1] = I1[2] = 0.0;
    for (int e = 0; e < 3; ++e) {
        double lv[3], lhat[3], uhat[3], am[3], bm[3];
        sub3(vb[e], va[e], lv);
        const double len = norm3(lv);
        for (int d = 0; d < 3; ++d) lhat[d] = lv[d] / len;
        cross3(lhat, n, uhat);                 /* outward in-plane edge normal */
        sub3(va[e], rho, am);
        sub3(vb[e], rho, bm);
        const double lp = dot3(bm, lhat), lm = dot3(am, lhat);
        const double t = dot3(am, uhat);       /* signed distance to the edge line */
        const double R0sq = t * t + h * h;
        const double Rp = sqrt(R0sq + lp * lp), Rm = sqrt(R0sq + lm * lm);
        double f = 0.0, beta = 0.0;
        if (R0sq > 1e-28 * len * len) {
            f = edge_log(lp, lm, Rp, Rm, R0sq);
            beta = atan2(t * lp, R0sq + ah * Rp) - atan2(t * lm, R0sq + ah * Rm);
        }
        *I0 += t * f - ah * beta;
        const double s = 0.5 * (R0sq * f + lp * Rp - lm * Rm);
        for (int d = 0; d < 3; ++d) I1[d] += s * uhat[d];
    }
}

int oracle_static_potential(const double *r, const double *tri9, double *I0, double *I1, double *rho)
{
    static_potential(r, tri9, tri9 + 3, tri9 + 6, I0, I1, rho);
    return 0;
}

/* ------------------------------------------------------ Green function --- */
/* (exp(ikR) - 1) / R, bounded at R = 0 (limit ik) */
static cplx g_smooth(double k, double R)
{
    const double x = k * R;
    if (x < 1e-8) return I * k - 0.5 * k * k * R;
    const double s = sin(0.5 * x);
    return (-2.0 * s * s + I * sin(x)) / R;
}

static cplx g_full(double k, double R) { return cexp(I * k * R) / R; }

/*
 * Inner potentials of source triangle s at point r:
 *   P0 = int_s g(|r - r'|) dS',   P1 = int_s r' g(|r - r'|) dS'  (vector)
 * with singularity extraction when `singular` is set.
 */
static void tri_potential(const mesh_t *M, const double *r, int s, double k, int singular,
                          cplx *P0, cplx *P1)
{
    const double A = M->area[s];
    cplx p0 = 0.0, p1[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < 7; ++q) {
        const double *rq = M->qp + 21 * s + 3 * q;
        double d[3];
        sub3(r, rq, d);
        const double R = norm3(d);
        const cplx g = singular ? g_smooth(k, R) : g_full(k, R);
        const cplx wg = A * Q7[q][3] * g;
        p0 += wg;
        for (int c = 0; c < 3; ++c) p1[c] += wg * rq[c];
    }
    if (singular) {
        const double *v = M->V;
        const int32_t *t = M->T + 3 * s;
        double I0, I1[3], rho[3];
        static_potential(r, v + 3 * t[0], v + 3 * t[1], v + 3 * t[2], &I0, I1, rho);
        p0 += I0;
        for (int c = 0; c < 3; ++c) p1[c] += I1[c] + rho[c] * I0;
    }
    *P0 = p0;
    for (int c = 0; c < 3; ++c) P1[c] = p1[c];
}

int oracle_tri_potential(int nv, const double *V, int nt, const int32_t *T, const double *r, int s,
                         double k, int singular, double *out /* P0 re,im; P1 x,y,z re,im */)
{
    (void)nv;
    mesh_t M;
    if (mesh_init(&M, nt, V, T)) return -1;
    cplx P0, P1[3];
    tri_potential(&M, r, s, k, singular, &P0, P1);
    out[0] = creal(P0); out[1] = cimag(P0);
    for (int c = 0; c < 3; ++c) { out[2 + 2 * c] = creal(P1[c]); out[3 + 2 * c] = cimag(P1[c]); }
    mesh_free(&M);
    return 0;
}

int oracle_pair_is_singular(int nv, const double *V, int nt, const int32_t *T, int t, int s)
{
    (void)nv;
    mesh_t M;
    if (mesh_init(&M, nt, V, T)) return -1;
    int r = pair_is_singular(&M, t, s);
    mesh_free(&M);
    return r;
}

/* ---------------------------------------------------------------- RWG --- */
typedef struct {
    int n;
    const int32_t *tri;   /* [n][2]  T+, T- */
    const int32_t *vfree; /* [n][2]  v+, v- */
    const double *len;    /* [n] */
} rwg_t;

/* ordered entry: f_i outer (test), f_j inner (source) */
static cplx z_raw(const mesh_t *M, const rwg_t *B, int i, int j, double k)
{
    cplx acc = 0.0;
    const double li = B->len[i], lj = B->len[j];
    for (int a = 0; a < 2; ++a) {
        const int t = B->tri[2 * i + a];
        const double si = a == 0 ? 1.0 : -1.0;
        const double *vi = M->V + 3 * B->vfree[2 * i + a];
        const double At = M->area[t];
        const double Di = si * li / At;
        for (int b = 0; b < 2; ++b) {
            const int s = B->tri[2 * j + b];
            const double sj = b == 0 ? 1.0 : -1.0;
            const double *vj = M->V + 3 * B->vfree[2 * j + b];
            const double As = M->area[s];
            const double Dj = sj * lj / As;
            const int sing = pair_is_singular(M, t, s);
            for (int q = 0; q < 7; ++q) {
                const double *r = M->qp + 21 * t + 3 * q;
                cplx P0, P1[3];
                tri_potential(M, r, s, k, sing, &P0, P1);
                /* f_i(r) . int f_j g  -  Di Dj / k^2 int g */
                cplx vec = 0.0;
                for (int c = 0; c < 3; ++c) {
                    const double fi = si * li / (2.0 * At) * (r[c] - vi[c]);
                    const cplx Fj = sj * lj / (2.0 * As) * (P1[c] - vj[c] * P0);
                    vec += fi * Fj;
                }
                acc += At * Q7[q][3] * (vec - Di * Dj * P0 / (k * k));
            }
        }
    }
    return acc;
}

static void rwg_from_args(rwg_t *B, int n, const int32_t *tri, const int32_t *vfree, const double *len)
{
    B->n = n; B->tri = tri; B->vfree = vfree; B->len = len;
}

/*
 * Ordered entry of dZ/dk.  With A = <f_i, g, f_j>, Phi = <div f_i, g, div f_j>
 * (both as in Z, with the same singularity extraction) and the k-derivatives
 * of the kernel, dg/dk = i exp(ikR) (bounded, plain seven-point rule):
 *   Z = i k eta A - (i eta / k) Phi
 *   dZ/dk = i eta A + i k eta A' + (i eta / k^2) Phi - (i eta / k) Phi'.
 */
static cplx dz_raw(const mesh_t *M, const rwg_t *B, int i, int j, double k, double eta)
{
    cplx A = 0.0, Phi = 0.0, Ad = 0.0, Phid = 0.0;
    const double li = B->len[i], lj = B->len[j];
    for (int a = 0; a < 2; ++a) {
        const int t = B->tri[2 * i + a];
        const double si = a == 0 ? 1.0 : -1.0;
        const double *vi = M->V + 3 * B->vfree[2 * i + a];
        const double At = M->area[t];
        const double Di = si * li / At;
        for (int b = 0; b < 2; ++b) {
            const int s = B->tri[2 * j + b];
            const double sj = b == 0 ? 1.0 : -1.0;
            const double *vj = M->V + 3 * B->vfree[2 * j + b];
            const double As = M->area[s];
            const double Dj = sj * lj / As;
            const int sing = pair_is_singular(M, t, s);
            for (int q = 0; q < 7; ++q) {
                const double *r = M->qp + 21 * t + 3 * q;
                const double wo = At * Q7[q][3];
                cplx P0, P1[3];
                tri_potential(M, r, s, k, sing, &P0, P1);
                cplx vec = 0.0;
                for (int c = 0; c < 3; ++c) {
                    const double fi = si * li / (2.0 * At) * (r[c] - vi[c]);
                    vec += fi * (sj * lj / (2.0 * As) * (P1[c] - vj[c] * P0));
                }
                A += wo * vec;
                Phi += wo * Di * Dj * P0;
                /* derivative kernel i exp(ikR): smooth, plain rule */
                for (int p = 0; p < 7; ++p) {
                    const double *rp = M->qp + 21 * s + 3 * p;
                    double d[3];
                    sub3(r, rp, d);
                    const cplx gd = I * cexp(I * k * norm3(d));
                    const double wi = As * Q7[p][3];
                    double ff = 0.0;
                    for (int c = 0; c < 3; ++c)
                        ff += (si * li / (2.0 * At) * (r[c] - vi[c])) * (sj * lj / (2.0 * As) * (rp[c] - vj[c]));
                    Ad += wo * wi * ff * gd;
                    Phid += wo * wi * Di * Dj * gd;
                }
            }
        }
    }
    return I * eta * A + I * k * eta * Ad + I * eta / (k * k) * Phi - I * eta / k * Phid;
}

/* Dense symmetric dZ/dk [n][n] complex (interleaved), row-major. */
int oracle_dzfill(int nv, const double *V, int nt, const int32_t *T,
                  int n, const int32_t *tri, const int32_t *vfree, const double *len,
                  double k, double eta, double *Z, int nthreads)
{
    (void)nv;
    mesh_t M;
    if (mesh_init(&M, nt, V, T)) return -1;
    rwg_t B;
    rwg_from_args(&B, n, tri, vfree, len);
    cplx *Zc = (cplx *)Z;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            Zc[(size_t)i * n + j] = dz_raw(&M, &B, i, j, k, eta);
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            const cplx s = 0.5 * (Zc[(size_t)i * n + j] + Zc[(size_t)j * n + i]);
            Zc[(size_t)i * n + j] = s;
            Zc[(size_t)j * n + i] = s;
        }
    mesh_free(&M);
    return 0;
}

/*
 * Dense symmetric Z [n][n] complex (interleaved re, im), row-major.
 */
int oracle_zfill(int nv, const double *V, int nt, const int32_t *T,
                 int n, const int32_t *tri, const int32_t *vfree, const double *len,
                 double k, double eta, double *Z, int nthreads)
{
    (void)nv;
    mesh_t M;
    if (mesh_init(&M, nt, V, T)) return -1;
    rwg_t B;
    rwg_from_args(&B, n, tri, vfree, len);
    cplx *Zc = (cplx *)Z;
    const cplx pref = I * k * eta;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            Zc[(size_t)i * n + j] = pref * z_raw(&M, &B, i, j, k);
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            const cplx s = 0.5 * (Zc[(size_t)i * n + j] + Zc[(size_t)j * n + i]);
            Zc[(size_t)i * n + j] = s;
            Zc[(size_t)j * n + i] = s;
        }
    mesh_free(&M);
    return 0;
}

/*
 * Selected rows of the symmetric Z: out[r][j] = (Zraw_ij + Zraw_ji) / 2 for
 * i = rows[r]; [nrows][n] complex interleaved.
 */
int oracle_zrows(int nv, const double *V, int nt, const int32_t *T,
                 int n, const int32_t *tri, const int32_t *vfree, const double *len,
                 double k, double eta, int nrows, const int64_t *rows, double *out, int nthreads)
{
    (void)nv;
    mesh_t M;
    if (mesh_init(&M, nt, V, T)) return -1;
    rwg_t B;
    rwg_from_args(&B, n, tri, vfree, len);
    cplx *O = (cplx *)out;
    const cplx pref = I * k * eta;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) collapse(2)
#endif
    for (int r = 0; r < nrows; ++r)
        for (int j = 0; j < n; ++j) {
            const int i = (int)rows[r];
            O[(size_t)r * n + j] = pref * 0.5 * (z_raw(&M, &B, i, j, k) + z_raw(&M, &B, j, i, k));
        }
    mesh_free(&M);
    return 0;
}

/* Rows of the symmetric dZ/dk (each entry the mean of both orders, as in
 * oracle_dzfill): out [nrows][n] complex. */
int oracle_dzrows(int nv, const double *V, int nt, const int32_t *T,
                  int n, const int32_t *tri, const int32_t *vfree, const double *len,
                  double k, double eta, int nrows, const int64_t *rows, double *out, int nthreads)
{
    (void)nv;
    mesh_t M;
    if (mesh_init(&M, nt, V, T)) return -1;
    rwg_t B;
    rwg_from_args(&B, n, tri, vfree, len);
    cplx *O = (cplx *)out;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) collapse(2)
#endif
    for (int r = 0; r < nrows; ++r)
        for (int j = 0; j < n; ++j) {
            const int i = (int)rows[r];
            O[(size_t)r * n + j] = 0.5 * (dz_raw(&M, &B, i, j, k, eta) + dz_raw(&M, &B, j, i, k, eta));
        }
    mesh_free(&M);
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
