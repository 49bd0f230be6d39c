/*
 * oracle.c -- plain, slow FP64 CPU oracle for the Galerkin boundary operators
 * of the OSRC-preconditioned PMCHWT formulation for acoustic transmission
 * (van 't Wout, Haqshenas, Gelat, Betcke, Saffari, JCP 2022; arXiv 2104.04609).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; it is used by the tests, by __graft_entry__.smoke() and by
 * the CPU-baseline leg of bench.py.  It shares no code, header or table with
 * the CUDA library.
 *
 * What it computes (each item cites the passage of the paper it follows):
 *  - Green's function G(x,y) = exp(ik|x-y|) / (4 pi |x-y|)            (Sec. 2.2)
 *  - Galerkin matrices on P1 x P1 for the four boundary operators of Sec. 2.2:
 *      V_ij = int int phi_i(x) G(x,y) phi_j(y)
 *      K_ij = int int phi_i(x) dG/dn_y(x,y) phi_j(y)       (double layer)
 *      T_ij = int int phi_i(x) dG/dn_x(x,y) phi_j(y)       (adjoint double layer)
 *      D_ij = int int G(x,y) [curl phi_i(x) . curl phi_j(y)
 *                             - k^2 (n_x . n_y) phi_i(x) phi_j(y)]
 *    (D = -d/dn_x of the double-layer potential, written in the
 *    integrated-by-parts form of Maue / Nedelec; P1 spaces as in Sec. 2.3.)
 *  - Quadrature: the 6-point degree-4 symmetric triangle rule (Strang & Fix;
 *    Dunavant 1985) on both triangles for pairs that share no vertex, and the
 *    Sauter-Schwab regularising transformations (Sauter & Schwab, Boundary
 *    Element Methods, Sec. 5.2) with n Gauss-Legendre points per cube
 *    dimension for pairs that share a vertex, an edge or are identical.
 *    The paper itself is silent on quadrature (it uses BEMPP defaults).
 *  - P1 mass and Laplace-Beltrami stiffness element matrices (Sec. 2.6: the
 *    OSRC operators are surface Helmholtz problems discretised with P1).
 *  - Right-hand sides <gamma_D u_inc, phi_i>, <gamma_N u_inc, phi_i> (Sec. 2.7)
 *    for a plane wave exp(i k d.x) and a point source G(x, x0).
 *
 * Conventions: triangles are counter-clockwise seen from outside, so the
 * element normal (P1-P0)x(P2-P0)/|..| points to the exterior (Sec. 2.1).
 * Complex numbers are C99 double complex, returned interleaved (re, im).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_PI 3.14159265358979323846

/* ---------------------------------------------------------------------- */
/* 6-point degree-4 rule: barycentric points (a,a,1-2a) and permutations.  */
/* ---------------------------------------------------------------------- */
static const double Q6_A1 = 0.44594849091596488632;
static const double Q6_W1 = 0.22338158967801146570;
static const double Q6_A2 = 0.09157621350977074346;
static const double Q6_W2 = 0.10995174365532186764;

int orc_quad6(double *bary /* 6x3 */, double *w /* 6 */)
{
    const double a[2] = {Q6_A1, Q6_A2}, ww[2] = {Q6_W1, Q6_W2};
    int p = 0;
    for (int g = 0; g < 2; ++g) {
        double b = 1.0 - 2.0 * a[g];
        double pts[3][3] = {{b, a[g], a[g]}, {a[g], b, a[g]}, {a[g], a[g], b}};
        for (int i = 0; i < 3; ++i, ++p) {
            for (int j = 0; j < 3; ++j) bary[3 * p + j] = pts[i][j];
            w[p] = ww[g];
        }
    }
    return 6;
}

/* Gauss-Legendre nodes and weights on [0,1], by Newton's method on P_n. */
int orc_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1) return -1;
    for (int i = 0; i < n; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
    return n;
}

/* ---------------------------------------------------------------------- */
/* Sauter-Schwab transformations.  Reference triangle That = {0<=x2<=x1<=1}, */
/* mapped to a physical triangle (P0,P1,P2) by P0 + x1 (P1-P0) + x2 (P2-P1).  */
/* kase 3: identical triangles; 2: common edge P0P1 in both; 1: common     */
/* vertex P0 in both.  Each map sends (xi, e1, e2, e3) in [0,1]^4 to a pair */
/* (xhat, yhat); jac is the Jacobian of that map.  Sum of jac over the     */
/* maps integrates to |That|^2 = 1/4.                                      */
/* ---------------------------------------------------------------------- */
static int ss_maps(int kase, double xi, double e1, double e2, double e3,
                   double xh[6][2], double yh[6][2], double jac[6])
{
    if (kase == 3) {
        double J = xi * xi * xi * e1 * e1 * e2;
        double ax[2] = {xi, xi * (1.0 - e1 + e1 * e2)};
        double ay[2] = {xi * (1.0 - e1 * e2 * e3), xi * (1.0 - e1)};
        double bx[2] = {xi, xi * e1 * (1.0 - e2 + e2 * e3)};
        double by[2] = {xi * (1.0 - e1 * e2), xi * e1 * (1.0 - e2)};
        double cx[2] = {xi * (1.0 - e1 * e2 * e3), xi * e1 * (1.0 - e2 * e3)};
        double cy[2] = {xi, xi * e1 * (1.0 - e2)};
        const double *X[6] = {ax, ay, bx, by, cx, cy};
        const double *Y[6] = {ay, ax, by, bx, cy, cx};
        for (int m = 0; m < 6; ++m) {
            xh[m][0] = X[m][0]; xh[m][1] = X[m][1];
            yh[m][0] = Y[m][0]; yh[m][1] = Y[m][1];
            jac[m] = J;
        }
        return 6;
    }
    if (kase == 2) {
        double J1 = xi * xi * xi * e1 * e1, J = J1 * e2;
        xh[0][0] = xi;                          xh[0][1] = xi * e1 * e3;
        yh[0][0] = xi * (1.0 - e1 * e2);        yh[0][1] = xi * e1 * (1.0 - e2);
        jac[0] = J1;
        xh[1][0] = xi;                          xh[1][1] = xi * e1;
        yh[1][0] = xi * (1.0 - e1 * e2 * e3);   yh[1][1] = xi * e1 * e2 * (1.0 - e3);
        jac[1] = J;
        xh[2][0] = xi * (1.0 - e1 * e2);        xh[2][1] = xi * e1 * (1.0 - e2);
        yh[2][0] = xi;                          yh[2][1] = xi * e1 * e2 * e3;
        jac[2] = J;
        xh[3][0] = xi * (1.0 - e1 * e2 * e3);   xh[3][1] = xi * e1 * e2 * (1.0 - e3);
        yh[3][0] = xi;                          yh[3][1] = xi * e1;
        jac[3] = J;
        xh[4][0] = xi * (1.0 - e1 * e2 * e3);   xh[4][1] = xi * e1 * (1.0 - e2 * e3);
        yh[4][0] = xi;                          yh[4][1] = xi * e1 * e2;
        jac[4] = J;
        return 5;
    }
    if (kase == 1) {
        double J = xi * xi * xi * e2;
        xh[0][0] = xi;            xh[0][1] = xi * e1;
        yh[0][0] = xi * e2;       yh[0][1] = xi * e2 * e3;
        jac[0] = J;
        xh[1][0] = xi * e2;       xh[1][1] = xi * e2 * e3;
        yh[1][0] = xi;            yh[1][1] = xi * e1;
        jac[1] = J;
        return 2;
    }
    return 0;
}

/* The full Sauter-Schwab point set for one case: out[N][4] = (x1,x2,y1,y2),  */
/* wout[N] = Gauss weight x Jacobian.  Returns N, or -1 if cap is too small. */
int orc_ss_rule(int kase, int n, double *out, double *wout, int cap)
{
    double gx[64], gw[64];
    if (n < 1 || n > 64) return -1;
    orc_gauss_legendre(n, gx, gw);
    int N = 0;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            for (int c = 0; c < n; ++c)
                for (int d = 0; d < n; ++d) {
                    double xh[6][2], yh[6][2], jac[6];
                    int nm = ss_maps(kase, gx[a], gx[b], gx[c], gx[d], xh, yh, jac);
                    double w = gw[a] * gw[b] * gw[c] * gw[d];
                    for (int m = 0; m < nm; ++m) {
                        if (N >= cap) return -1;
                        out[4 * N + 0] = xh[m][0];
                        out[4 * N + 1] = xh[m][1];
                        out[4 * N + 2] = yh[m][0];
                        out[4 * N + 3] = yh[m][1];
                        wout[N] = w * jac[m];
                        ++N;
                    }
                }
    return N;
}

/* ---------------------------------------------------------------------- */
/* Geometry of one flat triangle.                                          */
/* ---------------------------------------------------------------------- */
typedef struct {
    double P[3][3];     /* vertices */
    double n[3];        /* unit outward normal */
    double area;
    double grad[3][3];  /* surface gradient of the P1 hat functions */
    double curl[3][3];  /* surface curl n x grad */
} tri_geom;

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void make_geom(const double *verts, const int *tri, tri_geom *g)
{
    for (int a = 0; a < 3; ++a)
        for (int j = 0; j < 3; ++j) g->P[a][j] = verts[3 * tri[a] + j];
    double e1[3], e2[3], c[3];
    for (int j = 0; j < 3; ++j) {
        e1[j] = g->P[1][j] - g->P[0][j];
        e2[j] = g->P[2][j] - g->P[0][j];
    }
    cross3(e1, e2, c);
    double len = sqrt(dot3(c, c));
    g->area = 0.5 * len;
    for (int j = 0; j < 3; ++j) g->n[j] = c[j] / len;
    /* grad lambda_a = n x (P_{a+2} - P_{a+1}) / (2 area) */
    for (int a = 0; a < 3; ++a) {
        double e[3], t[3];
        for (int j = 0; j < 3; ++j) e[j] = g->P[(a + 2) % 3][j] - g->P[(a + 1) % 3][j];
        cross3(g->n, e, t);
        for (int j = 0; j < 3; ++j) g->grad[a][j] = t[j] / (2.0 * g->area);
        cross3(g->n, g->grad[a], g->curl[a]);
    }
}

/* Vertex-sharing type of two triangles: 0 none, 1 vertex, 2 edge, 3 same.  */
/* pt/ps give the local orders that put the shared vertices first, in the  */
/* same order in both triangles.                                            */
static int touching(const int *t, const int *s, int pt[3], int ps[3])
{
    int nsh = 0, shT[3], shS[3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (t[a] == s[b]) { shT[nsh] = a; shS[nsh] = b; ++nsh; }
    if (nsh == 3) {
        /* identical triangle: use s's order matching t's vertex by vertex */
        for (int a = 0; a < 3; ++a) {
            pt[a] = a;
            for (int b = 0; b < 3; ++b) if (s[b] == t[a]) ps[a] = b;
        }
        return 3;
    }
    if (nsh == 0) {
        for (int a = 0; a < 3; ++a) { pt[a] = a; ps[a] = a; }
        return 0;
    }
    /* shared first, then the rest in cyclic order */
    int used_t[3] = {0, 0, 0}, used_s[3] = {0, 0, 0}, k = 0;
    for (int i = 0; i < nsh; ++i) {
        pt[k] = shT[i]; ps[k] = shS[i];
        used_t[shT[i]] = 1; used_s[shS[i]] = 1; ++k;
    }
    int kt = k, ks = k;
    for (int a = 0; a < 3; ++a) if (!used_t[a]) pt[kt++] = a;
    for (int b = 0; b < 3; ++b) if (!used_s[b]) ps[ks++] = b;
    return nsh;
}

/* Accumulate one quadrature point pair into the four 3x3 local matrices.  */
static inline void accum_point(const tri_geom *gt, const tri_geom *gs,
                               const double *x, const double *y,
                               const double la[3], const double lb[3],
                               const int pt[3], const int ps[3],
                               double w, cplx k, const double cc[3][3], double nn,
                               cplx V[3][3], cplx K[3][3], cplx T[3][3], cplx D[3][3])
{
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r = sqrt(dot3(d, d));
    cplx e = cexp(I * k * r);
    cplx G = e / (4.0 * ORC_PI * r);
    cplx H = e * (I * k * r - 1.0) / (4.0 * ORC_PI * r * r * r);
    double dny = -dot3(d, gs->n);  /* (y - x) . n_y */
    double dnx = dot3(d, gt->n);   /* (x - y) . n_x */
    cplx k2 = k * k;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            int A = pt[a], B = ps[b];
            double ll = la[a] * lb[b] * w;
            V[A][B] += G * ll;
            K[A][B] += H * dny * ll;
            T[A][B] += H * dnx * ll;
            D[A][B] += G * (cc[A][B] * w - k2 * nn * ll);
        }
}

/* Local 3x3 matrices (original local vertex order of t and s) for one pair. */
static void pair_local(const tri_geom *gt, const tri_geom *gs, int kase,
                       const int pt[3], const int ps[3], cplx k,
                       int nss, const double *gx, const double *gw,
                       cplx V[3][3], cplx K[3][3], cplx T[3][3], cplx D[3][3])
{
    double cc[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            cc[a][b] = dot3(gt->curl[a], gs->curl[b]);
            V[a][b] = K[a][b] = T[a][b] = D[a][b] = 0.0;
        }
    double nn = dot3(gt->n, gs->n);
    if (kase == 0) {
        double bary[18], w6[6];
        orc_quad6(bary, w6);
        double scale = gt->area * gs->area;
        for (int p = 0; p < 6; ++p) {
            double x[3];
            for (int j = 0; j < 3; ++j)
                x[j] = bary[3 * p] * gt->P[0][j] + bary[3 * p + 1] * gt->P[1][j] +
                       bary[3 * p + 2] * gt->P[2][j];
            for (int q = 0; q < 6; ++q) {
                double y[3];
                for (int j = 0; j < 3; ++j)
                    y[j] = bary[3 * q] * gs->P[0][j] + bary[3 * q + 1] * gs->P[1][j] +
                           bary[3 * q + 2] * gs->P[2][j];
                accum_point(gt, gs, x, y, &bary[3 * p], &bary[3 * q], pt, ps,
                            w6[p] * w6[q] * scale, k, cc, nn, V, K, T, D);
            }
        }
        return;
    }
    /* permuted vertices: shared ones first */
    double Pt[3][3], Ps[3][3];
    for (int a = 0; a < 3; ++a)
        for (int j = 0; j < 3; ++j) {
            Pt[a][j] = gt->P[pt[a]][j];
            Ps[a][j] = gs->P[ps[a]][j];
        }
    double scale = 4.0 * gt->area * gs->area;
    for (int i0 = 0; i0 < nss; ++i0)
        for (int i1 = 0; i1 < nss; ++i1)
            for (int i2 = 0; i2 < nss; ++i2)
                for (int i3 = 0; i3 < nss; ++i3) {
                    double xh[6][2], yh[6][2], jac[6];
                    int nm = ss_maps(kase, gx[i0], gx[i1], gx[i2], gx[i3], xh, yh, jac);
                    double w = gw[i0] * gw[i1] * gw[i2] * gw[i3] * scale;
                    for (int m = 0; m < nm; ++m) {
                        double la[3] = {1.0 - xh[m][0], xh[m][0] - xh[m][1], xh[m][1]};
                        double lb[3] = {1.0 - yh[m][0], yh[m][0] - yh[m][1], yh[m][1]};
                        double x[3], y[3];
                        for (int j = 0; j < 3; ++j) {
                            x[j] = Pt[0][j] + xh[m][0] * (Pt[1][j] - Pt[0][j]) +
                                   xh[m][1] * (Pt[2][j] - Pt[1][j]);
                            y[j] = Ps[0][j] + yh[m][0] * (Ps[1][j] - Ps[0][j]) +
                                   yh[m][1] * (Ps[2][j] - Ps[1][j]);
                        }
                        accum_point(gt, gs, x, y, la, lb, pt, ps, w * jac[m], k, cc, nn,
                                    V, K, T, D);
                    }
                }
}

/* Local matrices of one triangle pair, for tests: out = 4 x 3 x 3 complex   */
/* (V, K, T, D), interleaved.  Returns the touching case (0..3).             */
int orc_pair_matrices(const double *verts, const int *tris, int t, int s,
                      double kre, double kim, int nss, double *out)
{
    double gx[64], gw[64];
    if (nss < 1 || nss > 64) return -1;
    orc_gauss_legendre(nss, gx, gw);
    tri_geom gt, gs;
    make_geom(verts, &tris[3 * t], &gt);
    make_geom(verts, &tris[3 * s], &gs);
    int pt[3], ps[3];
    int kase = touching(&tris[3 * t], &tris[3 * s], pt, ps);
    cplx V[3][3], K[3][3], T[3][3], D[3][3];
    pair_local(&gt, &gs, kase, pt, ps, kre + I * kim, nss, gx, gw, V, K, T, D);
    cplx *M[4] = {&V[0][0], &K[0][0], &T[0][0], &D[0][0]};
    for (int o = 0; o < 4; ++o)
        for (int i = 0; i < 9; ++i) {
            out[2 * (9 * o + i)] = creal(M[o][i]);
            out[2 * (9 * o + i) + 1] = cimag(M[o][i]);
        }
    return kase;
}

/* Dense assembly of V, K, T, D (each n_v x n_v complex, interleaved) for one */
/* wavenumber.  part: 1 = pairs sharing no vertex (6x6 rule) only,          */
/* 2 = touching pairs (Sauter-Schwab) only, 3 = all pairs.                   */
int orc_assemble(const double *verts, int nv, const int *tris, int nt,
                 double kre, double kim, int nss, int part, double *out)
{
    double gx[64], gw[64];
    if (nss < 1 || nss > 64) return -1;
    orc_gauss_legendre(nss, gx, gw);
    cplx k = kre + I * kim;
    size_t nn2 = (size_t)nv * nv;
    memset(out, 0, sizeof(double) * 2 * 4 * nn2);
    tri_geom *geo = (tri_geom *)malloc(sizeof(tri_geom) * (size_t)nt);
    if (!geo) return -2;
    for (int t = 0; t < nt; ++t) make_geom(verts, &tris[3 * t], &geo[t]);
    /* chunks of test triangles computed in parallel, scattered in order */
    size_t per_t = (size_t)nt * 36;
    int chunk = (int)(200000000 / (per_t * sizeof(cplx)));
    if (chunk < 1) chunk = 1;
    if (chunk > nt) chunk = nt;
    cplx *slab = (cplx *)malloc(sizeof(cplx) * per_t * (size_t)chunk);
    if (!slab) { free(geo); return -2; }
    for (int t0 = 0; t0 < nt; t0 += chunk) {
        int t1 = t0 + chunk < nt ? t0 + chunk : nt;
#pragma omp parallel for schedule(dynamic, 1)
        for (int t = t0; t < t1; ++t) {
            cplx *dst = slab + per_t * (size_t)(t - t0);
            for (int s = 0; s < nt; ++s) {
                int pt[3], ps[3];
                int kase = touching(&tris[3 * t], &tris[3 * s], pt, ps);
                cplx *L = dst + 36 * (size_t)s;
                int use = (kase == 0) ? (part & 1) : (part & 2);
                if (!use) {
                    for (int i = 0; i < 36; ++i) L[i] = 0.0;
                    continue;
                }
                cplx V[3][3], K[3][3], T[3][3], D[3][3];
                pair_local(&geo[t], &geo[s], kase, pt, ps, k, nss, gx, gw, V, K, T, D);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        L[0 * 9 + 3 * a + b] = V[a][b];
                        L[1 * 9 + 3 * a + b] = K[a][b];
                        L[2 * 9 + 3 * a + b] = T[a][b];
                        L[3 * 9 + 3 * a + b] = D[a][b];
                    }
            }
        }
        for (int t = t0; t < t1; ++t) {
            const cplx *src = slab + per_t * (size_t)(t - t0);
            for (int s = 0; s < nt; ++s) {
                const cplx *L = src + 36 * (size_t)s;
                for (int o = 0; o < 4; ++o)
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) {
                            size_t idx = (size_t)o * nn2 +
                                         (size_t)tris[3 * t + a] * nv + tris[3 * s + b];
                            out[2 * idx] += creal(L[9 * o + 3 * a + b]);
                            out[2 * idx + 1] += cimag(L[9 * o + 3 * a + b]);
                        }
            }
        }
    }
    free(slab);
    free(geo);
    return 0;
}

/* Selected rows of V, K, T, D: out[r][op][n_v] complex for test vertex      */
/* rows[r]; same quadrature and parts as orc_assemble.  Used where the dense */
/* matrices are too large: each row sums over the triangles around rows[r]. */
int orc_assemble_rows(const double *verts, int nv, const int *tris, int nt,
                      double kre, double kim, int nss, int part,
                      const int *rows, int nrows, double *out)
{
    double gx[64], gw[64];
    if (nss < 1 || nss > 64) return -1;
    orc_gauss_legendre(nss, gx, gw);
    cplx k = kre + I * kim;
    tri_geom *geo = (tri_geom *)malloc(sizeof(tri_geom) * (size_t)nt);
    if (!geo) return -2;
    for (int t = 0; t < nt; ++t) make_geom(verts, &tris[3 * t], &geo[t]);
    memset(out, 0, sizeof(double) * 2 * 4 * (size_t)nv * nrows);
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < nrows; ++r) {
        int i = rows[r];
        double *dst = out + 2 * 4 * (size_t)nv * r;
        for (int t = 0; t < nt; ++t) {
            int a = -1;
            for (int j = 0; j < 3; ++j) if (tris[3 * t + j] == i) a = j;
            if (a < 0) continue;
            for (int s = 0; s < nt; ++s) {
                int pt[3], ps[3];
                int kase = touching(&tris[3 * t], &tris[3 * s], pt, ps);
                int use = (kase == 0) ? (part & 1) : (part & 2);
                if (!use) continue;
                cplx V[3][3], K[3][3], T[3][3], D[3][3];
                pair_local(&geo[t], &geo[s], kase, pt, ps, k, nss, gx, gw, V, K, T, D);
                cplx *M[4] = {&V[a][0], &K[a][0], &T[a][0], &D[a][0]};
                for (int o = 0; o < 4; ++o)
                    for (int b = 0; b < 3; ++b) {
                        size_t idx = (size_t)o * nv + tris[3 * s + b];
                        dst[2 * idx] += creal(M[o][b]);
                        dst[2 * idx + 1] += cimag(M[o][b]);
                    }
            }
        }
    }
    free(geo);
    return 0;
}

/* P1 mass and stiffness element contributions as COO triplets: 9 per     */
/* triangle, rows/cols/values; duplicates are to be summed by the caller.  */
/*   M_ab = |t|/12 (1 + delta_ab),   S_ab = |t| grad phi_a . grad phi_b     */
int orc_mass_stiffness_coo(const double *verts, const int *tris, int nt,
                           int *ri, int *ci, double *mv, double *sv)
{
    for (int t = 0; t < nt; ++t) {
        tri_geom g;
        make_geom(verts, &tris[3 * t], &g);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                int e = 9 * t + 3 * a + b;
                ri[e] = tris[3 * t + a];
                ci[e] = tris[3 * t + b];
                mv[e] = g.area / 12.0 * (a == b ? 2.0 : 1.0);
                sv[e] = g.area * dot3(g.grad[a], g.grad[b]);
            }
    }
    return 0;
}

/* Right-hand side of Sec. 2.7, tested against P1 with the 6-point rule:    */
/*   b1_i = int u_inc phi_i,   b2_i = int du_inc/dn phi_i                   */
/* kind 0: plane wave exp(i k d.x), src = direction d (unit)                 */
/* kind 1: point source exp(ik|x-x0|)/(4 pi |x-x0|), src = x0                */
/* out: 2 n_v complex interleaved, [b1; b2].                                  */
int orc_rhs(const double *verts, int nv, const int *tris, int nt,
            double kre, double kim, int kind, const double *src, double *out)
{
    double bary[18], w6[6];
    orc_quad6(bary, w6);
    cplx k = kre + I * kim;
    cplx *b = (cplx *)calloc((size_t)2 * nv, sizeof(cplx));
    if (!b) return -2;
    for (int t = 0; t < nt; ++t) {
        tri_geom g;
        make_geom(verts, &tris[3 * t], &g);
        for (int p = 0; p < 6; ++p) {
            double x[3];
            for (int j = 0; j < 3; ++j)
                x[j] = bary[3 * p] * g.P[0][j] + bary[3 * p + 1] * g.P[1][j] +
                       bary[3 * p + 2] * g.P[2][j];
            cplx u, dudn;
            if (kind == 0) {
                double dx = dot3(src, x);
                u = cexp(I * k * dx);
                dudn = I * k * dot3(src, g.n) * u;
            } else {
                double d[3] = {x[0] - src[0], x[1] - src[1], x[2] - src[2]};
                double R = sqrt(dot3(d, d));
                cplx e = cexp(I * k * R);
                u = e / (4.0 * ORC_PI * R);
                dudn = e * (I * k * R - 1.0) / (4.0 * ORC_PI * R * R * R) * dot3(d, g.n);
            }
            double w = w6[p] * g.area;
            for (int a = 0; a < 3; ++a) {
                int i = tris[3 * t + a];
                b[i] += w * bary[3 * p + a] * u;
                b[nv + i] += w * bary[3 * p + a] * dudn;
            }
        }
    }
    for (int i = 0; i < 2 * nv; ++i) {
        out[2 * i] = creal(b[i]);
        out[2 * i + 1] = cimag(b[i]);
    }
    free(b);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Single- and double-layer potentials at points off the surface (Sec. 2.2,  */
/* the representation formulas): for densities psi, phi given as P1          */
/* coefficients (n_v complex each),                                          */
/*   slp(x) = int G(x, y) psi(y) dy,                                          */
/*   dlp(x) = int dG(x, y)/dn_y phi(y) dy,                                    */
/*   dG/dn_y = exp(ikr) (ikr - 1) (y - x).n_y / (4 pi r^3),                   */
/* each integral by the 6-point rule on every triangle.  out_slp, out_dlp:   */
/* npts complex interleaved.                                                  */
/* ------------------------------------------------------------------------ */
int orc_potentials(const double *verts, int nv, const int *tris, int nt,
                   double kre, double kim, const double *psi, const double *phi,
                   const double *pts, int npts, double *out_slp, double *out_dlp)
{
    (void)nv;
    double bary[18], w6[6];
    orc_quad6(bary, w6);
    cplx k = kre + I * kim;
    const cplx *ps = (const cplx *)psi, *ph = (const cplx *)phi;
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < npts; ++i) {
        const double *x = pts + 3 * i;
        cplx S = 0.0, D = 0.0;
        for (int t = 0; t < nt; ++t) {
            tri_geom g;
            make_geom(verts, &tris[3 * t], &g);
            const int *v = &tris[3 * t];
            for (int q = 0; q < 6; ++q) {
                double y[3];
                for (int j = 0; j < 3; ++j)
                    y[j] = bary[3 * q] * g.P[0][j] + bary[3 * q + 1] * g.P[1][j] +
                           bary[3 * q + 2] * g.P[2][j];
                cplx psq = bary[3 * q] * ps[v[0]] + bary[3 * q + 1] * ps[v[1]] +
                           bary[3 * q + 2] * ps[v[2]];
                cplx phq = bary[3 * q] * ph[v[0]] + bary[3 * q + 1] * ph[v[1]] +
                           bary[3 * q + 2] * ph[v[2]];
                double d[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};  /* y - x */
                double r = sqrt(dot3(d, d));
                cplx e = cexp(I * k * r);
                double w = w6[q] * g.area;
                S += w * e / (4.0 * ORC_PI * r) * psq;
                D += w * e * (I * k * r - 1.0) / (4.0 * ORC_PI * r * r * r) * dot3(d, g.n) * phq;
            }
        }
        out_slp[2 * i] = creal(S);
        out_slp[2 * i + 1] = cimag(S);
        out_dlp[2 * i] = creal(D);
        out_dlp[2 * i + 1] = cimag(D);
    }
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
