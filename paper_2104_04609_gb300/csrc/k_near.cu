// k_near.cu -- near-field (touching triangle pairs) in FP64 by Sauter-Schwab
// quadrature, assembled on the device into a vertex-pair CSR of 2x2 complex
// blocks of the permuted PMCHWT operator (Sec. 2.7); and the dense FP64
// system of the assembled path.
//
// Sauter-Schwab (Sauter & Schwab, Boundary Element Methods, Sec. 5.2): the
// reference triangle is That = {0 <= x2 <= x1 <= 1}, mapped to a flat
// triangle (P0, P1, P2) by P0 + x1 (P1 - P0) + x2 (P2 - P1), so that the hat
// functions are (1 - x1, x1 - x2, x2).  Touching pairs are re-ordered so that
// the shared vertices come first in both triangles; then the singular set is
// the origin (common vertex), the edge x2 = 0 (common edge) or the diagonal
// (identical triangles).  Each case splits [0,1]^4 into 2, 5 or 6 regions
// whose Jacobians (xi^3 eta2, xi^3 eta1^2 [eta2], xi^3 eta1^2 eta2) cancel the
// 1/r and 1/r^2 singularities, leaving integrands that tensor Gauss-Legendre
// rules integrate with exponential convergence.
#include "ffmath.cuh"
#include <algorithm>
#include <vector>

#include "osrc_internal.cuh"
#include "dense_sched.cuh"

namespace {

__device__ __forceinline__ int ss_nmaps(int kase) { return kase == 3 ? 6 : (kase == 2 ? 5 : 2); }

// Map m of case kase: (xi, e1, e2, e3) -> (xh, yh) with Jacobian jac.
__device__ __forceinline__ void ss_map(int kase, int m, double xi, double e1, double e2, double e3,
                                       double xh[2], double yh[2], double &jac) {
    if (kase == 3) {
        jac = xi * xi * xi * e1 * e1 * e2;
        double ax, ay, bx, by;  // first point, second point
        double cx, cy, dx, dy;
        const int pm = m >> 1;
        if (pm == 0) {
            ax = xi;                          ay = xi * (1.0 - e1 + e1 * e2);
            bx = xi * (1.0 - e1 * e2 * e3);   by = xi * (1.0 - e1);
        } else if (pm == 1) {
            ax = xi;                          ay = xi * e1 * (1.0 - e2 + e2 * e3);
            bx = xi * (1.0 - e1 * e2);        by = xi * e1 * (1.0 - e2);
        } else {
            ax = xi * (1.0 - e1 * e2 * e3);   ay = xi * e1 * (1.0 - e2 * e3);
            bx = xi;                          by = xi * e1 * (1.0 - e2);
        }
        if (m & 1) { cx = bx; cy = by; dx = ax; dy = ay; }
        else       { cx = ax; cy = ay; dx = bx; dy = by; }
        xh[0] = cx; xh[1] = cy; yh[0] = dx; yh[1] = dy;
        return;
    }
    if (kase == 2) {
        const double J1 = xi * xi * xi * e1 * e1;
        switch (m) {
            case 0:
                xh[0] = xi;                        xh[1] = xi * e1 * e3;
                yh[0] = xi * (1.0 - e1 * e2);      yh[1] = xi * e1 * (1.0 - e2);
                jac = J1; return;
            case 1:
                xh[0] = xi;                        xh[1] = xi * e1;
                yh[0] = xi * (1.0 - e1 * e2 * e3); yh[1] = xi * e1 * e2 * (1.0 - e3);
                jac = J1 * e2; return;
            case 2:
                xh[0] = xi * (1.0 - e1 * e2);      xh[1] = xi * e1 * (1.0 - e2);
                yh[0] = xi;                        yh[1] = xi * e1 * e2 * e3;
                jac = J1 * e2; return;
            case 3:
                xh[0] = xi * (1.0 - e1 * e2 * e3); xh[1] = xi * e1 * e2 * (1.0 - e3);
                yh[0] = xi;                        yh[1] = xi * e1;
                jac = J1 * e2; return;
            default:
                xh[0] = xi * (1.0 - e1 * e2 * e3); xh[1] = xi * e1 * (1.0 - e2 * e3);
                yh[0] = xi;                        yh[1] = xi * e1 * e2;
                jac = J1 * e2; return;
        }
    }
    jac = xi * xi * xi * e2;
    if (m == 0) {
        xh[0] = xi;       xh[1] = xi * e1;
        yh[0] = xi * e2;  yh[1] = xi * e2 * e3;
    } else {
        xh[0] = xi * e2;  xh[1] = xi * e2 * e3;
        yh[0] = xi;       yh[1] = xi * e1;
    }
}

struct NearConst {
    double k0, k1, rho;
    int nss;
    const ObjMat *obj;  // disjoint objects: material per object (else k1, rho)
    const int *tcomp;   // object of each triangle
    double sgn;         // sign of the interior terms: +1 PMCHWT, -1 Mueller
    double k1i;         // attenuation: Im k1 (objects: their own, from obj)
};

constexpr int NEAR_WARPS = 4;
constexpr double kInv4Pi = 0.079577471545947667884;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One warp per touching pair.  out[pair][36]: blocks (V0 + rho V1),
// -(K0 + K1), (T0 + T1), (D0 + D1/rho), each 3x3 in the original local
// vertex order of (test, source) triangle.
__global__ void __launch_bounds__(32 * NEAR_WARPS)
near_ss_kernel(const NearPair *__restrict__ pairs, long long npairs,
               const double *__restrict__ verts, const int *__restrict__ tris,
               const double *__restrict__ tgeo, const double *__restrict__ gl,
               NearConst c, double2 *__restrict__ out) {
    __shared__ double sx[16], sw[16];
    if (threadIdx.x < c.nss) {
        sx[threadIdx.x] = gl[threadIdx.x];
        sw[threadIdx.x] = gl[16 + threadIdx.x];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long pi = (long long)blockIdx.x * NEAR_WARPS + (threadIdx.x >> 5);
    if (pi >= npairs) return;
    const NearPair pr = pairs[pi];
    double k1 = c.k1, rho = c.rho, k1i = c.k1i;  // touching triangles lie on one object
    if (c.obj) {
        const ObjMat o = c.obj[c.tcomp[pr.t]];
        k1 = o.k1;
        rho = o.rho;
        k1i = o.k1i;
    }
    int pt[3], ps[3];
    for (int a = 0; a < 3; ++a) {
        pt[a] = (pr.perm >> (2 * a)) & 3;
        ps[a] = (pr.perm >> (6 + 2 * a)) & 3;
    }
    double Pt[3][3], Ps[3][3];
    for (int a = 0; a < 3; ++a) {
        const int vt = tris[3 * pr.t + pt[a]], vs = tris[3 * pr.s + ps[a]];
        for (int j = 0; j < 3; ++j) {
            Pt[a][j] = verts[3 * vt + j];
            Ps[a][j] = verts[3 * vs + j];
        }
    }
    const double *gt = tgeo + 16 * (size_t)pr.t, *gs = tgeo + 16 * (size_t)pr.s;
    const double nt0 = gt[1], nt1 = gt[2], nt2 = gt[3];
    const double ns0 = gs[1], ns1 = gs[2], ns2 = gs[3];
    const double nn = nt0 * ns0 + nt1 * ns1 + nt2 * ns2;
    const double scale = 4.0 * gt[0] * gs[0];
    const int n = c.nss, n2 = n * n, n4 = n2 * n2;
    const int total = ss_nmaps(pr.kase) * n4;

    double vr[9], vi[9], kr_[9], ki_[9], tr_[9], ti_[9], dr[9], di[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) vr[i] = vi[i] = kr_[i] = ki_[i] = tr_[i] = ti_[i] = dr[i] = di[i] = 0.0;
    double dcr = 0.0, dci = 0.0;

    for (int idx = lane; idx < total; idx += 32) {
        const int m = idx / n4;
        int rem = idx - m * n4;
        const int i0 = rem / (n2 * n);
        rem -= i0 * n2 * n;
        const int i1 = rem / n2;
        rem -= i1 * n2;
        const int i2 = rem / n, i3 = rem - (rem / n) * n;
        double xh[2], yh[2], jac;
        ss_map(pr.kase, m, sx[i0], sx[i1], sx[i2], sx[i3], xh, yh, jac);
        const double w = sw[i0] * sw[i1] * sw[i2] * sw[i3] * jac * scale;
        double x[3], y[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            x[j] = Pt[0][j] + xh[0] * (Pt[1][j] - Pt[0][j]) + xh[1] * (Pt[2][j] - Pt[1][j]);
            y[j] = Ps[0][j] + yh[0] * (Ps[1][j] - Ps[0][j]) + yh[1] * (Ps[2][j] - Ps[1][j]);
        }
        const double la[3] = {1.0 - xh[0], xh[0] - xh[1], xh[1]};
        const double lb[3] = {1.0 - yh[0], yh[0] - yh[1], yh[1]};
        const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
        const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
        const double r = sqrt(r2);
        const double ri = 1.0 / r;
        double s0, c0, s1, c1;
        sincos(c.k0 * r, &s0, &c0);
        sincos(k1 * r, &s1, &c1);
        // k1 = k1 + i k1i: e^{i k1 r} damped by e^{-k1i r}; (i k1 r - 1) gains -k1i r
        const double br = k1i * r, damp = c.sgn * (k1i != 0.0 ? exp(-br) : 1.0);
        s1 *= damp;
        c1 *= damp;
        const double kr0 = c.k0 * r, kr1 = k1 * r;
        const double f = kInv4Pi * ri, f3 = f * ri * ri;
        const double g0r = c0 * f, g0i = s0 * f, g1r = c1 * f, g1i = s1 * f;
        const double hsr = (-c0 - kr0 * s0 - c1 - kr1 * s1 - br * c1) * f3;
        const double hsi = (kr0 * c0 - s0 + kr1 * c1 - s1 - br * s1) * f3;
        const double gpr = g0r + rho * g1r, gpi = g0i + rho * g1i;
        const double gdr = g0r + g1r / rho, gdi = g0i + g1i / rho;
        const double dk0 = c.k0 * c.k0, dk1 = (k1 * k1 - k1i * k1i) / rho, dk1i = 2.0 * k1 * k1i / rho;
        const double gkr = dk0 * g0r + dk1 * g1r - dk1i * g1i, gki = dk0 * g0i + dk1 * g1i + dk1i * g1r;
        const double dny = -(d0 * ns0 + d1 * ns1 + d2 * ns2);  // (y - x).n_y
        const double dnx = d0 * nt0 + d1 * nt1 + d2 * nt2;     // (x - y).n_x
        dcr += gdr * w;
        dci += gdi * w;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double wa = la[a] * w;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const double ll = wa * lb[b];
                const int i = 3 * a + b;
                vr[i] += gpr * ll;
                vi[i] += gpi * ll;
                kr_[i] -= hsr * dny * ll;
                ki_[i] -= hsi * dny * ll;
                tr_[i] += hsr * dnx * ll;
                ti_[i] += hsi * dnx * ll;
                dr[i] += gkr * ll;
                di[i] += gki * ll;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        vr[i] = warp_sum(vr[i]);
        vi[i] = warp_sum(vi[i]);
        kr_[i] = warp_sum(kr_[i]);
        ki_[i] = warp_sum(ki_[i]);
        tr_[i] = warp_sum(tr_[i]);
        ti_[i] = warp_sum(ti_[i]);
        dr[i] = warp_sum(dr[i]);
        di[i] = warp_sum(di[i]);
    }
    dcr = warp_sum(dcr);
    dci = warp_sum(dci);
    if (lane == 0) {
        double2 *o = out + 36 * (size_t)pi;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const int A = pt[a], B = ps[b], i = 3 * a + b, j = 3 * A + B;
                const double *ca = gt + 4 + 3 * A, *cb = gs + 4 + 3 * B;
                const double cc = ca[0] * cb[0] + ca[1] * cb[1] + ca[2] * cb[2];
                o[j] = cd(vr[i], vi[i]);
                o[9 + j] = cd(kr_[i], ki_[i]);
                o[18 + j] = cd(tr_[i], ti_[i]);
                o[27 + j] = cd(dcr * cc - nn * dr[i], dci * cc - nn * di[i]);
            }
    }
}

// CSR value of entry e = sum of its contributions (pair * 9 + 3 A + B).
__global__ void near_csr_kernel(int nnz, const int *__restrict__ cptr, const int *__restrict__ cidx,
                                const double2 *__restrict__ buf, double2 *__restrict__ val) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    double2 s[4] = {cd(0, 0), cd(0, 0), cd(0, 0), cd(0, 0)};
    for (int k = cptr[e]; k < cptr[e + 1]; ++k) {
        const long long c = cidx[k];
        const long long pair = c / 9, ab = c % 9;
        const double2 *b = buf + 36 * pair + ab;
        for (int o = 0; o < 4; ++o) s[o] = cadd(s[o], b[9 * o]);
    }
    for (int o = 0; o < 4; ++o) val[4 * (size_t)e + o] = s[o];
}

// ---------------------------------------------------------------------------
// dense FP64 system (assembled path): far pairs with the 6-point rule,
// accumulated with FP64 atomics.  Each unordered pair {t, s} (t < s, sharing
// no vertex) is evaluated once and written in both orientations: V and D are
// symmetric in (x, y), and with the point roles swapped the K integrand of
// the reversed pair is minus the T integrand of the forward pair (and vice
// versa), so the reversed 3x3 blocks are V^T, -T^T, -K^T, D^T.
// Six threads per pair, one per test point p: each sums over the source
// points q into the three source vertices (Z_p[b] = sum_q phi_b(y_q) w_pq f_pq),
// the six partial rows meet in shared memory, and block entry (a, b) is
// sum_p phi_a(x_p) Z_p[b] (the 6x6 -> 3x3 contraction done in two steps).
// ---------------------------------------------------------------------------
constexpr double kDa1 = 0.445948490915965, kDw1 = 0.223381589678011;
constexpr double kDa2 = 0.091576213509771, kDw2 = 0.109951743655322;
constexpr int DA_PAIRS = 16;  // triangle pairs per block (6 threads each)

// Deterministic accumulation of the dense matrix without atomics.  The
// triangles are coloured so that no two of one colour share a vertex; the
// unordered far pairs are visited colour pair by colour pair (ca <= cb, one
// launch each).  Within a launch every matrix entry (row of a vertex of the
// test triangle, column of a vertex of the source triangle) then has at most
// one contributing pair, so the kernel adds with plain loads and stores.
// For ca == cb the pair's reverse orientation (test s, source t) is written
// in the same launch: an entry gets a forward contribution only from the
// pair whose first triangle has the smaller index in the colour list and a
// reverse one only from the other order, never both.  For ca < cb the reverse
// values go to a stash and a second launch (dense_reverse_kernel) adds them.
// Every entry therefore receives its contributions in a fixed order and the
// assembled matrix is the same bit for bit from run to run.
struct DenseSched {
    const int *la, *lb;  // triangles of colour ca and cb
    int na, nb;
    int diag;            // ca == cb
    double2 *stash;      // ca < cb: [na * nb][9][4] reverse values
};

// pair of launch block (bx, by), slot lp: triangles t (from la), s (from lb)
// and the stash row; false when out of range
__device__ __forceinline__ bool dense_pair(const DenseSched &sc, int lp, int &t, int &s, long long &row) {
    if (sc.diag) {  // folded triangular enumeration of i < k within one list
        int i, k;
        if (!dense_diag_pair((int)blockIdx.y, (long long)blockIdx.x * DA_PAIRS + lp, sc.na, &i, &k)) return false;
        t = sc.la[i];
        s = sc.la[k];
        row = -1;
        return true;
    }
    const int i = blockIdx.y;
    const int k = blockIdx.x * DA_PAIRS + lp;
    if (i >= sc.na || k >= sc.nb) return false;
    t = sc.la[i];
    s = sc.lb[k];
    row = (long long)i * sc.nb + k;
    return true;
}

// Adds the values of entry (a, b) of pair (t, s) to the four blocks, forward
// and (same launch, or stashed) reversed; reversed K and T blocks are the
// negated T and K values.
// Adds v to the entry: within one launch every entry has at most one
// writer (the colour-pair schedule), so the sum of each entry forms in the
// fixed launch order whichever way the add is issued; OSRC_DENSE_RED issues
// it as a reduction (no value returned) instead of a load and a store.
#ifndef OSRC_DENSE_RED
#define OSRC_DENSE_RED 1
#endif
__device__ __forceinline__ void dense_add(double2 *q, double x, double y) {
#if OSRC_DENSE_RED
    atomicAdd(&q->x, x);
    atomicAdd(&q->y, y);
#else
    q->x += x;
    q->y += y;
#endif
}

__device__ __forceinline__ void dense_emit(const DenseSched &sc, long long row, int e, double2 *__restrict__ A,
                                           int nv, size_t ra, size_t rb, double2 v, double2 k, double2 tt,
                                           double2 dd) {
    const size_t n2 = 2 * (size_t)nv;
    dense_add(&A[ra * n2 + rb], v.x, v.y);
    dense_add(&A[ra * n2 + nv + rb], k.x, k.y);
    dense_add(&A[(nv + ra) * n2 + rb], tt.x, tt.y);
    dense_add(&A[(nv + ra) * n2 + nv + rb], dd.x, dd.y);
    if (sc.diag) {
        dense_add(&A[rb * n2 + ra], v.x, v.y);
        dense_add(&A[rb * n2 + nv + ra], -tt.x, -tt.y);
        dense_add(&A[(nv + rb) * n2 + ra], -k.x, -k.y);
        dense_add(&A[(nv + rb) * n2 + nv + ra], dd.x, dd.y);
    } else {
        double2 *o = sc.stash + (row * 9 + e) * 4;
        o[0] = v;
        o[1] = cd(-tt.x, -tt.y);
        o[2] = cd(-k.x, -k.y);
        o[3] = dd;
    }
}

// zero stash rows of pairs that contribute nothing (touching pairs), so that
// the reverse launch can add every row
__device__ __forceinline__ void dense_emit_zero(const DenseSched &sc, long long row, int p) {
    if (sc.diag) return;
    for (int e = p; e < 9; e += 6) {
        double2 *o = sc.stash + (row * 9 + e) * 4;
        o[0] = o[1] = o[2] = o[3] = cd(0, 0);
    }
}

// Reverse orientation of colour pair (ca < cb): entry (vertex b of s, vertex
// a of t) of the four blocks, one thread per (pair, entry).
__global__ void dense_reverse_kernel(int nv, const int *__restrict__ tris, DenseSched sc,
                                     double2 *__restrict__ A) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long npairs = (long long)sc.na * sc.nb;
    if (g >= npairs * 9) return;
    const long long row = g / 9;
    const int e = (int)(g - row * 9);
    const int i = (int)(row / sc.nb), k = (int)(row - (long long)i * sc.nb);
    const int t = sc.la[i], s = sc.lb[k];
    const size_t ra = tris[3 * t + e / 3], rb = tris[3 * s + e % 3];
    const size_t n2 = 2 * (size_t)nv;
    const double2 *o = sc.stash + g * 4;
    dense_add(&A[rb * n2 + ra], o[0].x, o[0].y);
    dense_add(&A[rb * n2 + nv + ra], o[1].x, o[1].y);
    dense_add(&A[(nv + rb) * n2 + ra], o[2].x, o[2].y);
    dense_add(&A[(nv + rb) * n2 + nv + ra], o[3].x, o[3].y);
}

__device__ __forceinline__ double dense_bary(int q, int j) {
    const double a = q < 3 ? kDa1 : kDa2;
    return (j == q % 3) ? 1.0 - 2.0 * a : a;
}

__device__ __forceinline__ double dense_w(int q) { return q < 3 ? kDw1 : kDw2; }

// One launch per colour pair (DenseSched): each unordered far pair once, six
// threads per pair (one per test rule point).
__global__ void __launch_bounds__(DA_PAIRS * 6)
dense_far_kernel(int nv, int nt, const double *__restrict__ verts, const int *__restrict__ tris,
                 const double *__restrict__ tgeo, NearConst c, DenseSched sc, double2 *__restrict__ A) {
    __shared__ double2 zs[DA_PAIRS][6][13];  // per pair, per test point: V[3], K[3], T[3], D[3], dc
    const int lp = threadIdx.x / 6, p = threadIdx.x % 6;
    int t = -1, s = -1;
    long long row = -1;
    const bool inrange = dense_pair(sc, lp, t, s, row);
    bool live = inrange;
    int vt[3] = {0, 0, 0}, vs[3] = {0, 0, 0};
    if (live) {
        for (int a = 0; a < 3; ++a) {
            vt[a] = tris[3 * t + a];
            vs[a] = tris[3 * s + a];
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                if (vt[a] == vs[b]) live = false;  // touching: near field
    }
    const double *gt = tgeo + 16 * (size_t)(live ? t : 0), *gs = tgeo + 16 * (size_t)(live ? s : 0);
    // disjoint objects: the pair's object material; interior terms only
    // within one object
    double k1 = c.k1, rho = c.rho, on1 = c.sgn, k1i = c.k1i;
    if (c.obj && live) {
        const int ct = c.tcomp[t], cs = c.tcomp[s];
        const ObjMat o = c.obj[ct];
        k1 = o.k1;
        rho = o.rho;
        k1i = o.k1i;
        if (ct != cs) on1 = 0.0;
    }
    double2 Z[13];
    for (int i = 0; i < 13; ++i) Z[i] = cd(0, 0);
    if (live) {
        double X[3], Vs[3][3];
        for (int k = 0; k < 3; ++k)
            for (int b = 0; b < 3; ++b) Vs[b][k] = verts[3 * vs[b] + k];
        for (int k = 0; k < 3; ++k)
            X[k] = dense_bary(p, 0) * verts[3 * vt[0] + k] + dense_bary(p, 1) * verts[3 * vt[1] + k] +
                   dense_bary(p, 2) * verts[3 * vt[2] + k];
        const double scale = gt[0] * gs[0] * dense_w(p);
        const double dk0 = c.k0 * c.k0, dk1 = (k1 * k1 - k1i * k1i) / rho, dk1i = 2.0 * k1 * k1i / rho;
        for (int q = 0; q < 6; ++q) {
            const double b0 = dense_bary(q, 0), b1 = dense_bary(q, 1), b2 = dense_bary(q, 2);
            const double d0 = X[0] - (b0 * Vs[0][0] + b1 * Vs[1][0] + b2 * Vs[2][0]);
            const double d1 = X[1] - (b0 * Vs[0][1] + b1 * Vs[1][1] + b2 * Vs[2][1]);
            const double d2 = X[2] - (b0 * Vs[0][2] + b1 * Vs[1][2] + b2 * Vs[2][2]);
            const double w = dense_w(q) * scale;
            const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2), ri = 1.0 / r;
            double s0, c0, s1, c1;
            sincos(c.k0 * r, &s0, &c0);
            sincos(k1 * r, &s1, &c1);
            const double br = k1i * r, damp = on1 * (k1i != 0.0 ? exp(-br) : 1.0);
            s1 *= damp;
            c1 *= damp;
            const double kr0 = c.k0 * r, kr1 = k1 * r;
            const double fw = kInv4Pi * ri * w, f3 = fw * ri * ri;
            const double2 g0 = cd(c0 * fw, s0 * fw), g1 = cd(c1 * fw, s1 * fw);
            const double2 hs = cd((-c0 - kr0 * s0 - c1 - kr1 * s1 - br * c1) * f3,
                                  (kr0 * c0 - s0 + kr1 * c1 - s1 - br * s1) * f3);
            const double2 gp = cadd(g0, cscale(g1, rho));
            const double2 gk = cadd(cscale(g0, dk0), cmul(g1, cd(dk1, dk1i)));
            const double2 hk = cscale(hs, d0 * gs[1] + d1 * gs[2] + d2 * gs[3]);  // -hs (y - x).n_y
            const double2 ht = cscale(hs, d0 * gt[1] + d1 * gt[2] + d2 * gt[3]);  //  hs (x - y).n_x
            Z[12] = cadd(Z[12], cadd(g0, cscale(g1, 1.0 / rho)));
            const double bq[3] = {b0, b1, b2};
            for (int b = 0; b < 3; ++b) {
                Z[b] = cadd(Z[b], cscale(gp, bq[b]));
                Z[3 + b] = cadd(Z[3 + b], cscale(hk, bq[b]));
                Z[6 + b] = cadd(Z[6 + b], cscale(ht, bq[b]));
                Z[9 + b] = cadd(Z[9 + b], cscale(gk, bq[b]));
            }
        }
    }
    for (int i = 0; i < 13; ++i) zs[lp][p][i] = Z[i];
    __syncthreads();
    if (!live) {
        if (inrange) dense_emit_zero(sc, row, p);
        return;
    }
    const double nn = gt[1] * gs[1] + gt[2] * gs[2] + gt[3] * gs[3];
    double2 dc = cd(0, 0);
    for (int pp = 0; pp < 6; ++pp) dc = cadd(dc, zs[lp][pp][12]);
    // thread p writes entries (a, b) = (e / 3, e % 3) for e = p, p + 6 (the 9
    // entries of the four blocks: 36 values over 6 threads)
    for (int e = p; e < 9; e += 6) {
        const int a = e / 3, b = e % 3;
        double2 v = cd(0, 0), k = cd(0, 0), tt = cd(0, 0), d = cd(0, 0);
        for (int pp = 0; pp < 6; ++pp) {
            const double ba = dense_bary(pp, a);
            v = cadd(v, cscale(zs[lp][pp][b], ba));
            k = cadd(k, cscale(zs[lp][pp][3 + b], ba));
            tt = cadd(tt, cscale(zs[lp][pp][6 + b], ba));
            d = cadd(d, cscale(zs[lp][pp][9 + b], ba));
        }
        const double *ca = gt + 4 + 3 * a, *cb = gs + 4 + 3 * b;
        const double cc = ca[0] * cb[0] + ca[1] * cb[1] + ca[2] * cb[2];
        const double2 dd = csub(cscale(dc, cc), cscale(d, nn));
        dense_emit(sc, row, e, A, nv, vt[a], vs[b], v, k, tt, dd);
    }
}

// ---------------------------------------------------------------------------
// The same dense far-pair assembly in float-float arithmetic (ffmath.cuh,
// about 48 significant bits) on the FP32 pipes, which on this part issue
// 64 times the FP64 rate.  Same pairs, threads, contraction and FP64
// atomics as dense_far_kernel; the geometry comes from a per-triangle
// float-float table (area, normal, surface curls, the six rule points) and
// the phases k r from float-float sine / cosine.  Lossless materials only.
// ---------------------------------------------------------------------------
constexpr int DFF_GEOM = 31;  // float-float values per triangle in the table

struct FFMat {
    ff k1, rho, irho, dk1;  // interior wavenumber, rho, 1/rho, k1^2 / rho
};

struct DenseFFConst {
    ff k0, dk0, inv4pi;
    FFMat m;             // the material (one object)
    const FFMat *obj;    // disjoint objects: material per object (else m)
    const int *tcomp;    // object of each triangle
    float sgn;           // sign of the interior terms: +1 PMCHWT, -1 Mueller
};

// Per triangle: [0] area, [1..3] unit normal, [4..12] the surface curls of
// the three hat functions, [13..30] the six rule points (x, y, z each).
__global__ void dense_geom_ff_kernel(int nt, const double *__restrict__ verts, const int *__restrict__ tris,
                                     const double *__restrict__ tgeo, ff *__restrict__ G) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    ff *o = G + DFF_GEOM * (size_t)t;
    for (int i = 0; i < 13; ++i) o[i] = ff_make(tgeo[16 * (size_t)t + i]);
    for (int p = 0; p < 6; ++p)
        for (int k = 0; k < 3; ++k) {
            const double x = dense_bary(p, 0) * verts[3 * tris[3 * t] + k] +
                             dense_bary(p, 1) * verts[3 * tris[3 * t + 1] + k] +
                             dense_bary(p, 2) * verts[3 * tris[3 * t + 2] + k];
            o[13 + 3 * p + k] = ff_make(x);
        }
}

__global__ void __launch_bounds__(DA_PAIRS * 6)
dense_far_ff_kernel(int nv, int nt, const int *__restrict__ tris, const ff *__restrict__ G, DenseFFConst c,
                    DenseSched sc, double2 *__restrict__ A) {
    // complex values as ff2 with (re, im) in the two lanes
    __shared__ ff2 zs[DA_PAIRS][6][13];  // per pair, per test point: V[3], K[3], T[3], D[3], dc
    const int lp = threadIdx.x / 6, p = threadIdx.x % 6;
    int t = -1, s = -1;
    long long row = -1;
    const bool inrange = dense_pair(sc, lp, t, s, row);
    bool live = inrange;
    int vt[3] = {0, 0, 0}, vs[3] = {0, 0, 0};
    if (live) {
        for (int a = 0; a < 3; ++a) {
            vt[a] = tris[3 * t + a];
            vs[a] = tris[3 * s + a];
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                if (vt[a] == vs[b]) live = false;  // touching: near field
    }
    const ff *gt = G + DFF_GEOM * (size_t)(live ? t : 0), *gs = G + DFF_GEOM * (size_t)(live ? s : 0);
    // rule constants (kDw*, kDa*, 1 - 2 kDa* split into float pairs): weights
    // and the two barycentric values of each orbit
    const ff w1{0.22338159382343292f, -4.1454217836189855e-09f}, w2{0.10995174199342728f, 1.6618947329405387e-09f};
    const ff a1{0.4459484815597534f, 9.356211805311432e-09f}, a2{0.09157621115446091f, 2.355310169122049e-09f};
    const ff b1{0.10810301452875137f, 3.6393186242378306e-09f}, b2{0.816847562789917f, 1.0190540855603558e-08f};
    FFMat m = c.m;
    float on1 = c.sgn;
    if (c.obj && live) {
        const int ct = c.tcomp[t], cs = c.tcomp[s];
        m = c.obj[ct];
        if (ct != cs) on1 = 0.f;
    }
    const ff2 zero{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    ff2 Z[13];
    for (int i = 0; i < 13; ++i) Z[i] = zero;
    if (live) {
        const ff X[3] = {gt[13 + 3 * p], gt[14 + 3 * p], gt[15 + 3 * p]};
        const ff scale = ff_mul(ff_mul(gt[0], gs[0]), p < 3 ? w1 : w2);
        const ff2 k01 = ff2_make(c.k0, m.k1);
#pragma unroll 1
        for (int q = 0; q < 6; ++q) {  // not unrolled: the body is long enough
            const ff d[3] = {ff_sub(X[0], gs[13 + 3 * q]), ff_sub(X[1], gs[14 + 3 * q]),
                             ff_sub(X[2], gs[15 + 3 * q])};
            const ff r = ff_sqrt(ff_dot3(d, d));
            const ff ri = ff_rcp(r);
            const ff2 kr = ff2_mul(k01, ff2_dup(r));  // (k0 r, k1 r)
            ff2 sn, cs;                               // (sin k0 r, sin k1 r), (cos ..)
            ff2_sincos(kr, sn, cs);
            sn.hi.y *= on1;
            sn.lo.y *= on1;
            cs.hi.y *= on1;
            cs.lo.y *= on1;
            const ff fw = ff_mul(ff_mul(c.inv4pi, ri), ff_mul(q < 3 ? w1 : w2, scale));
            const ff f3 = ff_mul(ff_mul(fw, ri), ri);
            const ff2 fw2 = ff2_dup(fw);
            const ff2 cw = ff2_mul(cs, fw2), sw = ff2_mul(sn, fw2);
            const ff2 g0 = ff2_make(ff2_x(cw), ff2_x(sw)), g1 = ff2_make(ff2_y(cw), ff2_y(sw));
            // H = e^{ikr}(ikr - 1)/r^3 summed over both wavenumbers, negated:
            // re = -(sum c + kr s) f3, im = (sum kr c - s) f3
            const ff2 ha = ff2_fma(kr, sn, cs), hb = ff2_sub(ff2_mul(kr, cs), sn);
            const ff2 hs = ff2_mul(ff2_make(ff_neg(ff_add(ff2_x(ha), ff2_y(ha))), ff_add(ff2_x(hb), ff2_y(hb))),
                                   ff2_dup(f3));
            const ff2 gp = ff2_fma(ff2_dup(m.rho), g1, g0);
            const ff2 gk = ff2_fma(ff2_dup(m.dk1), g1, ff2_mul(ff2_dup(c.dk0), g0));
            const ff2 hk = ff2_mul(hs, ff2_dup(ff_dot3(d, gs + 1)));  // -hs (y - x).n_y
            const ff2 ht = ff2_mul(hs, ff2_dup(ff_dot3(d, gt + 1)));  //  hs (x - y).n_x
            Z[12] = ff2_add(Z[12], ff2_fma(ff2_dup(m.irho), g1, g0));
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const ff2 bq = ff2_dup((b == q % 3) ? (q < 3 ? b1 : b2) : (q < 3 ? a1 : a2));
                Z[b] = ff2_fma(bq, gp, Z[b]);
                Z[3 + b] = ff2_fma(bq, hk, Z[3 + b]);
                Z[6 + b] = ff2_fma(bq, ht, Z[6 + b]);
                Z[9 + b] = ff2_fma(bq, gk, Z[9 + b]);
            }
        }
    }
    for (int i = 0; i < 13; ++i) zs[lp][p][i] = Z[i];
    __syncthreads();
    if (!live) {
        if (inrange) dense_emit_zero(sc, row, p);
        return;
    }
    const ff nn = ff_dot3(gt + 1, gs + 1);
    ff2 dc = zs[lp][0][12];
    for (int pp = 1; pp < 6; ++pp) dc = ff2_add(dc, zs[lp][pp][12]);
    for (int e = p; e < 9; e += 6) {
        const int a = e / 3, b = e % 3;
        ff2 v = zero, k = zero, tt = zero, d = zero;
        for (int pp = 0; pp < 6; ++pp) {
            const ff2 ba = ff2_dup((a == pp % 3) ? (pp < 3 ? b1 : b2) : (pp < 3 ? a1 : a2));
            v = ff2_fma(ba, zs[lp][pp][b], v);
            k = ff2_fma(ba, zs[lp][pp][3 + b], k);
            tt = ff2_fma(ba, zs[lp][pp][6 + b], tt);
            d = ff2_fma(ba, zs[lp][pp][9 + b], d);
        }
        const ff cc = ff_dot3(gt + 4 + 3 * a, gs + 4 + 3 * b);
        const ff2 dd = ff2_sub(ff2_mul(dc, ff2_dup(cc)), ff2_mul(d, ff2_dup(nn)));
        const double vx = ff_to_double(ff2_x(v)), vy = ff_to_double(ff2_y(v));
        const double kx = ff_to_double(ff2_x(k)), ky = ff_to_double(ff2_y(k));
        const double tx = ff_to_double(ff2_x(tt)), ty = ff_to_double(ff2_y(tt));
        const double dx = ff_to_double(ff2_x(dd)), dy = ff_to_double(ff2_y(dd));
        dense_emit(sc, row, e, A, nv, vt[a], vs[b], cd(vx, vy), cd(kx, ky), cd(tx, ty), cd(dx, dy));
    }
}

// Adds the near CSR blocks into the dense matrix (one thread per vertex row).
__global__ void dense_add_near_kernel(int nv, const int *__restrict__ ptr, const int *__restrict__ col,
                                      const double2 *__restrict__ val, double2 *__restrict__ A) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const size_t n2 = 2 * (size_t)nv;
    for (int e = ptr[v]; e < ptr[v + 1]; ++e) {
        const int j = col[e];
        const double2 *B = val + 4 * (size_t)e;
        A[(size_t)v * n2 + j] = cadd(A[(size_t)v * n2 + j], B[0]);
        A[(size_t)v * n2 + nv + j] = cadd(A[(size_t)v * n2 + nv + j], B[1]);
        A[(size_t)(nv + v) * n2 + j] = cadd(A[(size_t)(nv + v) * n2 + j], B[2]);
        A[(size_t)(nv + v) * n2 + nv + j] = cadd(A[(size_t)(nv + v) * n2 + nv + j], B[3]);
    }
}

// y = A x, one warp per row, coalesced row reads.
__global__ void dense_gemv_kernel(int n, const double2 *__restrict__ A, const double2 *__restrict__ x,
                                  double2 *__restrict__ y) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const double2 *a = A + (size_t)row * n;
    // four independent loads in flight per lane (the row is streamed once)
    double sr[4] = {0.0, 0.0, 0.0, 0.0}, si[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j0 = lane; j0 < n; j0 += 128) {
        double2 u[4], v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = j0 + 32 * k;
            u[k] = j < n ? __ldcs(a + j) : cd(0, 0);
            v[k] = j < n ? x[j] : cd(0, 0);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            sr[k] += u[k].x * v[k].x - u[k].y * v[k].y;
            si[k] += u[k].x * v[k].y + u[k].y * v[k].x;
        }
    }
    double tr = (sr[0] + sr[1]) + (sr[2] + sr[3]), ti = (si[0] + si[1]) + (si[2] + si[3]);
    tr = warp_sum(tr);
    ti = warp_sum(ti);
    if (lane == 0) y[row] = cd(tr, ti);
}

// Gauss-Legendre nodes and weights on [0,1] (Newton on the three-term
// recurrence of the Legendre polynomials).
void gauss_legendre01(int n, double *x, double *w) {
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double pm = 1.0, pc = z;
            for (int j = 2; j <= n; ++j) {
                const double pn = ((2.0 * j - 1.0) * z * pc - (j - 1.0) * pm) / j;
                pm = pc;
                pc = pn;
            }
            if (n == 1) { pc = z; pm = 1.0; }
            dp = n * (z * pc - pm) / (z * z - 1.0);
            const double dz = pc / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double pm = 1.0, pc = z;
        for (int j = 2; j <= n; ++j) {
            const double pn = ((2.0 * j - 1.0) * z * pc - (j - 1.0) * pm) / j;
            pm = pc;
            pc = pn;
        }
        if (n == 1) { pc = z; pm = 1.0; }
        dp = n * (z * pc - pm) / (z * z - 1.0);
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
}

}  // namespace

int near_build(osrc_problem *pb, const std::vector<NearPair> &pairs,
               const std::vector<int> &cptr, const std::vector<int> &cidx, cudaStream_t st) {
    osrc_mesh *m = pb->mesh;
    osrc_ctx *ctx = m->ctx;
    const long long np = (long long)pairs.size();
    pb->near_pairs = np;
    const int nnz = pb->near_nnz;
    DBuf<NearPair> d_pairs;
    DBuf<double2> d_buf;
    DBuf<int> d_cptr, d_cidx;
    DBuf<double> d_gl;
    OSRC_TRY(d_pairs.alloc(ctx, np));
    OSRC_TRY(d_buf.alloc(ctx, 36 * (size_t)np));
    OSRC_TRY(d_cptr.alloc(ctx, cptr.size()));
    OSRC_TRY(d_cidx.alloc(ctx, cidx.size()));
    OSRC_TRY(d_gl.alloc(ctx, 32));
    OSRC_TRY(pb->d_nr_val.alloc(ctx, 4 * (size_t)nnz));
    double gl[32] = {0};
    gauss_legendre01(pb->p.n_ss, gl, gl + 16);
    OSRC_CK(cudaMemcpyAsync(d_pairs.p, pairs.data(), np * sizeof(NearPair), cudaMemcpyHostToDevice, st));
    OSRC_CK(cudaMemcpyAsync(d_cptr.p, cptr.data(), cptr.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    OSRC_CK(cudaMemcpyAsync(d_cidx.p, cidx.data(), cidx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    OSRC_CK(cudaMemcpyAsync(d_gl.p, gl, sizeof(gl), cudaMemcpyHostToDevice, st));
    NearConst c{pb->p.k_ext, pb->p.k_int, pb->p.rho_ratio, pb->p.n_ss, pb->multi ? pb->d_obj.p : nullptr,
                 pb->mesh->d_tcomp.p, pb->p.formulation == OSRC_MULLER ? -1.0 : 1.0, pb->p.k_int_im};
    const long long blocks = (np + NEAR_WARPS - 1) / NEAR_WARPS;
    if (blocks > 0) {
        near_ss_kernel<<<(unsigned)blocks, 32 * NEAR_WARPS, 0, st>>>(
            d_pairs.p, np, m->d_verts.p, m->d_tris.p, pb->d_tgeo.p, d_gl.p, c, d_buf.p);
        pb->launches++;
        OSRC_CK(cudaGetLastError());
    }
    if (nnz > 0) {
        near_csr_kernel<<<(nnz + 255) / 256, 256, 0, st>>>(nnz, d_cptr.p, d_cidx.p, d_buf.p,
                                                           pb->d_nr_val.p);
        pb->launches++;
        OSRC_CK(cudaGetLastError());
    }
    // the temporaries are released when this function returns: finish first
    OSRC_CK(cudaStreamSynchronize(st));
    return OSRC_OK;
}

int dense_assemble(osrc_problem *pb, cudaStream_t st) {
    osrc_mesh *m = pb->mesh;
    const int nv = pb->nv, nt = pb->nt;
    const size_t n2 = 2 * (size_t)nv;
    OSRC_TRY(pb->d_dense.alloc(m->ctx, n2 * n2));
    OSRC_CK(cudaMemsetAsync(pb->d_dense.p, 0, n2 * n2 * sizeof(double2), st));
    NearConst c{pb->p.k_ext, pb->p.k_int, pb->p.rho_ratio, pb->p.n_ss, pb->multi ? pb->d_obj.p : nullptr,
                 pb->mesh->d_tcomp.p, pb->p.formulation == OSRC_MULLER ? -1.0 : 1.0, pb->p.k_int_im};
    // colours: greedy, in triangle order, so that triangles sharing a vertex
    // differ; lists of each colour's triangles (ascending)
    std::vector<int> col;
    const int ncol = dense_colour(nt, m->tris.data(), m->vt_ptr.data(), m->vt_idx.data(), col);
    std::vector<int> cbeg(ncol + 1, 0), order(nt);
    for (int t = 0; t < nt; ++t) cbeg[col[t] + 1]++;
    for (int c = 0; c < ncol; ++c) cbeg[c + 1] += cbeg[c];
    {
        std::vector<int> fill(cbeg.begin(), cbeg.end() - 1);
        for (int t = 0; t < nt; ++t) order[fill[col[t]]++] = t;
    }
    int cmax = 0;
    for (int c = 0; c < ncol; ++c) cmax = std::max(cmax, cbeg[c + 1] - cbeg[c]);
    if ((cmax + 1) / 2 > 65535) {
        osrc_set_error("dense assembly: too many triangles for the dense path");
        return OSRC_UNSUPPORTED;
    }
    DBuf<int> d_order;
    DBuf<double2> stash;
    OSRC_TRY(d_order.alloc(m->ctx, nt));
    OSRC_CK(cudaMemcpyAsync(d_order.p, order.data(), nt * sizeof(int), cudaMemcpyHostToDevice, st));
    if (ncol > 1) OSRC_TRY(stash.alloc(m->ctx, (size_t)cmax * cmax * 36));
    // launches: colour pairs in a fixed order; launch(sched) runs one pair
    // kernel, then the stashed reverse values for ca < cb
    auto for_each_pair = [&](auto launch) -> int {
        for (int ca = 0; ca < ncol; ++ca)
            for (int cb = ca; cb < ncol; ++cb) {
                DenseSched sc{};
                sc.la = d_order.p + cbeg[ca];
                sc.lb = d_order.p + cbeg[cb];
                sc.na = cbeg[ca + 1] - cbeg[ca];
                sc.nb = cbeg[cb + 1] - cbeg[cb];
                sc.diag = ca == cb;
                sc.stash = stash.p;
                if (sc.diag && sc.na < 2) continue;
                if (sc.na < 1 || sc.nb < 1) continue;
                const dim3 grid = sc.diag ? dim3((unsigned)((sc.na - 1 + DA_PAIRS - 1) / DA_PAIRS),
                                                 (unsigned)((sc.na + 1) / 2))
                                          : dim3((unsigned)((sc.nb + DA_PAIRS - 1) / DA_PAIRS), (unsigned)sc.na);
                launch(sc, grid);
                pb->launches++;
                if (!sc.diag) {
                    const long long work = (long long)sc.na * sc.nb * 9;
                    dense_reverse_kernel<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(nv, m->d_tris.p, sc,
                                                                                          pb->d_dense.p);
                    pb->launches++;
                }
                OSRC_CK(cudaGetLastError());
            }
        return OSRC_OK;
    };
    // float-float assembly on request, for lossless materials
    const bool use_ff = pb->p.dense_assembly == OSRC_ASSEMBLE_FF && !pb->absorb;
    DBuf<ff> geo;
    DBuf<FFMat> fobj;
    if (nt > 1 && use_ff) {
        OSRC_TRY(geo.alloc(m->ctx, DFF_GEOM * (size_t)nt));
        dense_geom_ff_kernel<<<(nt + 127) / 128, 128, 0, st>>>(nt, m->d_verts.p, m->d_tris.p, pb->d_tgeo.p,
                                                               geo.p);
        pb->launches++;
        auto mat = [](double k1, double rho) {
            return FFMat{ff_make(k1), ff_make(rho), ff_make(1.0 / rho), ff_make(k1 * k1 / rho)};
        };
        DenseFFConst fc{};
        fc.k0 = ff_make(pb->p.k_ext);
        fc.dk0 = ff_make(pb->p.k_ext * pb->p.k_ext);
        fc.inv4pi = ff_make(kInv4Pi);
        fc.m = mat(pb->p.k_int, pb->p.rho_ratio);
        fc.sgn = pb->p.formulation == OSRC_MULLER ? -1.f : 1.f;
        fc.tcomp = pb->mesh->d_tcomp.p;
        if (pb->multi) {
            std::vector<FFMat> h(pb->obj.size());
            for (size_t i = 0; i < h.size(); ++i) h[i] = mat(pb->obj[i].k1, pb->obj[i].rho);
            OSRC_TRY(fobj.alloc(m->ctx, h.size()));
            OSRC_CK(cudaMemcpyAsync(fobj.p, h.data(), h.size() * sizeof(FFMat), cudaMemcpyHostToDevice, st));
            fc.obj = fobj.p;
        }
        OSRC_TRY(for_each_pair([&](const DenseSched &sc, dim3 grid) {
            dense_far_ff_kernel<<<grid, DA_PAIRS * 6, 0, st>>>(nv, nt, m->d_tris.p, geo.p, fc, sc, pb->d_dense.p);
        }));
    } else if (nt > 1) {
        OSRC_TRY(for_each_pair([&](const DenseSched &sc, dim3 grid) {
            dense_far_kernel<<<grid, DA_PAIRS * 6, 0, st>>>(nv, nt, m->d_verts.p, m->d_tris.p, pb->d_tgeo.p, c, sc,
                                                             pb->d_dense.p);
        }));
    }
    dense_add_near_kernel<<<(nv + 127) / 128, 128, 0, st>>>(nv, pb->d_nr_ptr.p, pb->d_nr_col.p,
                                                            pb->d_nr_val.p, pb->d_dense.p);
    pb->launches++;
    OSRC_CK(cudaGetLastError());
    // the colour lists, stash and float-float tables are released on return
    OSRC_CK(cudaStreamSynchronize(st));
    return OSRC_OK;
}

int dense_apply(osrc_problem *pb, const double2 *x, double2 *y, cudaStream_t st) {
    const int n = 2 * pb->nv;
    dense_gemv_kernel<<<(n + 7) / 8, 256, 0, st>>>(n, pb->d_dense.p, x, y);
    pb->launches++;
    OSRC_CK(cudaGetLastError());
    return OSRC_OK;
}

// Mueller formulation: the identity blocks, + M_ij added to the (1,2) and
// (2,1) entries of the touching-pair CSR (vertices sharing a triangle are
// touching, so every mass entry has a place there).  One thread per row.
__global__ void near_add_mass_kernel(int nv, const int *__restrict__ mptr, const int *__restrict__ mcol,
                                     const double *__restrict__ M, const int *__restrict__ nptr,
                                     const int *__restrict__ ncol, double2 *__restrict__ val) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    for (int e = mptr[i]; e < mptr[i + 1]; ++e) {
        const int j = mcol[e];
        int lo = nptr[i], hi = nptr[i + 1] - 1;
        while (lo < hi) {  // first position with ncol >= j (rows are sorted)
            const int mid = (lo + hi) >> 1;
            if (ncol[mid] < j) lo = mid + 1;
            else hi = mid;
        }
        if (lo < nptr[i + 1] && ncol[lo] == j) {
            val[4 * (size_t)lo + 1].x += M[e];
            val[4 * (size_t)lo + 2].x += M[e];
        }
    }
}

int near_add_mass(osrc_problem *pb, cudaStream_t st) {
    const int nv = pb->nv;
    near_add_mass_kernel<<<(nv + 127) / 128, 128, 0, st>>>(nv, pb->d_ms_ptr.p, pb->d_ms_col.p, pb->d_M.p,
                                                           pb->d_nr_ptr.p, pb->d_nr_col.p, pb->d_nr_val.p);
    pb->launches++;
    OSRC_CK(cudaGetLastError());
    return OSRC_OK;
}
