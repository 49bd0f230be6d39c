// k_far.cu -- matrix-free FP32 far-field apply of the permuted PMCHWT
// operator (Sec. 2.7) for all triangle pairs that share no vertex, with the
// 6-point degree-4 triangle rule (Strang & Fix / Dunavant) on both triangles.
//
// Structure of one apply y = B_far x:
//   1. far_prep_kernel   (per source triangle)  densities at the 6 source
//      points and the surface-curl vector of the phi density, FP32;
//   2. far_kernel        (per test point)       N-body sum over all source
//      points staged through shared memory in tiles of triangles; both
//      wavenumbers are evaluated from one distance; the source range is split
//      over gridDim.y so that the grid fills every SM; partial sums per test
//      point go to d_part (no atomics);
//   3. gather_kernel     (per vertex)           sums the partials of the test
//      points of the incident triangles with the test weights (FP64) and adds
//      the near-field CSR product (touching pairs, Sauter-Schwab values).
//
// Kernel identities (G = e^{ikr}/(4 pi r), d = x - y, r = |d|):
//   dG/dn_y = H (y - x).n_y,  dG/dn_x = H (x - y).n_x,
//   H = e^{ikr} (ikr - 1) / (4 pi r^3);
//   D (Maue form) = G [curl phi_i . curl phi_j - k^2 (n_x.n_y) phi_i phi_j].
// Because every source point of a flat triangle lies in its plane,
// (x - y).n_y = x.n_y - n_y.P0 is constant over the triangle's six points,
// and so is n_x.n_y; the surface curl of the P1 density is constant per
// triangle.  These per-triangle factors are applied once per (test point,
// source triangle), not per point pair.
#include <algorithm>

#include "osrc_internal.cuh"

namespace {

// 6-point symmetric rule: barycentric (1-2a, a, a) and permutations.
constexpr double kQa1 = 0.445948490915965;
constexpr double kQw1 = 0.223381589678011;
constexpr double kQa2 = 0.091576213509771;
constexpr double kQw2 = 0.109951743655322;

__host__ __device__ inline void rule_point(int q, double bary[3], double &w) {
    const double a = q < 3 ? kQa1 : kQa2;
    w = q < 3 ? kQw1 : kQw2;
    const int i = q % 3;
    for (int j = 0; j < 3; ++j) bary[j] = (j == i) ? 1.0 - 2.0 * a : a;
}

constexpr int FAR_THREADS = 128;
// resident blocks per SM the one-right-hand-side kernel is compiled for
// (registers per thread = 65536 / (FAR_THREADS x FAR_MIN_BLOCKS))
#ifndef OSRC_FAR_MIN_BLOCKS
#define OSRC_FAR_MIN_BLOCKS 4
#endif
// largest k_max x (bounding-box diagonal) for the plain (FP32 k r) variant
constexpr double FAR_PLAIN_MAX_PHASE = 32.0 * 3.14159265358979323846;
constexpr int FAR_TS = 64;  // source triangles per shared-memory tile

__global__ void far_geom_kernel(const double *__restrict__ verts, const int *__restrict__ tris,
                                int nt, float4 *__restrict__ pt, float4 *__restrict__ poff,
                                float4 *__restrict__ cen, float4 *__restrict__ tn,
                                int4 *__restrict__ tv, double *__restrict__ tgeo) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double P[3][3];
    int v[3];
    for (int a = 0; a < 3; ++a) {
        v[a] = tris[3 * t + a];
        for (int j = 0; j < 3; ++j) P[a][j] = verts[3 * v[a] + j];
    }
    double e1[3], e2[3], c[3];
    for (int j = 0; j < 3; ++j) {
        e1[j] = P[1][j] - P[0][j];
        e2[j] = P[2][j] - P[0][j];
    }
    c[0] = e1[1] * e2[2] - e1[2] * e2[1];
    c[1] = e1[2] * e2[0] - e1[0] * e2[2];
    c[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double len = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    const double area = 0.5 * len;
    double n[3] = {c[0] / len, c[1] / len, c[2] / len};
    double cc[3];
    for (int j = 0; j < 3; ++j) cc[j] = (P[0][j] + P[1][j] + P[2][j]) / 3.0;
    for (int q = 0; q < 6; ++q) {
        double b[3], w;
        rule_point(q, b, w);
        double x[3];
        for (int j = 0; j < 3; ++j) x[j] = b[0] * P[0][j] + b[1] * P[1][j] + b[2] * P[2][j];
        pt[6 * t + q] = make_float4((float)x[0], (float)x[1], (float)x[2], (float)(w * area));
        poff[6 * t + q] = make_float4((float)(x[0] - cc[0]), (float)(x[1] - cc[1]),
                                      (float)(x[2] - cc[2]), (float)(w * area));
    }
    // centroid as an unevaluated float pair (hi + lo), about 48 significant bits
    float hi[3], lo[3];
    for (int j = 0; j < 3; ++j) {
        hi[j] = (float)cc[j];
        lo[j] = (float)(cc[j] - (double)hi[j]);
    }
    cen[2 * t] = make_float4(hi[0], hi[1], hi[2], 0.f);
    cen[2 * t + 1] = make_float4(lo[0], lo[1], lo[2], 0.f);
    const double h = n[0] * P[0][0] + n[1] * P[0][1] + n[2] * P[0][2];
    tn[t] = make_float4((float)n[0], (float)n[1], (float)n[2], (float)h);
    tv[t] = make_int4(v[0], v[1], v[2], 0);
    double *g = tgeo + 16 * (size_t)t;
    g[0] = area;
    g[1] = n[0];
    g[2] = n[1];
    g[3] = n[2];
    // curl phi_a = n x grad phi_a = (P_{a+1} - P_{a+2}) / (2 area)
    for (int a = 0; a < 3; ++a)
        for (int j = 0; j < 3; ++j)
            g[4 + 3 * a + j] = (P[(a + 1) % 3][j] - P[(a + 2) % 3][j]) / (2.0 * area);
    g[13] = g[14] = g[15] = 0.0;
}

// Source data of one apply, duplicated into (value, value) pairs and stored
// with both signs, so that the far kernel's packed FP32 instructions (two
// test points per thread) take every operand of a complex multiply-add
// straight from shared memory, without moves or negations:
//   sP[5k]   = (-y.x, -y.x, -y.y, -y.y)     sP[5k+1] = (-y.z, -y.z, psi.re, psi.re)
//   sP[5k+2] = (psi.im, psi.im, -psi.re, -psi.re)
//   sP[5k+3] = (-psi.im, -psi.im, phi.re, phi.re)
//   sP[5k+4] = (phi.im, phi.im, -phi.re, -phi.re)   sP5[k] = (-phi.im, -phi.im)
// with psi_q = w_q |s| sum_b lambda_b(q) psi_b (the same for phi); per
// triangle c_s = |s| sum_b phi_b curl phi_b as
//   sC[5t] = (cx.re, cx.re, cx.im, cx.im)   sC[5t+1] = (-cx.im, -cx.im, cy.re, cy.re)
//   sC[5t+2] = (cy.im, cy.im, -cy.im, -cy.im)   sC[5t+3] = (cz.re, cz.re, cz.im, cz.im)
//   sC[5t+4] = (-cz.im, -cz.im, 0, 0)
__global__ void far_prep_kernel(const double2 *__restrict__ x, int nv, int nt,
                                const int *__restrict__ tris, const float4 *__restrict__ pt,
                                const double *__restrict__ tgeo, float4 *__restrict__ sP,
                                float2 *__restrict__ sP5, float4 *__restrict__ sC) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double2 ps[3], ph[3];
    for (int a = 0; a < 3; ++a) {
        const int v = tris[3 * t + a];
        ps[a] = x[v];
        ph[a] = x[nv + v];
    }
    const double *g = tgeo + 16 * (size_t)t;
    const double area = g[0];
    for (int q = 0; q < 6; ++q) {
        double b[3], w;
        rule_point(q, b, w);
        const double W = w * area;
        double2 s = cd(0, 0), f = cd(0, 0);
        for (int a = 0; a < 3; ++a) {
            s = cadd(s, cscale(ps[a], b[a]));
            f = cadd(f, cscale(ph[a], b[a]));
        }
        const float4 p = pt[6 * t + q];
        const float psr = (float)(W * s.x), psi = (float)(W * s.y);
        const float phr = (float)(W * f.x), phi = (float)(W * f.y);
        const size_t k = 6 * (size_t)t + q;
        float4 *d = sP + 5 * k;
        d[0] = make_float4(-p.x, -p.x, -p.y, -p.y);
        d[1] = make_float4(-p.z, -p.z, psr, psr);
        d[2] = make_float4(psi, psi, -psr, -psr);
        d[3] = make_float4(-psi, -psi, phr, phr);
        d[4] = make_float4(phi, phi, -phr, -phr);
        sP5[k] = make_float2(-phi, -phi);
    }
    float cr[3], ci[3];
    for (int j = 0; j < 3; ++j) {
        double2 cv = cd(0, 0);
        for (int a = 0; a < 3; ++a) cv = cadd(cv, cscale(ph[a], g[4 + 3 * a + j]));
        cr[j] = (float)(cv.x * area);
        ci[j] = (float)(cv.y * area);
    }
    float4 *c = sC + 5 * (size_t)t;
    c[0] = make_float4(cr[0], cr[0], ci[0], ci[0]);
    c[1] = make_float4(-ci[0], -ci[0], cr[1], cr[1]);
    c[2] = make_float4(ci[1], ci[1], -ci[1], -ci[1]);
    c[3] = make_float4(cr[2], cr[2], ci[2], ci[2]);
    c[4] = make_float4(-ci[2], -ci[2], 0.f, 0.f);
}

typedef float2 f2;
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ f2 hi2(const float4 &v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ f2 dup2(float a) { return make_float2(a, a); }

// Constants as (value, value) pairs for the packed instructions.  The D
// normal term k0^2 G0 + (k1^2/rho) G1 is evaluated as dks (G0 + dk1 G1):
// dk0 holds the scale dks (applied once per source triangle) and dk1 the
// ratio (k1^2/rho) / dks.
struct FarConst2 {
    f2 k0, k1, nk0, nk1, rho, irho, dk0, dk1;
};

// Accumulators of the two test points of a thread, packed (point a, point b):
// tile sums of u1, u2 (complex) and of the curl vector A (3 complex), and
// the per-source-triangle sums T1n = -sum_q Hs phi_q, U = sum_q Gk phi_q,
// T3 = sum_q w_q Gd.
struct PairAcc {
    f2 u1r, u1i, u2r, u2i, axr, axi, ayr, ayi, azr, azi;
    f2 t1r, t1i, ur, ui, t3r, t3i;
};

// Per (test triangle, source triangle) data of the centred (large k r)
// variant: D = c_x - c_y (centroid difference, FP32 rounding of a
// float-float value), r_c = |D| and the phase k r_c as a fraction of a
// revolution in [-1/2, 1/2], from float-float arithmetic (about 48 bits).
struct CenterPair {
    f2 Dx, Dy, Dz, rc, b0, b1;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float v = s - a;
    e = (a - (s - v)) + (b - v);
}

// a - b for float-float a = (ah, al), b = (bh, bl); result (h, l)
__device__ __forceinline__ void ff_sub(float ah, float al, float bh, float bl, float &h, float &l) {
    float s, e;
    two_sum(ah, -bh, s, e);
    e += al - bl;
    h = s + e;
    l = e - (h - s);
}

// frac(r (kh + kl)) in revolutions for float-float r = (rh, rl)
__device__ __forceinline__ float ff_phase_rev(float rh, float rl, float kh, float kl) {
    const float p = rh * kh;
    const float pe = fmaf(rh, kh, -p) + fmaf(rh, kl, rl * kh);
    const float n = rintf(p);
    return (p - n) + pe;
}

// 1/x to about one ulp (PTX rcp.approx), used where the result scales a
// small quantity
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ CenterPair center_pair(const float4 &cth, const float4 &ctl,
                                                  const float4 &csh, const float4 &csl,
                                                  float k0h, float k0l, float k1h, float k1l) {
    float dh[3], dl[3];
    ff_sub(cth.x, ctl.x, csh.x, csl.x, dh[0], dl[0]);
    ff_sub(cth.y, ctl.y, csh.y, csl.y, dh[1], dl[1]);
    ff_sub(cth.z, ctl.z, csh.z, csl.z, dh[2], dl[2]);
    // |D|^2 as float-float: exact squares of the high parts plus cross terms
    float sh = 0.f, sl = 0.f;
    for (int i = 0; i < 3; ++i) {
        const float p = dh[i] * dh[i];
        const float e = fmaf(dh[i], dh[i], -p) + 2.f * dh[i] * dl[i];
        float s, t;
        two_sum(sh, p, s, t);
        sh = s;
        sl += t + e;
    }
    // square root with one Newton correction (the correction only needs a
    // few significant bits of 1/(2 sqrt(sh)), so approximate rsqrt suffices)
    const float y = rsqrtf(sh);
    const float rs = sh * y;
    const float corr = (fmaf(-rs, rs, sh) + sl) * (0.5f * y);
    const float rh = rs + corr;
    const float rl = corr - (rh - rs);
    CenterPair c;
    c.Dx = dup2(dh[0]);
    c.Dy = dup2(dh[1]);
    c.Dz = dup2(dh[2]);
    c.rc = dup2(rh);
    // reduced centroid phases in radians (in [-pi, pi])
    c.b0 = dup2(6.28318530717958647692f * ff_phase_rev(rh, rl, k0h, k0l));
    c.b1 = dup2(6.28318530717958647692f * ff_phase_rev(rh, rl, k1h, k1l));
    return c;
}

// One source point against the two test points of the thread, both
// wavenumbers, packed FP32 arithmetic.  P[0..4], P5 hold the signed
// duplicated source data; (mnx, mny, mnz) is the negated test-triangle
// normal; wq2 the rule weight.  Plain variant: (X, Y, Z) are the test points
// and the source coordinates absolute; the MUFU sine / cosine take k r
// directly (their own argument scaling has the same FP32 rounding as an
// explicit reduction).  CENTRED variant (large k r): coordinates are offsets
// from the triangle centroids, x - y = D + delta, and the phase is
// k r = k r_c + k (2 D.delta + delta.delta) / (r + r_c) with k r_c reduced in
// float-float arithmetic once per triangle pair.
// MULTI: m1 multiplies the interior terms (0: source on another object, -1:
// Mueller); k1i / dk1i: imaginary parts of k1 and k1^2 / rho (attenuation).
template <bool CENTRED, bool MULTI, bool ABSORB>
__device__ __forceinline__ void far_pair2(f2 X, f2 Y, f2 Z, const float4 *P, const f2 &P5, f2 mnx,
                                          f2 mny, f2 mnz, f2 wq2, const FarConst2 &c,
                                          const CenterPair &cp, f2 m1, f2 k1i, f2 dk1i, PairAcc &A) {
    const float4 P0 = P[0], P1 = P[1], P2 = P[2], P3 = P[3], P4 = P[4];
    f2 dx, dy, dz, ddx, ddy, ddz;
    if (CENTRED) {
        ddx = add2(X, lo2(P0));  // delta = a - b
        ddy = add2(Y, hi2(P0));
        ddz = add2(Z, lo2(P1));
        dx = add2(ddx, cp.Dx);
        dy = add2(ddy, cp.Dy);
        dz = add2(ddz, cp.Dz);
    } else {
        dx = add2(X, lo2(P0));  // x - y
        dy = add2(Y, hi2(P0));
        dz = add2(Z, lo2(P1));
    }
    f2 r2 = mul2(dx, dx);
    r2 = fma2(dy, dy, r2);
    r2 = fma2(dz, dz, r2);
    const f2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const f2 r = mul2(r2, ri);
    const f2 ri2 = mul2(ri, ri);
    f2 dnxn = mul2(dx, mnx);  // (y - x).n_x
    dnxn = fma2(dy, mny, dnxn);
    dnxn = fma2(dz, mnz, dnxn);
    f2 s0, c0, s1, c1;
    if (CENTRED) {
        f2 num = mul2(ddx, ddx);
        num = fma2(ddy, ddy, num);
        num = fma2(ddz, ddz, num);
        f2 dd = mul2(ddx, cp.Dx);
        dd = fma2(ddy, cp.Dy, dd);
        dd = fma2(ddz, cp.Dz, dd);
        num = fma2(dd, dup2(2.f), num);  // r^2 - r_c^2
        const f2 den = add2(r, cp.rc);
        const f2 dlt = mul2(num, make_float2(rcp_approx(den.x), rcp_approx(den.y)));  // r - r_c
        const f2 ph0 = fma2(c.k0, dlt, cp.b0);
        const f2 ph1 = fma2(c.k1, dlt, cp.b1);
        __sincosf(ph0.x, &s0.x, &c0.x);
        __sincosf(ph0.y, &s0.y, &c0.y);
        __sincosf(ph1.x, &s1.x, &c1.x);
        __sincosf(ph1.y, &s1.y, &c1.y);
    } else {
        const f2 kr0 = mul2(r, c.k0), kr1 = mul2(r, c.k1);
        __sincosf(kr0.x, &s0.x, &c0.x);
        __sincosf(kr0.y, &s0.y, &c0.y);
        __sincosf(kr1.x, &s1.x, &c1.x);
        __sincosf(kr1.y, &s1.y, &c1.y);
    }
    f2 br = make_float2(0.f, 0.f);
    constexpr bool absorb = MULTI && ABSORB;
    if (MULTI) {  // e^{i k1 r} with k1 = k1r + i k1i: damping e^{-k1i r}, and m1
        f2 damp = m1;
        if (absorb) {
            br = mul2(r, k1i);
            damp = mul2(m1, make_float2(__expf(-br.x), __expf(-br.y)));
        }
        c1 = mul2(c1, damp);
        s1 = mul2(s1, damp);
    }
    const f2 psr = hi2(P1), psi = lo2(P2), mpsr = hi2(P2), mpsi = lo2(P3);
    const f2 phr = hi2(P3), phi = lo2(P4), mphr = hi2(P4), mphi = P5;
    (void)mpsr;
    (void)mphr;
    // cos and sin scaled by 1/r once: G = (c + i s)/r for every kernel below
    const f2 c0r = mul2(c0, ri), s0r = mul2(s0, ri), c1r = mul2(c1, ri), s1r = mul2(s1, ri);
    // V block (G0 + rho G1) psi, without 1/(4 pi)
    const f2 gpr = fma2(c.rho, c1r, c0r), gpi = fma2(c.rho, s1r, s0r);
    A.u1r = fma2(gpr, psr, fma2(gpi, mpsi, A.u1r));
    A.u1i = fma2(gpr, psi, fma2(gpi, psr, A.u1i));
    // D normal term (k0^2 G0 + k1^2/rho G1) phi, as (G0 + dk1 G1) phi; the
    // scale dks is applied per source triangle
    f2 gkr = fma2(c.dk1, c1r, c0r), gki = fma2(c.dk1, s1r, s0r);
    if (absorb) {  // complex k1^2 / (rho dks)
        gkr = fma2(mul2(dk1i, s1r), dup2(-1.f), gkr);
        gki = fma2(dk1i, c1r, gki);
    }
    A.ur = fma2(gkr, phr, fma2(gki, mphi, A.ur));
    A.ui = fma2(gkr, phi, fma2(gki, phr, A.ui));
    // D curl term: sum_q w_q (G0 + G1/rho)
    A.t3r = fma2(fma2(c.irho, c1r, c0r), wq2, A.t3r);
    A.t3i = fma2(fma2(c.irho, s1r, s0r), wq2, A.t3i);
    // -(H0 + H1), H = e^{ikr} (i k r - 1) / r^3, written with the scaled c, s:
    //   re = (c0/r + c1/r + k0 s0 + k1 s1) / r^2,  im = (s0/r + s1/r - k0 c0 - k1 c1) / r^2
    f2 hp0 = fma2(c.k1, s1, fma2(c.k0, s0, add2(c0r, c1r)));
    f2 hq0 = fma2(c.nk1, c1, fma2(c.nk0, c0, add2(s0r, s1r)));
    if (absorb) {  // (i k1 r - 1) with Im k1: + k1i r (c1, s1) / r
        hp0 = fma2(k1i, c1, hp0);
        hq0 = fma2(k1i, s1, hq0);
    }
    const f2 hp = mul2(hp0, ri2);
    const f2 hq = mul2(hq0, ri2);
    A.t1r = fma2(hp, phr, fma2(hq, mphi, A.t1r));  // T1n = -sum Hs phi
    A.t1i = fma2(hp, phi, fma2(hq, phr, A.t1i));
    // T block: (H0 + H1)(x - y).n_x psi = (-(H0 + H1)) (y - x).n_x psi
    const f2 hxp = mul2(hp, dnxn), hxq = mul2(hq, dnxn);
    A.u2r = fma2(hxp, psr, fma2(hxq, mpsi, A.u2r));
    A.u2i = fma2(hxp, psi, fma2(hxq, psr, A.u2i));
}

// One thread per pair of test points (2j, 2j+1) of test triangle 2j / 6,
// packed into the two lanes of FP32x2 instructions.  Output
// part[(split * 10 + c) * npts + p], c = u1 (re, im), u2 (re, im),
// A (x re, x im, y re, y im, z re, z im):
//   u1 = sum [ (G0 + rho G1) psi_q + (x.n_y - h_y)(H0 + H1) phi_q ]
//   u2 = sum [ (H0 + H1)(x - y).n_x psi_q - (n_x.n_y)(k0^2 G0 + k1^2/rho G1) phi_q ]
//   A  = sum_s (sum_q w_q (G0 + G1/rho)) c_s
// with G, H here without the factor 1/(4 pi) (applied in the gather).  Sums
// run per 64-triangle tile, then tile sums are added to running sums kept in
// part.
// CENTRED: pt holds offsets from the test-triangle centroid and cen the
// float-float centroids (see far_pair2).
// MULTI: disjoint objects (Sec. 2.2) or the Mueller formulation; the interior
// constants are the test triangle's object's, interior terms vanish for
// sources on other objects and change sign for Mueller.  ABSORB (with MULTI):
// complex interior wavenumbers (attenuation).
template <bool CENTRED, bool MULTI, bool ABSORB>
__global__ void __launch_bounds__(FAR_THREADS, OSRC_FAR_MIN_BLOCKS)
far_kernel(const float4 *__restrict__ pt, const float4 *__restrict__ cen,
           const float4 *__restrict__ tn, const int4 *__restrict__ tv,
           const float4 *__restrict__ sP, const float2 *__restrict__ sP5,
           const float4 *__restrict__ sC, int nt, int npts, int tris_per_split, FarConst2 c0,
           float4 kff0, const int *__restrict__ tcomp, const FarObj *__restrict__ fobj,
           float *__restrict__ part) {
    __shared__ float4 shP[FAR_TS * 6 * 5];
    __shared__ float2 shP5[FAR_TS * 6];
    __shared__ float4 shN[FAR_TS];
    __shared__ float4 shC[FAR_TS * 5];
    __shared__ int4 shV[FAR_TS];
    __shared__ float4 shCen[CENTRED ? 2 * FAR_TS : 1];
    __shared__ int shComp[MULTI ? FAR_TS : 1];

    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int split = blockIdx.y;
    const int s_begin = split * tris_per_split;
    const int s_end = min(nt, s_begin + tris_per_split);
    const bool active = 2 * j < npts;
    const int p0 = active ? 2 * j : 0;
    const int tau = p0 / 6;
    const float4 xa = pt[p0], xb = pt[p0 + 1];
    const f2 X = make_float2(xa.x, xb.x), Y = make_float2(xa.y, xb.y), Z = make_float2(xa.z, xb.z);
    const float4 n4 = tn[tau];
    const int4 vt = tv[tau];
    const f2 mnx = dup2(-n4.x), mny = dup2(-n4.y), mnz = dup2(-n4.z);
    const f2 W1 = dup2((float)kQw1), W2 = dup2((float)kQw2);
    FarConst2 c = c0;
    float4 kff = kff0;
    int ct = 0;
    float sgn = 1.f;  // sign of the interior terms (-1: Mueller)
    f2 k1i = make_float2(0.f, 0.f), dk1i = k1i;
    if (MULTI) {
        ct = tcomp[tau];
        const FarObj o = fobj[ct];
        c.k1 = dup2(o.k1);
        c.nk1 = dup2(o.nk1);
        c.rho = dup2(o.rho);
        c.irho = dup2(o.irho);
        c.dk1 = dup2(o.dk1);
        kff.z = o.k1h;
        kff.w = o.k1l;
        sgn = o.sgn;
        k1i = dup2(o.k1i);
        dk1i = dup2(o.dk1i);
    }
    float4 cth = make_float4(0.f, 0.f, 0.f, 0.f), ctl = cth;
    if (CENTRED) {
        cth = cen[2 * tau];
        ctl = cen[2 * tau + 1];
    }

    for (int t0 = s_begin; t0 < s_end; t0 += FAR_TS) {
        const int cnt = min(FAR_TS, s_end - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt * 30; i += blockDim.x) shP[i] = sP[30 * (size_t)t0 + i];
        for (int i = threadIdx.x; i < cnt * 6; i += blockDim.x) shP5[i] = sP5[6 * (size_t)t0 + i];
        for (int i = threadIdx.x; i < cnt * 5; i += blockDim.x) shC[i] = sC[5 * (size_t)t0 + i];
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const float4 ns = tn[t0 + i];
            shN[i] = make_float4(-ns.x, -ns.y, -ns.z, ns.w);
            shV[i] = tv[t0 + i];
        }
        if (CENTRED)
            for (int i = threadIdx.x; i < 2 * cnt; i += blockDim.x) shCen[i] = cen[2 * (size_t)t0 + i];
        if (MULTI)
            for (int i = threadIdx.x; i < cnt; i += blockDim.x) shComp[i] = tcomp[t0 + i];
        __syncthreads();

        PairAcc A;
        A.u1r = A.u1i = A.u2r = A.u2i = make_float2(0.f, 0.f);
        A.axr = A.axi = A.ayr = A.ayi = A.azr = A.azi = make_float2(0.f, 0.f);
        for (int s = 0; s < cnt; ++s) {
            const int4 vs = shV[s];
            const bool touch = (vs.x == vt.x) | (vs.x == vt.y) | (vs.x == vt.z) |
                               (vs.y == vt.x) | (vs.y == vt.y) | (vs.y == vt.z) |
                               (vs.z == vt.x) | (vs.z == vt.y) | (vs.z == vt.z);
            if (touch) continue;
            const float4 mns = shN[s];  // (-n_y, n_y.P0)
            CenterPair cp;
            f2 xnyn;  // -(x - y).n_y, constant over the source triangle
            if (CENTRED) {
                cp = center_pair(cth, ctl, shCen[2 * s], shCen[2 * s + 1], kff.x, kff.y, kff.z, kff.w);
                // (x - y).n_y = (c_x - c_y + a).n_y since c_y lies in the source plane
                const float dn = cp.Dx.x * mns.x + cp.Dy.x * mns.y + cp.Dz.x * mns.z;
                xnyn = fma2(Z, dup2(mns.z), fma2(Y, dup2(mns.y), fma2(X, dup2(mns.x), dup2(dn))));
            } else {
                xnyn = fma2(Z, dup2(mns.z), fma2(Y, dup2(mns.y), fma2(X, dup2(mns.x), dup2(mns.w))));
            }
            const float nxnyn = n4.x * mns.x + n4.y * mns.y + n4.z * mns.z;  // -n_x.n_y
            A.t1r = A.t1i = A.ur = A.ui = A.t3r = A.t3i = make_float2(0.f, 0.f);
            const f2 m1 = dup2(MULTI ? (shComp[s] != ct ? 0.f : sgn) : 1.f);
#pragma unroll
            for (int q = 0; q < 6; ++q)
                far_pair2<CENTRED, MULTI, ABSORB>(X, Y, Z, &shP[30 * s + 5 * q], shP5[6 * s + q], mnx, mny, mnz,
                                          q < 3 ? W1 : W2, c, cp, m1, k1i, dk1i, A);
            // u1 += (x - y).n_y T1 = (-(x - y).n_y)(-T1);  u2 += (-n_x.n_y) U
            A.u1r = fma2(xnyn, A.t1r, A.u1r);
            A.u1i = fma2(xnyn, A.t1i, A.u1i);
            const f2 nn = dup2(nxnyn * c.dk0.x);
            A.u2r = fma2(nn, A.ur, A.u2r);
            A.u2i = fma2(nn, A.ui, A.u2i);
            const float4 C0 = shC[5 * s], C1 = shC[5 * s + 1], C2 = shC[5 * s + 2];
            const float4 C3 = shC[5 * s + 3], C4 = shC[5 * s + 4];
            A.axr = fma2(A.t3r, lo2(C0), fma2(A.t3i, lo2(C1), A.axr));
            A.axi = fma2(A.t3r, hi2(C0), fma2(A.t3i, lo2(C0), A.axi));
            A.ayr = fma2(A.t3r, hi2(C1), fma2(A.t3i, hi2(C2), A.ayr));
            A.ayi = fma2(A.t3r, lo2(C2), fma2(A.t3i, hi2(C1), A.ayi));
            A.azr = fma2(A.t3r, lo2(C3), fma2(A.t3i, lo2(C4), A.azr));
            A.azi = fma2(A.t3r, hi2(C3), fma2(A.t3i, lo2(C3), A.azi));
        }
        // running sums live in the output: the first tile stores, later
        // tiles add (the thread's own entries; registers stay free for the
        // pair loop)
        if (active) {
            const f2 v[10] = {A.u1r, A.u1i, A.u2r, A.u2i, A.axr, A.axi, A.ayr, A.ayi, A.azr, A.azi};
            f2 *pp = reinterpret_cast<f2 *>(part);
#pragma unroll
            for (int i = 0; i < 10; ++i) {
                const size_t o = (((size_t)split * 10 + i) * npts + p0) / 2;
                pp[o] = t0 == s_begin ? v[i] : add2(pp[o], v[i]);
            }
        }
    }
    if (active && s_begin >= s_end) {  // empty split: zero sums
        f2 *pp = reinterpret_cast<f2 *>(part);
#pragma unroll
        for (int i = 0; i < 10; ++i) pp[(((size_t)split * 10 + i) * npts + p0) / 2] = make_float2(0.f, 0.f);
    }
}

// Per vertex v: y1_v = (1/4pi) sum_{(t,a) incident} |t| sum_q w_q lambda_a(q) u1(t,q)
//               y2_v = (1/4pi) sum |t| [sum_q w_q lambda_a(q) u2(t,q) + curl_a . sum_q w_q A(t,q)]
// plus the near-field CSR rows (2x2 complex blocks) applied to x.
__global__ void gather_kernel(int nv, int npts, int nsplit, const int *__restrict__ vt_ptr,
                              const int *__restrict__ vt_idx, const double *__restrict__ tgeo,
                              const float *__restrict__ part, int use_far,
                              const int *__restrict__ nr_ptr, const int *__restrict__ nr_col,
                              const double2 *__restrict__ nr_val, int use_near,
                              const double2 *__restrict__ x, double2 *__restrict__ y) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double2 y1 = cd(0, 0), y2 = cd(0, 0);
    if (use_far) {
        for (int e = vt_ptr[v]; e < vt_ptr[v + 1]; ++e) {
            const int t = vt_idx[e] / 3, a = vt_idx[e] % 3;
            const double *g = tgeo + 16 * (size_t)t;
            double2 s1 = cd(0, 0), s2 = cd(0, 0), ax = cd(0, 0), ay = cd(0, 0), az = cd(0, 0);
            for (int q = 0; q < 6; ++q) {
                double b[3], w;
                rule_point(q, b, w);
                const double wl = w * b[a];
                const size_t p = 6 * (size_t)t + q;
                for (int sp = 0; sp < nsplit; ++sp) {
                    const float *P = part + (size_t)sp * 10 * npts + p;
                    s1 = cadd(s1, cd(wl * P[0], wl * P[(size_t)npts]));
                    s2 = cadd(s2, cd(wl * P[2 * (size_t)npts], wl * P[3 * (size_t)npts]));
                    ax = cadd(ax, cd(w * P[4 * (size_t)npts], w * P[5 * (size_t)npts]));
                    ay = cadd(ay, cd(w * P[6 * (size_t)npts], w * P[7 * (size_t)npts]));
                    az = cadd(az, cd(w * P[8 * (size_t)npts], w * P[9 * (size_t)npts]));
                }
            }
            const double *cu = g + 4 + 3 * a;
            s2 = cadd(s2, cadd(cadd(cscale(ax, cu[0]), cscale(ay, cu[1])), cscale(az, cu[2])));
            y1 = cadd(y1, cscale(s1, g[0]));
            y2 = cadd(y2, cscale(s2, g[0]));
        }
        const double inv4pi = 0.079577471545947667884;
        y1 = cscale(y1, inv4pi);
        y2 = cscale(y2, inv4pi);
    }
    if (use_near) {
        for (int e = nr_ptr[v]; e < nr_ptr[v + 1]; ++e) {
            const int j = nr_col[e];
            const double2 xa = x[j], xb = x[nv + j];
            const double2 *B = nr_val + 4 * (size_t)e;
            y1 = cadd(y1, cadd(cmul(B[0], xa), cmul(B[1], xb)));
            y2 = cadd(y2, cadd(cmul(B[2], xa), cmul(B[3], xb)));
        }
    }
    y[v] = y1;
    y[nv + v] = y2;
}

// ---------------------------------------------------------------------------
// Multi-right-hand-side far field: one launch applies B_far to R vectors.
// Everything that depends only on the point pair (distance, 1/r, the four
// sine / cosine values, the kernel combinations) is computed once and shared
// by the R right-hand sides; only the accumulations scale with R.  To keep
// per-right-hand-side state small, the per-source-triangle factors of the
// K and D-normal terms ((x - y).n_y and n_x.n_y) are folded into the pair's
// kernel values, so each right-hand side has just the two complex sums
//   u1 = sum [ (G0 + rho G1) psi_q + (x - y).n_y (H0 + H1) phi_q ]
//   u2 = sum [ (H0 + H1)(x - y).n_x psi_q - (n_x.n_y)(k0^2 G0 + k1^2/rho G1) phi_q ]
// per test point, kept in registers over the whole source range.  The D
// curl term A = sum_s (sum_q w_q (G0 + G1/rho)) c_s needs only
// W(tau, s) = sum_p w_p sum_q w_q (G0 + G1/rho), which does not depend on the
// right-hand side: each thread's share of it goes to shared memory per
// source triangle, and after each tile the three threads of a test triangle
// contract it with the right-hand sides' curl sources c_s (each thread a
// third of the right-hand sides).
//
// Block: FARM_THREADS = 384 threads = 128 test triangles, thread j holds test
// points 2 (j mod 3), 2 (j mod 3) + 1 of triangle j / 3 packed in FP32x2
// lanes.  Source data (per point, duplicated pairs for the packed lanes):
//   sG [6nt][2]   (-y.x, -y.x, -y.y, -y.y), (-y.z, -y.z, w_q, w_q)   (static)
//   sD [nt][6][R][2]  (psi.re, psi.re, psi.im, psi.im), (phi.re, ..., phi.im)
//   sCm [nt][R][3]    c_s components (complex)
// Outputs (no atomics; gridDim.y splits the source range):
//   part  [ns][R][4][npts]  u1 (re, im), u2 (re, im) per test point
//   partA [ns][R][6][nt]    sum_p w_p A(x_p) per test triangle (x, y, z; re, im)
// ---------------------------------------------------------------------------
// 384 threads = 12 warps, 3 on each of the SM's four schedulers (a block
// whose warps spread unevenly over the schedulers waits at every tile
// barrier for its most crowded scheduler); one block per SM at <= 170
// registers per thread
#ifndef OSRC_FARM_THREADS
#define OSRC_FARM_THREADS 384
#endif
constexpr int FARM_THREADS = OSRC_FARM_THREADS;
#ifndef OSRC_FARM_MIN_BLOCKS
#define OSRC_FARM_MIN_BLOCKS 1
#endif
#ifndef OSRC_FARM_QUNROLL
#define OSRC_FARM_QUNROLL 2
#endif
constexpr int FARM_QUNROLL = OSRC_FARM_QUNROLL;  // unroll of the rule-point loop
constexpr int FARM_TRIS = FARM_THREADS / 3;  // test triangles per block
constexpr int FARM_TS = 16;                  // source triangles per shared-memory tile
constexpr int FARM_MAX_R = 8;

struct VecPtrs {
    const double2 *p[FARM_MAX_R];
};
struct OutPtrs {
    double2 *p[FARM_MAX_R];
};

// one shared-memory tile buffer: sG, sD, sCm, normals, vertex ids, centroids
constexpr size_t farm_buf_bytes(int R, bool centred) {
    return (size_t)FARM_TS * (12 * 16 + 12 * 16 * R + 24 * R + 16 + 16 + (centred ? 32 : 0));
}

size_t farm_smem_bytes(int R, bool centred) {
    return 2 * farm_buf_bytes(R, centred) + (size_t)FARM_TS * FARM_THREADS * sizeof(float2) + 2 * sizeof(uint64_t);
}

constexpr unsigned long long FARM_TIMEOUT_NS = 2000000000ULL;

__device__ __forceinline__ uint32_t farm_saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long farm_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// waits for phase `parity` of the mbarrier, at most FARM_TIMEOUT_NS of global time
__device__ __forceinline__ bool farm_wait(uint64_t *bar, uint32_t parity) {
    const unsigned long long t0 = farm_ns();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(farm_saddr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (farm_ns() - t0 > FARM_TIMEOUT_NS) return false;
    }
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple
// of 16), completion counted on the mbarrier
__device__ __forceinline__ void farm_bulk(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            farm_saddr(dst)),
        "l"((uint64_t)src), "r"(bytes), "r"(farm_saddr(bar))
        : "memory");
}

// static source geometry of the multi kernel: coordinates (absolute, or
// offsets from the triangle centroid for the centred variant) negated and
// duplicated, and the rule weight w_q
__global__ void farm_geom_kernel(const float4 *__restrict__ pts, int npts, float4 *__restrict__ sG) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npts) return;
    const float4 p = pts[k];
    const int q = k % 6;
    const float w = (float)(q < 3 ? kQw1 : kQw2);
    sG[2 * (size_t)k] = make_float4(-p.x, -p.x, -p.y, -p.y);
    sG[2 * (size_t)k + 1] = make_float4(-p.z, -p.z, w, w);
}

// densities of R right-hand sides at the source rule points and the curl
// sources c_s, one thread per (source triangle, right-hand side)
__global__ void farm_prep_kernel(VecPtrs x, int R, int nv, int nt, const int *__restrict__ tris,
                                 const double *__restrict__ tgeo, float4 *__restrict__ sD,
                                 float2 *__restrict__ sCm) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (t >= nt || r >= R) return;
    const double2 *xr = x.p[r];
    double2 ps[3], ph[3];
    for (int a = 0; a < 3; ++a) {
        const int v = tris[3 * t + a];
        ps[a] = xr[v];
        ph[a] = xr[nv + v];
    }
    const double *g = tgeo + 16 * (size_t)t;
    const double area = g[0];
    for (int q = 0; q < 6; ++q) {
        double b[3], w;
        rule_point(q, b, w);
        const double W = w * area;
        double2 sv = cd(0, 0), fv = cd(0, 0);
        for (int a = 0; a < 3; ++a) {
            sv = cadd(sv, cscale(ps[a], b[a]));
            fv = cadd(fv, cscale(ph[a], b[a]));
        }
        const float psr = (float)(W * sv.x), psi = (float)(W * sv.y);
        const float phr = (float)(W * fv.x), phi = (float)(W * fv.y);
        float4 *d = sD + 2 * ((6 * (size_t)t + q) * R + r);
        d[0] = make_float4(psr, psr, psi, psi);
        d[1] = make_float4(phr, phr, phi, phi);
    }
    for (int j = 0; j < 3; ++j) {
        double2 cv = cd(0, 0);
        for (int a = 0; a < 3; ++a) cv = cadd(cv, cscale(ph[a], g[4 + 3 * a + j]));
        sCm[3 * ((size_t)t * R + r) + j] = make_float2((float)(cv.x * area), (float)(cv.y * area));
    }
}

// One source point against the thread's two test points, R right-hand sides.
template <int R, bool CENTRED>
__device__ __forceinline__ void farm_pair(f2 X, f2 Y, f2 Z, const float4 G0, const float4 G1,
                                          const float4 *__restrict__ D, f2 mnx, f2 mny, f2 mnz, f2 xnyn,
                                          f2 nn, const FarConst2 &c, const CenterPair &cp, f2 &t3r,
                                          f2 &t3i, f2 (&u1r)[R], f2 (&u1i)[R], f2 (&u2r)[R],
                                          f2 (&u2i)[R]) {
    f2 dx, dy, dz, ddx, ddy, ddz;
    if (CENTRED) {
        ddx = add2(X, lo2(G0));
        ddy = add2(Y, hi2(G0));
        ddz = add2(Z, lo2(G1));
        dx = add2(ddx, cp.Dx);
        dy = add2(ddy, cp.Dy);
        dz = add2(ddz, cp.Dz);
    } else {
        dx = add2(X, lo2(G0));
        dy = add2(Y, hi2(G0));
        dz = add2(Z, lo2(G1));
    }
    f2 r2 = mul2(dx, dx);
    r2 = fma2(dy, dy, r2);
    r2 = fma2(dz, dz, r2);
    const f2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const f2 r = mul2(r2, ri);
    const f2 ri2 = mul2(ri, ri);
    f2 dnxn = mul2(dx, mnx);  // (y - x).n_x
    dnxn = fma2(dy, mny, dnxn);
    dnxn = fma2(dz, mnz, dnxn);
    f2 s0, c0, s1, c1;
    if (CENTRED) {
        f2 num = mul2(ddx, ddx);
        num = fma2(ddy, ddy, num);
        num = fma2(ddz, ddz, num);
        f2 dd = mul2(ddx, cp.Dx);
        dd = fma2(ddy, cp.Dy, dd);
        dd = fma2(ddz, cp.Dz, dd);
        num = fma2(dd, dup2(2.f), num);
        const f2 den = add2(r, cp.rc);
        const f2 dlt = mul2(num, make_float2(rcp_approx(den.x), rcp_approx(den.y)));
        const f2 ph0 = fma2(c.k0, dlt, cp.b0);
        const f2 ph1 = fma2(c.k1, dlt, cp.b1);
        __sincosf(ph0.x, &s0.x, &c0.x);
        __sincosf(ph0.y, &s0.y, &c0.y);
        __sincosf(ph1.x, &s1.x, &c1.x);
        __sincosf(ph1.y, &s1.y, &c1.y);
    } else {
        const f2 kr0 = mul2(r, c.k0), kr1 = mul2(r, c.k1);
        __sincosf(kr0.x, &s0.x, &c0.x);
        __sincosf(kr0.y, &s0.y, &c0.y);
        __sincosf(kr1.x, &s1.x, &c1.x);
        __sincosf(kr1.y, &s1.y, &c1.y);
    }
    const f2 c0r = mul2(c0, ri), s0r = mul2(s0, ri), c1r = mul2(c1, ri), s1r = mul2(s1, ri);
    // V: G0 + rho G1
    const f2 gpr = fma2(c.rho, c1r, c0r), gpi = fma2(c.rho, s1r, s0r);
    // D normal: (-n_x.n_y) dks (G0 + dk1 G1), nn = -n_x.n_y dks
    const f2 gkr = mul2(nn, fma2(c.dk1, c1r, c0r)), gki = mul2(nn, fma2(c.dk1, s1r, s0r));
    // D curl weight: sum_q w_q (G0 + G1/rho)
    const f2 wq = hi2(G1);
    t3r = fma2(fma2(c.irho, c1r, c0r), wq, t3r);
    t3i = fma2(fma2(c.irho, s1r, s0r), wq, t3i);
    // -(H0 + H1) with the scaled c, s (see far_pair2)
    const f2 hp = mul2(fma2(c.k1, s1, fma2(c.k0, s0, add2(c0r, c1r))), ri2);
    const f2 hq = mul2(fma2(c.nk1, c1, fma2(c.nk0, c0, add2(s0r, s1r))), ri2);
    // K: (x - y).n_y (H0 + H1) = (-(x - y).n_y)(-(H0 + H1));  T: (H0 + H1)(x - y).n_x
    const f2 kr = mul2(xnyn, hp), ki = mul2(xnyn, hq);
    const f2 tr = mul2(dnxn, hp), ti = mul2(dnxn, hq);
    const f2 m1 = dup2(-1.f);
    const f2 ngpi = mul2(gpi, m1), nki = mul2(ki, m1), nti = mul2(ti, m1), ngki = mul2(gki, m1);
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
        const float4 Ps = D[2 * rr], Ph = D[2 * rr + 1];
        const f2 psr = lo2(Ps), psi = hi2(Ps), phr = lo2(Ph), phi = hi2(Ph);
        u1r[rr] = fma2(gpr, psr, fma2(ngpi, psi, fma2(kr, phr, fma2(nki, phi, u1r[rr]))));
        u1i[rr] = fma2(gpr, psi, fma2(gpi, psr, fma2(kr, phi, fma2(ki, phr, u1i[rr]))));
        u2r[rr] = fma2(tr, psr, fma2(nti, psi, fma2(gkr, phr, fma2(ngki, phi, u2r[rr]))));
        u2i[rr] = fma2(tr, psi, fma2(ti, psr, fma2(gkr, phi, fma2(gki, phr, u2i[rr]))));
    }
}

template <int R, bool CENTRED>
struct FarmBuf {
    float4 *G;   // [TS*6][2]
    float4 *D;   // [TS*6][R][2]
    float2 *C;   // [TS][R][3]
    float4 *N;   // [TS] normal, plane offset
    int4 *V;     // [TS] vertex ids
    float4 *Cen; // [2 TS] (centred)
    __device__ FarmBuf(unsigned char *base) {
        G = reinterpret_cast<float4 *>(base);
        D = G + FARM_TS * 12;
        C = reinterpret_cast<float2 *>(D + FARM_TS * 12 * R);
        N = reinterpret_cast<float4 *>(C + FARM_TS * 3 * R);
        V = reinterpret_cast<int4 *>(N + FARM_TS);
        Cen = reinterpret_cast<float4 *>(V + FARM_TS);
    }
};

// Source tiles are staged by 1-D TMA bulk copies (cp.async.bulk) into a
// two-buffer shared-memory ring: thread 0 issues tile k + 1 while every
// thread computes tile k, and an mbarrier per buffer counts the bytes in.
// Every wait is bounded (FARM_TIMEOUT_NS of global time); a thread that
// gives up sets *err, stops waiting, and writes NaN instead of its sums, and
// thread 0 waits (bounded) for the copies it issued before the block exits.
template <int R, bool CENTRED>
__global__ void __launch_bounds__(FARM_THREADS, OSRC_FARM_MIN_BLOCKS)
farm_kernel(const float4 *__restrict__ pt, const float4 *__restrict__ cen, const float4 *__restrict__ tn,
            const int4 *__restrict__ tv, const float4 *__restrict__ sG, const float4 *__restrict__ sD,
            const float2 *__restrict__ sCm, int nt, int npts, int tris_per_split, FarConst2 c,
            float4 kff, float *__restrict__ part, float *__restrict__ partA, int *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char farm_smem[];
    constexpr size_t BUF = farm_buf_bytes(R, CENTRED);
    float2 *shW = reinterpret_cast<float2 *>(farm_smem + 2 * BUF);  // [TS][threads]
    uint64_t *bar = reinterpret_cast<uint64_t *>(shW + FARM_TS * FARM_THREADS);

    const int j = threadIdx.x;
    const int lt = j / 3, sub = j - 3 * (j / 3);
    const int tau_raw = blockIdx.x * FARM_TRIS + lt;
    const bool active = tau_raw < nt;
    const int tau = active ? tau_raw : 0;
    const int p0 = 6 * tau + 2 * sub;
    const int split = blockIdx.y;
    const int s_begin = split * tris_per_split;
    const int s_end = min(nt, s_begin + tris_per_split);
    const int ntiles = s_end > s_begin ? (s_end - s_begin + FARM_TS - 1) / FARM_TS : 0;
    const float4 xa = pt[p0], xb = pt[p0 + 1];
    const f2 X = make_float2(xa.x, xb.x), Y = make_float2(xa.y, xb.y), Z = make_float2(xa.z, xb.z);
    const float4 n4 = tn[tau];
    const int4 vt = tv[tau];
    const f2 mnx = dup2(-n4.x), mny = dup2(-n4.y), mnz = dup2(-n4.z);
    const float wa = (float)(2 * sub < 3 ? kQw1 : kQw2), wb = (float)(2 * sub + 1 < 3 ? kQw1 : kQw2);
    float4 cth = make_float4(0.f, 0.f, 0.f, 0.f), ctl = cth;
    if (CENTRED) {
        cth = cen[2 * tau];
        ctl = cen[2 * tau + 1];
    }
    f2 u1r[R], u1i[R], u2r[R], u2i[R];
#pragma unroll
    for (int rr = 0; rr < R; ++rr) u1r[rr] = u1i[rr] = u2r[rr] = u2i[rr] = make_float2(0.f, 0.f);

    // thread 0: the copies of tile k into buffer k & 1
    auto issue = [&](int k) {
        const int t0 = s_begin + k * FARM_TS;
        const int cnt = min(FARM_TS, s_end - t0);
        FarmBuf<R, CENTRED> fb(farm_smem + (k & 1) * BUF);
        uint64_t *mb = &bar[k & 1];
        const uint32_t bytes = (uint32_t)cnt * (12 * 16 + 12 * 16 * R + 24 * R + 16 + 16 + (CENTRED ? 32 : 0));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(farm_saddr(mb)), "r"(bytes)
                     : "memory");
        farm_bulk(fb.G, sG + 12 * (size_t)t0, (uint32_t)cnt * 12 * 16, mb);
        farm_bulk(fb.D, sD + 12 * (size_t)R * t0, (uint32_t)cnt * 12 * 16 * R, mb);
        farm_bulk(fb.C, sCm + 3 * (size_t)R * t0, (uint32_t)cnt * 24 * R, mb);
        farm_bulk(fb.N, tn + t0, (uint32_t)cnt * 16, mb);
        farm_bulk(fb.V, tv + t0, (uint32_t)cnt * 16, mb);
        if (CENTRED) farm_bulk(fb.Cen, cen + 2 * (size_t)t0, (uint32_t)cnt * 32, mb);
    };
    if (j == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(farm_saddr(&bar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(farm_saddr(&bar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (j == 0 && ntiles > 0) issue(0);
    bool dead = false;      // a bounded wait gave up
    int issued = ntiles > 0 ? 1 : 0;  // tiles issued (thread 0)

    for (int k = 0; k < ntiles; ++k) {
        const int t0 = s_begin + k * FARM_TS;
        const int cnt = min(FARM_TS, s_end - t0);
        FarmBuf<R, CENTRED> fb(farm_smem + (k & 1) * BUF);
        if (!dead && !farm_wait(&bar[k & 1], (uint32_t)(k >> 1) & 1u)) {
            dead = true;
            atomicExch(err, 1);
        }
        // the other buffer held tile k - 1, released by the barrier that ended it
        if (j == 0 && !dead && k + 1 < ntiles) {
            issue(k + 1);
            issued = k + 2;
        }
        for (int s = 0; s < cnt; ++s) {
            const int4 vs = fb.V[s];
            const bool touch = (vs.x == vt.x) | (vs.x == vt.y) | (vs.x == vt.z) |
                               (vs.y == vt.x) | (vs.y == vt.y) | (vs.y == vt.z) |
                               (vs.z == vt.x) | (vs.z == vt.y) | (vs.z == vt.z);
            if (touch) {
                shW[s * FARM_THREADS + j] = make_float2(0.f, 0.f);
                continue;
            }
            const float4 ns = fb.N[s];
            const float4 mns = make_float4(-ns.x, -ns.y, -ns.z, ns.w);
            CenterPair cp;
            f2 xnyn;
            if (CENTRED) {
                cp = center_pair(cth, ctl, fb.Cen[2 * s], fb.Cen[2 * s + 1], kff.x, kff.y, kff.z, kff.w);
                const float dn = cp.Dx.x * mns.x + cp.Dy.x * mns.y + cp.Dz.x * mns.z;
                xnyn = fma2(Z, dup2(mns.z), fma2(Y, dup2(mns.y), fma2(X, dup2(mns.x), dup2(dn))));
            } else {
                xnyn = fma2(Z, dup2(mns.z), fma2(Y, dup2(mns.y), fma2(X, dup2(mns.x), dup2(mns.w))));
            }
            const f2 nn = dup2((n4.x * mns.x + n4.y * mns.y + n4.z * mns.z) * c.dk0.x);
            f2 t3r = make_float2(0.f, 0.f), t3i = t3r;
#pragma unroll FARM_QUNROLL
            for (int q = 0; q < 6; ++q)
                farm_pair<R, CENTRED>(X, Y, Z, fb.G[12 * s + 2 * q], fb.G[12 * s + 2 * q + 1],
                                      &fb.D[2 * R * (6 * s + q)], mnx, mny, mnz, xnyn, nn, c, cp, t3r,
                                      t3i, u1r, u1i, u2r, u2i);
            shW[s * FARM_THREADS + j] = make_float2(wa * t3r.x + wb * t3r.y, wa * t3i.x + wb * t3i.y);
        }
        __syncthreads();
        // curl term of this tile: thread (lt, sub) takes right-hand sides sub, sub + 3, ...
        if (active) {
            for (int rr = sub; rr < R; rr += 3) {
                float ar[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int s = 0; s < cnt; ++s) {
                    const float2 *w3 = shW + s * FARM_THREADS + 3 * lt;
                    const float wr = w3[0].x + w3[1].x + w3[2].x, wi = w3[0].y + w3[1].y + w3[2].y;
                    const float2 *cc = fb.C + 3 * (s * R + rr);
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const float2 cv = cc[d];
                        ar[2 * d] += wr * cv.x - wi * cv.y;
                        ar[2 * d + 1] += wr * cv.y + wi * cv.x;
                    }
                }
                float *pa = partA + (((size_t)split * R + rr) * 6) * nt + tau;
#pragma unroll
                for (int d = 0; d < 6; ++d) pa[(size_t)d * nt] = k == 0 ? ar[d] : pa[(size_t)d * nt] + ar[d];
            }
        }
        __syncthreads();
    }
    if (j == 0 && dead) {  // copies still in flight land before the block exits: the
                           // last tile issued into each buffer
        for (int k = max(0, issued - 2); k < issued; ++k)
            if (!farm_wait(&bar[k & 1], (uint32_t)(k >> 1) & 1u)) break;
    }
    if (active) {
        f2 *pp = reinterpret_cast<f2 *>(part);
        const f2 nan2 = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
#pragma unroll
        for (int rr = 0; rr < R; ++rr) {
            const size_t base = (((size_t)split * R + rr) * 4) * npts + p0;
            pp[base / 2] = dead ? nan2 : u1r[rr];
            pp[(base + (size_t)npts) / 2] = dead ? nan2 : u1i[rr];
            pp[(base + 2 * (size_t)npts) / 2] = dead ? nan2 : u2r[rr];
            pp[(base + 3 * (size_t)npts) / 2] = dead ? nan2 : u2i[rr];
        }
        if (ntiles == 0)  // empty split: zero curl sums
            for (int rr = sub; rr < R; rr += 3)
                for (int d = 0; d < 6; ++d) partA[(((size_t)split * R + rr) * 6 + d) * nt + tau] = 0.f;
    }
}

// Per (vertex, right-hand side): the far-field partial sums gathered with the
// test weights, plus the near-field CSR product (as gather_kernel).
__global__ void farm_gather_kernel(int nv, int nt, int npts, int nsplit, int R, const int *__restrict__ vt_ptr,
                                   const int *__restrict__ vt_idx, const double *__restrict__ tgeo,
                                   const float *__restrict__ part, const float *__restrict__ partA,
                                   int use_far, const int *__restrict__ nr_ptr, const int *__restrict__ nr_col,
                                   const double2 *__restrict__ nr_val, int use_near, VecPtrs x, OutPtrs y) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const int rr = blockIdx.y;
    if (v >= nv || rr >= R) return;
    double2 y1 = cd(0, 0), y2 = cd(0, 0);
    if (use_far) {
        for (int e = vt_ptr[v]; e < vt_ptr[v + 1]; ++e) {
            const int t = vt_idx[e] / 3, a = vt_idx[e] % 3;
            const double *g = tgeo + 16 * (size_t)t;
            double2 s1 = cd(0, 0), s2 = cd(0, 0), ax = cd(0, 0), ay = cd(0, 0), az = cd(0, 0);
            for (int sp = 0; sp < nsplit; ++sp) {
                const float *P = part + (((size_t)sp * R + rr) * 4) * npts;
                for (int q = 0; q < 6; ++q) {
                    double b[3], w;
                    rule_point(q, b, w);
                    const double wl = w * b[a];
                    const size_t p = 6 * (size_t)t + q;
                    s1 = cadd(s1, cd(wl * P[p], wl * P[p + (size_t)npts]));
                    s2 = cadd(s2, cd(wl * P[p + 2 * (size_t)npts], wl * P[p + 3 * (size_t)npts]));
                }
                const float *PA = partA + (((size_t)sp * R + rr) * 6) * nt + t;
                ax = cadd(ax, cd(PA[0], PA[(size_t)nt]));
                ay = cadd(ay, cd(PA[2 * (size_t)nt], PA[3 * (size_t)nt]));
                az = cadd(az, cd(PA[4 * (size_t)nt], PA[5 * (size_t)nt]));
            }
            const double *cu = g + 4 + 3 * a;
            s2 = cadd(s2, cadd(cadd(cscale(ax, cu[0]), cscale(ay, cu[1])), cscale(az, cu[2])));
            y1 = cadd(y1, cscale(s1, g[0]));
            y2 = cadd(y2, cscale(s2, g[0]));
        }
        const double inv4pi = 0.079577471545947667884;
        y1 = cscale(y1, inv4pi);
        y2 = cscale(y2, inv4pi);
    }
    if (use_near) {
        const double2 *xr = x.p[rr];
        for (int e = nr_ptr[v]; e < nr_ptr[v + 1]; ++e) {
            const int jc = nr_col[e];
            const double2 xa = xr[jc], xb = xr[nv + jc];
            const double2 *Bk = nr_val + 4 * (size_t)e;
            y1 = cadd(y1, cadd(cmul(Bk[0], xa), cmul(Bk[1], xb)));
            y2 = cadd(y2, cadd(cmul(Bk[2], xa), cmul(Bk[3], xb)));
        }
    }
    y.p[rr][v] = y1;
    y.p[rr][nv + v] = y2;
}

}  // namespace

int far_setup_geometry(osrc_problem *pb, cudaStream_t st) {
    osrc_mesh *m = pb->mesh;
    const int nt = pb->nt;
    OSRC_TRY(pb->d_pt.alloc(m->ctx, 6 * (size_t)nt));
    OSRC_TRY(pb->d_poff.alloc(m->ctx, 6 * (size_t)nt));
    OSRC_TRY(pb->d_cen.alloc(m->ctx, 2 * (size_t)nt));
    OSRC_TRY(pb->d_tn.alloc(m->ctx, nt));
    OSRC_TRY(pb->d_tv.alloc(m->ctx, nt));
    OSRC_TRY(pb->d_tgeo.alloc(m->ctx, 16 * (size_t)nt));
    OSRC_TRY(pb->d_sP.alloc(m->ctx, 30 * (size_t)nt));
    OSRC_TRY(pb->d_sP5.alloc(m->ctx, 6 * (size_t)nt));
    OSRC_TRY(pb->d_sC.alloc(m->ctx, 5 * (size_t)nt));
    far_geom_kernel<<<(nt + 127) / 128, 128, 0, st>>>(m->d_verts.p, m->d_tris.p, nt, pb->d_pt.p,
                                                      pb->d_poff.p, pb->d_cen.p, pb->d_tn.p,
                                                      pb->d_tv.p, pb->d_tgeo.p);
    pb->launches++;
    OSRC_CK(cudaGetLastError());
    // largest phase k r over the mesh (bounding-box diagonal): beyond
    // FAR_PLAIN_MAX_PHASE radians the centred variant with float-float
    // phases is used.  The plain variant's FP32 phase error grows linearly
    // with k r: measured 1.04e-5 relative (operator apply) at
    // k_max x diagonal = 63 pi, so the switch sits at 32 pi (about 5e-6)
    {
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int i = 0; i < m->nv; ++i)
            for (int d = 0; d < 3; ++d) {
                lo[d] = fmin(lo[d], m->verts[3 * i + d]);
                hi[d] = fmax(hi[d], m->verts[3 * i + d]);
            }
        const double diag = sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                 (hi[2] - lo[2]) * (hi[2] - lo[2]));
        double kmax = fmax(pb->p.k_ext, pb->p.k_int);
        for (const ObjMat &o : pb->obj) kmax = fmax(kmax, o.k1);
        pb->far_reduce = kmax * diag > FAR_PLAIN_MAX_PHASE;
    }
    // split the source range so that the grid covers the GPU several times
    int dev = m->ctx->device, sms = 0, per_sm = 0;
    OSRC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (pb->far_reduce)
        OSRC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, far_kernel<true, false, false>, FAR_THREADS, 0));
    else
        OSRC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, far_kernel<false, false, false>, FAR_THREADS, 0));
    if (per_sm < 1) per_sm = 1;
    const int bx = (pb->npts / 2 + FAR_THREADS - 1) / FAR_THREADS;
    const int slots = sms * per_sm;
    int ns = (4 * slots + bx - 1) / bx;
    const int max_ns = (nt + FAR_TS - 1) / FAR_TS;
    if (ns > max_ns) ns = max_ns;
    if (ns < 1) ns = 1;
    pb->nsplit = ns;
    OSRC_TRY(pb->d_part.alloc(m->ctx, (size_t)ns * 10 * pb->npts));
    return OSRC_OK;
}

// Adds the duration of the last timed far-kernel launch to the statistics.
int far_prof_collect(osrc_problem *pb) {
    if (!pb->prof_pending) return OSRC_OK;
    OSRC_CK(cudaEventSynchronize(pb->prof_ev[1]));
    float ms = 0.f;
    OSRC_CK(cudaEventElapsedTime(&ms, pb->prof_ev[0], pb->prof_ev[1]));
    pb->prof_ms += ms;
    pb->prof_launches++;
    pb->prof_rhs += pb->prof_rhs_pending;
    pb->prof_rhs_pending = 1;
    pb->prof_pending = false;
    return OSRC_OK;
}

int far_apply(osrc_problem *pb, const double2 *x, double2 *y, int part, cudaStream_t st) {
    osrc_mesh *m = pb->mesh;
    const int nt = pb->nt, nv = pb->nv, npts = pb->npts;
    const int use_far = (part & OSRC_PART_FAR) ? 1 : 0;
    const int use_near = (part & OSRC_PART_NEAR) ? 1 : 0;
    if (use_far) {
        const float4 *src_pts = pb->far_reduce ? pb->d_poff.p : pb->d_pt.p;
        far_prep_kernel<<<(nt + 127) / 128, 128, 0, st>>>(x, nv, nt, m->d_tris.p, src_pts,
                                                          pb->d_tgeo.p, pb->d_sP.p, pb->d_sP5.p,
                                                          pb->d_sC.p);
        pb->launches++;
        const double k0 = pb->p.k_ext, k1 = pb->p.k_int, rho = pb->p.rho_ratio;
        const double inv2pi = 0.15915494309189533577;
        auto d2 = [](double v) { return make_float2((float)v, (float)v); };
        FarConst2 c;
        c.k0 = d2(k0);
        c.k1 = d2(k1);
        c.nk0 = d2(-k0);
        c.nk1 = d2(-k1);
        c.rho = d2(rho);
        c.irho = d2(1.0 / rho);
        c.dk0 = d2(pb->far_dks);
        c.dk1 = d2(k1 * k1 / rho / pb->far_dks);
        // k / (2 pi) as float pairs (hi, lo) for the float-float phases
        const double q0 = k0 * inv2pi, q1 = k1 * inv2pi;
        const float q0h = (float)q0, q1h = (float)q1;
        const float4 kff = make_float4(q0h, (float)(q0 - (double)q0h), q1h, (float)(q1 - (double)q1h));
        const int ns = pb->nsplit;
        const int tps = (nt + ns - 1) / ns;
        dim3 grid((npts / 2 + FAR_THREADS - 1) / FAR_THREADS, ns);
        if (pb->prof_on) {
            OSRC_TRY(far_prof_collect(pb));
            OSRC_CK(cudaEventRecord(pb->prof_ev[0], st));
        }
        const float4 *pts = pb->far_reduce ? pb->d_poff.p : pb->d_pt.p;
        const int *tc = m->d_tcomp.p;
        const FarObj *fo = pb->d_fobj.p;
        float *prt = pb->d_part.p;
        const bool ab = pb->absorb;
#define OSRC_FAR_LAUNCH(C, M, A)                                                                               \
    far_kernel<C, M, A><<<grid, FAR_THREADS, 0, st>>>(pts, pb->d_cen.p, pb->d_tn.p, pb->d_tv.p, pb->d_sP.p,      \
                                                      pb->d_sP5.p, pb->d_sC.p, nt, npts, tps, c, kff, tc, fo, prt)
        if (pb->far_reduce && pb->far_obj && ab) OSRC_FAR_LAUNCH(true, true, true);
        else if (pb->far_reduce && pb->far_obj) OSRC_FAR_LAUNCH(true, true, false);
        else if (pb->far_reduce) OSRC_FAR_LAUNCH(true, false, false);
        else if (pb->far_obj && ab) OSRC_FAR_LAUNCH(false, true, true);
        else if (pb->far_obj) OSRC_FAR_LAUNCH(false, true, false);
        else OSRC_FAR_LAUNCH(false, false, false);
#undef OSRC_FAR_LAUNCH
        pb->launches++;
        if (pb->prof_on) {
            OSRC_CK(cudaEventRecord(pb->prof_ev[1], st));
            pb->prof_pending = true;
        }
    }
    gather_kernel<<<(nv + 127) / 128, 128, 0, st>>>(
        nv, npts, pb->nsplit, m->d_vt_ptr.p, m->d_vt_idx.p, pb->d_tgeo.p, pb->d_part.p, use_far,
        pb->d_nr_ptr.p, pb->d_nr_col.p, pb->d_nr_val.p, use_near, x, y);
    pb->launches++;
    OSRC_CK(cudaGetLastError());
    return OSRC_OK;
}

// ---------------------------------------------------------------------------
// multi-right-hand-side apply: y_r = B_far x_r (+ near) for r < nrhs, in
// launches of up to FARM_MAX_R right-hand sides (chunks of 8, then 4, 2;
// a last single vector takes the one-right-hand-side kernel)
// ---------------------------------------------------------------------------
template <int R, bool C>
static int farm_setup_kernel_attr(size_t smem) {
    OSRC_CK(cudaFuncSetAttribute(farm_kernel<R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return OSRC_OK;
}

static PerDeviceOnce g_farm_once;

static int farm_prepare(osrc_problem *pb, int rmax, cudaStream_t st) {
    OSRC_TRY(per_device_once(g_farm_once, [](int) {
        int s = OSRC_OK;
        if (!s) s = farm_setup_kernel_attr<2, false>(farm_smem_bytes(2, false));
        if (!s) s = farm_setup_kernel_attr<4, false>(farm_smem_bytes(4, false));
        if (!s) s = farm_setup_kernel_attr<8, false>(farm_smem_bytes(8, false));
        if (!s) s = farm_setup_kernel_attr<2, true>(farm_smem_bytes(2, true));
        if (!s) s = farm_setup_kernel_attr<4, true>(farm_smem_bytes(4, true));
        if (!s) s = farm_setup_kernel_attr<8, true>(farm_smem_bytes(8, true));
        return s;
    }));
    osrc_ctx *ctx = pb->mesh->ctx;
    const int nt = pb->nt, npts = pb->npts;
    if (!pb->d_sG.p) {
        OSRC_TRY(pb->d_sG.alloc(ctx, 2 * (size_t)npts));
        const float4 *pts = pb->far_reduce ? pb->d_poff.p : pb->d_pt.p;
        farm_geom_kernel<<<(npts + 127) / 128, 128, 0, st>>>(pts, npts, pb->d_sG.p);
        pb->launches++;
        OSRC_CK(cudaGetLastError());
    }
    if (pb->farm_cap < rmax) {
        int dev = ctx->device, sms = 0, per_sm = 0;
        OSRC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const size_t sm8 = farm_smem_bytes(8, pb->far_reduce);
        if (pb->far_reduce)
            OSRC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, farm_kernel<8, true>, FARM_THREADS, sm8));
        else
            OSRC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, farm_kernel<8, false>, FARM_THREADS, sm8));
        if (per_sm < 1) per_sm = 1;
        // source splits: at least four blocks per resident slot, and among
        // the counts up to twice that, the one whose last wave is fullest
        const int bx = (nt + FARM_TRIS - 1) / FARM_TRIS;
        const int slots = sms * per_sm;
        const int max_ns = std::max(1, (nt + 4 * FARM_TS - 1) / (4 * FARM_TS));
        int ns0 = std::min(max_ns, std::max(1, (4 * slots + bx - 1) / bx));
        int ns = ns0;
        double best = -1.0;
        for (int cand = ns0; cand <= std::min(max_ns, 2 * ns0); ++cand) {
            const long long blocks = (long long)bx * cand;
            const long long waves = (blocks + slots - 1) / slots;
            const double eff = (double)blocks / (double)(waves * slots);
            if (eff > best + 1e-9) {
                best = eff;
                ns = cand;
            }
        }
        pb->farm_ns = ns;
        pb->d_sD.release();
        pb->d_sCm.release();
        pb->d_partm.release();
        pb->d_partA.release();
        OSRC_TRY(pb->d_sD.alloc(ctx, 12 * (size_t)nt * FARM_MAX_R));
        OSRC_TRY(pb->d_sCm.alloc(ctx, 3 * (size_t)nt * FARM_MAX_R));
        OSRC_TRY(pb->d_partm.alloc(ctx, (size_t)ns * FARM_MAX_R * 4 * npts));
        OSRC_TRY(pb->d_partA.alloc(ctx, (size_t)ns * FARM_MAX_R * 6 * nt));
        if (!pb->d_farm_err.p) {
            OSRC_TRY(pb->d_farm_err.alloc(ctx, 1));
            OSRC_CK(cudaMemsetAsync(pb->d_farm_err.p, 0, sizeof(int), st));
        }
        pb->farm_cap = FARM_MAX_R;
    }
    return OSRC_OK;
}

static int farm_launch(osrc_problem *pb, const double2 *const *xs, double2 *const *ys, int R, int part,
                       cudaStream_t st) {
    osrc_mesh *m = pb->mesh;
    const int nt = pb->nt, nv = pb->nv, npts = pb->npts;
    const int use_far = (part & OSRC_PART_FAR) ? 1 : 0;
    const int use_near = (part & OSRC_PART_NEAR) ? 1 : 0;
    VecPtrs xp{};
    OutPtrs yp{};
    for (int r = 0; r < R; ++r) {
        xp.p[r] = xs[r];
        yp.p[r] = ys[r];
    }
    const int ns = pb->farm_ns;
    if (use_far) {
        farm_prep_kernel<<<dim3((nt + 127) / 128, R), 128, 0, st>>>(xp, R, nv, nt, m->d_tris.p, pb->d_tgeo.p,
                                                                   pb->d_sD.p, pb->d_sCm.p);
        pb->launches++;
        const double k0 = pb->p.k_ext, k1 = pb->p.k_int, rho = pb->p.rho_ratio;
        const double inv2pi = 0.15915494309189533577;
        auto d2 = [](double v) { return make_float2((float)v, (float)v); };
        FarConst2 c;
        c.k0 = d2(k0);
        c.k1 = d2(k1);
        c.nk0 = d2(-k0);
        c.nk1 = d2(-k1);
        c.rho = d2(rho);
        c.irho = d2(1.0 / rho);
        c.dk0 = d2(pb->far_dks);
        c.dk1 = d2(k1 * k1 / rho / pb->far_dks);
        const double q0 = k0 * inv2pi, q1 = k1 * inv2pi;
        const float q0h = (float)q0, q1h = (float)q1;
        const float4 kff = make_float4(q0h, (float)(q0 - (double)q0h), q1h, (float)(q1 - (double)q1h));
        const int tps = (nt + ns - 1) / ns;
        dim3 grid((nt + FARM_TRIS - 1) / FARM_TRIS, ns);
        const float4 *pts = pb->far_reduce ? pb->d_poff.p : pb->d_pt.p;
        const size_t smem = farm_smem_bytes(R, pb->far_reduce);
        if (pb->prof_on) {
            OSRC_TRY(far_prof_collect(pb));
            OSRC_CK(cudaEventRecord(pb->prof_ev[0], st));
        }
#define OSRC_FARM_LAUNCH(RR, C)                                                                          \
    farm_kernel<RR, C><<<grid, FARM_THREADS, smem, st>>>(pts, pb->d_cen.p, pb->d_tn.p, pb->d_tv.p, pb->d_sG.p, \
                                                         pb->d_sD.p, pb->d_sCm.p, nt, npts, tps, c, kff,    \
                                                         pb->d_partm.p, pb->d_partA.p, pb->d_farm_err.p)
        if (pb->far_reduce) {
            if (R == 8) OSRC_FARM_LAUNCH(8, true);
            else if (R == 4) OSRC_FARM_LAUNCH(4, true);
            else OSRC_FARM_LAUNCH(2, true);
        } else {
            if (R == 8) OSRC_FARM_LAUNCH(8, false);
            else if (R == 4) OSRC_FARM_LAUNCH(4, false);
            else OSRC_FARM_LAUNCH(2, false);
        }
#undef OSRC_FARM_LAUNCH
        pb->launches++;
        OSRC_CK(cudaGetLastError());
        if (pb->prof_on) {
            OSRC_CK(cudaEventRecord(pb->prof_ev[1], st));
            pb->prof_pending = true;
            pb->prof_rhs_pending = R;
        }
    }
    farm_gather_kernel<<<dim3((nv + 127) / 128, R), 128, 0, st>>>(
        nv, nt, npts, ns, R, m->d_vt_ptr.p, m->d_vt_idx.p, pb->d_tgeo.p, pb->d_partm.p, pb->d_partA.p, use_far,
        pb->d_nr_ptr.p, pb->d_nr_col.p, pb->d_nr_val.p, use_near, xp, yp);
    pb->launches++;
    OSRC_CK(cudaGetLastError());
    return OSRC_OK;
}

// OSRC_TIMEOUT if a several-right-hand-side far kernel gave up a bounded
// wait since the last check (the flag is cleared); synchronises the stream
int far_multi_check(osrc_problem *pb, cudaStream_t st) {
    if (!pb->d_farm_err.p) return OSRC_OK;
    int h = 0;
    OSRC_CK(cudaMemcpyAsync(&h, pb->d_farm_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    OSRC_CK(cudaStreamSynchronize(st));
    if (h) {
        OSRC_CK(cudaMemsetAsync(pb->d_farm_err.p, 0, sizeof(int), st));
        osrc_set_error("far kernel: a bounded wait for a staged source tile gave up");
        return OSRC_TIMEOUT;
    }
    return OSRC_OK;
}

bool far_multi_supported(const osrc_problem *pb) {
    return pb->p.precision == OSRC_FP32_MATFREE && !pb->far_obj;
}

int far_apply_multi(osrc_problem *pb, const double2 *const *xs, double2 *const *ys, int nrhs, int part,
                    cudaStream_t st) {
    if (nrhs < 1) return OSRC_INVALID_ARG;
    if (nrhs == 1 || !far_multi_supported(pb) || !(part & OSRC_PART_FAR)) {
        for (int r = 0; r < nrhs; ++r) OSRC_TRY(far_apply(pb, xs[r], ys[r], part, st));
        return OSRC_OK;
    }
    OSRC_TRY(farm_prepare(pb, FARM_MAX_R, st));
    int r0 = 0;
    while (r0 < nrhs) {
        const int left = nrhs - r0;
        const int R = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        if (R == 1) OSRC_TRY(far_apply(pb, xs[r0], ys[r0], part, st));
        else OSRC_TRY(farm_launch(pb, xs + r0, ys + r0, R, part, st));
        r0 += R;
    }
    return OSRC_OK;
}
