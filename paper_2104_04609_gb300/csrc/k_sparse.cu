// k_sparse.cu -- P1 mass M and Laplace-Beltrami stiffness S (CSR, FP64), the
// mass preconditioner M^-1 (Sec. 2.4) and the OSRC preconditioner (Sec. 2.6,
// 2.7) by batched Krylov solves.
//
// Every inner system has the form (alpha M + beta S) w = f on the shared
// vertex-graph pattern.  One thread-block cluster (up to 8 CTAs) solves one
// system: each CTA owns a contiguous block of rows, the SpMV reads the search
// direction of the other CTAs from global memory after a cluster barrier,
// and dot products are reduced over the cluster through distributed shared
// memory, so a solve needs no host round trip and no grid-wide barrier.
// Rows owned by other CTAs are read with L2-only loads (__ldcg) after the
// cluster barrier, so no stale L1 line of an earlier iteration is used.
// Systems with real SPD matrices (M) use Hermitian CG; the complex-symmetric
// shifted OSRC systems use COCG (conjugate orthogonal CG, van der Vorst &
// Melissen 1990) with the unconjugated bilinear form x^T y.  Both are
// Jacobi-preconditioned and stop at |r| <= tol |f|.  All loops are bounded by
// the iteration cap; every CTA of a cluster takes the same branch because
// the decisions are made from cluster-reduced values summed in rank order.
// Two kernels share this layout: kmix_kernel (FP32 inner solves refined in
// FP64, used whenever a CTA's rows and FP32 entries fit) and kry_kernel
// (all FP64: larger meshes, in-place systems, the allocation-free entry).
#include <cooperative_groups.h>
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "osrc_internal.cuh"

namespace cg = cooperative_groups;

namespace {

__global__ void ms_element_kernel(int nt, const double *__restrict__ tgeo,
                                  const double *__restrict__ verts, const int *__restrict__ tris,
                                  double *__restrict__ bm, double *__restrict__ bs) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double *g = tgeo + 16 * (size_t)t;
    const double area = g[0];
    // grad phi_a = curl phi_a x n has the same length, and grad.grad = curl.curl
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const double *ca = g + 4 + 3 * a, *cb = g + 4 + 3 * b;
            bm[9 * (size_t)t + 3 * a + b] = area / 12.0 * (a == b ? 2.0 : 1.0);
            bs[9 * (size_t)t + 3 * a + b] = area * (ca[0] * cb[0] + ca[1] * cb[1] + ca[2] * cb[2]);
        }
}

__global__ void csr_sum_kernel(int nnz, const int *__restrict__ cptr, const int *__restrict__ cidx,
                               const double *__restrict__ bm, const double *__restrict__ bs,
                               double *__restrict__ M, double *__restrict__ S) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    double m = 0.0, s = 0.0;
    for (int k = cptr[e]; k < cptr[e + 1]; ++k) {
        m += bm[cidx[k]];
        s += bs[cidx[k]];
    }
    M[e] = m;
    S[e] = s;
}

constexpr int KRY_THREADS = 256;
constexpr int KRY_MAX_SYS = 40;

struct KrySys {
    double2 alpha, beta;  // system matrix alpha M + beta S
    const double2 *f;     // right-hand side
    double2 *x;           // solution
    int conj;             // 1: Hermitian CG, 0: COCG
    // disjoint objects: row i uses beta * bscale[vcomp[i]] (S has no entries
    // between objects, so the matrix stays complex symmetric); null: beta
    const double2 *bscale;
};

struct KryBatch {
    int nsys;
    const int *vcomp;  // object of each row (with KrySys::bscale)
    KrySys s[KRY_MAX_SYS];
};

__device__ __forceinline__ double2 dot_term(double2 a, double2 b, int conj) {
    // conj: conj(a) b, else a b
    return conj ? cd(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x) : cmul(a, b);
}

// Cluster-wide sum of three doubles.  Each warp reduces with shuffles, warp
// leaders write to `red`, thread 0 adds the warps and publishes the CTA sum
// in `slot`; after a cluster barrier lanes 0..cs-1 of warp 0 fetch the
// CTA sums of every rank through distributed shared memory and thread 0 adds
// them in rank order (the same order in every CTA, so all CTAs hold
// bit-identical sums).  The result is left in out[0..2] (shared memory),
// valid for every thread of the CTA after the final __syncthreads.
__device__ void cluster_sum3(cg::cluster_group &cl, double v0, double v1, double v2, double *red,
                             double *slot, double *gath, double *out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
    }
    if (lane == 0) {
        red[3 * wid] = v0;
        red[3 * wid + 1] = v1;
        red[3 * wid + 2] = v2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int w = 0; w < nw; ++w) {
            a += red[3 * w];
            b += red[3 * w + 1];
            c += red[3 * w + 2];
        }
        slot[0] = a;
        slot[1] = b;
        slot[2] = c;
    }
    cl.sync();
    const unsigned cs = cl.num_blocks();
    if (threadIdx.x < cs) {
        const double *rem = cl.map_shared_rank(slot, threadIdx.x);
        gath[3 * threadIdx.x] = rem[0];
        gath[3 * threadIdx.x + 1] = rem[1];
        gath[3 * threadIdx.x + 2] = rem[2];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (unsigned r = 0; r < cs; ++r) {
            a += gath[3 * r];
            b += gath[3 * r + 1];
            c += gath[3 * r + 2];
        }
        out[0] = a;
        out[1] = b;
        out[2] = c;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(KRY_THREADS)
kry_kernel(KryBatch batch, int n, const int *__restrict__ ptr, const int *__restrict__ col,
           const double *__restrict__ M, const double *__restrict__ S, double2 *__restrict__ work,
           double tol, int maxit, int *__restrict__ stat, double *__restrict__ res_out) {
    __shared__ double red[3 * 32];
    __shared__ double slotA[4], slotB[4], slotC[4];
    __shared__ double gath[3 * 16];
    __shared__ double sums[4];
    __shared__ double2 scal[2];  // alpha, beta of the current iteration
    __shared__ int flag;         // 0 continue, 1 converged, 2 breakdown
    cg::cluster_group cl = cg::this_cluster();
    const unsigned cs = cl.num_blocks();
    const unsigned rank = cl.block_rank();
    const int sid = blockIdx.x / cs;
    const KrySys sy = batch.s[sid];
    const int rows = (n + cs - 1) / cs;
    const int r0 = min(n, (int)rank * rows), r1 = min(n, r0 + rows);
    double2 *r = work + (5 * (size_t)sid + 0) * n;
    double2 *z = work + (5 * (size_t)sid + 1) * n;
    double2 *p = work + (5 * (size_t)sid + 2) * n;
    double2 *q = work + (5 * (size_t)sid + 3) * n;
    double2 *dinv = work + (5 * (size_t)sid + 4) * n;
    double2 *x = sy.x;
    const int cj = sy.conj;

    double v0 = 0.0, v1 = 0.0, v2 = 0.0;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        double md = 0.0, sd = 0.0;
        for (int e = ptr[i]; e < ptr[i + 1]; ++e)
            if (col[e] == i) { md = M[e]; sd = S[e]; }
        const double2 bi = sy.bscale ? cmul(sy.beta, sy.bscale[batch.vcomp[i]]) : sy.beta;
        const double2 d = cadd(cscale(sy.alpha, md), cscale(bi, sd));
        const double2 di = cdiv(cd(1.0, 0.0), d);
        const double2 b = sy.f[i];
        dinv[i] = di;
        x[i] = cd(0.0, 0.0);
        r[i] = b;
        const double2 zi = cmul(di, b);
        z[i] = zi;
        p[i] = zi;
        const double2 t = dot_term(b, zi, cj);
        v0 += t.x;
        v1 += t.y;
        v2 += cabs2(b);
    }
    cluster_sum3(cl, v0, v1, v2, red, slotA, gath, sums);
    double2 rho = cd(sums[0], sums[1]);
    const double bb = sums[2];
    double rr = bb;
    int its = 0, status = 0;  // 0 converged, 1 not converged, 2 breakdown
    if (bb > 0.0) {
        cl.sync();  // p complete everywhere
        status = 1;
        for (int it = 1; it <= maxit; ++it) {
            double w0 = 0.0, w1 = 0.0;
            for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
                double2 mp = cd(0.0, 0.0), sp = cd(0.0, 0.0);
                for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
                    const double2 pj = __ldcg(&p[col[e]]);
                    const double me = M[e], se = S[e];
                    mp.x += me * pj.x;
                    mp.y += me * pj.y;
                    sp.x += se * pj.x;
                    sp.y += se * pj.y;
                }
                const double2 bi = sy.bscale ? cmul(sy.beta, sy.bscale[batch.vcomp[i]]) : sy.beta;
                const double2 acc = cadd(cmul(sy.alpha, mp), cmul(bi, sp));
                q[i] = acc;
                const double2 t = dot_term(p[i], acc, cj);
                w0 += t.x;
                w1 += t.y;
            }
            cluster_sum3(cl, w0, w1, 0.0, red, slotB, gath, sums);
            if (threadIdx.x == 0) {
                const double2 pq = cd(sums[0], sums[1]);
                flag = (cabs2(pq) > 0.0) ? 0 : 2;
                scal[0] = flag ? cd(0.0, 0.0) : cdiv(rho, pq);
            }
            __syncthreads();
            if (flag) { status = 2; its = it; break; }
            const double2 al = scal[0];
            double u0 = 0.0, u1 = 0.0, u2 = 0.0;
            for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
                x[i] = cadd(x[i], cmul(al, p[i]));
                const double2 ri = csub(r[i], cmul(al, q[i]));
                r[i] = ri;
                const double2 zi = cmul(dinv[i], ri);
                z[i] = zi;
                const double2 t = dot_term(ri, zi, cj);
                u0 += t.x;
                u1 += t.y;
                u2 += cabs2(ri);
            }
            cluster_sum3(cl, u0, u1, u2, red, slotC, gath, sums);
            rr = sums[2];
            its = it;
            if (rr <= tol * tol * bb) { status = 0; break; }
            if (threadIdx.x == 0) {
                const double2 rn = cd(sums[0], sums[1]);
                flag = (cabs2(rho) > 0.0) ? 0 : 2;
                scal[1] = flag ? cd(0.0, 0.0) : cdiv(rn, rho);
                scal[0] = rn;
            }
            __syncthreads();
            if (flag) { status = 2; break; }
            const double2 be = scal[1];
            rho = scal[0];
            for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) p[i] = cadd(z[i], cmul(be, p[i]));
            cl.sync();
        }
    } else {
        rr = 0.0;
    }
    cl.sync();  // keep shared memory alive until every CTA has read it
    if (rank == 0 && threadIdx.x == 0) {
        stat[sid] = status == 0 ? its : (status == 1 ? -its : -1000000 - its);
        res_out[sid] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    }
}

// ---- mixed-precision refinement ---------------------------------------------
// The same systems (alpha M + beta S) w = f, solved by iterative refinement
// in the same cluster layout: an FP32 Jacobi-CG/COCG solve of A d = r, with
// the FP32 copy of A built once per launch in shared memory and r scaled to
// unit norm, reduces the residual by KMIX_INNER_TOL; then the FP64 solution
// is updated, x += d, and the FP64 residual r = f - A x decides: stop when
// |r| <= tol |f| (the criterion of kry_kernel, here on the true residual),
// else refine again.  Most arithmetic runs on the FP32 pipe, which on this
// part issues 64 times the FP64 rate; a refinement costs one FP64 product.
// Refinement converges while cond(D^-1 A) * 2^-24 stays well below one (the
// OSRC and mass systems sit near cond 10..100); a refinement that fails to
// halve the residual norm ends the solve as not converged.
constexpr int KMIX_THREADS = 512;          // at most, per CTA (two CTAs per SM)
constexpr int KMIX_ROWS_PER_THREAD = 2;    // rows a thread owns, at most
constexpr float KMIX_INNER_TOL = 1e-5f;    // residual reduction of one FP32 solve
constexpr int KMIX_MAX_REFINE = 40;
constexpr size_t KMIX_SMEM_MAX = 200 * 1024;

// Cluster-wide sums of NV values, identical in every thread of every CTA of
// the cluster: butterflies within each warp, the warp sums added by a
// butterfly in warp 0, then the CTA sums of all ranks (lane r reads rank r's
// slot through distributed shared memory) added by a butterfly in warp 0.
// IEEE addition is commutative, so every lane of a butterfly ends with the
// same bits, and every CTA adds the same rank-ordered values.  A slot may be
// written again once every CTA has passed one more cluster barrier.
template <typename T, int NV>
__device__ __forceinline__ void kmix_csum(cg::cluster_group &cl, T (&v)[NV], T *wred, T *slot, T *out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) wred[NV * wid + k] = v[k];
    __syncthreads();
    if (wid == 0) {
        T w[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) w[k] = lane < nw ? wred[NV * lane + k] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < NV; ++k) w[k] += __shfl_xor_sync(0xffffffffu, w[k], o);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < NV; ++k) slot[k] = w[k];
    }
    cl.sync();
    if (wid == 0) {
        const unsigned cs = cl.num_blocks();
        T w[NV];
        if ((unsigned)lane < cs) {
            const T *rem = cl.map_shared_rank(slot, lane);
#pragma unroll
            for (int k = 0; k < NV; ++k) w[k] = rem[k];
        } else {
#pragma unroll
            for (int k = 0; k < NV; ++k) w[k] = T(0);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < NV; ++k) w[k] += __shfl_xor_sync(0xffffffffu, w[k], o);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < NV; ++k) out[k] = w[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = out[k];
}

__device__ __forceinline__ float2 f2mul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 f2dot(float2 a, float2 b, int conj) {
    return conj ? make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x) : f2mul(a, b);
}
__device__ __forceinline__ float2 f2div(float2 a, float2 b) {
    const float den = b.x * b.x + b.y * b.y;
    return make_float2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

// One cluster per system, rows [r0, r1) per CTA, row r0 + tid + k blockDim.x
// for k < RPT per thread.  Dynamic shared memory: the CTA's CSR entries of
// A in FP32 (float2) followed by their columns.  work32: n float2 per
// system, the published FP32 search direction.  sy.x holds the published
// FP64 solution.  Status and residual as kry_kernel; the iteration count is
// the number of FP32 iterations over all refinements.
template <int RPT>
__global__ void __launch_bounds__(KMIX_THREADS, 2)
kmix_kernel(KryBatch batch, int n, const int *__restrict__ ptr, const int *__restrict__ col,
            const double *__restrict__ M, const double *__restrict__ S, float2 *__restrict__ work32,
            double tol, int maxit, int *__restrict__ stat, double *__restrict__ res_out) {
    extern __shared__ __align__(16) unsigned char kmix_dyn[];
    __shared__ float wredf[3 * 32];
    __shared__ double wredd[32];
    __shared__ float slotP[2], slotR[3], slotI[3], outf[3];
    __shared__ double slotD[1], slotB[1], outd[1];
    cg::cluster_group cl = cg::this_cluster();
    const unsigned cs = cl.num_blocks();
    const unsigned rank = cl.block_rank();
    const int sid = blockIdx.x / cs;
    const KrySys sy = batch.s[sid];
    const int rows = (n + cs - 1) / cs;
    const int r0 = min(n, (int)rank * rows), r1 = min(n, r0 + rows);
    const int ebase = r0 < n ? ptr[r0] : 0;
    const int ne = r0 < r1 ? ptr[r1] - ebase : 0;
    float2 *As = reinterpret_cast<float2 *>(kmix_dyn);
    int *Cs = reinterpret_cast<int *>(kmix_dyn + sizeof(float2) * (size_t)((ne + 1) & ~1));
    float2 *pg = work32 + (size_t)sid * n;
    double2 *xg = sy.x;
    const int cj = sy.conj;

    // per row: the FP64 residual and the FP32 state (the FP64 solution
    // lives in sy.x, the right-hand side is read again when needed)
    int row[RPT];
    bool ok[RPT];
    double2 r64[RPT];
    float2 dinv[RPT], d[RPT], r[RPT], z[RPT], p[RPT], q[RPT];
    double bb = 0.0;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        row[k] = r0 + threadIdx.x + k * blockDim.x;
        ok[k] = row[k] < r1;
        r64[k] = cd(0.0, 0.0);
        dinv[k] = make_float2(0.f, 0.f);
        if (ok[k]) {
            const int i = row[k];
            const double2 bi = sy.bscale ? cmul(sy.beta, sy.bscale[batch.vcomp[i]]) : sy.beta;
            double2 dg = cd(0.0, 0.0);
            for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
                const double2 a = cadd(cscale(sy.alpha, M[e]), cscale(bi, S[e]));
                As[e - ebase] = make_float2((float)a.x, (float)a.y);
                Cs[e - ebase] = col[e];
                if (col[e] == i) dg = a;
            }
            const double2 di = cdiv(cd(1.0, 0.0), dg);
            dinv[k] = make_float2((float)di.x, (float)di.y);
            r64[k] = sy.f[i];
            bb += cabs2(r64[k]);
            xg[i] = cd(0.0, 0.0);
        }
    }
    {
        double v[1] = {bb};
        kmix_csum<double, 1>(cl, v, wredd, slotB, outd);  // its barrier also orders the shared-memory fill
        bb = v[0];
    }
    double rr = bb;
    int its = 0, status = 0;  // 0 converged, 1 not converged, 2 breakdown
    if (bb > 0.0) {
        status = 1;
        for (int ref = 0; ref < KMIX_MAX_REFINE && its < maxit; ++ref) {
            // FP32 solve of A d = r / |r|
            const double sc = 1.0 / sqrt(rr);
            float v3[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                r[k] = make_float2((float)(r64[k].x * sc), (float)(r64[k].y * sc));
                z[k] = f2mul(dinv[k], r[k]);
                p[k] = z[k];
                d[k] = make_float2(0.f, 0.f);
                if (ok[k]) {
                    pg[row[k]] = p[k];
                    const float2 t = f2dot(r[k], z[k], cj);
                    v3[0] += t.x;
                    v3[1] += t.y;
                    v3[2] += r[k].x * r[k].x + r[k].y * r[k].y;
                }
            }
            kmix_csum<float, 3>(cl, v3, wredf, slotI, outf);  // also publishes p
            float2 rho = make_float2(v3[0], v3[1]);
            const float rr0 = v3[2];
            bool brk = false;
            while (its < maxit) {
                float v2[2] = {0.f, 0.f};
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    float2 acc = make_float2(0.f, 0.f);
                    if (ok[k]) {
                        const int eb = ptr[row[k]] - ebase, ee = ptr[row[k] + 1] - ebase;
#pragma unroll 4
                        for (int e = eb; e < ee; ++e) {
                            const float2 a = As[e], pj = __ldcg(&pg[Cs[e]]);
                            acc.x = fmaf(a.x, pj.x, fmaf(-a.y, pj.y, acc.x));
                            acc.y = fmaf(a.x, pj.y, fmaf(a.y, pj.x, acc.y));
                        }
                        const float2 t = f2dot(p[k], acc, cj);
                        v2[0] += t.x;
                        v2[1] += t.y;
                    }
                    q[k] = acc;
                }
                kmix_csum<float, 2>(cl, v2, wredf, slotP, outf);
                const float2 pq = make_float2(v2[0], v2[1]);
                if (!(pq.x * pq.x + pq.y * pq.y > 0.f)) { brk = true; break; }
                const float2 al = f2div(rho, pq);
                float w3[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    d[k] = make_float2(fmaf(al.x, p[k].x, fmaf(-al.y, p[k].y, d[k].x)),
                                       fmaf(al.x, p[k].y, fmaf(al.y, p[k].x, d[k].y)));
                    r[k] = make_float2(fmaf(-al.x, q[k].x, fmaf(al.y, q[k].y, r[k].x)),
                                       fmaf(-al.x, q[k].y, fmaf(-al.y, q[k].x, r[k].y)));
                    z[k] = f2mul(dinv[k], r[k]);
                    if (ok[k]) {
                        const float2 t = f2dot(r[k], z[k], cj);
                        w3[0] += t.x;
                        w3[1] += t.y;
                        w3[2] += r[k].x * r[k].x + r[k].y * r[k].y;
                    }
                }
                kmix_csum<float, 3>(cl, w3, wredf, slotR, outf);
                ++its;
                if (w3[2] <= KMIX_INNER_TOL * KMIX_INNER_TOL * rr0) break;
                if (!(rho.x * rho.x + rho.y * rho.y > 0.f)) { brk = true; break; }
                const float2 rz = make_float2(w3[0], w3[1]);
                const float2 be = f2div(rz, rho);
                rho = rz;
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    p[k] = make_float2(fmaf(be.x, p[k].x, fmaf(-be.y, p[k].y, z[k].x)),
                                       fmaf(be.x, p[k].y, fmaf(be.y, p[k].x, z[k].y)));
                    if (ok[k]) pg[row[k]] = p[k];
                }
                cl.sync();  // p published
            }
            if (brk) { status = 2; break; }
            // FP64 update and residual
            const double back = sqrt(rr);
#pragma unroll
            for (int k = 0; k < RPT; ++k)
                if (ok[k]) xg[row[k]] = cadd(xg[row[k]], cd((double)d[k].x * back, (double)d[k].y * back));
            cl.sync();  // x published
            double rn = 0.0;
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                if (!ok[k]) continue;
                const int i = row[k];
                double2 mx = cd(0.0, 0.0), sx = cd(0.0, 0.0);
                for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
                    const double2 xj = __ldcg(&xg[col[e]]);
                    const double me = M[e], se = S[e];
                    mx.x += me * xj.x;
                    mx.y += me * xj.y;
                    sx.x += se * xj.x;
                    sx.y += se * xj.y;
                }
                const double2 bi = sy.bscale ? cmul(sy.beta, sy.bscale[batch.vcomp[i]]) : sy.beta;
                r64[k] = csub(sy.f[i], cadd(cmul(sy.alpha, mx), cmul(bi, sx)));
                rn += cabs2(r64[k]);
            }
            double v[1] = {rn};
            kmix_csum<double, 1>(cl, v, wredd, slotD, outd);
            const double rprev = rr;
            rr = v[0];
            if (rr <= tol * tol * bb) { status = 0; break; }
            if (!(rr <= 0.25 * rprev)) break;  // refinement stagnates (or NaN): not converged
        }
    } else {
        rr = 0.0;
    }
    cl.sync();  // keep shared memory alive until every CTA has read it
    if (rank == 0 && threadIdx.x == 0) {
        stat[sid] = status == 0 ? its : (status == 1 ? -its : -1000000 - its);
        res_out[sid] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    }
}

// y = M u on both block rows (turns a strong-form vector into the weak one)
__global__ void mass_spmv_kernel(int n, const int *__restrict__ ptr, const int *__restrict__ col,
                                 const double *__restrict__ M, const double2 *__restrict__ u,
                                 double2 *__restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 a = cd(0, 0), b = cd(0, 0);
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
        const int j = col[e];
        a = cadd(a, cscale(u[j], M[e]));
        b = cadd(b, cscale(u[n + j], M[e]));
    }
    y[i] = a;
    y[n + i] = b;
}

struct OsrcComb {
    int np;
    double2 ik, iik;  // i k and 1/(i k)
    const double2 *ik_obj;  // disjoint objects: i k of each object (else ik)
    const int *vcomp;
    double2 cu;       // C0 + sum_j A_j / B_j
    double2 g0;
    double2 a[16];    // A_j / B_j
    double2 g[16];
};

// sol[0] = u1 = M^-1 y1, sol[1..np] = v_j, sol[np+1] = v'_0, sol[np+2..2np+1] = v'_j:
//   z1 = i k [(C0 + sum_j A_j/B_j) u1 - sum_j (A_j/B_j) v_j]
//   z2 = [g0 v'_0 + sum_j g_j v'_j] / (i k)
__global__ void osrc_combine_kernel(int n, OsrcComb c, const double2 *__restrict__ sol,
                                    double2 *__restrict__ z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 a = cmul(c.cu, sol[i]);
    for (int j = 0; j < c.np; ++j) a = csub(a, cmul(c.a[j], sol[(size_t)(1 + j) * n + i]));
    double2 b = cmul(c.g0, sol[(size_t)(c.np + 1) * n + i]);
    for (int j = 0; j < c.np; ++j) b = cadd(b, cmul(c.g[j], sol[(size_t)(c.np + 2 + j) * n + i]));
    const double2 ik = c.ik_obj ? c.ik_obj[c.vcomp[i]] : c.ik;
    const double2 iik = c.ik_obj ? cdiv(cd(1.0, 0.0), ik) : c.iik;
    z[i] = cmul(ik, a);
    z[n + i] = cmul(iik, b);
}

// Largest cluster the kernels may use on each device: 16 CTAs (a
// non-portable size that the kernel opts into) if the device can schedule
// it, else 8; 0 until kry_opt_in has run on that device.
int g_kry_max_cluster[OSRC_MAX_DEVICES] = {};

int kry_opt_in() {
    static PerDeviceOnce once;
    return per_device_once(once, [](int dev) -> int {
        g_kry_max_cluster[dev] = 8;
        if (cudaFuncSetAttribute(kry_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
            (void)cudaGetLastError();
            return (int)OSRC_OK;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16, 1, 1);
        cfg.blockDim = dim3(KRY_THREADS, 1, 1);
        int size = 0;
        if (cudaOccupancyMaxPotentialClusterSize(&size, kry_kernel, &cfg) == cudaSuccess && size >= 16)
            g_kry_max_cluster[dev] = 16;
        (void)cudaGetLastError();
        return (int)OSRC_OK;
    });
}

// CTAs per system: about 640 rows each, at most the device's largest
// cluster (call after kry_opt_in).
int cluster_size_for(int n) {
    int dev = 0;
    const int mx = cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < OSRC_MAX_DEVICES &&
                           g_kry_max_cluster[dev] > 0
                       ? g_kry_max_cluster[dev]
                       : 8;
    int cs = (n + 639) / 640;
    if (cs < 1) cs = 1;
    if (cs > mx) cs = mx;
    return cs;
}

template <int RPT>
int kmix_attrs() {
    OSRC_CK(cudaFuncSetAttribute(kmix_kernel<RPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    OSRC_CK(cudaFuncSetAttribute(kmix_kernel<RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)KMIX_SMEM_MAX));
    return OSRC_OK;
}

// Decides once per problem whether the mixed-precision kernel serves its
// systems: every CTA's rows within KMIX_THREADS x KMIX_ROWS_PER_THREAD, its
// FP32 entries within KMIX_SMEM_MAX, and the device able to hold one cluster
// of that shape.
int kmix_decide(osrc_problem *pb, int cs) {
    if (pb->kmix_state >= 0) return OSRC_OK;
    pb->kmix_state = 0;
    const int n = pb->nv;
    if ((int)pb->ms_ptr_h.size() != n + 1) return OSRC_OK;
    const int rows = (n + cs - 1) / cs;
    const int rpt = (rows + KMIX_THREADS - 1) / KMIX_THREADS;
    if (rpt < 1 || rpt > KMIX_ROWS_PER_THREAD) return OSRC_OK;
    size_t smem = 0;
    for (int k = 0; k < cs; ++k) {
        const int r0 = std::min(n, k * rows), r1 = std::min(n, r0 + rows);
        const size_t ne = (size_t)(pb->ms_ptr_h[r1] - pb->ms_ptr_h[r0]);
        smem = std::max(smem, sizeof(float2) * ((ne + 1) & ~(size_t)1) + sizeof(int) * ne);
    }
    if (smem > KMIX_SMEM_MAX) return OSRC_OK;
    const int threads = ((rows + rpt - 1) / rpt + 31) / 32 * 32;
    static PerDeviceOnce once;
    const int attr_status = per_device_once(once, [](int) -> int {
        int st = kmix_attrs<1>();
        if (st == OSRC_OK) st = kmix_attrs<2>();
        return st;
    });
    if (attr_status != OSRC_OK) {  // no opt-in on this device: the FP64 kernel serves
        (void)cudaGetLastError();
        return OSRC_OK;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    const cudaError_t e = rpt == 1 ? cudaOccupancyMaxActiveClusters(&nclusters, kmix_kernel<1>, &cfg)
                                   : cudaOccupancyMaxActiveClusters(&nclusters, kmix_kernel<2>, &cfg);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return OSRC_OK;
    }
    if (nclusters < 1) return OSRC_OK;
    pb->kmix_state = 1;
    pb->kmix_rpt = rpt;
    pb->kmix_threads = threads;
    pb->kmix_smem = smem;
    return OSRC_OK;
}

static bool ranges_overlap(const double2 *a, const double2 *b, int n) {
    return a < b + n && b < a + n;
}

int launch_kry(osrc_problem *pb, const KryBatch &batch, cudaStream_t st) {
    OSRC_TRY(kry_opt_in());
    const int n = pb->nv;
    const int cs = cluster_size_for(n);
    OSRC_TRY(kmix_decide(pb, cs));
    bool mix = pb->kmix_state == 1;
    for (int k = 0; k < batch.nsys && mix; ++k)  // in-place systems stay on the FP64 kernel
        if (ranges_overlap(batch.s[k].f, batch.s[k].x, n)) mix = false;
    if (mix) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(batch.nsys * cs, 1, 1);
        cfg.blockDim = dim3(pb->kmix_threads, 1, 1);
        cfg.dynamicSmemBytes = pb->kmix_smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        float2 *w32 = reinterpret_cast<float2 *>(pb->d_kry.p);
        const int *ptr = pb->d_ms_ptr.p, *col = pb->d_ms_col.p;
        if (pb->kmix_rpt == 1)
            OSRC_CK(cudaLaunchKernelEx(&cfg, kmix_kernel<1>, batch, n, ptr, col, (const double *)pb->d_M.p,
                                       (const double *)pb->d_S.p, w32, pb->p.inner_tol, pb->p.inner_maxit,
                                       pb->d_kry_stat.p, pb->d_kry_res.p));
        else
            OSRC_CK(cudaLaunchKernelEx(&cfg, kmix_kernel<2>, batch, n, ptr, col, (const double *)pb->d_M.p,
                                       (const double *)pb->d_S.p, w32, pb->p.inner_tol, pb->p.inner_maxit,
                                       pb->d_kry_stat.p, pb->d_kry_res.p));
        pb->launches++;
        return OSRC_OK;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(batch.nsys * cs, 1, 1);
    cfg.blockDim = dim3(KRY_THREADS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    OSRC_CK(cudaLaunchKernelEx(&cfg, kry_kernel, batch, n, (const int *)pb->d_ms_ptr.p,
                               (const int *)pb->d_ms_col.p, (const double *)pb->d_M.p,
                               (const double *)pb->d_S.p, pb->d_kry.p, pb->p.inner_tol,
                               pb->p.inner_maxit, pb->d_kry_stat.p, pb->d_kry_res.p));
    pb->launches++;
    return OSRC_OK;
}

// Reads back the inner solver status (one small copy; the caller's stream is
// synchronised) and turns non-convergence into a status code.
int check_kry(osrc_problem *pb, int nsys, cudaStream_t st) {
    int stat[KRY_MAX_SYS];
    OSRC_CK(cudaMemcpyAsync(stat, pb->d_kry_stat.p, nsys * sizeof(int), cudaMemcpyDeviceToHost, st));
    OSRC_CK(cudaStreamSynchronize(st));
    return kry_status_host(pb, stat, nsys);
}

}  // namespace

int ms_build(osrc_problem *pb, const std::vector<int> &cptr, const std::vector<int> &cidx,
             cudaStream_t st) {
    osrc_mesh *m = pb->mesh;
    osrc_ctx *ctx = m->ctx;
    const int nt = pb->nt, nnz = pb->ms_nnz;
    DBuf<double> bm, bs;
    DBuf<int> d_cptr, d_cidx;
    OSRC_TRY(bm.alloc(ctx, 9 * (size_t)nt));
    OSRC_TRY(bs.alloc(ctx, 9 * (size_t)nt));
    OSRC_TRY(d_cptr.alloc(ctx, cptr.size()));
    OSRC_TRY(d_cidx.alloc(ctx, cidx.size()));
    OSRC_TRY(pb->d_M.alloc(ctx, nnz));
    OSRC_TRY(pb->d_S.alloc(ctx, nnz));
    OSRC_CK(cudaMemcpyAsync(d_cptr.p, cptr.data(), cptr.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    OSRC_CK(cudaMemcpyAsync(d_cidx.p, cidx.data(), cidx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    ms_element_kernel<<<(nt + 127) / 128, 128, 0, st>>>(nt, pb->d_tgeo.p, m->d_verts.p, m->d_tris.p,
                                                        bm.p, bs.p);
    csr_sum_kernel<<<(nnz + 255) / 256, 256, 0, st>>>(nnz, d_cptr.p, d_cidx.p, bm.p, bs.p, pb->d_M.p,
                                                      pb->d_S.p);
    pb->launches += 2;
    OSRC_CK(cudaGetLastError());
    // inner solver workspace: 2 N_Pade + 2 systems of 5 vectors, plus the
    // weak-form input and the solutions
    const int nsys = 2 * pb->p.n_pade + 2;
    OSRC_TRY(pb->d_kry.alloc(ctx, 5 * (size_t)nsys * pb->nv));
    OSRC_TRY(pb->d_kry_rhs.alloc(ctx, (size_t)(2 + nsys) * pb->nv));
    OSRC_TRY(pb->d_kry_stat.alloc(ctx, KRY_MAX_SYS));
    OSRC_TRY(pb->d_kry_res.alloc(ctx, KRY_MAX_SYS));
    OSRC_CK(cudaStreamSynchronize(st));
    return OSRC_OK;
}

int mass_solve(osrc_problem *pb, const double2 *x, double2 *y, cudaStream_t st) {
    const int n = pb->nv;
    KryBatch b{};
    b.nsys = 2;
    for (int k = 0; k < 2; ++k) {
        b.s[k].alpha = cd(1.0, 0.0);
        b.s[k].beta = cd(0.0, 0.0);
        b.s[k].f = x + (size_t)k * n;
        b.s[k].x = y + (size_t)k * n;
        b.s[k].conj = 1;
    }
    OSRC_TRY(launch_kry(pb, b, st));
    return check_kry(pb, 2, st);
}

// z = P M^-1 y for a weak-form vector y = [y1; y2] (Sec. 2.4, 2.6, 2.7).
// With u = M^-1 y and X = -M^-1 S / k_eps^2 the Pade terms are rewritten so
// that no system waits for another:
//   X (1 + B_j X)^-1 u1 = (u1 - v_j) / B_j,  (M - B_j S / k_eps^2) v_j = y1
//   (1 + B X)^-1 u2 = (M - B S / k_eps^2)^-1 y2
// so the mass solve of row 1 and all 2 N_Pade + 1 shifted systems run as one
// batched launch (row 2 needs no mass solve at all).
int osrc_precond_nsys(const osrc_problem *pb) {
    return pb->p.precond == OSRC_PRECOND_OSRC ? 2 * pb->p.n_pade + 2 : 2;
}

// both block rows of M^-1 y; rows swapped in the output when swap is set
static int mass_solve_async(osrc_problem *pb, const double2 *y, double2 *z, bool swap, cudaStream_t st) {
    const int n = pb->nv;
    KryBatch b{};
    b.nsys = 2;
    for (int k = 0; k < 2; ++k) {
        b.s[k].alpha = cd(1.0, 0.0);
        b.s[k].beta = cd(0.0, 0.0);
        b.s[k].f = y + (size_t)k * n;
        b.s[k].x = z + (size_t)(swap ? 1 - k : k) * n;
        b.s[k].conj = 1;
    }
    return launch_kry(pb, b, st);
}

int kry_status_host(osrc_problem *pb, const int *stat, int nsys) {
    int worst = 0;
    for (int i = 0; i < nsys; ++i) {
        if (stat[i] <= -1000000) return OSRC_BREAKDOWN;
        if (stat[i] < 0) return OSRC_NOT_CONVERGED;
        if (stat[i] > worst) worst = stat[i];
    }
    if (worst > pb->inner_last_max) pb->inner_last_max = worst;
    return OSRC_OK;
}

int osrc_precond_fused(osrc_problem *pb, const double2 *y, double2 *z, cudaStream_t st) {
    OSRC_TRY(osrc_precond_fused_async(pb, y, z, st));
    return check_kry(pb, osrc_precond_nsys(pb), st);
}

int osrc_precond_fused_async(osrc_problem *pb, const double2 *y, double2 *z, cudaStream_t st) {
    const int n = pb->nv, np = pb->p.n_pade;
    if (pb->p.precond == OSRC_PRECOND_MASS) return mass_solve_async(pb, y, z, false, st);
    if (pb->p.precond == OSRC_PRECOND_CALDERON) {
        // z = M^-1 B Pi M^-1 y: the first mass solve writes its rows swapped
        double2 *t = pb->d_kry_rhs.p + 2 * (size_t)n, *w = pb->d_tmp2.p + 2 * (size_t)n;
        OSRC_TRY(mass_solve_async(pb, y, t, true, st));
        if (pb->p.precision == OSRC_FP64_DENSE) OSRC_TRY(dense_apply(pb, t, w, st));
        else OSRC_TRY(far_apply(pb, t, w, OSRC_PART_ALL, st));
        return mass_solve_async(pb, w, z, false, st);
    }
    const double2 ke2 = cmul(pb->k_eps, pb->k_eps);
    // disjoint objects: 1/k_eps^2 of each row's object via KrySys::bscale
    const double2 inv_ke2 = pb->multi ? cd(1.0, 0.0) : cdiv(cd(1.0, 0.0), ke2);
    const double2 *bscale = pb->multi ? pb->d_obj_ike.p + pb->mesh->ncomp : nullptr;
    double2 *sol = pb->d_kry_rhs.p + 2 * (size_t)n;
    const double2 *y1 = y, *y2 = y + n;
    KryBatch b{};
    b.nsys = 2 * np + 2;
    b.vcomp = pb->mesh->d_vcomp.p;
    {   // M u1 = y1 (Hermitian CG)
        KrySys &s = b.s[0];
        s.alpha = cd(1.0, 0.0);
        s.beta = cd(0.0, 0.0);
        s.f = y1;
        s.x = sol;
        s.conj = 1;
    }
    for (int j = 0; j < np; ++j) {  // DtN: (M - B_j S / k_eps^2) v_j = y1
        KrySys &s = b.s[1 + j];
        s.alpha = cd(1.0, 0.0);
        s.beta = cscale(cmul(pb->B[j], inv_ke2), -1.0);
        s.bscale = bscale;
        s.f = y1;
        s.x = sol + (size_t)(1 + j) * n;
        s.conj = 0;
    }
    {   // NtD: (M - S / k_eps^2) v'_0 = y2
        KrySys &s = b.s[np + 1];
        s.alpha = cd(1.0, 0.0);
        s.beta = cscale(inv_ke2, -1.0);
        s.bscale = bscale;
        s.f = y2;
        s.x = sol + (size_t)(np + 1) * n;
        s.conj = 0;
    }
    for (int j = 0; j < np; ++j) {  // NtD: (M - B_j S / k_eps^2) v'_j = y2
        KrySys &s = b.s[np + 2 + j];
        s.alpha = cd(1.0, 0.0);
        s.beta = cscale(cmul(pb->B[j], inv_ke2), -1.0);
        s.bscale = bscale;
        s.f = y2;
        s.x = sol + (size_t)(np + 2 + j) * n;
        s.conj = 0;
    }
    OSRC_TRY(launch_kry(pb, b, st));
    OsrcComb c{};
    c.np = np;
    c.ik = cd(-pb->k_osrc_i, pb->k_osrc);  // i k_osrc (complex with attenuation)
    c.iik = cdiv(cd(1.0, 0.0), c.ik);
    c.ik_obj = pb->multi ? pb->d_obj_ike.p : nullptr;
    c.vcomp = pb->mesh->d_vcomp.p;
    double2 cu = pb->C0;
    for (int j = 0; j < np; ++j) {
        c.a[j] = cdiv(pb->A[j], pb->B[j]);
        cu = cadd(cu, c.a[j]);
        c.g[j] = pb->g[j];
    }
    c.cu = cu;
    c.g0 = pb->g0;
    osrc_combine_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, c, sol, z);
    pb->launches++;
    OSRC_CK(cudaGetLastError());
    return OSRC_OK;
}

// P x for a strong-form vector x: P x = P M^-1 (M x).
int osrc_precond(osrc_problem *pb, const double2 *x, double2 *y, cudaStream_t st) {
    const int n = pb->nv;
    double2 *mx = pb->d_kry_rhs.p;
    mass_spmv_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, pb->d_ms_ptr.p, pb->d_ms_col.p, pb->d_M.p, x,
                                                      mx);
    pb->launches++;
    OSRC_CK(cudaGetLastError());
    return osrc_precond_fused(pb, mx, y, st);
}

// ---------------------------------------------------------------------------
// Allocation-free batched shifted solve.
//
// Some callers cannot call cudaMalloc at the point where they need a solve:
// code that runs while a stream is being captured into a CUDA graph (an
// allocation there breaks or invalidates the capture), real-time or
// callback-driven hosts that forbid allocation after start-up, and
// frameworks whose device memory is owned by their own pool allocator.
// osrc_shifted_solve_noalloc serves them: it runs the same cluster-batched
// CG / COCG kernel as the library's mass and OSRC solves, but its Krylov
// workspace is the file-scope array below instead of memory from
// cudaMalloc, so the call allocates nothing.  The caller owns every input
// and output buffer.
//
// The array holds NOALLOC_MAX_ENTRIES complex entries per Krylov vector
// (5 vectors, 10 MiB in total) on every GPU that loads this library, until
// the process exits.  Every call on a device shares it, and it keeps the
// last call's contents; the kernel writes each scratch entry before reading
// it, so only the per-system status words need clearing, which every call
// does.  Calls whose kernels overlap on the GPU (two streams, or two host
// threads) race on the array: serialise them.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t NOALLOC_MAX_ENTRIES = 131072;  // nsys * n complex values per vector
constexpr int NOALLOC_MAX_SYS = 16;

static __device__ __align__(256) double2 g_noalloc_work[5 * NOALLOC_MAX_ENTRIES];
static __device__ __align__(256) int g_noalloc_stat[NOALLOC_MAX_SYS];
static __device__ __align__(256) double g_noalloc_res[NOALLOC_MAX_SYS];

struct NoAllocScratch {
    double2 *work = nullptr;
    int *stat = nullptr;
    double *res = nullptr;
    unsigned long long ctx_id = 0;  // context the addresses belong to
    bool ready = false;
};

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
NoAllocScratch g_noalloc[NOALLOC_MAX_DEVICES];

// Unique id of the context current on this host thread (driver entry
// points reached through the runtime, so no link against libcuda).  Ids are
// never reused, so a device reset, which replaces the primary context and
// with it the array's address, shows up as a new id.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);
int current_ctx_id(unsigned long long &id) {
    static PfnCtxGetCurrent get_cur = nullptr;
    static PfnCtxGetId get_id = nullptr;
    if (!get_cur || !get_id) {
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        OSRC_CK(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void **)&get_cur, 12000,
                                                 cudaEnableDefault, &q1));
        OSRC_CK(cudaGetDriverEntryPointByVersion("cuCtxGetId", (void **)&get_id, 12000,
                                                 cudaEnableDefault, &q2));
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !get_cur || !get_id) {
            osrc_set_error("driver entry points cuCtxGetCurrent / cuCtxGetId not found");
            return OSRC_UNSUPPORTED;
        }
    }
    CUcontext c = nullptr;
    if (get_cur(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) {
        osrc_set_error("no current CUDA context");
        return OSRC_CUDA_ERROR;
    }
    return OSRC_OK;
}

// Device address of the scratch array on the current device.  Looked up
// with cudaGetSymbolAddress (that device current) on the first call on a
// device and again whenever the device's context has changed since (after
// cudaDeviceReset), so a kernel is never given an address of a context that
// no longer exists.
int noalloc_scratch(int dev, NoAllocScratch &out) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return OSRC_UNSUPPORTED;
    // makes the device's primary context current (created if needed)
    OSRC_CK(cudaSetDevice(dev));
    unsigned long long id = 0;
    OSRC_TRY(current_ctx_id(id));
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocScratch &s = g_noalloc[dev];
    if (!s.ready || s.ctx_id != id) {
        s.ready = false;
        OSRC_CK(cudaGetSymbolAddress((void **)&s.work, g_noalloc_work));
        OSRC_CK(cudaGetSymbolAddress((void **)&s.stat, g_noalloc_stat));
        OSRC_CK(cudaGetSymbolAddress((void **)&s.res, g_noalloc_res));
        s.ctx_id = id;
        s.ready = true;
    }
    out = s;
    return OSRC_OK;
}

}  // namespace

extern "C" int osrc_shifted_solve_noalloc(int n, const int32_t *row_ptr, const int32_t *col_idx,
                                          const double *M_vals, const double *S_vals, int nsys,
                                          const double *alpha, const double *beta, const void *f,
                                          void *w, double tol, int maxit, int conj,
                                          int *iters_out, void *stream) {
    if (n < 1 || nsys < 1 || nsys > NOALLOC_MAX_SYS || !row_ptr || !col_idx || !M_vals ||
        !S_vals || !alpha || !beta || !f || !w || !(tol > 0.0) || tol > 1e-4 || maxit < 1 ||
        (conj != 0 && conj != 1)) {
        osrc_set_error("osrc_shifted_solve_noalloc: invalid argument");
        return OSRC_INVALID_ARG;
    }
    if ((size_t)n * (size_t)nsys > NOALLOC_MAX_ENTRIES) {
        osrc_set_error("osrc_shifted_solve_noalloc: nsys * n exceeds the static scratch "
                       "capacity of 131072 complex entries");
        return OSRC_INVALID_ARG;
    }
    int dev = 0;
    OSRC_CK(cudaGetDevice(&dev));
    NoAllocScratch sc;
    OSRC_TRY(noalloc_scratch(dev, sc));
    cudaStream_t st = (cudaStream_t)stream;
    KryBatch b{};
    b.nsys = nsys;
    for (int s = 0; s < nsys; ++s) {
        b.s[s].alpha = cd(alpha[2 * s], alpha[2 * s + 1]);
        b.s[s].beta = cd(beta[2 * s], beta[2 * s + 1]);
        b.s[s].f = (const double2 *)f + (size_t)s * n;
        b.s[s].x = (double2 *)w + (size_t)s * n;
        b.s[s].conj = conj;
    }
    OSRC_TRY(kry_opt_in());
    // status words start as "not written" so that a failed launch is seen
    OSRC_CK(cudaMemsetAsync(sc.stat, 0x80, nsys * sizeof(int), st));
    const int cs = cluster_size_for(n);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nsys * cs, 1, 1);
    cfg.blockDim = dim3(KRY_THREADS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    OSRC_CK(cudaLaunchKernelEx(&cfg, kry_kernel, b, n, (const int *)row_ptr, (const int *)col_idx,
                               M_vals, S_vals, sc.work, tol, maxit, sc.stat, sc.res));
    if (!iters_out) return OSRC_OK;
    OSRC_CK(cudaMemcpyAsync(iters_out, sc.stat, nsys * sizeof(int), cudaMemcpyDeviceToHost, st));
    OSRC_CK(cudaStreamSynchronize(st));
    int status = OSRC_OK;
    for (int s = 0; s < nsys; ++s) {
        if (iters_out[s] <= -1000000) status = OSRC_BREAKDOWN;
        else if (iters_out[s] < 0 && status == OSRC_OK) status = OSRC_NOT_CONVERGED;
    }
    return status;
}
