// k_field.cu -- total pressure at points off the surface from a solution of
// the permuted PMCHWT system (Sec. 2.2, representation formulas; the paper
// measures its accuracy this way on a grid through the object, Sec. 3.2).
//
// With psi = exterior normal derivative and phi = trace of the total field
// (outward normal), rho = rho_int / rho_ext:
//   outside: u = u_inc + DLP_0 phi - SLP_0 psi
//   inside:  u = rho SLP_1 psi - DLP_1 phi
//   SLP_k psi(x) = int G_k(x, y) psi(y) dy,  DLP_k phi(x) = int dG_k/dn_y phi(y) dy,
// each integral by the 6-point rule per triangle with the P1 densities
// interpolated at the rule points.  A point's region comes from the Laplace
// double layer of the constant 1 (Gauss: 1 inside, 0 outside), so each
// target needs one wavenumber only and a warp never diverges in the pair loop.
// Disjoint objects (Sec. 2.2): source points are stored object by object;
// a point inside object m (region m + 1) takes the interior representation
// over that object's surface with its own material.
// Pass 1 (region) runs in FP32; pass 2 (field) in FP64, source points staged
// through shared memory in tiles of FT.
#include "osrc_internal.cuh"

namespace {

constexpr double kFa1 = 0.445948490915965, kFw1 = 0.223381589678011;
constexpr double kFa2 = 0.091576213509771, kFw2 = 0.109951743655322;
constexpr double kFInv4Pi = 0.079577471545947667884;
constexpr int FT = 128;

// Source data per rule point (6 per triangle): {y, w |tau|}, {n, 0},
// {psi_q re, im, phi_q re, im}.
__global__ void field_src_kernel(int nt, int nv, const int *__restrict__ tris, const double *__restrict__ verts,
                                 const double *__restrict__ tgeo, const int *__restrict__ order,
                                 const double2 *__restrict__ x, double4 *__restrict__ src) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 6 * nt) return;
    const int t = order[idx / 6], q = idx % 6;
    const double al = q < 3 ? kFa1 : kFa2, w = q < 3 ? kFw1 : kFw2;
    double bc[3] = {al, al, al};
    bc[q % 3] = 1.0 - 2.0 * al;
    double y[3] = {0, 0, 0};
    double2 ps = cd(0, 0), ph = cd(0, 0);
    for (int a = 0; a < 3; ++a) {
        const int v = tris[3 * t + a];
        for (int j = 0; j < 3; ++j) y[j] += bc[a] * verts[3 * v + j];
        ps = cadd(ps, cscale(x[v], bc[a]));
        ph = cadd(ph, cscale(x[nv + v], bc[a]));
    }
    const double *g = tgeo + 16 * (size_t)t;
    src[3 * (size_t)idx] = make_double4(y[0], y[1], y[2], w * g[0]);
    src[3 * (size_t)idx + 1] = make_double4(g[1], g[2], g[3], 0.0);
    src[3 * (size_t)idx + 2] = make_double4(ps.x, ps.y, ph.x, ph.y);
}

// region[i] = m + 1 if the solid angle of object m's surface at the point,
// sum_q w_q (y_q - x).n_q / (4 pi r^3), exceeds 1/2 (inside object m), else 0.
// obeg: [nobj + 1] source-point ranges of the objects.
__global__ void __launch_bounds__(FT)
field_region_kernel(int npts, const double *__restrict__ pts, int nobj, const int *__restrict__ obeg,
                    const double4 *__restrict__ src, int *__restrict__ region) {
    __shared__ float4 sy[FT], sn[FT];
    const int i = blockIdx.x * FT + threadIdx.x;
    const bool valid = i < npts;
    const float x0 = valid ? (float)pts[3 * (size_t)i] : 0.f, x1 = valid ? (float)pts[3 * (size_t)i + 1] : 0.f,
                x2 = valid ? (float)pts[3 * (size_t)i + 2] : 0.f;
    int reg = 0;
    for (int m = 0; m < nobj; ++m) {
        const int b0 = obeg[m], b1 = obeg[m + 1];
        double total = 0.0;
        for (int base = b0; base < b1; base += FT) {
            const int j = base + threadIdx.x;
            if (j < b1) {
                const double4 a = src[3 * (size_t)j], b = src[3 * (size_t)j + 1];
                sy[threadIdx.x] = make_float4((float)a.x, (float)a.y, (float)a.z, (float)a.w);
                sn[threadIdx.x] = make_float4((float)b.x, (float)b.y, (float)b.z, 0.f);
            }
            __syncthreads();
            const int jn = min(FT, b1 - base);
            float acc = 0.f;
            for (int jj = 0; jj < jn; ++jj) {
                const float4 y = sy[jj], n = sn[jj];
                const float d0 = y.x - x0, d1 = y.y - x1, d2 = y.z - x2;
                const float ri = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
                acc += y.w * (d0 * n.x + d1 * n.y + d2 * n.z) * ri * ri * ri;
            }
            total += (double)acc;
            __syncthreads();
        }
        if (total * kFInv4Pi > 0.5) reg = m + 1;
    }
    if (valid) region[i] = reg;
}

struct FieldConst {
    double k0;
    int inc_kind;  // 0 none, 1 plane wave (s = direction), 2 point source (s = position)
    double s0, s1, s2;
};

__global__ void __launch_bounds__(FT)
field_kernel(int npts, const double *__restrict__ pts, int ns, const int *__restrict__ obeg,
             const ObjMat *__restrict__ obj, const double4 *__restrict__ src, const int *__restrict__ region,
             FieldConst c, double2 *__restrict__ u) {
    __shared__ double4 sa[FT], sb[FT], sc[FT];
    const int i = blockIdx.x * FT + threadIdx.x;
    const bool valid = i < npts;
    const double x0 = valid ? pts[3 * (size_t)i] : 0.0, x1 = valid ? pts[3 * (size_t)i + 1] : 0.0,
                 x2 = valid ? pts[3 * (size_t)i + 2] : 0.0;
    const int ins = valid ? region[i] : 0;
    // outside: every source point, k0; inside object m: its own points, k_m
    const double k = ins ? obj[ins - 1].k1 : c.k0;
    const double ki = ins ? obj[ins - 1].k1i : 0.0;  // attenuation inside
    const int lo = ins ? obeg[ins - 1] : 0, hi = ins ? obeg[ins] : ns;
    double2 S = cd(0, 0), D = cd(0, 0);
    for (int base = 0; base < ns; base += FT) {
        const int j = base + threadIdx.x;
        if (j < ns) {
            sa[threadIdx.x] = src[3 * (size_t)j];
            sb[threadIdx.x] = src[3 * (size_t)j + 1];
            sc[threadIdx.x] = src[3 * (size_t)j + 2];
        }
        __syncthreads();
        const int j0 = max(0, lo - base), j1 = min(FT, min(ns, hi) - base);
        for (int jj = j0; jj < j1; ++jj) {
            const double4 a = sa[jj], n = sb[jj], dv = sc[jj];
            const double d0 = a.x - x0, d1 = a.y - x1, d2 = a.z - x2;  // y - x
            const double ri = rsqrt(d0 * d0 + d1 * d1 + d2 * d2);
            const double r = (d0 * d0 + d1 * d1 + d2 * d2) * ri;
            double sn_, cs_;
            sincos(k * r, &sn_, &cs_);
            const double f = a.w * kFInv4Pi * ri * (ki != 0.0 ? exp(-ki * r) : 1.0);
            const double2 g = cd(cs_ * f, sn_ * f);                        // w G
            S = cadd(S, cmul(g, cd(dv.x, dv.y)));                          // w G psi_q
            const double dn = (d0 * n.x + d1 * n.y + d2 * n.z) * ri * ri;  // (y - x).n / r^2
            const double2 h = cscale(cmul(g, cd(-1.0 - ki * r, k * r)), dn);  // w dG/dn_y
            D = cadd(D, cmul(h, cd(dv.z, dv.w)));
        }
        __syncthreads();
    }
    if (!valid) return;
    double2 out;
    if (ins) {
        out = csub(cscale(S, obj[ins - 1].rho), D);
    } else {
        double2 inc = cd(0, 0);
        if (c.inc_kind == 1) {
            double sn_, cs_;
            sincos(c.k0 * (c.s0 * x0 + c.s1 * x1 + c.s2 * x2), &sn_, &cs_);
            inc = cd(cs_, sn_);
        } else if (c.inc_kind == 2) {
            const double e0 = x0 - c.s0, e1 = x1 - c.s1, e2 = x2 - c.s2;
            const double R = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
            double sn_, cs_;
            sincos(c.k0 * R, &sn_, &cs_);
            inc = cd(cs_ * kFInv4Pi / R, sn_ * kFInv4Pi / R);
        }
        out = csub(cadd(inc, D), S);
    }
    u[i] = out;
}

}  // namespace

extern "C" int osrc_field_eval(osrc_problem *pb, const void *x, const double *pts, int npts, int inc_kind,
                               const double *inc_param, void *u, int *region, void *stream) {
    if (!pb || !x || npts < 0 || inc_kind < 0 || inc_kind > 2 || (inc_kind && !inc_param))
        return OSRC_INVALID_ARG;
    if (npts == 0) return OSRC_OK;
    if (!pts || !u) return OSRC_INVALID_ARG;
    OSRC_CK(cudaSetDevice(pb->mesh->ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    osrc_mesh *m = pb->mesh;
    const int nt = pb->nt, ns = 6 * nt;
    if (pb->d_fsrc.n < 3 * (size_t)ns) OSRC_TRY(pb->d_fsrc.alloc(m->ctx, 3 * (size_t)ns));
    int *reg = region;
    if (!reg) {
        if (pb->d_freg.n < (size_t)npts) OSRC_TRY(pb->d_freg.alloc(m->ctx, npts));
        reg = pb->d_freg.p;
    }
    if (pb->d_fobeg.n < (size_t)m->ncomp + 1) {
        OSRC_TRY(pb->d_fobeg.alloc(m->ctx, m->ncomp + 1));
        std::vector<int> ob(m->ncomp + 1);
        for (int c = 0; c <= m->ncomp; ++c) ob[c] = 6 * m->comp_tbeg[c];
        OSRC_CK(cudaMemcpy(pb->d_fobeg.p, ob.data(), ob.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    field_src_kernel<<<(ns + 255) / 256, 256, 0, st>>>(nt, pb->nv, m->d_tris.p, m->d_verts.p, pb->d_tgeo.p,
                                                       m->d_tri_order.p, (const double2 *)x, pb->d_fsrc.p);
    const unsigned nb = (unsigned)((npts + FT - 1) / FT);
    field_region_kernel<<<nb, FT, 0, st>>>(npts, pts, m->ncomp, pb->d_fobeg.p, pb->d_fsrc.p, reg);
    FieldConst c{pb->p.k_ext, inc_kind, 0.0, 0.0, 0.0};
    if (inc_kind) {
        c.s0 = inc_param[0];
        c.s1 = inc_param[1];
        c.s2 = inc_param[2];
    }
    field_kernel<<<nb, FT, 0, st>>>(npts, pts, ns, pb->d_fobeg.p, pb->d_obj.p, pb->d_fsrc.p, reg, c,
                                    (double2 *)u);
    pb->launches += 3;
    OSRC_CK(cudaGetLastError());
    return OSRC_OK;
}
