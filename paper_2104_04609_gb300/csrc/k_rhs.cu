// k_rhs.cu -- right-hand side of the PMCHWT system (Sec. 2.7): the Dirichlet
// and Neumann traces of the incident field tested against the P1 hat
// functions, b = [<u_inc, phi_i>; <du_inc/dn, phi_i>], FP64, 6-point rule per
// triangle, gathered per vertex (no atomics).
#include "osrc_internal.cuh"

namespace {

constexpr double kRa1 = 0.445948490915965, kRw1 = 0.223381589678011;
constexpr double kRa2 = 0.091576213509771, kRw2 = 0.109951743655322;

// kind 0: plane wave exp(i k d.x), src = d;  kind 1: point source
// exp(i k |x - x0|) / (4 pi |x - x0|), src = x0.
__global__ void rhs_kernel(int nv, const int *__restrict__ vt_ptr, const int *__restrict__ vt_idx,
                           const int *__restrict__ tris, const double *__restrict__ verts,
                           const double *__restrict__ tgeo, double k, int kind, double s0,
                           double s1, double s2, double2 *__restrict__ b) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double2 b1 = cd(0, 0), b2 = cd(0, 0);
    for (int e = vt_ptr[v]; e < vt_ptr[v + 1]; ++e) {
        const int t = vt_idx[e] / 3, a = vt_idx[e] % 3;
        const double *g = tgeo + 16 * (size_t)t;
        const double area = g[0], n0 = g[1], n1 = g[2], n2 = g[3];
        const double *P0 = verts + 3 * tris[3 * t], *P1 = verts + 3 * tris[3 * t + 1],
                     *P2 = verts + 3 * tris[3 * t + 2];
        for (int q = 0; q < 6; ++q) {
            const double al = q < 3 ? kRa1 : kRa2, w = q < 3 ? kRw1 : kRw2;
            double bc[3] = {al, al, al};
            bc[q % 3] = 1.0 - 2.0 * al;
            double x[3];
            for (int j = 0; j < 3; ++j) x[j] = bc[0] * P0[j] + bc[1] * P1[j] + bc[2] * P2[j];
            double2 u, dn;
            if (kind == 0) {
                double sn, cs;
                sincos(k * (s0 * x[0] + s1 * x[1] + s2 * x[2]), &sn, &cs);
                u = cd(cs, sn);
                dn = cmul(cd(0.0, k * (s0 * n0 + s1 * n1 + s2 * n2)), u);
            } else {
                const double d0 = x[0] - s0, d1 = x[1] - s1, d2 = x[2] - s2;
                const double R = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                double sn, cs;
                sincos(k * R, &sn, &cs);
                const double f = 0.079577471545947667884 / R;
                u = cd(cs * f, sn * f);
                dn = cscale(cmul(u, cd(-1.0, k * R)), (d0 * n0 + d1 * n1 + d2 * n2) / (R * R));
            }
            const double wl = w * area * bc[a];
            b1 = cadd(b1, cscale(u, wl));
            b2 = cadd(b2, cscale(dn, wl));
        }
    }
    b[v] = b1;
    b[nv + v] = b2;
}

}  // namespace

int rhs_build(osrc_problem *pb, int kind, const double *src3, double2 *b, cudaStream_t st) {
    osrc_mesh *m = pb->mesh;
    const int nv = pb->nv;
    rhs_kernel<<<(nv + 127) / 128, 128, 0, st>>>(nv, m->d_vt_ptr.p, m->d_vt_idx.p, m->d_tris.p,
                                                 m->d_verts.p, pb->d_tgeo.p, pb->p.k_ext, kind,
                                                 src3[0], src3[1], src3[2], b);
    pb->launches++;
    OSRC_CK(cudaGetLastError());
    return OSRC_OK;
}
