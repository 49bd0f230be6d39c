// osrc_api.cu -- the C ABI (include/osrc_pmchwt.h): contexts, meshes,
// problems, operator applies and the GMRES driver.  Host code here builds
// the mesh topology (incidence, touching triangle pairs, CSR patterns and
// the deterministic contribution lists that the device kernels sum); all
// arithmetic of the method runs in the kernels of k_*.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "osrc_internal.cuh"

// ---------------------------------------------------------------------------
// errors and memory accounting
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;
void osrc_set_error(const std::string &msg) { g_last_error = msg; }

extern "C" const char *osrc_status_string(int s) {
    switch (s) {
        case OSRC_OK: return "OSRC_OK";
        case OSRC_INVALID_ARG: return "OSRC_INVALID_ARG";
        case OSRC_OUT_OF_MEMORY: return "OSRC_OUT_OF_MEMORY";
        case OSRC_CUDA_ERROR: return "OSRC_CUDA_ERROR";
        case OSRC_NOT_CONVERGED: return "OSRC_NOT_CONVERGED";
        case OSRC_BREAKDOWN: return "OSRC_BREAKDOWN";
        case OSRC_TIMEOUT: return "OSRC_TIMEOUT";
        case OSRC_UNSUPPORTED: return "OSRC_UNSUPPORTED";
        default: return "OSRC_UNKNOWN_STATUS";
    }
}

int ctx_alloc(osrc_ctx *ctx, void **p, size_t bytes) {
    *p = nullptr;
    // reserve against the budget first (atomically: allocations may come from
    // several host threads), give the reservation back if cudaMalloc fails
    size_t cur = ctx->used.load();
    do {
        if (ctx->budget && cur + bytes > ctx->budget) {
            osrc_set_error("device memory budget exceeded");
            return OSRC_OUT_OF_MEMORY;
        }
    } while (!ctx->used.compare_exchange_weak(cur, cur + bytes));
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        ctx->used -= bytes;
        osrc_set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return OSRC_OUT_OF_MEMORY;
    }
    return OSRC_OK;
}

void ctx_free(osrc_ctx *ctx, void *p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    ctx->used -= bytes;
}

extern "C" void osrc_params_default(osrc_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->k_ext = 1.0;
    p->k_int = 1.0;
    p->rho_ratio = 1.0;
    p->n_pade = 4;
    p->theta = M_PI / 3.0;
    p->damping_R = 0.0;
    p->osrc_side = 1;
    p->n_ss = 4;
    p->precision = OSRC_FP32_MATFREE;
    p->inner_tol = 1e-10;
    p->inner_maxit = 2000;
    p->precond = OSRC_PRECOND_OSRC;
    p->formulation = OSRC_PMCHWT;
    p->k_int_im = 0.0;
    p->dense_assembly = OSRC_ASSEMBLE_FP64;
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" int osrc_create(osrc_ctx **out, int device, size_t budget) {
    if (!out) return OSRC_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    OSRC_CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return OSRC_INVALID_ARG;
    OSRC_CK(cudaSetDevice(device));
    cudaDeviceProp prop;
    OSRC_CK(cudaGetDeviceProperties(&prop, device));
    if (prop.major < 10) {
        osrc_set_error("this library is built for sm_103a (GB300)");
        return OSRC_UNSUPPORTED;
    }
    osrc_ctx *c = new osrc_ctx;
    c->device = device;
    c->budget = budget;
    *out = c;
    return OSRC_OK;
}

extern "C" void osrc_destroy(osrc_ctx *ctx) { delete ctx; }
extern "C" size_t osrc_mem_used(const osrc_ctx *ctx) { return ctx ? ctx->used.load() : 0; }

// ---------------------------------------------------------------------------
// mesh
// ---------------------------------------------------------------------------
extern "C" int osrc_mesh_validate(const double *verts, int32_t nv, const int32_t *tris, int32_t nt) {
    if (!verts || !tris || nv < 4 || nt < 4) {
        osrc_set_error("mesh needs at least 4 vertices and 4 triangles");
        return OSRC_INVALID_ARG;
    }
    for (long long i = 0; i < 3LL * nv; ++i)
        if (!std::isfinite(verts[i])) {
            osrc_set_error("non-finite vertex coordinate");
            return OSRC_INVALID_ARG;
        }
    std::vector<char> used(nv, 0);
    std::unordered_map<uint64_t, int> edges;
    edges.reserve(3 * (size_t)nt * 2);
    for (int t = 0; t < nt; ++t) {
        const int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
        if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) {
            osrc_set_error("triangle index out of range");
            return OSRC_INVALID_ARG;
        }
        if (a == b || b == c || a == c) {
            osrc_set_error("triangle with a repeated vertex");
            return OSRC_INVALID_ARG;
        }
        used[a] = used[b] = used[c] = 1;
        const double *P0 = verts + 3 * a, *P1 = verts + 3 * b, *P2 = verts + 3 * c;
        double e1[3], e2[3];
        for (int j = 0; j < 3; ++j) {
            e1[j] = P1[j] - P0[j];
            e2[j] = P2[j] - P0[j];
        }
        const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                     cz = e1[0] * e2[1] - e1[1] * e2[0];
        const double l1 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
        const double l2 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
        const double a2 = cx * cx + cy * cy + cz * cz;
        if (!(a2 > 1e-24 * l1 * l2) || l1 == 0.0 || l2 == 0.0) {
            osrc_set_error("zero-area triangle");
            return OSRC_INVALID_ARG;
        }
        const int vv[3] = {a, b, c};
        for (int k = 0; k < 3; ++k) {
            const uint64_t key = ((uint64_t)(uint32_t)vv[k] << 32) | (uint32_t)vv[(k + 1) % 3];
            if (++edges[key] > 1) {
                osrc_set_error("directed edge used twice: inconsistent orientation or non-manifold");
                return OSRC_INVALID_ARG;
            }
        }
    }
    for (const auto &kv : edges) {
        const uint64_t rev = (kv.first << 32) | (kv.first >> 32);
        if (edges.find(rev) == edges.end()) {
            osrc_set_error("open mesh: an edge has no opposite triangle");
            return OSRC_INVALID_ARG;
        }
    }
    for (int i = 0; i < nv; ++i)
        if (!used[i]) {
            osrc_set_error("vertex not used by any triangle");
            return OSRC_INVALID_ARG;
        }
    return OSRC_OK;
}

extern "C" int osrc_mesh_create(osrc_ctx *ctx, const double *verts, int32_t nv,
                                const int32_t *tris, int32_t nt, osrc_mesh **out) {
    if (!ctx || !out) return OSRC_INVALID_ARG;
    *out = nullptr;
    OSRC_TRY(osrc_mesh_validate(verts, nv, tris, nt));
    OSRC_CK(cudaSetDevice(ctx->device));
    osrc_mesh *m = new osrc_mesh;
    m->ctx = ctx;
    m->nv = nv;
    m->nt = nt;
    m->verts.assign(verts, verts + 3 * (size_t)nv);
    m->tris.assign(tris, tris + 3 * (size_t)nt);
    // vertex -> (3 t + local) incidence, in triangle order
    m->vt_ptr.assign(nv + 1, 0);
    for (int k = 0; k < 3 * nt; ++k) m->vt_ptr[tris[k] + 1]++;
    for (int i = 0; i < nv; ++i) m->vt_ptr[i + 1] += m->vt_ptr[i];
    m->vt_idx.assign(3 * (size_t)nt, 0);
    {
        std::vector<int> fill(m->vt_ptr.begin(), m->vt_ptr.end() - 1);
        for (int k = 0; k < 3 * nt; ++k) m->vt_idx[fill[tris[k]]++] = k;
    }
    // mean edge length over unique edges
    double sum = 0.0;
    long long cnt = 0;
    for (int t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) {
            const int a = tris[3 * t + k], b = tris[3 * t + (k + 1) % 3];
            if (a < b) {
                double d2 = 0.0;
                for (int j = 0; j < 3; ++j) {
                    const double d = verts[3 * a + j] - verts[3 * b + j];
                    d2 += d * d;
                }
                sum += std::sqrt(d2);
                ++cnt;
            }
        }
    m->mean_edge = cnt ? sum / cnt : 0.0;
    // objects: union-find over vertices joined by triangle edges, numbered in
    // the order of each object's first triangle
    {
        std::vector<int> par(nv);
        for (int i = 0; i < nv; ++i) par[i] = i;
        auto root = [&](int a) {
            while (par[a] != a) a = par[a] = par[par[a]];
            return a;
        };
        for (int t = 0; t < nt; ++t)
            for (int k = 1; k < 3; ++k) {
                const int a = root(tris[3 * t]), b = root(tris[3 * t + k]);
                if (a != b) par[std::max(a, b)] = std::min(a, b);
            }
        std::vector<int> id(nv, -1);
        m->tcomp.assign(nt, 0);
        int nc = 0;
        for (int t = 0; t < nt; ++t) {
            const int r = root(tris[3 * t]);
            if (id[r] < 0) id[r] = nc++;
            m->tcomp[t] = id[r];
        }
        m->ncomp = nc;
        m->vcomp.assign(nv, 0);
        for (int v = 0; v < nv; ++v) m->vcomp[v] = id[root(v)];
        m->comp_tbeg.assign(nc + 1, 0);
        for (int t = 0; t < nt; ++t) m->comp_tbeg[m->tcomp[t] + 1]++;
        for (int c = 0; c < nc; ++c) m->comp_tbeg[c + 1] += m->comp_tbeg[c];
        m->tri_order.assign(nt, 0);
        std::vector<int> fill(m->comp_tbeg.begin(), m->comp_tbeg.end() - 1);
        for (int t = 0; t < nt; ++t) m->tri_order[fill[m->tcomp[t]]++] = t;
    }
    int s;
    if ((s = m->d_verts.alloc(ctx, 3 * (size_t)nv)) || (s = m->d_tris.alloc(ctx, 3 * (size_t)nt)) ||
        (s = m->d_vt_ptr.alloc(ctx, nv + 1)) || (s = m->d_vt_idx.alloc(ctx, 3 * (size_t)nt)) ||
        (s = m->d_tcomp.alloc(ctx, nt)) || (s = m->d_vcomp.alloc(ctx, nv)) ||
        (s = m->d_tri_order.alloc(ctx, nt))) {
        delete m;
        return s;
    }
    cudaError_t e = cudaMemcpy(m->d_verts.p, verts, 3 * (size_t)nv * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_tris.p, tris, 3 * (size_t)nt * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_vt_ptr.p, m->vt_ptr.data(), (nv + 1) * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_vt_idx.p, m->vt_idx.data(), 3 * (size_t)nt * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_tcomp.p, m->tcomp.data(), nt * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_vcomp.p, m->vcomp.data(), nv * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_tri_order.p, m->tri_order.data(), nt * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        osrc_set_error(std::string("mesh upload: ") + cudaGetErrorString(e));
        delete m;
        return OSRC_CUDA_ERROR;
    }
    *out = m;
    return OSRC_OK;
}

extern "C" void osrc_mesh_destroy(osrc_mesh *m) { delete m; }
extern "C" double osrc_mesh_mean_edge(const osrc_mesh *m) { return m ? m->mean_edge : 0.0; }
extern "C" int osrc_mesh_objects(const osrc_mesh *m) { return m ? m->ncomp : 0; }

// ---------------------------------------------------------------------------
// problem set-up: topology on the host, numerics on the device
// ---------------------------------------------------------------------------
namespace {

// Shared-vertex type of triangles t, s and the local orders that put the
// shared vertices first (same order in both), packed 2 bits per index.
int touch_case(const int *t, const int *s, int &perm) {
    int pt[3], ps[3], n = 0;
    bool ut[3] = {false, false, false}, us[3] = {false, false, false};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (t[a] == s[b]) {
                pt[n] = a;
                ps[n] = b;
                ut[a] = us[b] = true;
                ++n;
            }
    if (n == 0) return 0;
    int kt = n, ks = n;
    for (int a = 0; a < 3; ++a) if (!ut[a]) pt[kt++] = a;
    for (int b = 0; b < 3; ++b) if (!us[b]) ps[ks++] = b;
    perm = 0;
    for (int a = 0; a < 3; ++a) perm |= (pt[a] << (2 * a)) | (ps[a] << (6 + 2 * a));
    return n;
}

// Counting sort of (position, index) contributions into CSR-like lists.
void bucket(int nbuckets, const std::vector<int> &pos, const std::vector<int> &idx,
            std::vector<int> &ptr, std::vector<int> &out) {
    ptr.assign(nbuckets + 1, 0);
    for (int p : pos) ptr[p + 1]++;
    for (int i = 0; i < nbuckets; ++i) ptr[i + 1] += ptr[i];
    out.assign(pos.size(), 0);
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (size_t k = 0; k < pos.size(); ++k) out[fill[pos[k]]++] = idx[k];
}

int find_col(const std::vector<int> &ptr, const std::vector<int> &col, int i, int j) {
    auto b = col.begin() + ptr[i], e = col.begin() + ptr[i + 1];
    auto it = std::lower_bound(b, e, j);
    return (it != e && *it == j) ? (int)(it - col.begin()) : -1;
}

void pade_coefficients(int np, double theta, std::complex<double> &C0,
                       std::vector<std::complex<double>> &A, std::vector<std::complex<double>> &B) {
    using cdbl = std::complex<double>;
    const cdbl I(0.0, 1.0);
    const cdbl z0 = std::exp(-I * theta) - 1.0;
    cdbl R0 = 1.0;
    A.resize(np);
    B.resize(np);
    for (int j = 1; j <= np; ++j) {
        const double sj = std::sin(j * M_PI / (2.0 * np + 1.0));
        const double aj = 2.0 / (2.0 * np + 1.0) * sj * sj;
        const double cj = std::cos(j * M_PI / (2.0 * np + 1.0));
        const double bj = cj * cj;
        const cdbl den = 1.0 + bj * z0;
        R0 += aj * z0 / den;
        A[j - 1] = std::exp(-0.5 * I * theta) * aj / (den * den);
        B[j - 1] = std::exp(-I * theta) * bj / den;
    }
    C0 = std::exp(0.5 * I * theta) * R0;
}

}  // namespace

static int problem_create(osrc_mesh *mesh, const osrc_params *prm, const double *k_int_obj,
                          const double *rho_obj, osrc_problem **out, void *stream);

extern "C" int osrc_problem_create(osrc_mesh *mesh, const osrc_params *prm, osrc_problem **out,
                                   void *stream) {
    if (!mesh || !prm || !out) return OSRC_INVALID_ARG;
    std::vector<double> k(mesh->ncomp, prm->k_int), r(mesh->ncomp, prm->rho_ratio);
    return problem_create(mesh, prm, k.data(), r.data(), out, stream);
}

extern "C" int osrc_problem_create_objects(osrc_mesh *mesh, const osrc_params *prm, int nobj,
                                           const double *k_int, const double *rho_ratio, osrc_problem **out,
                                           void *stream) {
    if (!mesh || !prm || !out || !k_int || !rho_ratio) return OSRC_INVALID_ARG;
    if (nobj != mesh->ncomp) {
        osrc_set_error("osrc_problem_create_objects: nobj differs from the mesh's number of objects");
        return OSRC_INVALID_ARG;
    }
    for (int m = 0; m < nobj; ++m)
        if (!(k_int[m] > 0.0) || !std::isfinite(k_int[m]) || !(rho_ratio[m] > 0.0) || !std::isfinite(rho_ratio[m]))
            return OSRC_INVALID_ARG;
    osrc_params p = *prm;
    p.k_int = k_int[0];
    p.rho_ratio = rho_ratio[0];
    return problem_create(mesh, &p, k_int, rho_ratio, out, stream);
}

static int problem_create(osrc_mesh *mesh, const osrc_params *prm, const double *k_int_obj,
                          const double *rho_obj, osrc_problem **out, void *stream) {
    *out = nullptr;
    const osrc_params &p = *prm;
    if (!(p.k_ext > 0.0) || !(p.k_int > 0.0) || !std::isfinite(p.k_ext) || !std::isfinite(p.k_int) ||
        !(p.rho_ratio > 0.0) || !std::isfinite(p.rho_ratio) || p.n_pade < 1 || p.n_pade > 16 ||
        p.n_ss < 2 || p.n_ss > 12 || !(p.inner_tol > 0.0) || p.inner_tol > 1e-4 ||
        p.inner_maxit < 1 || (p.precision != OSRC_FP32_MATFREE && p.precision != OSRC_FP64_DENSE) ||
        p.precond < OSRC_PRECOND_OSRC || p.precond > OSRC_PRECOND_CALDERON ||
        (p.formulation != OSRC_PMCHWT && p.formulation != OSRC_MULLER) ||
        !(p.k_int_im >= 0.0) || !std::isfinite(p.k_int_im) ||
        (p.dense_assembly != OSRC_ASSEMBLE_FP64 && p.dense_assembly != OSRC_ASSEMBLE_FF) ||
        (p.osrc_side != 0 && p.osrc_side != 1) || !std::isfinite(p.theta)) {
        osrc_set_error("invalid problem parameters");
        return OSRC_INVALID_ARG;
    }
    osrc_ctx *ctx = mesh->ctx;
    OSRC_CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    osrc_problem *pb = new osrc_problem;
    pb->mesh = mesh;
    pb->p = p;
    pb->nv = mesh->nv;
    pb->nt = mesh->nt;
    pb->npts = 6 * mesh->nt;
    int s = OSRC_OK;
    const int nv = pb->nv, nt = pb->nt;
    const int *tris = mesh->tris.data();
    do {
        // ---- per-object materials (one object: the single-material path) -------
        {
            const double R = p.damping_R > 0.0 ? p.damping_R : mesh->mean_edge;
            pb->multi = mesh->ncomp > 1;
            pb->absorb = p.k_int_im != 0.0;
            pb->far_obj = pb->multi || p.formulation == OSRC_MULLER || pb->absorb;
            const float sgn = p.formulation == OSRC_MULLER ? -1.f : 1.f;
            pb->obj.resize(mesh->ncomp);
            std::vector<FarObj> fo(mesh->ncomp);
            std::vector<double2> ike(2 * (size_t)mesh->ncomp);
            double dk1_max = 0.0;
            for (int m = 0; m < mesh->ncomp; ++m) {
                const std::complex<double> k1c(k_int_obj[m], p.k_int_im);
                dk1_max = std::fmax(dk1_max, std::abs(k1c * k1c / rho_obj[m]));
            }
            pb->far_dks = far_dnormal_scale(p.k_ext, dk1_max);
            for (int m = 0; m < mesh->ncomp; ++m) {
                ObjMat &o = pb->obj[m];
                o.k1 = k_int_obj[m];
                o.k1i = p.k_int_im;
                o.rho = rho_obj[m];
                o.k_osrc = p.osrc_side == 1 ? o.k1 : p.k_ext;
                o.k_osrc_i = p.osrc_side == 1 ? o.k1i : 0.0;
                const std::complex<double> ko(o.k_osrc, o.k_osrc_i);
                const std::complex<double> ke =
                    ko * (1.0 + std::complex<double>(0.0, 0.4) * std::pow(ko * R, -2.0 / 3.0));
                o.k_eps = cd(ke.real(), ke.imag());
                const std::complex<double> inv = 1.0 / (ke * ke);
                ike[m] = cd(-o.k_osrc_i, o.k_osrc);                 // i k_osrc
                ike[mesh->ncomp + m] = cd(inv.real(), inv.imag());  // 1 / k_eps^2
                const double q = o.k1 * 0.15915494309189533577;
                const std::complex<double> k1c(o.k1, o.k1i), dk1 = k1c * k1c / o.rho;
                fo[m] = FarObj{(float)o.k1, (float)-o.k1, (float)o.rho, (float)(1.0 / o.rho),
                               (float)(dk1.real() / pb->far_dks), (float)q, (float)(q - (double)(float)q),
                               sgn, (float)o.k1i, (float)(dk1.imag() / pb->far_dks)};
            }
            if ((s = pb->d_obj.alloc(ctx, mesh->ncomp)) || (s = pb->d_fobj.alloc(ctx, mesh->ncomp)) ||
                (s = pb->d_obj_ike.alloc(ctx, 2 * (size_t)mesh->ncomp)))
                break;
            if (cudaMemcpy(pb->d_obj.p, pb->obj.data(), mesh->ncomp * sizeof(ObjMat), cudaMemcpyHostToDevice) ||
                cudaMemcpy(pb->d_fobj.p, fo.data(), mesh->ncomp * sizeof(FarObj), cudaMemcpyHostToDevice) ||
                cudaMemcpy(pb->d_obj_ike.p, ike.data(), ike.size() * sizeof(double2), cudaMemcpyHostToDevice)) {
                s = OSRC_CUDA_ERROR;
                break;
            }
        }
        if ((s = far_setup_geometry(pb, st))) break;
        // ---- touching triangle pairs ----------------------------------------
        std::vector<NearPair> pairs;
        pairs.reserve(14 * (size_t)nt);
        std::vector<int> cand;
        for (int t = 0; t < nt; ++t) {
            cand.clear();
            for (int a = 0; a < 3; ++a) {
                const int v = tris[3 * t + a];
                for (int e = mesh->vt_ptr[v]; e < mesh->vt_ptr[v + 1]; ++e) cand.push_back(mesh->vt_idx[e] / 3);
            }
            std::sort(cand.begin(), cand.end());
            cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
            for (int sidx : cand) {
                int perm = 0;
                const int kase = touch_case(tris + 3 * t, tris + 3 * sidx, perm);
                if (kase > 0) pairs.push_back(NearPair{t, sidx, kase, perm});
            }
        }
        // ---- near CSR pattern: vertex pairs of touching triangles -------------
        std::vector<int> nptr(nv + 1, 0), ncol;
        {
            std::vector<std::vector<int>> rowsets(nv);
            for (const NearPair &pr : pairs)
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) rowsets[tris[3 * pr.t + a]].push_back(tris[3 * pr.s + b]);
            for (int i = 0; i < nv; ++i) {
                auto &r = rowsets[i];
                std::sort(r.begin(), r.end());
                r.erase(std::unique(r.begin(), r.end()), r.end());
                nptr[i + 1] = nptr[i] + (int)r.size();
            }
            ncol.reserve(nptr[nv]);
            for (int i = 0; i < nv; ++i) ncol.insert(ncol.end(), rowsets[i].begin(), rowsets[i].end());
        }
        pb->near_nnz = nptr[nv];
        std::vector<int> cpos, cidx;
        cpos.reserve(9 * pairs.size());
        cidx.reserve(9 * pairs.size());
        for (size_t k = 0; k < pairs.size(); ++k)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    cpos.push_back(find_col(nptr, ncol, tris[3 * pairs[k].t + a], tris[3 * pairs[k].s + b]));
                    cidx.push_back((int)(9 * k + 3 * a + b));
                }
        std::vector<int> cptr, clist;
        bucket(pb->near_nnz, cpos, cidx, cptr, clist);
        if ((s = pb->d_nr_ptr.alloc(ctx, nv + 1)) || (s = pb->d_nr_col.alloc(ctx, ncol.size()))) break;
        if (cudaMemcpy(pb->d_nr_ptr.p, nptr.data(), (nv + 1) * sizeof(int), cudaMemcpyHostToDevice) ||
            cudaMemcpy(pb->d_nr_col.p, ncol.data(), ncol.size() * sizeof(int), cudaMemcpyHostToDevice)) {
            s = OSRC_CUDA_ERROR;
            break;
        }
        if ((s = near_build(pb, pairs, cptr, clist, st))) break;
        // ---- mass / stiffness CSR (1-ring) -------------------------------------
        std::vector<int> mptr(nv + 1, 0), mcol;
        {
            std::vector<std::vector<int>> rowsets(nv);
            for (int t = 0; t < nt; ++t)
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) rowsets[tris[3 * t + a]].push_back(tris[3 * t + b]);
            for (int i = 0; i < nv; ++i) {
                auto &r = rowsets[i];
                std::sort(r.begin(), r.end());
                r.erase(std::unique(r.begin(), r.end()), r.end());
                mptr[i + 1] = mptr[i] + (int)r.size();
            }
            for (int i = 0; i < nv; ++i) mcol.insert(mcol.end(), rowsets[i].begin(), rowsets[i].end());
        }
        pb->ms_nnz = mptr[nv];
        pb->ms_ptr_h = mptr;
        cpos.clear();
        cidx.clear();
        for (int t = 0; t < nt; ++t)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    cpos.push_back(find_col(mptr, mcol, tris[3 * t + a], tris[3 * t + b]));
                    cidx.push_back(9 * t + 3 * a + b);
                }
        bucket(pb->ms_nnz, cpos, cidx, cptr, clist);
        if ((s = pb->d_ms_ptr.alloc(ctx, nv + 1)) || (s = pb->d_ms_col.alloc(ctx, mcol.size()))) break;
        if (cudaMemcpy(pb->d_ms_ptr.p, mptr.data(), (nv + 1) * sizeof(int), cudaMemcpyHostToDevice) ||
            cudaMemcpy(pb->d_ms_col.p, mcol.data(), mcol.size() * sizeof(int), cudaMemcpyHostToDevice)) {
            s = OSRC_CUDA_ERROR;
            break;
        }
        if ((s = ms_build(pb, cptr, clist, st))) break;
        if (p.formulation == OSRC_MULLER && (s = near_add_mass(pb, st))) break;
        // ---- OSRC constants (Sec. 2.6) ------------------------------------------
        pb->k_osrc = p.osrc_side == 1 ? p.k_int : p.k_ext;
        pb->k_osrc_i = p.osrc_side == 1 ? p.k_int_im : 0.0;
        const double R = p.damping_R > 0.0 ? p.damping_R : mesh->mean_edge;
        const std::complex<double> kos(pb->k_osrc, pb->k_osrc_i);
        const std::complex<double> ke =
            kos * (1.0 + std::complex<double>(0.0, 0.4) * std::pow(kos * R, -2.0 / 3.0));
        pb->k_eps = cd(ke.real(), ke.imag());
        std::complex<double> C0;
        std::vector<std::complex<double>> A, B;
        pade_coefficients(p.n_pade, p.theta, C0, A, B);
        pb->C0 = cd(C0.real(), C0.imag());
        std::complex<double> g0 = C0;
        pb->A.resize(p.n_pade);
        pb->B.resize(p.n_pade);
        pb->g.resize(p.n_pade);
        for (int j = 0; j < p.n_pade; ++j) {
            const std::complex<double> gj = A[j] / (1.0 - B[j]);
            g0 -= gj;
            pb->A[j] = cd(A[j].real(), A[j].imag());
            pb->B[j] = cd(B[j].real(), B[j].imag());
            pb->g[j] = cd(gj.real(), gj.imag());
        }
        pb->g0 = cd(g0.real(), g0.imag());
        // ---- workspace ------------------------------------------------------------
        if ((s = pb->d_tmp2.alloc(ctx, 4 * (size_t)nv))) break;
        if ((s = pb->d_scalars.alloc(ctx, 64))) break;
        if (p.precision == OSRC_FP64_DENSE && (s = dense_assemble(pb, st))) break;
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            s = OSRC_CUDA_ERROR;
            break;
        }
    } while (0);
    if (s != OSRC_OK) {
        delete pb;
        return s;
    }
    *out = pb;
    return OSRC_OK;
}

extern "C" void osrc_problem_destroy(osrc_problem *pb) {
    if (!pb) return;
    if (pb->h_res) cudaFreeHost(pb->h_res);
    for (auto &e : pb->prof_ev)
        if (e) cudaEventDestroy(e);
    if (pb->batched) batched_free(pb->batched);
    delete pb;
}

extern "C" int osrc_problem_nv(const osrc_problem *pb) { return pb ? pb->nv : 0; }
extern "C" long long osrc_launch_count(const osrc_problem *pb) { return pb ? pb->launches : 0; }
extern "C" int osrc_profile_enable(osrc_problem *pb, int on) {
    if (!pb) return OSRC_INVALID_ARG;
    OSRC_CK(cudaSetDevice(pb->mesh->ctx->device));
    for (auto &e : pb->prof_ev)
        if (!e) OSRC_CK(cudaEventCreate(&e));
    if (pb->prof_pending) OSRC_TRY(far_prof_collect(pb));
    pb->prof_on = on != 0;
    pb->prof_launches = 0;
    pb->prof_ms = 0.0;
    pb->prof_rhs = 0;
    return OSRC_OK;
}

extern "C" int osrc_far_kernel_stats(osrc_problem *pb, long long *launches, double *total_ms) {
    if (!pb || !launches || !total_ms) return OSRC_INVALID_ARG;
    OSRC_CK(cudaSetDevice(pb->mesh->ctx->device));
    OSRC_TRY(far_prof_collect(pb));
    *launches = pb->prof_launches;
    *total_ms = pb->prof_ms;
    return OSRC_OK;
}

extern "C" long long osrc_far_kernel_rhs(const osrc_problem *pb) { return pb ? pb->prof_rhs : 0; }

extern "C" long long osrc_far_pairs(const osrc_problem *pb) {
    return pb ? 36LL * ((long long)pb->nt * pb->nt - pb->near_pairs) : 0;
}

extern "C" long long osrc_near_pairs(const osrc_problem *pb) { return pb ? pb->near_pairs : 0; }
extern "C" long long osrc_near_nnz(const osrc_problem *pb) { return pb ? pb->near_nnz : 0; }

// ---------------------------------------------------------------------------
// right-hand sides
// ---------------------------------------------------------------------------
static int rhs_common(osrc_problem *pb, const double *src, int nrhs, void *b, void *stream, int kind) {
    if (!pb || !src || !b || nrhs < 1) return OSRC_INVALID_ARG;
    OSRC_CK(cudaSetDevice(pb->mesh->ctx->device));
    for (int r = 0; r < nrhs; ++r) {
        const double *s3 = src + 3 * r;
        if (!std::isfinite(s3[0]) || !std::isfinite(s3[1]) || !std::isfinite(s3[2])) return OSRC_INVALID_ARG;
        if (kind == 0 && std::fabs(s3[0] * s3[0] + s3[1] * s3[1] + s3[2] * s3[2] - 1.0) > 1e-9)
            return OSRC_INVALID_ARG;
        OSRC_TRY(rhs_build(pb, kind, s3, (double2 *)b + 2 * (size_t)pb->nv * r, (cudaStream_t)stream));
    }
    return OSRC_OK;
}

extern "C" int osrc_rhs_planewave(osrc_problem *pb, const double *dirs, int nrhs, void *b, void *stream) {
    return rhs_common(pb, dirs, nrhs, b, stream, 0);
}

extern "C" int osrc_rhs_pointsource(osrc_problem *pb, const double *srcs, int nrhs, void *b, void *stream) {
    return rhs_common(pb, srcs, nrhs, b, stream, 1);
}

// ---------------------------------------------------------------------------
// operators
// ---------------------------------------------------------------------------
static int apply_one(osrc_problem *pb, const double2 *x, double2 *y, int form, int part, cudaStream_t st) {
    double2 *dst = form == OSRC_STRONG ? pb->d_tmp2.p : y;
    if (pb->p.precision == OSRC_FP64_DENSE) {
        if (part != OSRC_PART_ALL) return OSRC_UNSUPPORTED;
        OSRC_TRY(dense_apply(pb, x, dst, st));
    } else {
        OSRC_TRY(far_apply(pb, x, dst, part, st));
    }
    if (form == OSRC_STRONG) OSRC_TRY(mass_solve(pb, dst, y, st));
    return OSRC_OK;
}

extern "C" int osrc_pmchwt_apply(osrc_problem *pb, const void *x, void *y, int nrhs, int form,
                                 int part, void *stream) {
    if (!pb || !x || !y || nrhs < 1 || (form != OSRC_WEAK && form != OSRC_STRONG) || part < 1 || part > 3)
        return OSRC_INVALID_ARG;
    if (x == y) return OSRC_INVALID_ARG;
    OSRC_CK(cudaSetDevice(pb->mesh->ctx->device));
    const size_t n = 2 * (size_t)pb->nv;
    if (nrhs > 1 && form == OSRC_WEAK && far_multi_supported(pb)) {
        // several right-hand sides per far-field launch
        std::vector<const double2 *> xs(nrhs);
        std::vector<double2 *> ys(nrhs);
        for (int r = 0; r < nrhs; ++r) {
            xs[r] = (const double2 *)x + n * r;
            ys[r] = (double2 *)y + n * r;
        }
        return far_apply_multi(pb, xs.data(), ys.data(), nrhs, part, (cudaStream_t)stream);
    }
    for (int r = 0; r < nrhs; ++r)
        OSRC_TRY(apply_one(pb, (const double2 *)x + n * r, (double2 *)y + n * r, form, part,
                           (cudaStream_t)stream));
    return OSRC_OK;
}

extern "C" int osrc_mass_solve(osrc_problem *pb, const void *x, void *y, int nrhs, void *stream) {
    if (!pb || !x || !y || nrhs < 1 || x == y) return OSRC_INVALID_ARG;
    OSRC_CK(cudaSetDevice(pb->mesh->ctx->device));
    const size_t n = 2 * (size_t)pb->nv;
    for (int r = 0; r < nrhs; ++r)
        OSRC_TRY(mass_solve(pb, (const double2 *)x + n * r, (double2 *)y + n * r, (cudaStream_t)stream));
    return OSRC_OK;
}

extern "C" int osrc_precond_apply(osrc_problem *pb, const void *x, void *y, int nrhs, void *stream) {
    if (!pb || !x || !y || nrhs < 1 || x == y) return OSRC_INVALID_ARG;
    OSRC_CK(cudaSetDevice(pb->mesh->ctx->device));
    const size_t n = 2 * (size_t)pb->nv;
    for (int r = 0; r < nrhs; ++r)
        OSRC_TRY(osrc_precond(pb, (const double2 *)x + n * r, (double2 *)y + n * r, (cudaStream_t)stream));
    return OSRC_OK;
}

// ---------------------------------------------------------------------------
// GMRES (Sec. 3.1): no restart, x0 = 0, preconditioned relative residual
// ---------------------------------------------------------------------------
// pinned host block of a workspace: doubles [0, 16), then status ints
static const int kHostDoubles = 16;
static const int kHostInts = 48;

static int *host_stat(osrc_problem *pb) { return (int *)(pb->h_res + kHostDoubles); }

int ensure_gmres_workspace(osrc_problem *pb, int maxit) {
    osrc_ctx *ctx = pb->mesh->ctx;
    const size_t n = 2 * (size_t)pb->nv;
    if (pb->basis_cap < maxit) {
        pb->d_basis.release();
        pb->d_h.release();
        pb->d_givens.release();
        OSRC_TRY(pb->d_basis.alloc(ctx, (size_t)(maxit + 1) * n));
        OSRC_TRY(pb->d_h.alloc(ctx, (size_t)(maxit + 1) * maxit));
        OSRC_TRY(pb->d_givens.alloc(ctx, 6 * (size_t)(maxit + 1)));
        pb->basis_cap = maxit;
    }
    if (!pb->d_w.p) {
        OSRC_TRY(pb->d_w.alloc(ctx, n));
        OSRC_TRY(pb->d_y.alloc(ctx, n));
        OSRC_TRY(pb->d_cvec.alloc(ctx, n));
        OSRC_TRY(pb->d_b1.alloc(ctx, n));
        OSRC_TRY(pb->d_x1.alloc(ctx, n));
    }
    if (!pb->h_res)
        OSRC_CK(cudaMallocHost((void **)&pb->h_res, kHostDoubles * sizeof(double) + kHostInts * sizeof(int)));
    return OSRC_OK;
}

GmresRun::~GmresRun() {
    if (ev) cudaEventDestroy(ev);
    for (auto &e : tev)
        if (e) cudaEventDestroy(e);
}

bool GmresRun::ready() const { return ev == nullptr || cudaEventQuery(ev) != cudaErrorNotReady; }

// Copies the status words of the last inner solve next to the scalars and
// marks the end of the enqueued step.
static int end_step(GmresRun &g) {
    osrc_problem *pb = g.pb;
    const int nsys = osrc_precond_nsys(pb);
    OSRC_CK(cudaMemcpyAsync(host_stat(pb), pb->d_kry_stat.p, nsys * sizeof(int), cudaMemcpyDeviceToHost, g.st));
    OSRC_CK(cudaEventRecord(g.ev, g.st));
    return OSRC_OK;
}

// one Arnoldi step: w = P M^-1 B v_j, CGS2 against v_0..v_j, Givens, |g_{j+1}|/beta.
// Split in two so that a batch of runs can share one several-right-hand-side
// apply: enqueue_apply (B v_j into d_tmp2) and enqueue_iteration_rest.
static int enqueue_apply(GmresRun &g) {
    osrc_problem *pb = g.pb;
    cudaStream_t st = g.st;
    const int n = 2 * pb->nv, j = g.j;
    double2 *V = pb->d_basis.p;
    OSRC_CK(cudaEventRecord(g.tev[0], st));
    if (pb->p.precision == OSRC_FP64_DENSE) OSRC_TRY(dense_apply(pb, V + (size_t)j * n, pb->d_tmp2.p, st));
    else OSRC_TRY(far_apply(pb, V + (size_t)j * n, pb->d_tmp2.p, OSRC_PART_ALL, st));
    OSRC_CK(cudaEventRecord(g.tev[1], st));
    return OSRC_OK;
}

static int enqueue_iteration_rest(GmresRun &g) {
    osrc_problem *pb = g.pb;
    cudaStream_t st = g.st;
    const int n = 2 * pb->nv, j = g.j, ldh = g.maxit + 1;
    double2 *V = pb->d_basis.p, *H = pb->d_h.p, *gv = pb->d_givens.p, *w = pb->d_w.p;
    double *sc = pb->d_scalars.p;
    OSRC_TRY(osrc_precond_fused_async(pb, pb->d_tmp2.p, w, st));
    OSRC_CK(cudaEventRecord(g.tev[2], st));
    double2 *hc = H + (size_t)ldh * j;
    double2 *h2 = gv + 4 * ldh;  // second-pass projections
    OSRC_TRY(vec_dots_conj(pb, V, j + 1, w, n, hc, st));
    OSRC_TRY(vec_update(pb, V, j + 1, hc, w, n, st));
    OSRC_TRY(vec_dots_conj(pb, V, j + 1, w, n, h2, st));
    OSRC_TRY(vec_update(pb, V, j + 1, h2, w, n, st));
    OSRC_TRY(vec_axpby(pb, cd(1, 0), hc, cd(1, 0), h2, hc, j + 1, st));
    OSRC_TRY(vec_norm(pb, w, n, sc + 1, st));
    OSRC_CK(cudaMemcpyAsync(hc + j + 1, sc + 1, sizeof(double), cudaMemcpyDeviceToDevice, st));
    OSRC_CK(cudaMemsetAsync((double *)(hc + j + 1) + 1, 0, sizeof(double), st));
    OSRC_TRY(vec_scale_copy(pb, w, sc + 1, V + (size_t)(j + 1) * n, n, st));
    OSRC_TRY(gmres_givens(pb, j, ldh, H, gv, sc + 2, g.beta, st));
    OSRC_CK(cudaMemcpyAsync(pb->h_res + 2, sc + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
    OSRC_CK(cudaEventRecord(g.tev[3], st));
    return end_step(g);
}

static int enqueue_iteration(GmresRun &g) {
    OSRC_TRY(enqueue_apply(g));
    return enqueue_iteration_rest(g);
}

// x = V y, then the true weak residual |b - B x| / |b|; split like the
// iteration: enqueue_finish_x (x = V y), the apply B x into d_w,
// enqueue_finish_rest
static int enqueue_finish_x(GmresRun &g) {
    osrc_problem *pb = g.pb;
    const int n = 2 * pb->nv;
    if (g.j > 0) {
        OSRC_TRY(gmres_finish(pb, g.j, g.maxit + 1, pb->d_h.p, pb->d_givens.p, pb->d_basis.p, g.x, n, g.st));
    } else {
        OSRC_CK(cudaMemsetAsync(g.x, 0, n * sizeof(double2), g.st));
    }
    return OSRC_OK;
}

static int enqueue_finish_rest(GmresRun &g) {
    osrc_problem *pb = g.pb;
    cudaStream_t st = g.st;
    const int n = 2 * pb->nv;
    double *sc = pb->d_scalars.p;
    double2 *t = pb->d_w.p;
    OSRC_TRY(vec_axpby(pb, cd(1, 0), g.b, cd(-1, 0), t, t, n, st));
    OSRC_TRY(vec_norm(pb, t, n, sc + 4, st));
    OSRC_TRY(vec_norm(pb, g.b, n, sc + 5, st));
    OSRC_CK(cudaMemcpyAsync(pb->h_res + 4, sc + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    OSRC_CK(cudaEventRecord(g.ev, st));
    return OSRC_OK;
}

static int enqueue_finish(GmresRun &g) {
    osrc_problem *pb = g.pb;
    OSRC_TRY(enqueue_finish_x(g));
    if (pb->p.precision == OSRC_FP64_DENSE) OSRC_TRY(dense_apply(pb, g.x, pb->d_w.p, g.st));
    else OSRC_TRY(far_apply(pb, g.x, pb->d_w.p, OSRC_PART_ALL, g.st));
    return enqueue_finish_rest(g);
}

// next step of a deferred run: the batch driver enqueues it (GmresRun::defer)
static int schedule_iteration(GmresRun &g) {
    if (g.defer) {
        g.next = 1;
        return OSRC_OK;
    }
    return enqueue_iteration(g);
}

static int schedule_finish(GmresRun &g) {
    if (g.defer) {
        g.next = 2;
        return OSRC_OK;
    }
    return enqueue_finish(g);
}

int GmresRun::start(osrc_problem *p, cudaStream_t s, const double2 *b_, double2 *x_, double tol_,
                    int maxit_) {
    pb = p;
    st = s;
    b = b_;
    x = x_;
    tol = tol_;
    maxit = maxit_;
    j = 0;
    beta = 0.0;
    res = 1.0;
    status = OSRC_OK;
    converged = false;
    info = osrc_solve_info{};
    OSRC_TRY(ensure_gmres_workspace(pb, maxit));
    if (!ev) OSRC_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    for (auto &e : tev)
        if (!e) OSRC_CK(cudaEventCreate(&e));
    const int n = 2 * pb->nv;
    double *sc = pb->d_scalars.p;
    // c = P M^-1 b, beta = |c|
    OSRC_TRY(osrc_precond_fused_async(pb, b, pb->d_cvec.p, st));
    OSRC_TRY(vec_norm(pb, pb->d_cvec.p, n, sc, st));
    OSRC_CK(cudaMemcpyAsync(pb->h_res, sc, sizeof(double), cudaMemcpyDeviceToHost, st));
    OSRC_TRY(end_step(*this));
    phase = 1;
    return OSRC_OK;
}

int GmresRun::advance() {
    const int n = 2 * pb->nv;
    const int ldh = maxit + 1;
    if (phase == 3) {  // final residual arrived
        info.true_residual = pb->h_res[5] > 0 ? pb->h_res[4] / pb->h_res[5] : 0.0;
        info.iterations = j;
        info.precond_residual = (j > 0) ? res : 0.0;
        info.converged = converged ? 1 : 0;
        info.total_iterations = j;
        phase = 4;
        return status;
    }
    int s = kry_status_host(pb, host_stat(pb), osrc_precond_nsys(pb));
    if (s != OSRC_OK) {
        status = s;
        phase = 4;
        return s;
    }
    if (phase == 1) {
        beta = pb->h_res[0];
        if (!std::isfinite(beta)) {
            status = OSRC_INVALID_ARG;
            phase = 4;
            return status;
        }
        if (!(beta > 0.0)) {  // zero right-hand side: x = 0
            converged = true;
            res = 0.0;
            OSRC_TRY(schedule_finish(*this));
            phase = 3;
            return OSRC_OK;
        }
        double2 *V = pb->d_basis.p, *H = pb->d_h.p, *gv = pb->d_givens.p;
        OSRC_TRY(vec_scale_copy(pb, pb->d_cvec.p, pb->d_scalars.p, V, n, st));
        OSRC_CK(cudaMemsetAsync(H, 0, (size_t)ldh * maxit * sizeof(double2), st));
        OSRC_CK(cudaMemsetAsync(gv, 0, 4 * (size_t)ldh * sizeof(double2), st));
        pb->h_res[6] = beta;  // g_0 = (beta, 0), copied from pinned memory
        pb->h_res[7] = 0.0;
        OSRC_CK(cudaMemcpyAsync(gv + 2 * ldh, pb->h_res + 6, sizeof(double2), cudaMemcpyHostToDevice, st));
        OSRC_TRY(schedule_iteration(*this));
        phase = 2;
        return OSRC_OK;
    }
    // phase 2: iteration j finished
    {
        float a = 0.f, bb = 0.f, c = 0.f;
        cudaEventElapsedTime(&a, tev[0], tev[1]);
        cudaEventElapsedTime(&bb, tev[1], tev[2]);
        cudaEventElapsedTime(&c, tev[2], tev[3]);
        info.ms_matvec += a;
        info.ms_precond += bb;
        info.ms_arnoldi += c;
    }
    res = pb->h_res[2];
    ++j;
    if (!std::isfinite(res)) {
        status = OSRC_BREAKDOWN;
        phase = 4;
        return status;
    }
    if (res <= tol) converged = true;
    if (converged || j >= maxit) {
        OSRC_TRY(schedule_finish(*this));
        phase = 3;
        return OSRC_OK;
    }
    OSRC_TRY(schedule_iteration(*this));
    return OSRC_OK;
}

int GmresRun::run_to_completion() {
    while (!done()) {
        OSRC_CK(cudaEventSynchronize(ev));
        const int s = advance();
        if (s != OSRC_OK) return s;
    }
    return status;
}

// ---------------------------------------------------------------------------
// problem clones: shared resident state, own workspace (serving slots)
// ---------------------------------------------------------------------------
int problem_clone(osrc_problem *m, osrc_problem **out) {
    *out = nullptr;
    osrc_ctx *ctx = m->mesh->ctx;
    osrc_problem *c = new osrc_problem;
    c->mesh = m->mesh;
    c->p = m->p;
    c->nv = m->nv;
    c->nt = m->nt;
    c->npts = m->npts;
    c->nsplit = m->nsplit;
    c->far_reduce = m->far_reduce;
    c->near_pairs = m->near_pairs;
    c->near_nnz = m->near_nnz;
    c->ms_nnz = m->ms_nnz;
    c->ms_ptr_h = m->ms_ptr_h;
    c->k_osrc = m->k_osrc;
    c->k_osrc_i = m->k_osrc_i;
    c->k_eps = m->k_eps;
    c->C0 = m->C0;
    c->g0 = m->g0;
    c->A = m->A;
    c->B = m->B;
    c->g = m->g;
    c->multi = m->multi;
    c->far_obj = m->far_obj;
    c->far_dks = m->far_dks;
    c->absorb = m->absorb;
    c->obj = m->obj;
    c->d_obj.borrow(m->d_obj);
    c->d_fobj.borrow(m->d_fobj);
    c->d_obj_ike.borrow(m->d_obj_ike);
    c->d_pt.borrow(m->d_pt);
    c->d_poff.borrow(m->d_poff);
    c->d_cen.borrow(m->d_cen);
    c->d_tn.borrow(m->d_tn);
    c->d_tv.borrow(m->d_tv);
    c->d_tgeo.borrow(m->d_tgeo);
    c->d_nr_ptr.borrow(m->d_nr_ptr);
    c->d_nr_col.borrow(m->d_nr_col);
    c->d_nr_val.borrow(m->d_nr_val);
    c->d_ms_ptr.borrow(m->d_ms_ptr);
    c->d_ms_col.borrow(m->d_ms_col);
    c->d_M.borrow(m->d_M);
    c->d_S.borrow(m->d_S);
    c->d_dense.borrow(m->d_dense);
    const int nt = m->nt, nv = m->nv;
    const int nsys = 2 * m->p.n_pade + 2;
    int s = OSRC_OK;
    if ((s = c->d_sP.alloc(ctx, 30 * (size_t)nt)) || (s = c->d_sP5.alloc(ctx, 6 * (size_t)nt)) ||
        (s = c->d_sC.alloc(ctx, 5 * (size_t)nt)) ||
        (s = c->d_part.alloc(ctx, (size_t)c->nsplit * 10 * c->npts)) ||
        (s = c->d_kry.alloc(ctx, 5 * (size_t)nsys * nv)) ||
        (s = c->d_kry_rhs.alloc(ctx, (size_t)(2 + nsys) * nv)) || (s = c->d_kry_stat.alloc(ctx, 40)) ||
        (s = c->d_kry_res.alloc(ctx, 40)) || (s = c->d_tmp2.alloc(ctx, 4 * (size_t)nv)) ||
        (s = c->d_scalars.alloc(ctx, 64))) {
        delete c;
        return s;
    }
    *out = c;
    return OSRC_OK;
}

size_t estimate_problem_bytes(int nv, int nt, const osrc_params &p) {
    size_t b = 0;
    b += (size_t)nt * (6 * 16 * 2 + 2 * 16 + 16 + 16 + 16 * 8);   // far geometry + FP64 triangle data
    b += (size_t)nv * 20 * (4 + 64) + (size_t)nv * 4;               // near CSR
    b += (size_t)nv * 8 * (4 + 16) + (size_t)nv * 4;                // M, S
    b += (size_t)nt * 14 * (576 + 16 + 9 * 8);                      // transient Sauter-Schwab build
    if (p.precision == OSRC_FP64_DENSE) {
        b += (size_t)4 * nv * nv * 16;
        const size_t cmax = (size_t)nt / 10 + 1;  // largest triangle colour (transient stash of the assembly)
        b += cmax * cmax * 36 * 16;
    }
    return b;
}

size_t estimate_work_bytes(int nv, int nt, const osrc_params &p, int maxit) {
    const size_t nsys = 2 * (size_t)p.n_pade + 2;
    size_t b = 0;
    b += (size_t)nt * (30 * 16 + 6 * 8 + 5 * 16);      // far source data
    const size_t ns = std::min<size_t>(64, (size_t)(nt + 63) / 64);
    b += ns * 10 * 6 * (size_t)nt * 4;                  // far partial sums
    b += nsys * nv * (5 + 1) * 16 + 2 * (size_t)nv * 16 + 4 * (size_t)nv * 16;  // inner solves
    b += (size_t)(maxit + 1) * 2 * nv * 16 + (size_t)(maxit + 1) * maxit * 16;   // Krylov basis
    b += (size_t)5 * 2 * nv * 16 + 6 * (size_t)(maxit + 1) * 16;
    return b;
}

// ---------------------------------------------------------------------------
// GMRES for several right-hand sides in lockstep: one run per right-hand
// side, each on a clone of the problem (own Krylov basis, Hessenberg matrix,
// inner-solver workspace; shared resident operator state), all on one
// stream.  Every iteration applies B to the newest basis vectors of all
// runs that are still iterating in one several-right-hand-side far-field
// launch (far_apply_multi), then each run does its own preconditioner,
// Gram-Schmidt and Givens steps.  Runs stop independently (a converged run
// drops out of the shared apply).  Up to kBatchRuns runs are in flight; more
// right-hand sides are taken in groups.
// ---------------------------------------------------------------------------
static const int kBatchRuns = 16;

struct CloneSet {
    std::vector<osrc_problem *> c;
    ~CloneSet() {
        for (osrc_problem *p : c) osrc_problem_destroy(p);
    }
};

static int gmres_solve_lockstep(osrc_problem *pb, const void *b, void *x, int nrhs, double tol, int maxit,
                                bool host, osrc_solve_info &info, cudaStream_t st) {
    const int n = 2 * pb->nv;
    const int G = std::min(nrhs, kBatchRuns);
    CloneSet cs;
    cs.c.assign(G, nullptr);
    for (int g = 0; g < G; ++g) OSRC_TRY(problem_clone(pb, &cs.c[g]));
    DBuf<double2> db, dx;
    if (host) {
        OSRC_TRY(db.alloc(pb->mesh->ctx, (size_t)G * n));
        OSRC_TRY(dx.alloc(pb->mesh->ctx, (size_t)G * n));
    }
    cudaEvent_t ea = nullptr, eb = nullptr;
    OSRC_CK(cudaEventCreate(&ea));
    OSRC_CK(cudaEventCreate(&eb));
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } evg{ea, eb};
    double ms_apply = 0.0;
    bool apply_pending = false;
    int last_its = 0;
    double last_pres = 0.0, last_tres = 0.0;
    for (int r0 = 0; r0 < nrhs; r0 += G) {
        const int R = std::min(G, nrhs - r0);
        std::vector<GmresRun> runs(R);
        for (int r = 0; r < R; ++r) {
            const double2 *br;
            double2 *xr;
            if (host) {
                OSRC_CK(cudaMemcpyAsync(db.p + (size_t)r * n, (const double2 *)b + (size_t)n * (r0 + r),
                                        n * sizeof(double2), cudaMemcpyHostToDevice, st));
                br = db.p + (size_t)r * n;
                xr = dx.p + (size_t)r * n;
            } else {
                br = (const double2 *)b + (size_t)n * (r0 + r);
                xr = (double2 *)x + (size_t)n * (r0 + r);
            }
            cs.c[r]->inner_last_max = 0;
            runs[r].defer = true;
            OSRC_TRY(runs[r].start(cs.c[r], st, br, xr, tol, maxit));
        }
        std::vector<const double2 *> xs;
        std::vector<double2 *> ys;
        std::vector<int> it, fin;
        for (;;) {
            OSRC_CK(cudaStreamSynchronize(st));
            OSRC_TRY(far_multi_check(pb, st));
            if (pb->cancel && pb->cancel->load()) {
                osrc_set_error("lockstep GMRES cancelled");
                return OSRC_TIMEOUT;
            }
            if (apply_pending) {
                float ms = 0.f;
                OSRC_CK(cudaEventElapsedTime(&ms, ea, eb));
                ms_apply += ms;
                apply_pending = false;
            }
            it.clear();
            fin.clear();
            for (int r = 0; r < R; ++r) {
                GmresRun &g = runs[r];
                if (g.done()) continue;
                g.next = 0;
                const int s = g.advance();
                if (s != OSRC_OK) return s;
                if (g.done()) continue;
                if (g.next == 1) it.push_back(r);
                else if (g.next == 2) fin.push_back(r);
            }
            if (it.empty() && fin.empty()) break;
            if (!it.empty()) {
                xs.clear();
                ys.clear();
                for (int r : it) {
                    osrc_problem *c = cs.c[r];
                    xs.push_back(c->d_basis.p + (size_t)runs[r].j * n);
                    ys.push_back(c->d_tmp2.p);
                }
                OSRC_CK(cudaEventRecord(ea, st));
                OSRC_TRY(far_apply_multi(pb, xs.data(), ys.data(), (int)it.size(), OSRC_PART_ALL, st));
                OSRC_CK(cudaEventRecord(eb, st));
                apply_pending = true;
                for (int r : it) {
                    // the shared apply's time is counted once by the driver
                    OSRC_CK(cudaEventRecord(runs[r].tev[0], st));
                    OSRC_CK(cudaEventRecord(runs[r].tev[1], st));
                    OSRC_TRY(enqueue_iteration_rest(runs[r]));
                }
            }
            if (!fin.empty()) {
                xs.clear();
                ys.clear();
                for (int r : fin) {
                    OSRC_TRY(enqueue_finish_x(runs[r]));
                    xs.push_back(runs[r].x);
                    ys.push_back(cs.c[r]->d_w.p);
                }
                OSRC_TRY(far_apply_multi(pb, xs.data(), ys.data(), (int)fin.size(), OSRC_PART_ALL, st));
                for (int r : fin) OSRC_TRY(enqueue_finish_rest(runs[r]));
            }
        }
        for (int r = 0; r < R; ++r) {
            const GmresRun &g = runs[r];
            if (host)
                OSRC_CK(cudaMemcpyAsync((double2 *)x + (size_t)n * (r0 + r), dx.p + (size_t)r * n,
                                        n * sizeof(double2), cudaMemcpyDeviceToHost, st));
            last_its = g.info.iterations;
            last_pres = g.info.precond_residual;
            last_tres = g.info.true_residual;
            info.ms_precond += g.info.ms_precond;
            info.ms_arnoldi += g.info.ms_arnoldi;
            info.total_iterations += g.info.iterations;
            info.inner_iterations_max = std::max(info.inner_iterations_max, cs.c[r]->inner_last_max);
            if (!g.converged) info.converged = 0;
        }
    }
    for (osrc_problem *c : cs.c) {  // the clones' launches count as the problem's
        pb->launches += c->launches;
        c->launches = 0;
    }
    OSRC_CK(cudaStreamSynchronize(st));
    info.iterations = last_its;
    info.precond_residual = last_pres;
    info.true_residual = last_tres;
    info.ms_matvec += ms_apply;
    return OSRC_OK;
}

extern "C" int osrc_gmres_solve(osrc_problem *pb, const void *b, void *x, int nrhs, double tol, int maxit,
                                int flags, osrc_solve_info *info_out, void *stream) {
    if (!pb || !b || !x || nrhs < 1 || !(tol > 0.0) || maxit < 1 || maxit > 100000) return OSRC_INVALID_ARG;
    OSRC_CK(cudaSetDevice(pb->mesh->ctx->device));
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)stream;
    OSRC_TRY(ensure_gmres_workspace(pb, maxit));
    const int n = 2 * pb->nv;
    osrc_solve_info info{};
    info.converged = 1;
    pb->inner_last_max = 0;
    const bool host = (flags & OSRC_HOST_BUFFERS) != 0;
    if (nrhs > 1 && far_multi_supported(pb) && pb->p.precond != OSRC_PRECOND_CALDERON) {
        OSRC_TRY(gmres_solve_lockstep(pb, b, x, nrhs, tol, maxit, host, info, st));
        info.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (info_out) *info_out = info;
        return info.converged ? OSRC_OK : OSRC_NOT_CONVERGED;
    }
    GmresRun run;
    for (int r = 0; r < nrhs; ++r) {
        const double2 *br;
        double2 *xr;
        if (host) {
            OSRC_CK(cudaMemcpyAsync(pb->d_b1.p, (const double2 *)b + (size_t)n * r, n * sizeof(double2),
                                    cudaMemcpyHostToDevice, st));
            br = pb->d_b1.p;
            xr = pb->d_x1.p;
        } else {
            br = (const double2 *)b + (size_t)n * r;
            xr = (double2 *)x + (size_t)n * r;
        }
        OSRC_TRY(run.start(pb, st, br, xr, tol, maxit));
        OSRC_TRY(run.run_to_completion());
        if (host)
            OSRC_CK(cudaMemcpyAsync((double2 *)x + (size_t)n * r, xr, n * sizeof(double2),
                                    cudaMemcpyDeviceToHost, st));
        info.iterations = run.info.iterations;
        info.precond_residual = run.info.precond_residual;
        info.true_residual = run.info.true_residual;
        info.ms_matvec += run.info.ms_matvec;
        info.ms_precond += run.info.ms_precond;
        info.ms_arnoldi += run.info.ms_arnoldi;
        info.total_iterations += run.info.iterations;
        if (!run.converged) info.converged = 0;
    }
    OSRC_CK(cudaStreamSynchronize(st));
    info.inner_iterations_max = pb->inner_last_max;
    info.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info_out) *info_out = info;
    return info.converged ? OSRC_OK : OSRC_NOT_CONVERGED;
}
