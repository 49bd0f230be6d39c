// osrc_internal.cuh -- internal state and kernel launchers of the GB300 OSRC
// PMCHWT library.  Not part of the ABI (see include/osrc_pmchwt.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <atomic>
#include <mutex>
#include <cmath>
#include <vector>

#include "../../include/osrc_pmchwt.h"

// ---------------------------------------------------------------------------
// error handling: every CUDA call is checked; failures become status codes
// ---------------------------------------------------------------------------
#define OSRC_CK(call)                                                       \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) {                                            \
            osrc_set_error(std::string(#call) + ": " + cudaGetErrorString(e_)); \
            return (e_ == cudaErrorMemoryAllocation) ? OSRC_OUT_OF_MEMORY   \
                                                     : OSRC_CUDA_ERROR;     \
        }                                                                   \
    } while (0)

#define OSRC_TRY(expr)                 \
    do {                               \
        int s_ = (expr);               \
        if (s_ != OSRC_OK) return s_;  \
    } while (0)

void osrc_set_error(const std::string &msg);

// ---------------------------------------------------------------------------
// complex helpers (double2 / float2 as complex numbers)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ double2 cd(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return cd(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return cd(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return cd(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return cd(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return cd(a.x, -a.y); }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    double d = b.x * b.x + b.y * b.y;
    return cd((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
// One-time set-up per device: kernel attributes (opt-ins, shared-memory
// limits) and occupancy-derived settings belong to the device that is current
// when they are made, so each call site keeps one result per device.
constexpr int OSRC_MAX_DEVICES = 64;
struct PerDeviceOnce {
    std::mutex m;
    bool done[OSRC_MAX_DEVICES] = {};
    int status[OSRC_MAX_DEVICES] = {};
};
template <typename F>
int per_device_once(PerDeviceOnce &o, F f) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return OSRC_CUDA_ERROR;
    if (dev < 0 || dev >= OSRC_MAX_DEVICES) return OSRC_UNSUPPORTED;
    std::lock_guard<std::mutex> g(o.m);
    if (!o.done[dev]) {
        o.status[dev] = f(dev);
        o.done[dev] = true;
    }
    return o.status[dev];
}

struct osrc_ctx {
    int device = 0;
    size_t budget = 0;               // 0 = unlimited
    std::atomic<size_t> used{0};     // allocations may come from several host threads
};

int ctx_alloc(osrc_ctx *ctx, void **p, size_t bytes);
void ctx_free(osrc_ctx *ctx, void *p, size_t bytes);

// A device buffer whose size is accounted to a context.
// A borrowed buffer (borrow()) points at another buffer's memory and never
// frees it; its owner must outlive it.
template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    osrc_ctx *ctx = nullptr;
    bool owned = true;
    int alloc(osrc_ctx *c, size_t count) {
        release();
        ctx = c;
        n = count;
        owned = true;
        if (count == 0) return OSRC_OK;
        return ctx_alloc(ctx, (void **)&p, count * sizeof(T));
    }
    void borrow(const DBuf &o) {
        release();
        p = o.p;
        n = o.n;
        ctx = o.ctx;
        owned = false;
    }
    void release() {
        if (p && owned) ctx_free(ctx, p, n * sizeof(T));
        p = nullptr;
        n = 0;
        owned = true;
    }
    ~DBuf() { release(); }
};

struct osrc_mesh {
    osrc_ctx *ctx = nullptr;
    int nv = 0, nt = 0;
    std::vector<double> verts;       // nv x 3
    std::vector<int> tris;           // nt x 3
    std::vector<int> vt_ptr, vt_idx; // vertex -> (3*triangle + local) incidence
    double mean_edge = 0.0;
    // objects: connected components (triangles sharing vertices), numbered in
    // the order of their first triangle
    int ncomp = 1;
    std::vector<int> tcomp, vcomp;   // per triangle / per vertex object
    std::vector<int> tri_order;      // triangles sorted by object (stable)
    std::vector<int> comp_tbeg;      // [ncomp + 1] ranges of tri_order
    DBuf<double> d_verts;
    DBuf<int> d_tris, d_vt_ptr, d_vt_idx;
    DBuf<int> d_tcomp, d_vcomp, d_tri_order;
};

// Material of one object (disjoint objects, Sec. 2.2): interior wavenumber,
// density ratio rho_m / rho_0, OSRC wavenumber and its damped version.
struct ObjMat {
    double k1, rho, k_osrc, k1i;  // k1i: imaginary part of the interior wavenumber
    double2 k_eps;
    double k_osrc_i, pad;         // imaginary part of the OSRC wavenumber
};

// FP32 constants of one object for the far kernel (duplicated-pair form is
// built per thread): k1, -k1, rho, 1/rho, k1^2/rho, k1/(2 pi) as float-float.
struct FarObj {
    float k1, nk1, rho, irho, dk1, k1h, k1l, sgn;  // sgn: +1 PMCHWT, -1 Mueller
    float k1i, dk1i;  // attenuation: Im k1; dk1, dk1i: Re and Im of (k1^2 / rho) / far_dks
};

// Scale dks of the far kernel's D normal term k0^2 G0 + (k1^2/rho) G1 =
// dks (G0 + (k1^2/rho)/dks G1): k0^2, raised to 1e-20 max|k1^2/rho| so that
// the ratio stays below 1e20 (a G0 coefficient changed by less than 1e-20 of
// the G1 coefficient is below FP32 resolution).
inline double far_dnormal_scale(double k0, double dk1_abs_max) {
    return std::fmax(k0 * k0, 1e-20 * dk1_abs_max);
}

// Touching triangle pair for the Sauter-Schwab kernel.
struct NearPair {
    int t, s;      // test, source triangle
    int kase;      // 1 vertex, 2 edge, 3 identical
    int perm;      // pt[0..2] | ps[0..2] << 6, 2 bits each
};

struct BatchedState;
void batched_free(BatchedState *s);

struct osrc_problem {
    osrc_mesh *mesh = nullptr;
    BatchedState *batched = nullptr;  // dense batched-solve state (k_batched.cu)
    osrc_params p{};
    int nv = 0, nt = 0, npts = 0;
    long long launches = 0;

    // ---- far field (FP32): static geometry -----------------------------
    DBuf<float4> d_pt;   // [6nt]  point x, y, z, quadrature weight * area
    DBuf<float4> d_poff; // [6nt]  point minus triangle centroid, quadrature weight * area
    DBuf<float4> d_cen;  // [2nt]  triangle centroid as float pairs (hi, lo)
    DBuf<float4> d_tn;   // [nt]   outward normal, plane offset n.P0
    DBuf<int4> d_tv;     // [nt]   vertex indices
    // ---- far field: per-apply workspace ----------------------------------
    DBuf<float4> d_sP;   // [6nt][5] source points: -y, psi, phi with both signs, duplicated pairs
    DBuf<float2> d_sP5;  // [6nt] (-phi.im, -phi.im)
    DBuf<float4> d_sC;   // [nt][5] c_sigma components with both signs, duplicated pairs
    DBuf<float> d_part;       // [nsplit][6nt][10] per test point partial sums
    int nsplit = 1;
    // ---- far field, several right-hand sides per launch (k_far.cu farm_*) ----
    DBuf<float4> d_sG;        // [6nt][2] static source geometry (coordinates, rule weight)
    DBuf<float4> d_sD;        // [nt][6][R][2] densities of R right-hand sides
    DBuf<float2> d_sCm;       // [nt][R][3] curl sources
    DBuf<float> d_partm;      // [ns][R][4][6nt] u1, u2 partial sums
    DBuf<float> d_partA;      // [ns][R][6][nt] curl-term partial sums per test triangle
    DBuf<int> d_farm_err;     // set when the kernel gave up a bounded wait
    // when set and true, a lockstep GMRES on this problem stops at its next
    // iteration with OSRC_TIMEOUT (the serving loop's shutdown)
    const std::atomic<bool> *cancel = nullptr;
    int farm_ns = 1, farm_cap = 0;
    bool far_reduce = false;  // centred far kernel with float-float phases (large k r)
    // ---- FP64 per-triangle geometry: area, normal, curls of the hat functions
    DBuf<double> d_tgeo;      // [nt][16]
    // ---- near field CSR (vertex pairs of touching triangles), FP64 --------
    long long near_pairs = 0;
    int near_nnz = 0;
    DBuf<int> d_nr_ptr, d_nr_col;
    DBuf<double2> d_nr_val;   // [nnz][4]: blocks (1,1) (1,2) (2,1) (2,2)
    // ---- sparse mass / stiffness (1-ring CSR), FP64 ----------------------
    int ms_nnz = 0;
    DBuf<int> d_ms_ptr, d_ms_col;
    std::vector<int> ms_ptr_h;  // host copy of the CSR row pointers (shared-memory sizing)
    DBuf<double> d_M, d_S;
    // ---- dense FP64 system (OSRC_FP64_DENSE) -------------------------------
    DBuf<double2> d_dense;    // [2nv][2nv] row-major
    // ---- OSRC constants (Sec. 2.6) -------------------------------------------
    double k_osrc = 0.0, k_osrc_i = 0.0;  // OSRC wavenumber (complex with attenuation)
    double2 k_eps{};
    double2 C0{}, g0{};
    std::vector<double2> A, B, g;
    // ---- inner solver workspace ------------------------------------------------
    DBuf<double2> d_kry;      // batched CG/COCG vectors
    DBuf<double2> d_kry_rhs;  // right-hand sides of the shifted systems
    DBuf<double2> d_tmp2;     // [2][2nv] temporaries
    DBuf<int> d_kry_stat;     // per-system iteration count / status
    DBuf<double> d_kry_res;   // per-system final relative residual
    int inner_last_max = 0;
    // mixed-precision inner solver (k_sparse.cu): -1 not yet decided, 0 not
    // usable for this problem, 1 usable with kmix_rpt rows per thread,
    // kmix_threads threads and kmix_smem bytes of dynamic shared memory
    int kmix_state = -1, kmix_rpt = 0, kmix_threads = 0;
    size_t kmix_smem = 0;
    // ---- GMRES workspace --------------------------------------------------------
    DBuf<double2> d_basis;    // (maxit+1) x 2nv
    int basis_cap = 0;
    DBuf<double2> d_h;        // Hessenberg (maxit+1) x maxit, column-major
    DBuf<double2> d_givens;   // cs (as .x), sn, g vectors
    DBuf<double> d_scalars;   // reduction scratch
    DBuf<double2> d_w, d_y, d_x1, d_b1, d_cvec;  // 2nv vectors
    double *h_res = nullptr;  // pinned host block: doubles [0, 16), then ints (inner status)
    // ---- disjoint objects with their own materials --------------------------------
    bool multi = false;          // more than one object: interior terms within objects only
    double far_dks = 1.0;        // scale of the far kernel's D normal term (far_dnormal_scale)
    bool far_obj = false;        // far kernel with per-object constants (objects or Mueller)
    bool absorb = false;         // some object has a complex interior wavenumber
    std::vector<ObjMat> obj;     // [ncomp]
    DBuf<ObjMat> d_obj;
    DBuf<FarObj> d_fobj;
    DBuf<double2> d_obj_ike;     // [2][ncomp]: i k_osrc, then 1 / k_eps^2 per object (OSRC)
    // ---- field evaluation off the surface (k_field.cu) -------------------------
    DBuf<double4> d_fsrc;     // [6nt][3] rule points, normals, densities
    DBuf<int> d_freg;         // region scratch when the caller passes none
    DBuf<int> d_fobeg;        // [objects + 1] source-point ranges of the objects
    // ---- far-kernel event timing -------------------------------------------------
    bool prof_on = false, prof_pending = false;
    int prof_rhs_pending = 1;    // right-hand sides of the last timed far launch
    long long prof_rhs = 0;      // right-hand sides summed over the timed launches
    cudaEvent_t prof_ev[2] = {nullptr, nullptr};
    long long prof_launches = 0;
    double prof_ms = 0.0;
};

int far_prof_collect(osrc_problem *pb);

// ---------------------------------------------------------------------------
// kernel launchers (each returns an osrc_status; all work on `st`)
// ---------------------------------------------------------------------------
// far field (k_far.cu)
int far_setup_geometry(osrc_problem *pb, cudaStream_t st);
int far_apply(osrc_problem *pb, const double2 *x, double2 *y, int part, cudaStream_t st);
// y_r = B x_r for nrhs vectors (far part of several right-hand sides per launch
// where the problem allows it: one object, PMCHWT, lossless interior)
int far_apply_multi(osrc_problem *pb, const double2 *const *xs, double2 *const *ys, int nrhs, int part,
                    cudaStream_t st);
bool far_multi_supported(const osrc_problem *pb);
int far_multi_check(osrc_problem *pb, cudaStream_t st);

// near field (k_near.cu)
int near_build(osrc_problem *pb, const std::vector<NearPair> &pairs,
               const std::vector<int> &contrib_ptr, const std::vector<int> &contrib_idx,
               cudaStream_t st);

// dense FP64 (k_near.cu)
int dense_assemble(osrc_problem *pb, cudaStream_t st);
int near_add_mass(osrc_problem *pb, cudaStream_t st);  // Mueller: + M in blocks (1,2), (2,1)
int dense_apply(osrc_problem *pb, const double2 *x, double2 *y, cudaStream_t st);

// sparse M, S and the inner solvers (k_sparse.cu)
int ms_build(osrc_problem *pb, const std::vector<int> &contrib_ptr,
             const std::vector<int> &contrib_idx, cudaStream_t st);
int mass_solve(osrc_problem *pb, const double2 *x, double2 *y, cudaStream_t st);
int osrc_precond(osrc_problem *pb, const double2 *x, double2 *y, cudaStream_t st);
int osrc_precond_fused(osrc_problem *pb, const double2 *y, double2 *z, cudaStream_t st);
// the same without waiting: the inner status is left in d_kry_stat
int osrc_precond_fused_async(osrc_problem *pb, const double2 *y, double2 *z, cudaStream_t st);
int osrc_precond_nsys(const osrc_problem *pb);
// turns a host copy of the inner status words into a status code
int kry_status_host(osrc_problem *pb, const int *stat, int nsys);

// GMRES helpers (k_gmres.cu)
int vec_dots_conj(osrc_problem *pb, const double2 *V, int nvec, const double2 *w, int n,
                  double2 *out, cudaStream_t st);
int vec_update(osrc_problem *pb, const double2 *V, int nvec, const double2 *h, double2 *w,
               int n, cudaStream_t st);
int vec_norm(osrc_problem *pb, const double2 *w, int n, double *out, cudaStream_t st);
int vec_scale_copy(osrc_problem *pb, const double2 *w, const double *nrm, double2 *out,
                   int n, cudaStream_t st);
int gmres_givens(osrc_problem *pb, int j, int ldh, double2 *H, double2 *gv, double *res_out,
                 double beta_norm_for_rel, cudaStream_t st);
int gmres_finish(osrc_problem *pb, int j, int ldh, const double2 *H, const double2 *gv,
                 const double2 *V, double2 *x, int n, cudaStream_t st);
int vec_axpby(osrc_problem *pb, double2 a, const double2 *x, double2 b, const double2 *y,
              double2 *out, int n, cudaStream_t st);

// right-hand sides (k_rhs.cu)
int rhs_build(osrc_problem *pb, int kind, const double *src3, double2 *b, cudaStream_t st);

// ---------------------------------------------------------------------------
// resumable GMRES (osrc_api.cu): one right-hand side, advanced one iteration
// at a time without blocking the host, so that several runs overlap on the
// GPU (the serving loop) or are driven to completion synchronously
// (osrc_gmres_solve).
// ---------------------------------------------------------------------------
struct GmresRun {
    osrc_problem *pb = nullptr;
    cudaStream_t st = nullptr;
    const double2 *b = nullptr;
    double2 *x = nullptr;
    double tol = 1e-5;
    int maxit = 100;
    int j = 0;          // completed iterations
    double beta = 0.0;  // |P M^-1 b|
    double res = 1.0;   // relative preconditioned residual estimate
    int phase = 0;      // 0 idle, 1 initial norm, 2 iteration, 3 final residual, 4 done
    int status = OSRC_OK;
    bool converged = false;
    cudaEvent_t ev = nullptr;
    cudaEvent_t tev[4] = {nullptr, nullptr, nullptr, nullptr};
    osrc_solve_info info{};
    // deferred mode (batches of runs sharing one several-right-hand-side
    // apply): advance() only records the next step, 1 iteration or 2 finish,
    // and the batch driver enqueues it
    bool defer = false;
    int next = 0;
    int start(osrc_problem *p, cudaStream_t s, const double2 *b_, double2 *x_, double tol_, int maxit_);
    bool ready() const;   // the work enqueued last has finished
    int advance();        // consumes the finished step and enqueues the next
    bool done() const { return phase == 4; }
    int run_to_completion();
    ~GmresRun();
};

int ensure_gmres_workspace(osrc_problem *pb, int maxit);
// a problem that borrows the resident state of `master` and owns a fresh
// workspace (per-apply, inner-solver and GMRES buffers)
int problem_clone(osrc_problem *master, osrc_problem **out);
// device bytes of the resident state and of one workspace (estimates used
// for admission by device memory)
size_t estimate_problem_bytes(int nv, int nt, const osrc_params &p);
size_t estimate_work_bytes(int nv, int nt, const osrc_params &p, int maxit);
size_t estimate_batched_bytes(int nv, int n_pade, int nrhs, int maxit);
