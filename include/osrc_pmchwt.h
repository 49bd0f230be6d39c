/*
 * osrc_pmchwt.h -- C ABI of the GB300 (sm_103a) OSRC-preconditioned PMCHWT
 * library for harmonic acoustic transmission through a penetrable object
 * (van 't Wout, Haqshenas, Gelat, Betcke, Saffari, "Frequency-robust
 * preconditioning of boundary integral equations for acoustic transmission",
 * J. Comput. Phys. 2022, arXiv 2104.04609).
 *
 * The problem (Sec. 2.1, eq. "helmholtz"): exterior wavenumber k_ext, interior
 * wavenumber k_int, density ratio rho = rho_int / rho_ext, a closed surface
 * given as a flat-triangle mesh.  The unknowns are the P1 coefficients of
 * psi = gamma_N^+ u_tot and phi = gamma_D u_tot (Sec. 2.2), stored in the
 * permuted order of Sec. 2.7:  x = [psi_0 .. psi_{nv-1}, phi_0 .. phi_{nv-1}].
 * The system matrix is the permuted PMCHWT operator of Sec. 2.7,
 *     B = [[V0 + rho V1, -K0 - K1], [T0 + T1, D0 + D1 / rho]],
 * discretised with P1 Galerkin (Sec. 2.3), left-preconditioned by the mass
 * matrix (strong form, Sec. 2.4) and by the OSRC operator
 * diag(L_DtN, L_NtD) (Sec. 2.6, 2.7), and solved by GMRES without restart
 * (Sec. 3.1).
 *
 * Conventions for every entry point:
 *  - Complex vectors are interleaved double (re, im), i.e. C99
 *    "double complex" / cuDoubleComplex, one vector of 2*nv entries per
 *    right-hand side, right-hand sides stored one after another.
 *  - "device" pointers are CUDA global-memory pointers owned by the caller
 *    (for instance PyTorch tensors); "host" pointers are ordinary memory.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    All device work of a call is enqueued on that stream.
 *  - Every call returns an osrc_status.  No C++ exception and no device trap
 *    crosses the ABI.  On error the output buffers are unspecified and the
 *    handles stay valid.
 *  - Handles (osrc_ctx, osrc_mesh, osrc_problem) own the device memory they
 *    allocate.  A handle must not be used from two host threads at once.
 */
#ifndef OSRC_PMCHWT_H
#define OSRC_PMCHWT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
typedef enum osrc_status {
    OSRC_OK = 0,
    OSRC_INVALID_ARG = 1,     /* bad pointer, size, index, NaN, degenerate mesh */
    OSRC_OUT_OF_MEMORY = 2,   /* device allocation failed or memory budget exceeded */
    OSRC_CUDA_ERROR = 3,      /* a CUDA runtime call failed */
    OSRC_NOT_CONVERGED = 4,   /* an iterative solver reached its iteration limit */
    OSRC_BREAKDOWN = 5,       /* Krylov breakdown (zero pivot in COCG / GMRES) */
    OSRC_TIMEOUT = 6,         /* a bounded device wait gave up */
    OSRC_UNSUPPORTED = 7      /* option not implemented or device not capable */
} osrc_status;

/* Human-readable name of a status code (static string, never NULL). */
const char *osrc_status_string(int status);

/* ---- opaque handles ------------------------------------------------------- */
typedef struct osrc_ctx osrc_ctx;
typedef struct osrc_mesh osrc_mesh;
typedef struct osrc_problem osrc_problem;

/* Precision / operator path of a problem. */
enum {
    OSRC_FP32_MATFREE = 0,  /* matrix-free FP32 far field + FP64 near CSR (Sec. 2.2/2.3 operators) */
    OSRC_FP64_DENSE = 1     /* dense FP64 assembled 2nv x 2nv system */
};

/* Parameters of one transmission problem (Sec. 2.1, 2.6, 3.1). */
typedef struct osrc_params {
    double k_ext;        /* exterior wavenumber k_0 (> 0) */
    double k_int;        /* interior wavenumber k_1 (> 0) */
    double rho_ratio;    /* rho_1 / rho_0 (> 0) */
    int n_pade;          /* number of Pade terms N_Pade (1..16; paper: 4) */
    double theta;        /* branch-cut rotation angle (paper: pi/3) */
    double damping_R;    /* R in k_eps = k (1 + 0.4 i (k R)^(-2/3)); <= 0: mean edge length */
    int osrc_side;       /* wavenumber of the OSRC operator: 0 exterior, 1 interior */
    int n_ss;            /* Gauss points per dimension of the Sauter-Schwab rules (2..12) */
    int precision;       /* OSRC_FP32_MATFREE or OSRC_FP64_DENSE */
    double inner_tol;    /* relative residual of the inner mass / shifted solves (<= 1e-8);
                            checked on the true FP64 residual when the solves run
                            as FP32 iterations refined in FP64 (meshes whose
                            per-cluster-CTA slices fit shared memory) */
    int inner_maxit;     /* iteration cap of the inner solves */
    int precond;         /* preconditioner P of the GMRES solve: OSRC_PRECOND_* */
    int formulation;     /* OSRC_PMCHWT (default) or OSRC_MULLER */
    double k_int_im;     /* attenuation: imaginary part of the interior wavenumber
                            (>= 0; Sec. 3.1, k_m = 2 pi f / c_m + i alpha_m f^b_m),
                            added to every object's; the exterior stays lossless */
    int dense_assembly;  /* arithmetic of the OSRC_FP64_DENSE far-pair assembly:
                            OSRC_ASSEMBLE_FP64 (default) or OSRC_ASSEMBLE_FF */
} osrc_params;

/* Arithmetic of the dense assembly (the stored matrix is FP64 either way).
 * OSRC_ASSEMBLE_FF evaluates the far-pair integrands in float-float
 * arithmetic (pairs of FP32 numbers, about 48 significant bits; sine and
 * cosine by Cody-Waite reduction and Taylor series) on the FP32 pipes:
 * entries agree with the FP64 assembly to about 1e-13 relative at phases
 * k r of order 100.  Attenuating interiors (k_int_im > 0) keep FP64. */
enum { OSRC_ASSEMBLE_FP64 = 0, OSRC_ASSEMBLE_FF = 1 };

/* Boundary integral formulation (Sec. 2.2), both in the permuted ordering
 * [psi; phi] with the same right-hand side:
 *   OSRC_PMCHWT: [[V0 + rho V1, -K0 - K1], [T0 + T1, D0 + D1/rho]] (sum of the
 *                exterior and interior Calderon equations, first kind);
 *   OSRC_MULLER: [[V0 - rho V1, -K0 + K1 + M], [T0 - T1 + M, D0 - D1/rho]]
 *                (their difference plus the identity, M the P1 mass matrix;
 *                second kind without density contrast).
 * With several objects the interior terms are those of each object. */
enum { OSRC_PMCHWT = 0, OSRC_MULLER = 1 };

/* Preconditioners of the matrix-free and FP64 dense GMRES solves; GMRES runs
 * on P B x = P b with, for a weak-form vector y,
 *   OSRC_PRECOND_OSRC:     P y = diag(L_DtN, L_NtD) M^-1 y (Sec. 2.6, 2.7);
 *   OSRC_PRECOND_MASS:     P y = M^-1 y (mass preconditioning, Sec. 2.4);
 *   OSRC_PRECOND_CALDERON: P y = M^-1 B Pi M^-1 y, the block Calderon
 *     preconditioner of Sec. 2.5 for one object (the PMCHWT operator in its
 *     unpermuted ordering; Pi swaps the two block rows), one more operator
 *     apply and two mass solves per iteration.
 * The batched dense solve always uses OSRC. */
enum { OSRC_PRECOND_OSRC = 0, OSRC_PRECOND_MASS = 1, OSRC_PRECOND_CALDERON = 2 };

/* Fills p with the paper's defaults: n_pade 4, theta pi/3, interior OSRC
 * wavenumber, R = mean edge length, n_ss 4, FP32 matrix-free, inner_tol 1e-10,
 * OSRC preconditioner, PMCHWT formulation. */
void osrc_params_default(osrc_params *p);

/* Result record of osrc_gmres_solve (per right-hand side: the last one). */
typedef struct osrc_solve_info {
    int iterations;            /* GMRES iterations of the last right-hand side */
    int converged;             /* 1 if every right-hand side reached tol */
    double precond_residual;   /* |P M^-1 (b - B x)| / |P M^-1 b| (GMRES estimate) */
    double true_residual;      /* |b - B x| / |b|, weak form, recomputed at the end */
    double ms_total;           /* wall time of the call in ms */
    double ms_matvec;          /* time in B x (far + near), ms, summed */
    double ms_precond;         /* time in M^-1 and OSRC, ms, summed */
    double ms_arnoldi;         /* time in orthogonalisation, ms, summed */
    int inner_iterations_max;  /* largest inner CG/COCG iteration count seen (FP32
                                  iterations over all refinements when refined) */
    int total_iterations;      /* GMRES iterations summed over right-hand sides */
    double ms_queued;          /* server requests: submit to the start of the request's
                                  first GPU work, ms (0 for direct calls) */
} osrc_solve_info;

/* ---- context -------------------------------------------------------------- */
/* Creates a context on CUDA device `device`.  mem_budget_bytes caps the device
 * memory the library allocates through this context (0 = no cap); an
 * allocation beyond it fails with OSRC_OUT_OF_MEMORY. */
int osrc_create(osrc_ctx **out, int device, size_t mem_budget_bytes);
void osrc_destroy(osrc_ctx *ctx);
/* Device bytes currently allocated through the context. */
size_t osrc_mem_used(const osrc_ctx *ctx);

/* ---- mesh ----------------------------------------------------------------- */
/* Host-only check of a surface mesh (no device work): indices in range, no
 * repeated vertex in a triangle, no zero-area triangle, finite coordinates,
 * every edge shared by exactly two triangles with opposite orientation
 * (closed, consistently oriented 2-manifold).  verts: host, nv x 3 row-major;
 * tris: host, nt x 3, counter-clockwise seen from outside. */
int osrc_mesh_validate(const double *verts, int32_t nv, const int32_t *tris, int32_t nt);

/* Validates (as above), copies the mesh to the device and builds its
 * topology.  verts, tris: host, not retained. */
int osrc_mesh_create(osrc_ctx *ctx, const double *verts, int32_t nv,
                     const int32_t *tris, int32_t nt, osrc_mesh **out);
void osrc_mesh_destroy(osrc_mesh *mesh);
/* Mean edge length of the mesh (the default damping length R). */
double osrc_mesh_mean_edge(const osrc_mesh *mesh);

/* ---- problem (resident per-mesh, per-frequency state) ----------------------- */
/* Builds the resident state of one problem on the mesh: FP32 far-field
 * geometry, the near-field CSR of touching triangle pairs computed on the
 * device in FP64 by Sauter-Schwab quadrature, the P1 mass M and stiffness S
 * (CSR, FP64), the Pade constants of the OSRC operator (Sec. 2.6).  With
 * OSRC_FP64_DENSE it also assembles the dense system matrix.  The mesh must
 * outlive the problem. */
int osrc_problem_create(osrc_mesh *mesh, const osrc_params *params,
                        osrc_problem **out, void *stream);

/* Disjoint objects (Sec. 2.2, multiple scattering; the paper's four-sphere
 * experiment, Sec. 3.5): the objects are the connected components of the
 * mesh (triangles sharing vertices), numbered in the order of their first
 * triangle (osrc_mesh_objects gives their count).  Object m has its own
 * interior wavenumber k_int[m] and density ratio rho_ratio[m]; the system's
 * diagonal blocks are A_0,mm + A^_m (interior operators within the object),
 * its cross blocks A_0,mn exterior operators only; the OSRC preconditioner
 * is block diagonal with each object's wavenumber (interior side) and the
 * common damping length; the field inside object m uses its material.
 * prm->k_int and prm->rho_ratio are ignored.  nobj must equal the mesh's
 * object count (OSRC_INVALID_ARG otherwise).  osrc_problem_create on a mesh
 * with several objects gives every object prm's material. */
int osrc_problem_create_objects(osrc_mesh *mesh, const osrc_params *prm, int nobj,
                                const double *k_int, const double *rho_ratio, osrc_problem **out,
                                void *stream);
int osrc_mesh_objects(const osrc_mesh *mesh);
void osrc_problem_destroy(osrc_problem *pb);
int osrc_problem_nv(const osrc_problem *pb);

/* ---- right-hand sides (Sec. 2.7) --------------------------------------------- */
/* b[r] = [<u_inc, phi_i>; <du_inc/dn, phi_i>], 6-point rule per triangle.
 * Plane wave u_inc = exp(i k_ext d.x), dirs: host, nrhs x 3 unit vectors.
 * b: device, nrhs x 2nv complex. */
int osrc_rhs_planewave(osrc_problem *pb, const double *dirs, int nrhs, void *b, void *stream);
/* Point source u_inc = exp(i k_ext |x - x0|) / (4 pi |x - x0|); srcs: host,
 * nrhs x 3 positions off the surface. */
int osrc_rhs_pointsource(osrc_problem *pb, const double *srcs, int nrhs, void *b, void *stream);

/* ---- operators ------------------------------------------------------------------ */
enum { OSRC_WEAK = 0, OSRC_STRONG = 1 };
enum { OSRC_PART_FAR = 1, OSRC_PART_NEAR = 2, OSRC_PART_ALL = 3 };

/* y = B x (form OSRC_WEAK) or y = M^-1 B x (OSRC_STRONG), for nrhs vectors.
 * part selects the far-field (triangle pairs sharing no vertex, 6-point rule
 * on both triangles) and/or near-field (touching pairs, Sauter-Schwab) terms;
 * a partial apply is only meaningful with OSRC_WEAK.  x, y: device,
 * nrhs x 2nv complex, must not overlap. */
int osrc_pmchwt_apply(osrc_problem *pb, const void *x, void *y, int nrhs,
                      int form, int part, void *stream);

/* y = M^-1 x on both block rows (mass preconditioning, Sec. 2.4): CG on the
 * P1 mass matrix to params.inner_tol.  x, y: device, nrhs x 2nv complex. */
int osrc_mass_solve(osrc_problem *pb, const void *x, void *y, int nrhs, void *stream);

/* y = diag(L_DtN, L_NtD) x on strong-form coefficient vectors (Sec. 2.6, 2.7):
 *   L_DtN u = i k [C0 u + sum_j A_j w_j],  (M - B_j S / k_eps^2) w_j = -S u / k_eps^2
 *   L_NtD u = [g0 v_0 + sum_j g_j v_j] / (i k),
 *             (M - S / k_eps^2) v_0 = M u,  (M - B_j S / k_eps^2) v_j = M u
 * with the rotated-branch Pade coefficients C0, A_j, B_j of sqrt(1+z) and
 * the partial fractions g0, g_j of its product with (1+z)^-1.  The 2 N_Pade + 1
 * complex-symmetric shifted systems are solved together by a batched COCG to
 * params.inner_tol.  With params.precond = OSRC_PRECOND_MASS, y = x; with
 * OSRC_PRECOND_CALDERON, y = M^-1 B Pi x (see OSRC_PRECOND_*).  x, y:
 * device, nrhs x 2nv complex. */
int osrc_precond_apply(osrc_problem *pb, const void *x, void *y, int nrhs, void *stream);

/* ---- solve ----------------------------------------------------------------------- */
enum { OSRC_HOST_BUFFERS = 1 };

/* Solves B x = b for nrhs right-hand sides with GMRES without restart
 * (Sec. 3.1), x0 = 0, on the OSRC- and mass-preconditioned system
 * P M^-1 B x = P M^-1 b, stopping when the preconditioned relative residual
 * is <= tol or after maxit iterations (OSRC_NOT_CONVERGED).  Orthogonalisation
 * (classical Gram-Schmidt, twice) and the Givens updates are FP64 on the
 * device.  b, x: nrhs x 2nv complex; device pointers, or host pointers when
 * flags has OSRC_HOST_BUFFERS (the copies are then part of the call).
 * info may be NULL. */
int osrc_gmres_solve(osrc_problem *pb, const void *b, void *x, int nrhs, double tol,
                     int maxit, int flags, osrc_solve_info *info, void *stream);

/* ---- tensor-core GEMM (dense assembled path) ----------------------------------------- */
/* C = A B^T on the 5th-generation tensor cores (tcgen05 MMA, FP32 accumulator
 * in tensor memory, TMA-staged operands): the dense complex products of the
 * assembled path (Sec. 2.3 system applied to blocks of right-hand sides) run
 * through it in their real embedding.  A: device BF16, M x K row-major;
 * B: device BF16, N x K row-major (both K-major); C: device FP32, M x ldc,
 * ldc >= N.  M % 128 == 0, K % 64 == 0, 16 <= N <= 256 with N % 16 == 0,
 * rows 16-byte aligned; otherwise OSRC_INVALID_ARG.  The tile x K-slice work
 * is spread over one CTA per SM; tiles split between CTAs leave their pieces
 * in ws_dev (device, caller-owned, 16-byte aligned, at least
 * osrc_gemm_bf16_ws_bytes bytes; may be NULL when that is 0, else
 * OSRC_INVALID_ARG) and a second launch on the same stream sums them in a
 * fixed order, so C is identical from run to run.  Calls that share ws_dev
 * must not overlap on the GPU.  err_flag_dev: device int that the kernel
 * sets to 1 if a bounded wait gave up (then C is unspecified). */
int osrc_gemm_bf16(const void *A, int M, int K, const void *B, int N, float *C, int ldc,
                   void *ws_dev, size_t ws_bytes, int *err_flag_dev, void *stream);

/* Workspace bytes osrc_gemm_bf16 needs for this shape on the current device
 * (depends on its SM count; 0 when no tile is split).  Unsupported shapes:
 * OSRC_INVALID_ARG. */
int osrc_gemm_bf16_ws_bytes(int M, int N, int K, size_t *bytes);

/* ---- batched mixed-precision solve (dense assembled path) ---------------------------- */
typedef struct osrc_batched_info {
    int refinements;       /* outer FP64 refinement steps taken */
    int inner_iterations;  /* inner GMRES iterations summed over the steps */
    double residual;       /* largest |b_r - A x_r| / |b_r| over the right-hand sides (FP64) */
    double ms_total;
} osrc_batched_info;

/* Solves A x_r = b_r for up to 128 right-hand sides at once on a problem
 * created with OSRC_FP64_DENSE (A = the assembled permuted PMCHWT system of
 * Sec. 2.7): outer iterative refinement x += d (x in FP64), r = b - A x
 * (residual of the FP64 matrix in float-float arithmetic, about 48
 * significant bits), each correction solved approximately for all
 * right-hand sides together by GMRES on P M^-1 A d = P M^-1 r (OSRC and mass
 * preconditioning of Sec. 2.4-2.7, inner Krylov solves in FP32) whose
 * operator applies the far-field part of A in BF16 on the tensor cores (FP32
 * accumulation) and the touching-pair blocks exactly.  Stops when every
 * |b_r - A x_r| / |b_r| <= tol or after max_refine steps
 * (OSRC_NOT_CONVERGED).  inner_tol: relative tolerance of each inner solve
 * (e.g. 1e-3); inner_maxit <= 1000.  precond_tol: relative tolerance of the
 * FP32 shifted solves inside P M^-1 (at most 500 iterations each); <= 0
 * selects 0.1 inner_tol clamped to [1e-6, 1e-3].  b, x: device, nrhs x 2nv
 * complex FP64. */
int osrc_dense_batched_solve(osrc_problem *pb, const void *b, void *x, int nrhs, double tol,
                             int max_refine, double inner_tol, int inner_maxit, double precond_tol,
                             osrc_batched_info *info, void *stream);

/* The inner pieces of osrc_dense_batched_solve on nrhs (<= 128) vectors,
 * computed in FP32 / BF16 and returned in FP64: what 0 the inner operator
 * (far field BF16 on the tensor cores + exact touching-pair blocks), 1 the
 * FP32 preconditioner P M^-1 (Sec. 2.4, 2.6), 2 their product.  x, y:
 * device, nrhs x 2nv complex FP64.  Problem created with OSRC_FP64_DENSE. */
int osrc_dense_batched_apply(osrc_problem *pb, const void *x, void *y, int nrhs, int what,
                             void *stream);

/* Explicit preconditioner for the batched dense solve: P M^-1 (Sec. 2.4,
 * 2.6) is applied once to every unit vector (blocks of 128 columns, FP32
 * shifted solves to relative tolerance tol, at most maxit iterations each)
 * and stored as a 2nv x 2nv complex matrix in BF16, packed like the system
 * matrix (1 GB at nv = 8000).  From then on osrc_dense_batched_solve
 * applies the preconditioner as one tensor-core GEMM per inner iteration
 * instead of 2 N_p + 2 shifted Krylov solves.  The rounding of this matrix
 * changes the inner iteration count, not the solution: the inner GMRES
 * still solves A d = r, and the outer residual decides convergence.
 * Synchronises the stream.  osrc_dense_precond_drop frees the matrix and
 * returns to the iterative preconditioner. */
int osrc_dense_precond_build(osrc_problem *pb, double tol, int maxit, void *stream);
int osrc_dense_precond_drop(osrc_problem *pb);

/* As osrc_dense_batched_apply (which uses ptol 1e-6, pmaxit 1000), with the
 * relative tolerance ptol and iteration cap pmaxit of the FP32 shifted
 * solves inside P M^-1 (Sec. 2.6) given explicitly, and what 3: P M^-1
 * through the explicit BF16 matrix of osrc_dense_precond_build
 * (OSRC_UNSUPPORTED if it has not been built).  pits_max (host, may be
 * NULL): the largest iteration count any of those solves took; passing it
 * synchronises the stream. */
int osrc_dense_batched_apply_ex(osrc_problem *pb, const void *x, void *y, int nrhs, int what,
                                double ptol, int pmaxit, int *pits_max, void *stream);

/* ---- field evaluation --------------------------------------------------------------- */
enum { OSRC_INC_NONE = 0, OSRC_INC_PLANEWAVE = 1, OSRC_INC_POINTSOURCE = 2 };

/* Total pressure at npts points off the surface from one solution
 * x = [psi; phi] of the permuted PMCHWT system (Sec. 2.2, representation
 * formulas; the paper's accuracy measure evaluates it on a grid, Sec. 3.2):
 * outside u = u_inc + DLP_0 phi - SLP_0 psi, inside u = rho SLP_1 psi -
 * DLP_1 phi (rho = rho_int / rho_ext, interior Neumann trace rho psi), every
 * potential by the 6-point rule per triangle with the P1 densities.  A
 * point is inside when the Laplace double layer of 1 exceeds 1/2 (Gauss's
 * solid angle; unreliable within about one mesh size of the surface, where
 * the rule itself loses accuracy).  inc_kind / inc_param: the incident
 * field added outside (OSRC_INC_PLANEWAVE: unit direction d, u_inc =
 * exp(i k_ext d.x); OSRC_INC_POINTSOURCE: position x0, u_inc =
 * exp(i k_ext |x - x0|) / (4 pi |x - x0|); OSRC_INC_NONE: scattered field
 * only; inc_param host, 3 doubles).  x: device, 2nv complex FP64; pts:
 * device, npts x 3 FP64; u: device, npts complex FP64 (out); region:
 * device int[npts] (out: m + 1 inside object m, 0 outside) or NULL.  With
 * several objects a point inside object m takes the interior representation
 * over that object's surface with its material.  FP64 throughout
 * (region test in FP32).  Asynchronous on stream. */
int osrc_field_eval(osrc_problem *pb, const void *x, const double *pts, int npts, int inc_kind,
                    const double *inc_param, void *u, int *region, void *stream);

/* ---- serving loop ------------------------------------------------------------------ */
/* A continuous-batching server for solve requests of uneven mesh size and
 * frequency (the serving pattern that the solver is deployed in).  A worker
 * thread owns the GPU work; each request is split into one GMRES job per
 * right-hand side; jobs are admitted into at most max_active slots as slots
 * free up and as the context's device-memory budget (osrc_create) allows.
 * Every slot has its own stream and workspace, so jobs overlap on the device;
 * each result is bit-identical to solving the request alone because no kernel
 * or launch configuration depends on the mix.  Resident problem state (mesh
 * topology, near-field CSR, M, S, Pade constants) is cached by mesh and
 * parameters and shared by every right-hand side and request that matches;
 * unreferenced entries are evicted least-recently-used when memory is
 * needed.  While a server exists its worker is the only user of the context:
 * create no other handles on it.  Requests that cannot fit even alone finish
 * with OSRC_OUT_OF_MEMORY.
 *
 * Requests whose params.precision is OSRC_FP64_DENSE are not split: all their
 * right-hand sides (same mesh, same frequency) are solved together as one
 * block by the batched mixed-precision solve (see osrc_dense_batched_solve;
 * tol applies to the true residual, 1e-3 inner tolerance, at most 400 inner
 * iterations per refinement, blocks of up to 128), on the cached problem,
 * whose assembled system, BF16 matrices and explicit preconditioner stay
 * resident for later requests on the same mesh and frequency.  Such a block
 * runs on a host thread of its own with its slot's stream, so it overlaps
 * with the other slots' work; one block per resident problem at a time.
 * Results equal a direct osrc_dense_batched_solve of the same block within
 * the solve's tolerance, not bit for bit: the FP64 assembly accumulates with
 * atomics, so each assembly differs in the last bits. */
typedef struct osrc_server osrc_server;

typedef struct osrc_request {
    const double *verts;   /* host, nv x 3; copied at submit */
    int32_t nv;
    const int32_t *tris;   /* host, nt x 3, counter-clockwise from outside; copied */
    int32_t nt;
    osrc_params params;    /* wavenumbers, density ratio, OSRC and quadrature options */
    int rhs_kind;          /* 0: plane waves (src = unit directions), 1: point sources (src = positions) */
    const double *src;     /* host, nrhs x 3; copied */
    int nrhs;
    double tol;            /* GMRES tolerance (preconditioned relative residual) */
    int maxit;             /* GMRES iteration cap */
} osrc_request;

typedef struct osrc_server_stats {
    long long submitted, completed, failed, jobs_started;
    long long cache_hits, cache_misses, evictions;
    long long active_peak;  /* most slots busy at once */
    size_t mem_peak;        /* most device bytes allocated through the context */
    size_t mem_used;        /* device bytes allocated now */
    long long batched_jobs; /* requests solved as one block of right-hand sides */
} osrc_server_stats;

/* Starts a server with max_active slots (1..64) on the context. */
int osrc_server_create(osrc_ctx *ctx, int max_active, osrc_server **out);
/* Queues a request (validates the mesh on the host); *id identifies it. */
int osrc_server_submit(osrc_server *sv, const osrc_request *req, long long *id);
/* Non-blocking: *done = 1 once every right-hand side has finished; then
 * latency_ms (submit to completion, host clock) and info (worst residuals,
 * summed iterations and phase times) are filled and the request's status is
 * returned.  May be called until osrc_server_result releases the request. */
int osrc_server_poll(osrc_server *sv, long long id, int *done, double *latency_ms,
                     osrc_solve_info *info);
/* Blocks until the request finishes (its status) or timeout_s passes (OSRC_TIMEOUT). */
int osrc_server_wait(osrc_server *sv, long long id, double timeout_s);
/* Copies the solution (host, nrhs x 2nv complex, [psi; phi] per right-hand
 * side) and releases the request; OSRC_TIMEOUT if it has not finished. */
int osrc_server_result(osrc_server *sv, long long id, void *x_host);
int osrc_server_get_stats(osrc_server *sv, osrc_server_stats *out);
/* Stops the worker (jobs in flight finish their current step; queued
 * requests are dropped) and frees every resource of the server. */
void osrc_server_destroy(osrc_server *sv);

/* ---- allocation-free batched solve ------------------------------------------------- */
/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory when they need a solve: code running
 * during CUDA stream capture, real-time or callback-driven hosts that forbid
 * allocation after start-up, and frameworks that own device memory through
 * their own pool allocator.
 *
 * Solves the nsys systems (alpha_s M + beta_s S) w_s = f_s that share one CSR
 * pattern (n rows) with the library's cluster-batched Krylov kernel:
 * Hermitian CG when conj = 1 (real SPD systems), COCG when conj = 0
 * (complex-symmetric systems), Jacobi-preconditioned, to |r_s| <= tol |f_s|
 * (0 < tol <= 1e-4, else OSRC_INVALID_ARG) or maxit iterations.  All pointers except alpha, beta and iters_out are
 * device pointers owned by the caller: row_ptr (n+1), col_idx, M_vals,
 * S_vals (row_ptr[n] each, int32 / double), f and w (nsys x n complex,
 * interleaved).  alpha, beta: host, nsys complex each.
 *
 * The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine.  Its Krylov workspace is a static device array of 5 x 131072
 * complex entries (10 MiB) that every GPU loading this library holds until
 * process exit; requests with nsys * n > 131072 or nsys > 16 are rejected
 * with OSRC_INVALID_ARG.  The work runs on the calling thread's current
 * device.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture;
 * the address is looked up again when the device's context has changed
 * (after cudaDeviceReset), so the first call after a reset also belongs
 * outside a capture.
 * All calls on a device share the array and it keeps the last call's
 * contents: calls whose kernels overlap on the GPU race and must be
 * serialised by the caller.
 *
 * If iters_out (host, nsys ints) is non-NULL the call waits for the stream
 * and reports per system the iteration count (negative: not converged) and
 * returns OSRC_NOT_CONVERGED / OSRC_BREAKDOWN accordingly; with NULL it only
 * enqueues the work and returns OSRC_OK. */
int osrc_shifted_solve_noalloc(int n, const int32_t *row_ptr, const int32_t *col_idx,
                               const double *M_vals, const double *S_vals, int nsys,
                               const double *alpha, const double *beta, const void *f, void *w,
                               double tol, int maxit, int conj, int *iters_out, void *stream);

/* ---- introspection ---------------------------------------------------------------- */
/* Number of kernel launches the library has issued on this problem so far. */
long long osrc_launch_count(const osrc_problem *pb);
/* Enables (on != 0) or disables CUDA-event timing of the far-field kernel
 * launches of this problem; enabling resets the statistics. */
int osrc_profile_enable(osrc_problem *pb, int on);
/* Far-field kernel statistics since profiling was enabled: number of
 * launches and their summed device time in ms (events recorded on the
 * launching stream around each launch).  Waits for the last timed launch. */
int osrc_far_kernel_stats(osrc_problem *pb, long long *launches, double *total_ms);
/* Right-hand sides processed by the timed far-field launches (a launch of the
 * several-right-hand-side kernel counts each of its vectors). */
long long osrc_far_kernel_rhs(const osrc_problem *pb);
/* Number of far-field point pairs one apply evaluates: 36 x (number of
 * triangle pairs sharing no vertex). */
long long osrc_far_pairs(const osrc_problem *pb);
/* Number of touching triangle pairs (near-field pairs) and near CSR blocks. */
long long osrc_near_pairs(const osrc_problem *pb);
long long osrc_near_nnz(const osrc_problem *pb);

/* ---- measurement aid ----------------------------------------------------------------- */
/* Not part of the paper's method.  Measures the FP32 throughput of the
 * calling thread's current GPU, the denominator of the far-field kernel's
 * roofline: FFMA (scalar) and FP32x2 FMA (packed) loops over independent
 * chains at full occupancy with no memory traffic, each launched reps + 2
 * times on `stream` (the first two untimed); the fastest launch gives
 * *tflops_scalar and *tflops_packed (FMA = 2 flops).  Allocates and frees a
 * small device buffer.  reps in [1, 100]. */
int osrc_fp32_peak(int reps, double *tflops_scalar, double *tflops_packed, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* OSRC_PMCHWT_H */
