// k_gmres.cu -- FP64 device kernels of GMRES without restart (Sec. 3.1):
// classical Gram-Schmidt projections (applied twice by the caller), norms,
// the complex Givens rotation of the new Hessenberg column and the final
// triangular solve / solution update.  Scalars stay on the device; the host
// reads one residual estimate per iteration.
#include "osrc_internal.cuh"

namespace {

constexpr int RED_THREADS = 256;

__device__ double2 block_sum_c(double2 v, double2 *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double2 s = cd(0, 0);
    for (int w = 0; w < nw; ++w) s = cadd(s, red[w]);
    return s;
}

// out[i] (+)= V_i^H w, one block per basis vector i.
__global__ void dots_kernel(const double2 *__restrict__ V, size_t ldv, int nvec,
                            const double2 *__restrict__ w, int n, double2 *__restrict__ out,
                            int accumulate) {
    __shared__ double2 red[32];
    const int i = blockIdx.x;
    if (i >= nvec) return;
    const double2 *v = V + ldv * i;
    double2 s = cd(0, 0);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double2 a = v[k], b = w[k];
        s.x += a.x * b.x + a.y * b.y;
        s.y += a.x * b.y - a.y * b.x;
    }
    s = block_sum_c(s, red);
    if (threadIdx.x == 0) out[i] = accumulate ? cadd(out[i], s) : s;
}

// w -= sum_i h_i V_i
__global__ void update_kernel(const double2 *__restrict__ V, size_t ldv, int nvec,
                              const double2 *__restrict__ h, double2 *__restrict__ w, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double2 s = w[k];
    for (int i = 0; i < nvec; ++i) s = csub(s, cmul(h[i], V[ldv * i + k]));
    w[k] = s;
}

__global__ void norm_kernel(const double2 *__restrict__ w, int n, double *__restrict__ out) {
    __shared__ double2 red[32];
    double2 s = cd(0, 0);
    for (int k = threadIdx.x; k < n; k += blockDim.x) s.x += cabs2(w[k]);
    s = block_sum_c(s, red);
    if (threadIdx.x == 0) *out = sqrt(s.x);
}

__global__ void scale_copy_kernel(const double2 *__restrict__ w, const double *__restrict__ nrm,
                                  double2 *__restrict__ out, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double s = *nrm;
    out[k] = s > 0.0 ? cscale(w[k], 1.0 / s) : cd(0, 0);
}

// gv layout: gv[0 .. ldh) = (cs, 0), gv[ldh .. 2 ldh) = sn, gv[2 ldh .. 3 ldh) = g.
// Applies the j earlier rotations to column j of H, builds rotation j,
// updates g and writes |g_{j+1}| / beta to res.
__global__ void givens_kernel(int j, int ldh, double2 *__restrict__ H, double2 *__restrict__ gv,
                              double beta, double *__restrict__ res) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double2 *h = H + (size_t)ldh * j;
    double2 *cs = gv, *sn = gv + ldh, *g = gv + 2 * ldh;
    for (int i = 0; i < j; ++i) {
        const double c = cs[i].x;
        const double2 s = sn[i];
        const double2 t = cadd(cscale(h[i], c), cmul(s, h[i + 1]));
        h[i + 1] = cadd(cscale(cmul(cconj(s), h[i]), -1.0), cscale(h[i + 1], c));
        h[i] = t;
    }
    const double2 a = h[j], b = h[j + 1];
    const double aa = sqrt(cabs2(a)), bb = sqrt(cabs2(b));
    const double nu = hypot(aa, bb);
    double c;
    double2 s;
    if (aa == 0.0) {
        c = 0.0;
        s = cd(1.0, 0.0);
    } else {
        c = aa / nu;
        s = cscale(cmul(cscale(a, 1.0 / aa), cconj(b)), 1.0 / nu);
    }
    cs[j] = cd(c, 0.0);
    sn[j] = s;
    h[j] = cadd(cscale(a, c), cmul(s, b));
    h[j + 1] = cd(0, 0);
    const double2 gj = g[j];
    g[j + 1] = cscale(cmul(cconj(s), gj), -1.0);
    g[j] = cscale(gj, c);
    *res = sqrt(cabs2(g[j + 1])) / beta;
}

// y = H(0:m, 0:m)^-1 g(0:m) (upper triangular, back substitution), stored
// in gv[3 ldh ..]; single thread (m is the iteration count).
__global__ void backsub_kernel(int m, int ldh, const double2 *__restrict__ H, double2 *__restrict__ gv) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double2 *g = gv + 2 * ldh;
    double2 *y = gv + 3 * ldh;
    for (int i = m - 1; i >= 0; --i) {
        double2 s = g[i];
        for (int k = i + 1; k < m; ++k) s = csub(s, cmul(H[(size_t)ldh * k + i], y[k]));
        y[i] = cdiv(s, H[(size_t)ldh * i + i]);
    }
}

// x = sum_i y_i V_i
__global__ void combine_kernel(const double2 *__restrict__ V, size_t ldv, int m,
                               const double2 *__restrict__ y, double2 *__restrict__ x, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double2 s = cd(0, 0);
    for (int i = 0; i < m; ++i) s = cadd(s, cmul(y[i], V[ldv * i + k]));
    x[k] = s;
}

__global__ void axpby_kernel(double2 a, const double2 *__restrict__ x, double2 b,
                             const double2 *__restrict__ y, double2 *__restrict__ out, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    out[k] = cadd(cmul(a, x[k]), cmul(b, y[k]));
}

}  // namespace

int vec_dots_conj(osrc_problem *pb, const double2 *V, int nvec, const double2 *w, int n,
                  double2 *out, cudaStream_t st) {
    // accumulate flag is encoded by a negative nvec
    const int acc = nvec < 0 ? 1 : 0;
    if (nvec < 0) nvec = -nvec;
    dots_kernel<<<nvec, RED_THREADS, 0, st>>>(V, (size_t)n, nvec, w, n, out, acc);
    pb->launches++;
    OSRC_CK(cudaGetLastError());
    return OSRC_OK;
}

int vec_update(osrc_problem *pb, const double2 *V, int nvec, const double2 *h, double2 *w, int n,
               cudaStream_t st) {
    update_kernel<<<(n + 255) / 256, 256, 0, st>>>(V, (size_t)n, nvec, h, w, n);
    pb->launches++;
    OSRC_CK(cudaGetLastError());
    return OSRC_OK;
}

int vec_norm(osrc_problem *pb, const double2 *w, int n, double *out, cudaStream_t st) {
    norm_kernel<<<1, 1024, 0, st>>>(w, n, out);
    pb->launches++;
    OSRC_CK(cudaGetLastError());
    return OSRC_OK;
}

int vec_scale_copy(osrc_problem *pb, const double2 *w, const double *nrm, double2 *out, int n,
                   cudaStream_t st) {
    scale_copy_kernel<<<(n + 255) / 256, 256, 0, st>>>(w, nrm, out, n);
    pb->launches++;
    OSRC_CK(cudaGetLastError());
    return OSRC_OK;
}

int gmres_givens(osrc_problem *pb, int j, int ldh, double2 *H, double2 *gv, double *res_out,
                 double beta, cudaStream_t st) {
    givens_kernel<<<1, 32, 0, st>>>(j, ldh, H, gv, beta, res_out);
    pb->launches++;
    OSRC_CK(cudaGetLastError());
    return OSRC_OK;
}

int gmres_finish(osrc_problem *pb, int m, int ldh, const double2 *H, const double2 *gv,
                 const double2 *V, double2 *x, int n, cudaStream_t st) {
    backsub_kernel<<<1, 32, 0, st>>>(m, ldh, H, (double2 *)gv);
    combine_kernel<<<(n + 255) / 256, 256, 0, st>>>(V, (size_t)n, m, gv + 3 * ldh, x, n);
    pb->launches += 2;
    OSRC_CK(cudaGetLastError());
    return OSRC_OK;
}

int vec_axpby(osrc_problem *pb, double2 a, const double2 *x, double2 b, const double2 *y,
              double2 *out, int n, cudaStream_t st) {
    axpby_kernel<<<(n + 255) / 256, 256, 0, st>>>(a, x, b, y, out, n);
    pb->launches++;
    OSRC_CK(cudaGetLastError());
    return OSRC_OK;
}
