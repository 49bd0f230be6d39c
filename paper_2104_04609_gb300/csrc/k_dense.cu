// k_dense.cu -- dense mixed-precision building blocks of the assembled path:
// a BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05 MMA
// with the accumulator in tensor memory, operands staged by TMA), used by
// the batched dense solve for the far-field product and the explicit
// preconditioner matrix.
//
// GEMM: C[M x N] = A[M x K] * B[N x K]^T, A and B BF16 and K-major (row-major
// with K contiguous), C FP32.  The product is cut into 128-row tiles and
// 64-wide K slices.  The tile x slice iterations are dealt out in equal
// contiguous ranges to a persistent grid of one CTA per SM (stream-K), so
// every SM works to the end even when the number of tiles is not a multiple
// of the SM count (the 16000-row product of the 8000-vertex system has 125
// tiles for 152 SMs).  Per CTA of 192 threads:
//   - lane 0 of warp 4 issues TMA loads (128-byte swizzle) of the K slices of
//     A (evict-first in L2: it is streamed once) and B (evict-last: every CTA
//     re-reads it) into a shared-memory ring of as many stages as fit;
//   - lane 0 of warp 5 issues tcgen05.mma (kind::f16, M 128, N, K 16) into
//     one of two FP32 accumulators in tensor memory, releases each stage with
//     tcgen05.commit and signals the end of each tile segment;
//   - warps 0-3 read the accumulator of a finished segment (tcgen05.ld, warp
//     w owns lanes 32w..32w+31, a thread one row) and store it as 16-byte
//     vectors while the MMAs of the next segment fill the other accumulator.
// A CTA range that covers a whole tile writes C directly.  A tile split
// between CTAs has its pieces written to a workspace (slot 2c for the first
// segment of CTA c, 2c + 1 for its last) and summed by a second kernel in CTA
// order, so C is the same bit for bit from run to run (no atomics).
// Every mbarrier wait is bounded (2 s of global time): on timeout the kernel
// records an error flag, stops waiting, waits (bounded) for its own TMA loads
// and MMAs in flight, frees its tensor memory and returns.
//
// Complex products use the real embedding: with A_cat = [Re A | Im A]
// (M x 2K) and, for right-hand sides X_r, B rows [Re X_r | -Im X_r] (first
// half) and [Im X_r | Re X_r] (second half), C's first half is Re(A X) and
// its second half Im(A X).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "osrc_internal.cuh"
#include "stream_k.cuh"

namespace {

constexpr int UM_BM = 128;              // rows of a tile (one tensor-memory lane per row)
constexpr int UM_NBUF = 2;              // accumulators in tensor memory (2 x N <= 512 columns)
constexpr int UM_BK = 64;               // 64 BF16 = one 128-byte swizzle row
constexpr int UM_THREADS = 192;         // warps 0-3 epilogue, warp 4 TMA, warp 5 MMA
constexpr int UM_MIN_ITERS = 48;        // fewest K slices per CTA
constexpr int UM_MAX_STAGES = 8;
constexpr size_t UM_SMEM_MAX = 230400;  // dynamic shared memory per CTA (227 KB less the static part)
constexpr size_t UM_SMEM_FIXED = 1024 + 256;  // alignment slack, barriers
constexpr int UM_FIX_ROWS = 8;                  // rows of a split tile per block of the summing kernel
constexpr unsigned long long UM_TIMEOUT_NS = 2000000000ULL;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Waits for the completion of phase `parity`; false after the time limit.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > UM_TIMEOUT_NS) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar,
                                            uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of
// 1024 bytes (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;              // version
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulate, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// ncols = tensor-memory columns of one accumulator (a power of two >= N);
// two accumulators alternate between the tile segments of a CTA.
__global__ void __launch_bounds__(UM_THREADS, 1)
umma_sk_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, int M,
               int N, int KB, long long iters, int stages, uint32_t ncols, float *__restrict__ C, int ldc,
               float *__restrict__ ws, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int nbuf = UM_NBUF;
    const uint32_t a_bytes = UM_BM * UM_BK * 2, b_bytes = (uint32_t)N * UM_BK * 2;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    uint64_t *bars = (uint64_t *)(base + (size_t)stages * stage_bytes);
    uint64_t *full = bars, *empty = bars + stages, *accf = bars + 2 * stages, *acce = accf + 2, *drain = acce + 2;
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);
    __shared__ int timed_out;
    volatile int *vto = &timed_out;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = gridDim.x, cta = blockIdx.x;
    const long long it_begin = sk_begin(cta, iters, G), it_end = sk_begin(cta + 1, iters, G);
    const uint32_t tcols = (uint32_t)nbuf * ncols;

    if (threadIdx.x == 0) {
        timed_out = 0;
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4 * 32);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (warp == 4) {
        if (lane == 0) {
            // TMA producer
            uint64_t pol_a, pol_b;
            asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol_a));
            asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol_b));
            uint32_t g = 0;  // K slices issued
            bool ok = true;
            for (long long it = it_begin; it < it_end && ok;) {
                const SkSeg sg = sk_next(it, it_end, KB);
                for (int j = 0; j < sg.n; ++j) {
                    const uint32_t s = g % (uint32_t)stages, u = g / (uint32_t)stages;
                    if (g >= (uint32_t)stages && !mbar_wait(&empty[s], (u - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    if (*vto) {
                        ok = false;
                        break;
                    }
                    unsigned char *sa = base + (size_t)s * stage_bytes, *sb = sa + a_bytes;
                    const int kx = (sg.kb0 + j) * UM_BK;
                    mbar_expect_tx(&full[s], stage_bytes);
                    tma_load_2d(sa, &map_a, kx, sg.tile * UM_BM, &full[s], pol_a);
                    tma_load_2d(sb, &map_b, kx, 0, &full[s], pol_b);
                    ++g;
                }
                it += sg.n;
            }
            if (!ok) {
                *vto = 1;
                // let the loads already issued land before the CTA exits
                for (uint32_t j = g > (uint32_t)stages ? g - stages : 0; j < g; ++j)
                    mbar_wait(&full[j % stages], (j / stages) & 1);
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // MMA issuer
            const uint32_t idesc = instr_desc(UM_BM, N);
            uint32_t g = 0;
            int seg = 0;
            bool ok = true;
            for (long long it = it_begin; it < it_end && ok; ++seg) {
                const SkSeg sg = sk_next(it, it_end, KB);
                const int b = seg % nbuf;
                const uint32_t use = (uint32_t)(seg / nbuf);
                if (seg >= nbuf && !mbar_wait(&acce[b], (use - 1) & 1)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t acc = tmem + (uint32_t)b * ncols;
                for (int j = 0; j < sg.n; ++j, ++g) {
                    const uint32_t s = g % (uint32_t)stages, u = g / (uint32_t)stages;
                    if (!mbar_wait(&full[s], u & 1)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t sa = smem_u32(base + (size_t)s * stage_bytes), sb = sa + a_bytes;
                    const uint64_t da = smem_desc(sa), db = smem_desc(sb);
#pragma unroll
                    for (int k = 0; k < UM_BK / 16; ++k) {
                        // 16 BF16 = 32 bytes along K inside the swizzled rows
                        const uint32_t accum = (j | k) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\t"
                            "setp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc),
                            "l"(da + (uint64_t)(2 * k)), "l"(db + (uint64_t)(2 * k)), "r"(idesc), "r"(accum));
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            smem_u32(&empty[s]))
                        : "memory");
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&accf[b]))
                             : "memory");
                it += sg.n;
            }
            if (!ok) *vto = 1;
            // every MMA issued has finished before the tensor memory is freed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(drain))
                         : "memory");
            if (!mbar_wait(drain, 0)) *vto = 1;
        }
    } else {
        // epilogue: warps 0-3
        int seg = 0;
        for (long long it = it_begin; it < it_end; ++seg) {
            const SkSeg sg = sk_next(it, it_end, KB);
            const int b = seg % nbuf;
            const uint32_t use = (uint32_t)(seg / nbuf);
            // the warp decides together: tcgen05.ld below needs all 32 lanes
            if (!__all_sync(0xffffffffu, mbar_wait(&accf[b], use & 1))) {
                *vto = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            float *dst;
            int ld, rows;
            bool vec;
            if (sg.kb0 == 0 && sg.n == KB) {
                dst = C + (size_t)sg.tile * UM_BM * ldc;
                ld = ldc;
                rows = M - sg.tile * UM_BM;
                vec = (ldc & 3) == 0 && ((uintptr_t)C & 15) == 0;
            } else {
                dst = ws + (size_t)sk_slot(cta, seg) * UM_BM * N;
                ld = N;
                rows = UM_BM;
                vec = true;
            }
            {
                const int r0 = warp * 32;
                for (int c0 = 0; c0 < N; c0 += 32) {
                    uint32_t v[32];
                    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)b * ncols + (uint32_t)c0;
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
                        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
                        "%28, %29, %30, %31}, [%32];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
                          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
                          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
                          "=r"(v[31])
                        : "r"(taddr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    // lane l holds columns c0 .. c0 + 31 of row r0 + l
                    const int r = r0 + lane;
                    if (r < rows) {
                        float *o = dst + (size_t)r * ld + c0;
                        if (vec) {
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                if (c0 + 4 * q < N)
                                    reinterpret_cast<float4 *>(o)[q] =
                                        make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                                    __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
                        } else {
#pragma unroll
                            for (int q = 0; q < 32; ++q)
                                if (c0 + q < N) o[q] = __uint_as_float(v[q]);
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(&acce[b]);
            it += sg.n;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
    if (threadIdx.x == 0 && timed_out) atomicExch(err, 1);
}

// Sums the pieces of every tile split between CTAs, in CTA order, into C.
// CTA c owns iterations [c I / G, (c + 1) I / G); the CTAs that touch tile t
// are those owning its first and last iteration and the ones between.
// Block (t, y) takes rows UM_FIX_ROWS y .. of tile t, one float4 column group
// per thread.
__global__ void umma_sk_fixup_kernel(int M, int N, int bmt, int KB, long long iters, int G,
                                     const float *__restrict__ ws, float *__restrict__ C, int ldc, bool vec) {
    const int tile = blockIdx.x;
    int c_lo, c_hi;
    sk_tile_ctas(tile, KB, iters, G, &c_lo, &c_hi);
    if (c_lo == c_hi) return;  // one CTA covered the tile and wrote C itself
    const int rows = min(bmt, M - tile * bmt), n4 = N / 4;
    const int rbeg = blockIdx.y * UM_FIX_ROWS, rend = min(rows, rbeg + UM_FIX_ROWS);
    for (int e = threadIdx.x; e < (rend - rbeg) * n4; e += blockDim.x) {
        const int r = rbeg + e / n4, q = e % n4;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int c = c_lo; c <= c_hi; ++c) {
            const int slot = sk_piece_slot(c, tile, KB, iters, G);
            const float4 v = reinterpret_cast<const float4 *>(ws + ((size_t)slot * bmt + r) * N)[q];
            s.x += v.x;
            s.y += v.y;
            s.z += v.z;
            s.w += v.w;
        }
        float *o = C + (size_t)(tile * bmt + r) * ldc + 4 * q;
        if (vec) {
            *reinterpret_cast<float4 *>(o) = s;
        } else {
            o[0] = s.x;
            o[1] = s.y;
            o[2] = s.z;
            o[3] = s.w;
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

int get_encoder() {
    static std::once_flag once;
    static cudaError_t e = cudaSuccess;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        e = cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", (void **)&g_encode, cudaEnableDefault, &q);
        if (e == cudaSuccess && q != cudaDriverEntryPointSuccess) e = cudaErrorNotSupported;
    });
    OSRC_CK(e);
    return g_encode ? OSRC_OK : OSRC_UNSUPPORTED;
}

int make_map(CUtensorMap *m, const void *ptr, int rows, int cols, int box_rows) {
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)UM_BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        osrc_set_error("cuTensorMapEncodeTiled failed");
        return OSRC_INVALID_ARG;
    }
    return OSRC_OK;
}

int sm_count(int *n) {
    static PerDeviceOnce once;
    static int count[OSRC_MAX_DEVICES] = {};
    OSRC_TRY(per_device_once(once, [](int dev) -> int {
        OSRC_CK(cudaDeviceGetAttribute(&count[dev], cudaDevAttrMultiProcessorCount, dev));
        return OSRC_OK;
    }));
    int dev = 0;
    OSRC_CK(cudaGetDevice(&dev));
    *n = count[dev];
    return OSRC_OK;
}

}  // namespace

// Launch plan of one product: persistent grid, ring depth, accumulator
// columns and workspace (the pieces of split tiles).
struct UmmaPlan {
    int tiles = 0, KB = 0, grid = 0, stages = 0;
    uint32_t ncols = 32;
    long long iters = 0;
    bool split = false;
    size_t smem = 0, ws_floats = 0;
};

static bool umma_shape_ok(int M, int N, int K) {
    return M > 0 && M % UM_BM == 0 && K > 0 && K % UM_BK == 0 && N >= 16 && N <= 256 && N % 16 == 0;
}

// One CTA per SM, but at least UM_MIN_ITERS K slices each.
static int umma_plan(int M, int N, int K, UmmaPlan *p) {
    if (!umma_shape_ok(M, N, K)) {
        osrc_set_error("umma_gemm_bf16: unsupported shape");
        return OSRC_INVALID_ARG;
    }
    int nsm = 0;
    OSRC_TRY(sm_count(&nsm));
    UmmaPlan q;
    q.tiles = M / UM_BM;
    q.KB = K / UM_BK;
    q.iters = (long long)q.tiles * q.KB;
    long long g = q.iters / UM_MIN_ITERS;
    if (g > nsm) g = nsm;
    if (g < 1) g = 1;
    q.grid = (int)g;
    while (q.ncols < (uint32_t)N) q.ncols <<= 1;
    const size_t stage = (size_t)UM_BM * UM_BK * 2 + (size_t)N * UM_BK * 2;
    q.stages = (int)((UM_SMEM_MAX - UM_SMEM_FIXED) / stage);
    if (q.stages > UM_MAX_STAGES) q.stages = UM_MAX_STAGES;
    q.smem = UM_SMEM_FIXED + (size_t)q.stages * stage;
    for (int c = 1; c < q.grid && !q.split; ++c)
        if (sk_begin(c, q.iters, q.grid) % q.KB) q.split = true;
    q.ws_floats = q.split ? (size_t)2 * q.grid * UM_BM * N : 0;
    *p = q;
    return OSRC_OK;
}

size_t umma_gemm_ws_floats(int M, int N, int K) {
    UmmaPlan p;
    return umma_plan(M, N, K, &p) == OSRC_OK ? p.ws_floats : 0;
}

// C = A B^T for BF16 A (M x K), B (N x K), FP32 C (M x ldc); ws holds
// ws_floats >= umma_gemm_ws_floats(M, N, K) floats (may be null when that is
// 0).  err: device int set to 1 if a bounded wait gave up.
static int umma_gemm_run(const void *A, int M, int K, const void *Bm, int N, float *C, int ldc, float *ws,
                         size_t ws_floats, int *err, cudaStream_t st) {
    UmmaPlan p;
    OSRC_TRY(umma_plan(M, N, K, &p));
    if (ldc < N || !A || !Bm || !C || !err) return OSRC_INVALID_ARG;
    if (((uintptr_t)A & 15) || ((uintptr_t)Bm & 15)) return OSRC_INVALID_ARG;
    if (p.split && (!ws || ws_floats < p.ws_floats || ((uintptr_t)ws & 15))) {
        osrc_set_error("umma_gemm_bf16: workspace missing or too small");
        return OSRC_INVALID_ARG;
    }
    OSRC_TRY(get_encoder());
    CUtensorMap ma, mb;
    OSRC_TRY(make_map(&ma, A, M, K, UM_BM));
    OSRC_TRY(make_map(&mb, Bm, N, K, N));
    static PerDeviceOnce once;
    OSRC_TRY(per_device_once(once, [](int) -> int {
        OSRC_CK(cudaFuncSetAttribute(umma_sk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)UM_SMEM_MAX));
        return OSRC_OK;
    }));
    umma_sk_kernel<<<p.grid, UM_THREADS, p.smem, st>>>(ma, mb, M, N, p.KB, p.iters, p.stages, p.ncols, C, ldc,
                                                       ws, err);
    OSRC_CK(cudaGetLastError());
    if (p.split) {
        const dim3 fg(p.tiles, UM_BM / UM_FIX_ROWS);
        const bool vec = (ldc & 3) == 0 && ((uintptr_t)C & 15) == 0;
        umma_sk_fixup_kernel<<<fg, 256, 0, st>>>(M, N, UM_BM, p.KB, p.iters, p.grid, ws, C, ldc, vec);
        OSRC_CK(cudaGetLastError());
    }
    return OSRC_OK;
}

// Requirements: M % 128 == 0, K % 64 == 0, 16 <= N <= 256 and N % 16 == 0,
// 16-byte aligned rows, ldc >= N.
int umma_gemm_bf16(const void *A, int M, int K, const void *Bm, int N, float *C, int ldc, float *ws,
                   size_t ws_floats, int *err, cudaStream_t st) {
    return umma_gemm_run(A, M, K, Bm, N, C, ldc, ws, ws_floats, err, st);
}

extern "C" int osrc_gemm_bf16_ws_bytes(int M, int N, int K, size_t *bytes) {
    if (!bytes) return OSRC_INVALID_ARG;
    UmmaPlan p;
    OSRC_TRY(umma_plan(M, N, K, &p));
    *bytes = p.ws_floats * sizeof(float);
    return OSRC_OK;
}

extern "C" int osrc_gemm_bf16(const void *A, int M, int K, const void *B, int N, float *C, int ldc, void *ws_dev,
                              size_t ws_bytes, int *err_flag_dev, void *stream) {
    if (!A || !B || !C || !err_flag_dev) return OSRC_INVALID_ARG;
    return umma_gemm_bf16(A, M, K, B, N, C, ldc, (float *)ws_dev, ws_bytes / sizeof(float), err_flag_dev,
                          (cudaStream_t)stream);
}
