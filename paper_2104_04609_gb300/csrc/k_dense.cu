// k_dense.cu -- dense mixed-precision building blocks of the assembled path:
// a BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05 MMA
// with the accumulator in tensor memory, operands staged by TMA), used by
// the batched dense solve for the far-field product and the explicit
// preconditioner matrix.
//
// GEMM: C[M x N] = A[M x K] * B[N x K]^T, A and B BF16 and K-major (row-major
// with K contiguous), C FP32.  One CTA of 128 threads computes a 128 x N tile
// (N <= 256, a multiple of 16) over the whole K range:
//   - lane 0 of warp 0 issues TMA loads (128-byte swizzle) of 64-wide K
//     slices of A and B into a 4-stage shared-memory ring;
//   - lane 0 of warp 1 issues tcgen05.mma (kind::f16, M 128, N, K 16; four
//     per slice) into a 128-lane x N-column FP32 accumulator in tensor
//     memory and releases each stage with tcgen05.commit;
//   - all four warps then read the accumulator (tcgen05.ld, warp w owns
//     lanes 32w..32w+31) and store C.
// Every mbarrier wait is bounded (2 s of global time): on timeout the kernel
// records an error flag, stops waiting, frees its tensor memory and returns.
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

namespace {

constexpr int UM_BM = 128;
constexpr int UM_BK = 64;  // 64 BF16 = one 128-byte swizzle row
constexpr int UM_STAGES = 4;
constexpr int UM_THREADS = 128;
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

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
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

__global__ void __launch_bounds__(UM_THREADS, 1)
umma_gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                 int M, int N, int K, float *__restrict__ C, int ldc, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned ring of A (128 x 64) and B (N x 64) slices
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t a_bytes = UM_BM * UM_BK * 2, b_bytes = (uint32_t)N * UM_BK * 2;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    uint64_t *bars = (uint64_t *)(base + UM_STAGES * stage_bytes);
    uint64_t *full = bars, *empty = bars + UM_STAGES, *done = bars + 2 * UM_STAGES;
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * UM_STAGES + 1);
    __shared__ int timed_out;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * UM_BM;
    const int nk = K / UM_BK;
    if (threadIdx.x == 0) {
        timed_out = 0;
        for (int s = 0; s < UM_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t ncols = 32;
    while (ncols < (uint32_t)N) ncols <<= 1;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % UM_STAGES, use = kb / UM_STAGES;
            if (kb >= UM_STAGES && !mbar_wait(&empty[s], (use - 1) & 1)) {
                timed_out = 1;
                break;
            }
            unsigned char *sa = base + s * stage_bytes, *sb = sa + a_bytes;
            mbar_expect_tx(&full[s], stage_bytes);
            tma_load_2d(sa, &map_a, kb * UM_BK, m0, &full[s]);
            tma_load_2d(sb, &map_b, kb * UM_BK, 0, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = instr_desc(UM_BM, N);
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % UM_STAGES, use = kb / UM_STAGES;
            if (!mbar_wait(&full[s], use & 1)) {
                timed_out = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = smem_u32(base + s * stage_bytes), sb = sa + a_bytes;
            const uint64_t da = smem_desc(sa), db = smem_desc(sb);
#pragma unroll
            for (int k = 0; k < UM_BK / 16; ++k) {
                const uint32_t acc = (kb | k) ? 1u : 0u;
                // advance 16 BF16 = 32 bytes along K inside the swizzled rows
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(da + (uint64_t)(2 * k)), "l"(db + (uint64_t)(2 * k)), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(done))
                     : "memory");
    }
    __syncwarp();
    // epilogue: every warp waits for the accumulator, then reads its 32 lanes
    const bool ok = mbar_wait(done, 0);
    if (!ok) timed_out = 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int row = m0 + warp * 32 + lane;
    if (ok) {
        for (int c0 = 0; c0 < N; c0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
                "%30, %31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                  "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                  "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                  "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M)
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (c0 + j < N) C[(size_t)row * ldc + c0 + j] = __uint_as_float(v[j]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
    if (threadIdx.x == 0 && timed_out) atomicExch(err, 1);
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

}  // namespace

size_t umma_smem_bytes(int N) {
    return (size_t)UM_STAGES * (UM_BM * UM_BK * 2 + (size_t)N * UM_BK * 2) + 1024 + 256;
}

// C = A B^T for BF16 A (M x K), B (N x K), FP32 C (M x ldc); requirements:
// M % 128 == 0, K % 64 == 0, 16 <= N <= 256 and N % 16 == 0, 16-byte aligned
// rows.  err: device int set to 1 if a bounded wait gave up.
int umma_gemm_bf16(const void *A, int M, int K, const void *Bm, int N, float *C, int ldc, int *err,
                   cudaStream_t st) {
    if (M <= 0 || M % UM_BM || K <= 0 || K % UM_BK || N < 16 || N > 256 || N % 16 || ldc < N) {
        osrc_set_error("umma_gemm_bf16: unsupported shape");
        return OSRC_INVALID_ARG;
    }
    if (((uintptr_t)A & 15) || ((uintptr_t)Bm & 15)) return OSRC_INVALID_ARG;
    OSRC_TRY(get_encoder());
    CUtensorMap ma, mb;
    OSRC_TRY(make_map(&ma, A, M, K, UM_BM));
    OSRC_TRY(make_map(&mb, Bm, N, K, N));
    const size_t smem = umma_smem_bytes(N);
    static PerDeviceOnce once;
    OSRC_TRY(per_device_once(once, [](int) -> int {
        OSRC_CK(cudaFuncSetAttribute(umma_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)umma_smem_bytes(256)));
        return OSRC_OK;
    }));
    umma_gemm_kernel<<<M / UM_BM, UM_THREADS, smem, st>>>(ma, mb, M, N, K, C, ldc, err);
    OSRC_CK(cudaGetLastError());
    return OSRC_OK;
}

extern "C" int osrc_gemm_bf16(const void *A, int M, int K, const void *B, int N, float *C, int ldc,
                              int *err_flag_dev, void *stream) {
    if (!A || !B || !C || !err_flag_dev) return OSRC_INVALID_ARG;
    return umma_gemm_bf16(A, M, K, B, N, C, ldc, err_flag_dev, (cudaStream_t)stream);
}
