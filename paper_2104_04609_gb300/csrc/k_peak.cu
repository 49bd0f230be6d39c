// k_peak.cu -- measured FP32 throughput of the current GPU, the denominator
// of the far-field kernel's roofline (the far kernel is bound by the FP32
// pipe).  Not part of the paper's method: a measurement aid.
//
// Two loops over independent accumulator chains, no memory traffic, at full
// occupancy (2048 threads per SM):
//   scalar: FFMA only, 24 chains per thread;
//   packed: FP32x2 FMA (__ffma2_rn), 12 chains per thread, 4 flops each.
// Each is launched a few times after a warm-up and timed with CUDA events on
// the caller's stream; the best launch gives flops / time.
#include "osrc_internal.cuh"

namespace {

constexpr int PEAK_THREADS = 1024;

__global__ void __launch_bounds__(PEAK_THREADS) peak_ffma_kernel(float *out, int iters, float m) {
    float a[24];
#pragma unroll
    for (int i = 0; i < 24; ++i) a[i] = threadIdx.x * 1e-3f + i;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < 24; ++i) a[i] = fmaf(a[i], m, 1e-7f);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 24; ++i) s += a[i];
    if (s == 12345.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(PEAK_THREADS) peak_ffma2_kernel(float *out, int iters, float m) {
    float2 a[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) a[i] = make_float2(threadIdx.x * 1e-3f + i, 0.5f * i);
    const float2 mm = make_float2(m, m), cc = make_float2(1e-7f, 2e-7f);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < 12; ++i) a[i] = __ffma2_rn(a[i], mm, cc);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 12; ++i) s += a[i].x + a[i].y;
    if (s == 12345.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename K>
int best_ms(K kern, int blocks, int iters, int reps, float *out, cudaStream_t st, float &best) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    OSRC_CK(cudaEventCreate(&e0));
    OSRC_CK(cudaEventCreate(&e1));
    int s = OSRC_OK;
    best = 1e30f;
    for (int r = 0; r < reps + 2 && s == OSRC_OK; ++r) {
        if (cudaEventRecord(e0, st) != cudaSuccess) s = OSRC_CUDA_ERROR;
        kern<<<blocks, PEAK_THREADS, 0, st>>>(out, iters, 0.999f);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess)
            s = OSRC_CUDA_ERROR;
        float ms = 0.f;
        if (s == OSRC_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) s = OSRC_CUDA_ERROR;
        if (s == OSRC_OK && r >= 2) best = fminf(best, ms);  // the first two are warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != OSRC_OK) osrc_set_error("FP32 peak measurement failed");
    return s;
}

}  // namespace

extern "C" int osrc_fp32_peak(int reps, double *tflops_scalar, double *tflops_packed, void *stream) {
    if (!tflops_scalar || !tflops_packed || reps < 1 || reps > 100) return OSRC_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    OSRC_CK(cudaGetDevice(&dev));
    OSRC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 2 * sms;  // 2048 resident threads per SM
    // about 40 ms per launch at 70 TFLOP/s
    const int iters = 120000;
    float *out = nullptr;
    OSRC_CK(cudaMalloc(&out, (size_t)blocks * PEAK_THREADS * sizeof(float)));
    float ms1 = 0.f, ms2 = 0.f;
    int s = best_ms(peak_ffma_kernel, blocks, iters, reps, out, st, ms1);
    if (s == OSRC_OK) s = best_ms(peak_ffma2_kernel, blocks, iters, reps, out, st, ms2);
    cudaFree(out);
    if (s != OSRC_OK) return s;
    const double threads = (double)blocks * PEAK_THREADS;
    *tflops_scalar = threads * iters * 24.0 * 2.0 / (ms1 * 1e-3) / 1e12;
    *tflops_packed = threads * iters * 12.0 * 4.0 / (ms2 * 1e-3) / 1e12;
    return OSRC_OK;
}
