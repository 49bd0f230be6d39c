// Throughput of the FP32 pipe on this GPU for the far kernel's instruction
// mix.  Three loops, each over independent accumulator chains (no memory
// traffic, 4 CTAs of 128 threads per SM as the far kernel runs):
//   ffma2: packed FP32x2 FMA only;
//   ffma:  scalar FMA only;
//   mix:   per iteration 2 reciprocal square roots, 4 sine/cosine pairs and
//          54 packed FMA, the far kernel's count per thread and rule point
//          (two test points against one source point).
// Prints one JSON line: TFLOP/s counted from the FMA instructions only
// (4 flops per packed FMA, 2 per scalar FMA) and, for mix, the time per
// iteration in SM cycles at the clock the caller passes.
#include <cstdio>
#include <cuda_runtime.h>

namespace {
typedef float2 f2;
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }

__global__ void k_ffma2(float *out, int iters, float m) {
    f2 a[12];
    for (int i = 0; i < 12; ++i) a[i] = make_float2(threadIdx.x * 1e-3f + i, 0.5f * i);
    const f2 mm = make_float2(m, m), cc = make_float2(1e-7f, 2e-7f);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < 12; ++i) a[i] = fma2(a[i], mm, cc);
    float s = 0.f;
    for (int i = 0; i < 12; ++i) s += a[i].x + a[i].y;
    if (s == 12345.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_ffma(float *out, int iters, float m) {
    float a[24];
    for (int i = 0; i < 24; ++i) a[i] = threadIdx.x * 1e-3f + i;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < 24; ++i) a[i] = fmaf(a[i], m, 1e-7f);
    float s = 0.f;
    for (int i = 0; i < 24; ++i) s += a[i];
    if (s == 12345.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_mix(float *out, int iters, float m) {
    f2 a[9];
    for (int i = 0; i < 9; ++i) a[i] = make_float2(threadIdx.x * 1e-3f + i, 0.5f * i);
    const f2 mm = make_float2(m, m), cc = make_float2(1e-7f, 2e-7f);
    float u = 1.f + threadIdx.x * 1e-3f, v = 2.f;
    for (int it = 0; it < iters; ++it) {
        const float ra = rsqrtf(u), rb = rsqrtf(v);
        float s0, c0, s1, c1, s2, c2, s3, c3;
        __sincosf(ra, &s0, &c0);
        __sincosf(rb, &s1, &c1);
        __sincosf(ra * 1.3f, &s2, &c2);
        __sincosf(rb * 1.3f, &s3, &c3);
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int i = 0; i < 9; ++i) a[i] = fma2(a[i], mm, cc);
        u = 1.f + fabsf(s0 * c1 + s2 * c3);
        v = 2.f + fabsf(s1 * c0 + s3 * c2);
    }
    float s = u + v;
    for (int i = 0; i < 9; ++i) s += a[i].x + a[i].y;
    if (s == 12345.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename K>
double time_ms(K kern, int blocks, int threads, int iters, float *out) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int w = 0; w < 3; ++w) kern<<<blocks, threads>>>(out, iters, 0.999f);
    cudaEventRecord(e0);
    const int reps = 40;
    for (int r = 0; r < reps; ++r) kern<<<blocks, threads>>>(out, iters, 0.999f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms / reps;
}
}  // namespace

int main(int argc, char **argv) {
    const double mhz = argc > 1 ? atof(argv[1]) : 2070.0;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const int blocks = 4 * sms, threads = 128;
    float *out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(float)) != cudaSuccess) return 1;
    const double nthr = (double)blocks * threads;
    const int it_f2 = 80000, it_f = 80000, it_mix = 16000;
    const double t_f2 = time_ms(k_ffma2, blocks, threads, it_f2, out);
    const double t_f = time_ms(k_ffma, blocks, threads, it_f, out);
    const double t_mix = time_ms(k_mix, blocks, threads, it_mix, out);
    const cudaError_t e = cudaDeviceSynchronize();
    cudaFree(out);
    if (e != cudaSuccess) {
        printf("{\"error\": \"%s\"}\n", cudaGetErrorString(e));
        return 1;
    }
    const double tf_f2 = nthr * it_f2 * 12 * 4 / (t_f2 * 1e-3) / 1e12;
    const double tf_f = nthr * it_f * 24 * 2 / (t_f * 1e-3) / 1e12;
    const double tf_mix = nthr * it_mix * 54 * 4 / (t_mix * 1e-3) / 1e12;
    // cycles per warp-iteration on one SM sub-partition (4 per SM)
    const double warps_per_smsp = (double)blocks * threads / 32.0 / (4.0 * sms);
    const double cyc_mix = t_mix * 1e-3 * mhz * 1e6 / (it_mix * warps_per_smsp);
    printf("{\"sms\": %d, \"clock_mhz_assumed\": %.0f, \"ffma2_tflops\": %.2f, \"ffma_tflops\": %.2f, "
           "\"mix_tflops_fma_only\": %.2f, \"mix_cycles_per_warp_iteration\": %.1f, "
           "\"mix_fma2_per_iteration\": 54, \"mix_mufu_per_iteration\": 10}\n",
           sms, mhz, tf_f2, tf_f, tf_mix, cyc_mix);
    return 0;
}
