// Throughput probes of this GPU's arithmetic units, for the roofline that
// the benchmark reports against (no counterpart in the paper).  Each probe
// runs independent dependency chains on every lane of every SM long enough
// to hide latency, timed with CUDA events on the caller's stream:
//   HYDRO_PROBE_FP32: float fused multiply-adds, reported in TFLOP/s (2 per FMA)
//   HYDRO_PROBE_FP64: double fused multiply-adds, TFLOP/s (2 per FMA)
//   HYDRO_PROBE_MUFU: float reciprocal square roots on the special-function
//                     unit (rsqrt.approx), in Tops/s
#include <algorithm>

#include "hydro_internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fma(int iters, T seed, T *sink) {
    T a[PROBE_CHAINS];
    const T b = seed * T(0.999), c = seed * T(1e-3);
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; k++) a[k] = seed + T(threadIdx.x + k);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; k++) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; k++) s += a[k];
    // never true for the seeds used; keeps the chains live
    if (s == T(-12345.0)) sink[blockIdx.x] = s;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm volatile("rsqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_mufu(int iters, float seed, float *sink) {
    float a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; k++) a[k] = seed + (float)(threadIdx.x + k);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; k++) a[k] = rsqrt_approx(a[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; k++) s += a[k];
    if (s == -12345.f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" int hydro_probe_peak(int unit, double *value, hydro_stream stream) {
    if (!value || unit < HYDRO_PROBE_FP32 || unit > HYDRO_PROBE_MUFU) return HYDRO_EINVAL;
    *value = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HYDRO_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HYDRO_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    // enough blocks for every SM's warp slots; FP64 runs far fewer
    // operations per second, so fewer iterations keep its launch short
    const int blocks = sms * 8;
    const int iters = unit == HYDRO_PROBE_FP64 ? 256 : 4096;
    void *sink = nullptr;
    if (cudaMalloc(&sink, (size_t)blocks * sizeof(double)) != cudaSuccess) return HYDRO_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HYDRO_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = HYDRO_ECUDA;
    float best_ms = 0.f;
    for (int rep = 0; rep < 4 && rc == HYDRO_OK; rep++) {   // the first launch warms up
        cudaEventRecord(e0, st);
        if (unit == HYDRO_PROBE_FP32)
            k_probe_fma<float><<<blocks, PROBE_THREADS, 0, st>>>(iters, 1.0f, (float *)sink);
        else if (unit == HYDRO_PROBE_FP64)
            k_probe_fma<double><<<blocks, PROBE_THREADS, 0, st>>>(iters, 1.0, (double *)sink);
        else
            k_probe_mufu<<<blocks, PROBE_THREADS, 0, st>>>(iters, 2.0f, (float *)sink);
        if (hyd::launch_check() != cudaSuccess) { rc = HYDRO_ECUDA; break; }
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = HYDRO_ECUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc != HYDRO_OK) return rc;
    const double ops = (double)blocks * PROBE_THREADS * PROBE_CHAINS * iters;
    const double per = unit == HYDRO_PROBE_MUFU ? 1.0 : 2.0;   // an FMA is two flops
    *value = ops * per / (best_ms * 1e-3) / 1e12;
    return HYDRO_OK;
}
