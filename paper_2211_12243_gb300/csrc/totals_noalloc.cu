// Conserved totals without any allocation: the variant of the totals
// reduction whose scratch is a fixed array in the library's own device
// memory instead of a context buffer.
//
// Some callers cannot call cudaMalloc: a host application that owns every
// device allocation through its own pool allocator, or a plugin that must
// not change the device's memory footprint after it has started.  They can
// still check conservation with hydro_totals_noalloc(): it needs no context
// and allocates nothing; the caller passes the inputs and the output.
//
// The scratch array below holds one row of five partial sums per block of
// 4096 particles, 16384 rows (640 KiB), which caps n at 2^26 particles.
// Every GPU that loads the library keeps this array until the process
// exits.  All calls share it and it keeps the last call's contents: each
// call overwrites the rows it uses before reading them, so nothing has to
// start at zero, but two calls that overlap on the GPU (different streams,
// or different host threads) race on it and must be serialised by the
// caller.
#include <mutex>

#include "hydro_internal.cuh"

namespace {

constexpr int TOT_THREADS = 256;
constexpr int TOT_PER_BLOCK = 4096;
constexpr int TOT_MAX_BLOCKS = 16384;
constexpr int64_t TOT_MAX_N = (int64_t)TOT_MAX_BLOCKS * TOT_PER_BLOCK;

static __device__ __align__(256) double g_tot_scratch[TOT_MAX_BLOCKS * 5];

constexpr int TOT_MAX_DEVICES = 64;
std::mutex g_tot_mutex;
double *g_tot_ptr[TOT_MAX_DEVICES] = {nullptr};

struct KSum {
    double s, c;
};

__device__ __forceinline__ void ksum_add(KSum &k, double v) {
    double t = k.s + v;
    if (fabs(k.s) >= fabs(v)) k.c += (k.s - t) + v;
    else k.c += (v - t) + k.s;
    k.s = t;
}

// one row of partial sums per block of TOT_PER_BLOCK particles
__global__ void k_tot_partials(int64_t n, const double *__restrict__ m, const double *__restrict__ px,
                               const double *__restrict__ py, const double *__restrict__ pz,
                               const double *__restrict__ e, double *__restrict__ part) {
    const double *src[5] = {m, px, py, pz, e};
    KSum acc[5];
#pragma unroll
    for (int q = 0; q < 5; q++) acc[q] = {0.0, 0.0};
    const int64_t b0 = blockIdx.x * (int64_t)TOT_PER_BLOCK;
    const int64_t b1 = min(n, b0 + TOT_PER_BLOCK);
    for (int64_t i = b0 + threadIdx.x; i < b1; i += TOT_THREADS)
#pragma unroll
        for (int q = 0; q < 5; q++) ksum_add(acc[q], src[q][i]);
    __shared__ double sh[TOT_THREADS][5];
#pragma unroll
    for (int q = 0; q < 5; q++) sh[threadIdx.x][q] = acc[q].s + acc[q].c;
    __syncthreads();
    if (threadIdx.x < 5) {
        KSum k = {0.0, 0.0};
        for (int t = 0; t < TOT_THREADS; t++) ksum_add(k, sh[t][threadIdx.x]);
        part[blockIdx.x * 5 + threadIdx.x] = k.s + k.c;
    }
}

// five warps, one per quantity, fold the rows
__global__ void k_tot_final(int nb, const double *__restrict__ part, double *__restrict__ out) {
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (q >= 5) return;
    KSum k = {0.0, 0.0};
    for (int b = lane; b < nb; b += 32) ksum_add(k, part[b * 5 + q]);
    double s = k.s, c = k.c;
    for (int o = 16; o > 0; o >>= 1) {
        double s2 = __shfl_xor_sync(0xffffffffu, s, o);
        double c2 = __shfl_xor_sync(0xffffffffu, c, o);
        KSum m = {s, c};
        ksum_add(m, s2);
        s = m.s;
        c = m.c + c2;
    }
    if (lane == 0) out[q] = s + c;
}

}  // namespace

extern "C" int hydro_totals_noalloc(int64_t n, const double *mass, const double *px,
                                    const double *py, const double *pz, const double *etot,
                                    double *totals, hydro_stream stream) {
    if (n < 0 || !totals) return HYDRO_EINVAL;
    if (n > 0 && (!mass || !px || !py || !pz || !etot)) return HYDRO_EINVAL;
    if (n > TOT_MAX_N) return HYDRO_EINVAL;   // beyond the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HYDRO_ECUDA;
    if (dev < 0 || dev >= TOT_MAX_DEVICES) return HYDRO_EINVAL;
    double *scratch = nullptr;
    {
        // set-up, once per device, with that device current: the device
        // address of the scratch array (its host-side name is not one).
        // The first call on a device should precede any stream capture;
        // a cudaDeviceReset unloads the array and leaves this address
        // stale, so the entry point is not for use after a reset
        std::lock_guard<std::mutex> lock(g_tot_mutex);
        if (!g_tot_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_tot_scratch) != cudaSuccess || !p) return HYDRO_ECUDA;
            g_tot_ptr[dev] = static_cast<double *>(p);
        }
        scratch = g_tot_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (int)((n + TOT_PER_BLOCK - 1) / TOT_PER_BLOCK);
    if (nb > 0) {
        k_tot_partials<<<nb, TOT_THREADS, 0, st>>>(n, mass, px, py, pz, etot, scratch);
        if (hyd::launch_check() != cudaSuccess) return HYDRO_ECUDA;
    }
    k_tot_final<<<1, 160, 0, st>>>(nb, scratch, totals);
    if (hyd::launch_check() != cudaSuccess) return HYDRO_ECUDA;
    return HYDRO_OK;
}
