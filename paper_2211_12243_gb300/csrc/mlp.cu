// The learned starting pressure of the exact Riemann solver: a 12 -> 64 ->
// 64 -> 1 network on physics-based features of the face problem.
//
//   k_mlp_pack      float parameters -> packed bf16 tiles for the kernels.
//   k_mlp_predict   standalone inference on the 5th-generation tensor cores
//                   (the tile routine of mlp.cuh that the flux kernel also
//                   runs in front of its Riemann solves).
//   k_mlp_grad      training forward + backward of a minibatch (FP32 CUDA
//                   cores, optional BF16 rounding of the operands so that
//                   training sees the inference numerics).
//   k_mlp_adam      Adam update of the FP32 master parameters.
//   k_mlp_feat      features and targets of recorded face problems.
#include <algorithm>

#include "mlp.cuh"

namespace hyd {

namespace {

constexpr int GRAD_THREADS = 64;

__device__ __forceinline__ MlpTile &tile_of(unsigned char *raw) {
    return *reinterpret_cast<MlpTile *>((reinterpret_cast<uintptr_t>(raw) + 1023) &
                                        ~(uintptr_t)1023);
}

// float parameters -> the packed blob (bf16 K-major tiles + float vectors)
__global__ void k_mlp_pack(const float *__restrict__ theta, unsigned char *__restrict__ blob) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < MLP_NH * 16) {
        const int o = e >> 4, k = e & 15;
        const float v = k < MLP_NF ? theta[MLP_OFF_W1 + o * MLP_NF + k] : 0.f;
        *reinterpret_cast<__nv_bfloat16 *>(blob + MLP_W1_OFF + kmajor_off(o, k, 2)) =
            __float2bfloat16_rn(v);
        return;
    }
    const int e2 = e - MLP_NH * 16;
    if (e2 < MLP_NH * MLP_NH) {
        const int o = e2 >> 6, k = e2 & 63;
        *reinterpret_cast<__nv_bfloat16 *>(blob + MLP_W2_OFF + kmajor_off(o, k, 8)) =
            __float2bfloat16_rn(theta[MLP_OFF_W2 + e2]);
        return;
    }
    const int e3 = e2 - MLP_NH * MLP_NH;
    if (e3 < (int)(MLP_BLOB - MLP_F_OFF) / 4) {
        float v = 0.f;
        if (e3 < 64) v = theta[MLP_OFF_B1 + e3];
        else if (e3 < 128) v = theta[MLP_OFF_B2 + e3 - 64];
        else if (e3 < 192) v = theta[MLP_OFF_W3 + e3 - 128];
        else if (e3 < 204) v = theta[MLP_OFF_MEAN + e3 - 192];
        else if (e3 < 216) v = theta[MLP_OFF_SCALE + e3 - 204];
        else if (e3 == 216) v = theta[MLP_OFF_B3];
        else if (e3 == 217) v = theta[MLP_OFF_TMEAN];
        else if (e3 == 218) v = theta[MLP_OFF_TSCALE];
        else if (e3 < 231) v = theta[MLP_OFF_XMIN + e3 - 219];
        else if (e3 < 243) v = theta[MLP_OFF_XMAX + e3 - 231];
        reinterpret_cast<float *>(blob + MLP_F_OFF)[e3] = v;
    }
}

// Inference: faces (float rows rho_L, u_L, p_L, rho_R, u_R, p_R, row stride
// n) -> out[i] = p_TS exp(y), or -1 when the face is out of range (see
// mlp_guess); the caller then keeps its plain guess.
__global__ void __launch_bounds__(128) k_mlp_predict(int64_t n, const float *__restrict__ faces,
                                                     const unsigned char *__restrict__ blob,
                                                     GasK<float> K, float *__restrict__ out,
                                                     DevCounters *cnt, int stall) {
    extern __shared__ unsigned char smem_raw[];
    MlpTile &t = tile_of(smem_raw);
    const int tid = threadIdx.x;
    bool ok = mlp_tile_setup(t, blob, stall != 0);
    uint32_t phase = 0;
    const int64_t ntile = (n + 127) / 128;
    for (int64_t tile = blockIdx.x; ok && tile < ntile; tile += gridDim.x) {
        const int64_t i = tile * 128 + tid;
        float x[MLP_NF], pa = 1.f, lts = 0.f;
        bool in = false;
        if (i < n) {
            mlp_features(K, faces[i], faces[n + i], faces[2 * n + i], faces[3 * n + i],
                         faces[4 * n + i], faces[5 * n + i], x, pa);
            lts = x[9];
            in = mlp_standardise(t, x);
        } else {
#pragma unroll
            for (int k = 0; k < MLP_NF; k++) x[k] = 0.f;
        }
        mlp_put_row(t, tid, x);
        const float y = mlp_tile_eval(t, phase, &ok);
        if (ok && i < n) out[i] = mlp_guess(in, pa, lts, y);
    }
    if (!ok && tid == 0) atomicOr(&cnt->flags, ST_MLP);
    mlp_tile_teardown(t);
}

__device__ __forceinline__ float bfr(float v, bool q) {
    return q ? __bfloat162float(__float2bfloat16_rn(v)) : v;
}

// counter-based sample index (splitmix64 of seed, step, slot)
__device__ __forceinline__ int64_t sample_index(uint64_t seed, uint64_t step, uint64_t slot, int64_t n) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (step * 0x100000001B3ull + slot + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (int64_t)(z % (uint64_t)n);
}

// one block = GRAD_THREADS samples; gradient of 0.5 mean (y - t)^2 over
// the `nb` samples of the minibatch, summed into grad (float atomics)
__global__ void __launch_bounds__(GRAD_THREADS) k_mlp_grad(const float *__restrict__ theta,
                                                           const float *__restrict__ x,
                                                           const float *__restrict__ t, int64_t n,
                                                           int64_t nb, int random, uint64_t seed,
                                                           uint64_t step, int quant,
                                                           float *__restrict__ grad,
                                                           float *__restrict__ loss) {
    extern __shared__ float sg[];
    float *W1 = sg;                                   // 768
    float *W2 = W1 + MLP_NH * MLP_NF;                 // 4096
    float *pb = W2 + MLP_NH * MLP_NH;                 // b1 b2 w3 (192) b3 mean scale tmean tscale
    float *xs = pb + 3 * MLP_NH + 3 + 2 * MLP_NF;     // [64][13]
    float *h1 = xs + GRAD_THREADS * 13;               // [64][65]
    float *da = h1 + GRAD_THREADS * 65;               // [64][65]
    float *gw3 = da + GRAD_THREADS * 65;              // 64 + 1
    const int tid = threadIdx.x;
    const bool q = quant != 0;
    for (int e = tid; e < MLP_NH * MLP_NF; e += GRAD_THREADS) W1[e] = bfr(theta[MLP_OFF_W1 + e], q);
    for (int e = tid; e < MLP_NH * MLP_NH; e += GRAD_THREADS) W2[e] = bfr(theta[MLP_OFF_W2 + e], q);
    for (int e = tid; e < MLP_NH; e += GRAD_THREADS) {
        pb[e] = theta[MLP_OFF_B1 + e];
        pb[MLP_NH + e] = theta[MLP_OFF_B2 + e];
        pb[2 * MLP_NH + e] = theta[MLP_OFF_W3 + e];
        gw3[e] = 0.f;
    }
    if (tid == 0) {
        pb[3 * MLP_NH] = theta[MLP_OFF_B3];
        pb[3 * MLP_NH + 1 + 2 * MLP_NF] = theta[MLP_OFF_TMEAN];
        pb[3 * MLP_NH + 2 + 2 * MLP_NF] = theta[MLP_OFF_TSCALE];
        gw3[MLP_NH] = 0.f;
    }
    if (tid < MLP_NF) {
        pb[3 * MLP_NH + 1 + tid] = theta[MLP_OFF_MEAN + tid];
        pb[3 * MLP_NH + 1 + MLP_NF + tid] = theta[MLP_OFF_SCALE + tid];
    }
    __syncthreads();
    const float *b1 = pb, *b2 = pb + MLP_NH, *w3 = pb + 2 * MLP_NH;
    const float b3 = pb[3 * MLP_NH];
    const float *mean = pb + 3 * MLP_NH + 1, *scale = mean + MLP_NF;
    const float tmean = pb[3 * MLP_NH + 1 + 2 * MLP_NF], tscale = pb[3 * MLP_NH + 2 + 2 * MLP_NF];
    const int64_t slot = blockIdx.x * (int64_t)GRAD_THREADS + tid;
    bool active = slot < nb;
    const int64_t idx = active ? (random ? sample_index(seed, step, slot, n) : slot) : 0;
    // samples with a non-finite feature or target (an unphysical face) are skipped
    bool finite = active && isfinite(t[idx]);
    for (int k = 0; k < MLP_NF; k++) finite = finite && isfinite(x[idx * MLP_NF + k]);
    active = finite;
    float target = active ? t[idx] : 0.f;
    for (int k = 0; k < MLP_NF; k++)
        xs[tid * 13 + k] = active ? bfr((x[idx * MLP_NF + k] - mean[k]) / scale[k], q) : 0.f;
    for (int o = 0; o < MLP_NH; o++) {
        float a = b1[o];
        for (int k = 0; k < MLP_NF; k++) a += W1[o * MLP_NF + k] * xs[tid * 13 + k];
        h1[tid * 65 + o] = bfr(fmaxf(a, 0.f), q);
    }
    float z = b3;
    for (int o = 0; o < MLP_NH; o++) {
        float a = b2[o];
        for (int k = 0; k < MLP_NH; k++) a += W2[o * MLP_NH + k] * h1[tid * 65 + k];
        z += fmaxf(a, 0.f) * w3[o];
    }
    const float y = tmean + tscale * z;
    const float inv = 1.f / (float)nb;
    const float dy = active ? (y - target) * inv * tscale : 0.f;   // d loss / d z
    if (active) atomicAdd(loss, 0.5f * (y - target) * (y - target) * inv);
    for (int o = 0; o < MLP_NH; o++) {
        float a = b2[o];
        for (int k = 0; k < MLP_NH; k++) a += W2[o * MLP_NH + k] * h1[tid * 65 + k];
        float h2 = fmaxf(a, 0.f);
        da[tid * 65 + o] = a > 0.f ? dy * w3[o] : 0.f;
        atomicAdd(&gw3[o], h2 * dy);
    }
    atomicAdd(&gw3[MLP_NH], dy);
    __syncthreads();
    // dW2[o][k] = sum_s da2[s][o] h1[s][k]; db2[o] = sum_s da2[s][o]
    for (int e = tid; e < MLP_NH * MLP_NH; e += GRAD_THREADS) {
        int o = e >> 6, k = e & 63;
        float acc = 0.f;
        for (int s = 0; s < GRAD_THREADS; s++) acc += da[s * 65 + o] * h1[s * 65 + k];
        atomicAdd(&grad[MLP_OFF_W2 + e], acc);
    }
    {
        int o = tid;
        float acc = 0.f;
        for (int s = 0; s < GRAD_THREADS; s++) acc += da[s * 65 + o];
        atomicAdd(&grad[MLP_OFF_B2 + o], acc);
        atomicAdd(&grad[MLP_OFF_W3 + o], gw3[o]);
    }
    if (tid == 0) atomicAdd(&grad[MLP_OFF_B3], gw3[MLP_NH]);
    // da1 = (da2 W2) * relu'(a1), in place of da after everyone read it
    float d1[MLP_NH];
    for (int k = 0; k < MLP_NH; k++) {
        float acc = 0.f;
        for (int o = 0; o < MLP_NH; o++) acc += da[tid * 65 + o] * W2[o * MLP_NH + k];
        d1[k] = h1[tid * 65 + k] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    for (int k = 0; k < MLP_NH; k++) da[tid * 65 + k] = d1[k];
    __syncthreads();
    for (int e = tid; e < MLP_NH * MLP_NF; e += GRAD_THREADS) {
        int o = e / MLP_NF, k = e % MLP_NF;
        float acc = 0.f;
        for (int s = 0; s < GRAD_THREADS; s++) acc += da[s * 65 + o] * xs[s * 13 + k];
        atomicAdd(&grad[MLP_OFF_W1 + e], acc);
    }
    {
        int o = tid;
        float acc = 0.f;
        for (int s = 0; s < GRAD_THREADS; s++) acc += da[s * 65 + o];
        atomicAdd(&grad[MLP_OFF_B1 + o], acc);
    }
}

__global__ void k_mlp_adam(float *__restrict__ theta, float *__restrict__ grad, float *__restrict__ m,
                           float *__restrict__ v, float lr, float b1, float b2, float eps, int step) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= MLP_NTRAIN) return;
    float g = grad[e];
    float mm = b1 * m[e] + (1.f - b1) * g;
    float vv = b2 * v[e] + (1.f - b2) * g * g;
    m[e] = mm;
    v[e] = vv;
    float mh = mm / (1.f - powf(b1, (float)step));
    float vh = vv / (1.f - powf(b2, (float)step));
    theta[e] -= lr * mh / (sqrtf(vh) + eps);
    grad[e] = 0.f;
}

// features x[n][12] and targets ln(p*/p_a) of recorded faces [7][n]
__global__ void k_mlp_feat(int64_t n, const float *__restrict__ faces, GasK<float> K,
                           float *__restrict__ x, float *__restrict__ t) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float f[MLP_NF], pa;
    mlp_features(K, faces[i], faces[n + i], faces[2 * n + i], faces[3 * n + i], faces[4 * n + i],
                 faces[5 * n + i], f, pa);
    for (int k = 0; k < MLP_NF; k++) x[i * MLP_NF + k] = f[k];
    t[i] = logf(faces[6 * n + i] / pa) - f[9];   // ln(p* / p_TS)
}

// float <-> integer keys with the order of the floats (for atomicMin/Max)
__device__ __forceinline__ int ord_key(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord_val(int k) {
    return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff);
}

// per-feature and target mean and standard deviation (double accumulators:
// acc[0..11] sums, [12..23] sums of squares, [24], [25] the target's, [26]
// the count) and the feature box (box[0..11] min keys, [12..23] max keys),
// over the samples whose features and target are all finite
__global__ void k_mlp_stats(int64_t n, const float *__restrict__ x, const float *__restrict__ t,
                            double *__restrict__ acc, int *__restrict__ box) {
    double s[MLP_NF + 1], s2[MLP_NF + 1];
    float lo[MLP_NF], hi[MLP_NF];
    for (int k = 0; k <= MLP_NF; k++) s[k] = s2[k] = 0.0;
    for (int k = 0; k < MLP_NF; k++) { lo[k] = 3.0e38f; hi[k] = -3.0e38f; }
    double cnt = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        bool ok = isfinite(t[i]);
        for (int k = 0; k < MLP_NF; k++) ok = ok && isfinite(x[i * MLP_NF + k]);
        if (!ok) continue;
        cnt += 1.0;
        for (int k = 0; k <= MLP_NF; k++) {
            const float f = k < MLP_NF ? x[i * MLP_NF + k] : t[i];
            const double v = f;
            s[k] += v;
            s2[k] += v * v;
            if (k < MLP_NF) { lo[k] = fminf(lo[k], f); hi[k] = fmaxf(hi[k], f); }
        }
    }
    atomicAdd(&acc[2 * MLP_NF + 2], cnt);
    for (int k = 0; k < MLP_NF; k++) {
        atomicAdd(&acc[k], s[k]);
        atomicAdd(&acc[MLP_NF + k], s2[k]);
        atomicMin(&box[k], ord_key(lo[k]));
        atomicMax(&box[MLP_NF + k], ord_key(hi[k]));
    }
    atomicAdd(&acc[2 * MLP_NF], s[MLP_NF]);
    atomicAdd(&acc[2 * MLP_NF + 1], s2[MLP_NF]);
}

__global__ void k_mlp_box_init(int *box) {
    const int k = threadIdx.x;
    if (k < MLP_NF) {
        box[k] = ord_key(3.0e38f);
        box[MLP_NF + k] = ord_key(-3.0e38f);
    }
}

__global__ void k_mlp_set_norm(int64_t n, const double *__restrict__ acc, const int *__restrict__ box,
                               float *__restrict__ theta) {
    int k = threadIdx.x;
    if (k > MLP_NF) return;
    const double cnt = acc[2 * MLP_NF + 2] > 0.0 ? acc[2 * MLP_NF + 2] : 1.0;
    const double sum = k < MLP_NF ? acc[k] : acc[2 * MLP_NF];
    const double sq = k < MLP_NF ? acc[MLP_NF + k] : acc[2 * MLP_NF + 1];
    const double mu = sum / cnt;
    const double var = sq / cnt - mu * mu;
    const double sd = sqrt(var > 0.0 ? var : 0.0);
    if (k < MLP_NF) {
        theta[MLP_OFF_MEAN + k] = (float)mu;
        theta[MLP_OFF_SCALE + k] = (float)(sd + 1e-3);
        theta[MLP_OFF_XMIN + k] = ord_val(box[k]);
        theta[MLP_OFF_XMAX + k] = ord_val(box[MLP_NF + k]);
    } else {
        theta[MLP_OFF_TMEAN] = (float)mu;
        theta[MLP_OFF_TSCALE] = (float)(sd + 1e-6);
    }
}

size_t grad_smem() {
    return sizeof(float) * (MLP_NH * MLP_NF + MLP_NH * MLP_NH + 3 * MLP_NH + 3 + 2 * MLP_NF +
                            GRAD_THREADS * 13 + 2 * GRAD_THREADS * 65 + MLP_NH + 1);
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t mlp_pack(hydro_ctx *c, stream_t st) {
    HYD_CUDA(c->d_mlp_blob.ensure(MLP_BLOB));
    const int tot = MLP_NH * 16 + MLP_NH * MLP_NH + (int)(MLP_BLOB - MLP_F_OFF) / 4;
    k_mlp_pack<<<grid_for(tot, 256), 256, 0, st>>>(c->d_mlp.get(), c->d_mlp_blob.get());
    return launch_check();
}

cudaError_t mlp_predict(hydro_ctx *c, const float *faces, int64_t n, float *out, stream_t st) {
    const size_t smem = sizeof(MlpTile) + 1024;
    static bool configured = false;
    if (!configured) {
        HYD_CUDA(cudaFuncSetAttribute(k_mlp_predict, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        configured = true;
    }
    const int64_t ntile = (n + 127) / 128;
    const unsigned grid = (unsigned)std::min<int64_t>(ntile > 0 ? ntile : 1, 152 * 4);
    k_mlp_predict<<<grid, 128, smem, st>>>(n, faces, c->d_mlp_blob.get(),
                                           GasK<float>(c->cfg.gamma), out, c->d_cnt,
                                           c->mlp_stall);
    return launch_check();
}

cudaError_t mlp_features(hydro_ctx *c, const float *faces, int64_t n, float *x, float *t,
                         stream_t st) {
    k_mlp_feat<<<grid_for(n, 256), 256, 0, st>>>(n, faces, GasK<float>(c->cfg.gamma), x, t);
    return launch_check();
}

cudaError_t mlp_gradient(hydro_ctx *c, const float *x, const float *t, int64_t n, int64_t nb,
                         int random, uint64_t seed, uint64_t step, int quant, float *grad,
                         float *loss, stream_t st) {
    size_t smem = grad_smem();
    static bool configured = false;
    if (!configured) {
        HYD_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        configured = true;
    }
    k_mlp_grad<<<grid_for(nb, GRAD_THREADS), GRAD_THREADS, smem, st>>>(
        c->d_mlp.get(), x, t, n, nb, random, seed, step, quant, grad, loss);
    return launch_check();
}

cudaError_t mlp_adam(hydro_ctx *c, float *grad, float *m, float *v, float lr, int step,
                     stream_t st) {
    k_mlp_adam<<<grid_for(MLP_NTRAIN, 256), 256, 0, st>>>(c->d_mlp.get(), grad, m, v, lr, 0.9f,
                                                          0.999f, 1e-8f, step);
    return launch_check();
}

cudaError_t mlp_normalise(hydro_ctx *c, const float *x, const float *t, int64_t n, double *acc,
                          int *box, stream_t st) {
    HYD_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * (2 * MLP_NF + 3), st));
    k_mlp_box_init<<<1, 32, 0, st>>>(box);
    HYD_CUDA(launch_check());
    k_mlp_stats<<<256, 256, 0, st>>>(n, x, t, acc, box);
    HYD_CUDA(launch_check());
    k_mlp_set_norm<<<1, 32, 0, st>>>(n, acc, box, c->d_mlp.get());
    return launch_check();
}

}  // namespace hyd
static_assert(hyd::MLP_BLOB == hyd::MLP_BLOB_BYTES, "blob size");
