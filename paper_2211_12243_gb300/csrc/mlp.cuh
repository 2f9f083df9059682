// Star-pressure network shared pieces: face features and the tcgen05
// (5th-generation tensor core) helpers for the 12 -> 64 -> 64 -> 1 network
// that proposes the starting pressure of the exact Riemann solver.
#pragma once

#include <cuda_bf16.h>

#include "hydro_internal.cuh"
#include "riemann.cuh"

namespace hyd {

constexpr int MLP_NF = 12;
constexpr int MLP_NH = 64;
// packed float parameters: W1[64][12], b1[64], W2[64][64], b2[64], w3[64], b3,
// mean[12], scale[12] (feature standardisation), t_mean, t_scale (output:
// y = t_mean + t_scale (w3 . h2 + b3)), xmin[12], xmax[12] (the box of the
// training features: outside it the prediction is out of range)
constexpr int MLP_OFF_W1 = 0;
constexpr int MLP_OFF_B1 = MLP_OFF_W1 + MLP_NH * MLP_NF;
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_NH;
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_NH * MLP_NH;
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + MLP_NH;
constexpr int MLP_OFF_B3 = MLP_OFF_W3 + MLP_NH;
constexpr int MLP_OFF_MEAN = MLP_OFF_B3 + 1;
constexpr int MLP_OFF_SCALE = MLP_OFF_MEAN + MLP_NF;
constexpr int MLP_OFF_TMEAN = MLP_OFF_SCALE + MLP_NF;
constexpr int MLP_OFF_TSCALE = MLP_OFF_TMEAN + 1;
constexpr int MLP_OFF_XMIN = MLP_OFF_TSCALE + 1;
constexpr int MLP_OFF_XMAX = MLP_OFF_XMIN + MLP_NF;
constexpr int MLP_NPARAM = MLP_OFF_XMAX + MLP_NF;      // 5115
constexpr int MLP_NTRAIN = MLP_OFF_MEAN;               // trainable: W1..b3

// Features of one face problem (float): see the FP64 reference for the
// definitions.  pa receives (p_L + p_R)/2, the pressure scale of the target.
__device__ __forceinline__ void mlp_features(const GasK<float> &k, float rl, float ul, float pl,
                                             float rr, float ur, float pr, float x[MLP_NF],
                                             float &pa) {
    pa = 0.5f * (pl + pr);
    const float ra = 0.5f * (rl + rr);
    const float ca = sqrt_(k.g * __fdividef(pa, ra));
    const float cl = sqrt_(k.g * __fdividef(pl, rl));
    const float cr = sqrt_(k.g * __fdividef(pr, rr));
    const float du = ur - ul;
    const float ppv = 0.5f * (pl + pr) - 0.125f * du * (rl + rr) * (cl + cr);
    float num = cl + cr - 0.5f * k.gm1 * du;
    num = fmaxf(num, 1e-12f * (cl + cr));
    const float ptr = __powf(__fdividef(num, __fdividef(cl, __powf(pl, k.z)) + __fdividef(cr, __powf(pr, k.z))), k.zi);
    const float p0 = fmaxf(ppv, 0.f);
    const float gl = sqrt_(__fdividef(__fdividef(k.g5, rl), k.g6 * pl + p0));
    const float gr = sqrt_(__fdividef(__fdividef(k.g5, rr), k.g6 * pr + p0));
    const float pts = __fdividef(gl * pl + gr * pr - du, gl + gr);
    const float floor_ = 1e-6f * pa;
    const float ipa = __fdividef(1.f, pa);
    const float ira = __fdividef(1.f, ra);
    x[0] = __logf(pl * ipa);
    x[1] = __logf(pr * ipa);
    x[2] = __logf(rl * ira);
    x[3] = __logf(rr * ira);
    x[4] = fminf(fmaxf(__fdividef(du, ca), -8.f), 8.f);
    x[5] = __fdividef(cl, ca);
    x[6] = __fdividef(cr, ca);
    x[7] = __logf(fmaxf(ppv, floor_) * ipa);
    x[8] = __logf(fmaxf(ptr, floor_) * ipa);
    x[9] = __logf(fmaxf(pts, floor_) * ipa);
    x[10] = fabsf(__logf(__fdividef(pl, pr)));
    x[11] = __fdividef(pl - pr, pl + pr);
}

// ---------------------------------------------------------------------------
// tcgen05 helpers (sm_100a family).  Operands in shared memory use the
// no-swizzle K-major layout: 8-row x 16-byte core matrices, LBO = byte
// distance between core matrices adjacent along K, SBO = along M (or N).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of the sm_100 family
    // base offset 0, no swizzle
    return d;
}

// instruction descriptor, kind::f16: BF16 x BF16 -> F32, both K-major
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4)                        // D format F32
           | (1u << 7)                      // A format BF16
           | (1u << 10)                     // B format BF16
           | ((uint32_t)(N >> 3) << 17)     // N / 8
           | ((uint32_t)(M >> 4) << 24);    // M / 16
}

__device__ __forceinline__ void tmem_alloc(uint32_t smem_dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_dst),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                          uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        mbar));
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}

// wait for the phase with the given parity; gives up after max_spins
// polls and returns false (the caller records an error)
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int max_spins) {
    for (int i = 0; i < max_spins; i++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity));
        if (done) return true;
        if (i > 64) __nanosleep(64);
    }
    return false;
}

// non-blocking variant for the error-path test hook: test_wait never
// suspends, so max_polls bounds the time (about 0.1 us per poll)
__device__ __forceinline__ bool mbar_poll(uint32_t mbar, uint32_t parity, int max_polls) {
    for (int i = 0; i < max_polls; i++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity));
        if (done) return true;
        __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 16 consecutive 32-bit columns of the warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// byte offset of element (row, k) in a no-swizzle K-major tile whose core
// matrices are laid out (row/8) * kcm + (k/8), 128 bytes each
__device__ __forceinline__ uint32_t kmajor_off(int row, int k, int kcm) {
    return (uint32_t)((((row >> 3) * kcm + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
                 : "memory");
}

// bulk (non-tensor) TMA copy global -> shared, completion on mbar; both
// addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(mbar)
        : "memory");
}

// eight floats -> eight bf16 (round to nearest even) in one 16-byte store
__device__ __forceinline__ void store_bf16x8(unsigned char *dst, const float v[8]) {
    uint4 u;
    __nv_bfloat162 t0 = __floats2bfloat162_rn(v[0], v[1]);
    __nv_bfloat162 t1 = __floats2bfloat162_rn(v[2], v[3]);
    __nv_bfloat162 t2 = __floats2bfloat162_rn(v[4], v[5]);
    __nv_bfloat162 t3 = __floats2bfloat162_rn(v[6], v[7]);
    u.x = *reinterpret_cast<uint32_t *>(&t0);
    u.y = *reinterpret_cast<uint32_t *>(&t1);
    u.z = *reinterpret_cast<uint32_t *>(&t2);
    u.w = *reinterpret_cast<uint32_t *>(&t3);
    *reinterpret_cast<uint4 *>(dst) = u;
}

// ---------------------------------------------------------------------------
// One 128-row evaluation tile of the network on the tensor cores.
//
// Packed weights (device blob, MLP_BLOB_BYTES, written by mlp_pack): the
// bf16 W1 tile [64 x 16] (K padded 12 -> 16) and W2 tile [64 x 64] in the
// K-major core-matrix layout, then the floats b1[64], b2[64], w3[64],
// mean[12], scale[12], b3, t_mean, t_scale, xmin[12], xmax[12].  One bulk
// copy brings it into shared memory.
//
// A tile evaluates rows r = threadIdx.x (128 threads): the caller writes
// row r's standardised features with mlp_put_row, then every thread calls
// mlp_tile_eval, which runs layer 1 (M=128, N=64, K=16) and layer 2 (K=64
// in four K=16 steps) as tcgen05.mma with the FP32 accumulator in 64 TMEM
// columns, and returns the row's output y.  Warp w reads TMEM lanes
// 32w .. 32w+31, which are exactly its own rows.
// ---------------------------------------------------------------------------
constexpr uint32_t MLP_W1_OFF = 0, MLP_W2_OFF = 2048, MLP_F_OFF = 10240;
constexpr uint32_t MLP_BLOB = 11264;
constexpr int MLP_FB1 = 0, MLP_FB2 = 64, MLP_FW3 = 128, MLP_FMEAN = 192, MLP_FSCALE = 204,
              MLP_FB3 = 216, MLP_FTMEAN = 217, MLP_FTSCALE = 218, MLP_FXMIN = 219,
              MLP_FXMAX = 231;
constexpr uint32_t MLP_TMEM_COLS = 64;
constexpr int MLP_WAIT_SPINS = 1 << 22;   // ~0.3 s of polling before giving up
// the error-path test hook (hydro_test_mlp_stall): the weight copy is not
// issued, so the set-up's wait can never finish and gives up after this
// many polls (~0.3 ms); nothing is in flight when it does
constexpr int MLP_STALL_POLLS = 4096;

struct MlpTile {
    alignas(1024) unsigned char wb[MLP_BLOB];
    alignas(1024) unsigned char a1[128 * 16 * 2];
    alignas(1024) unsigned char a2[128 * 64 * 2];
    alignas(8) unsigned long long mbar_w, mbar_mma;
    uint32_t taddr;
};

__device__ __forceinline__ const float *mlp_f(const MlpTile &t) {
    return reinterpret_cast<const float *>(t.wb + MLP_F_OFF);
}

// all threads; returns false (and the tile is unusable) when the weight copy
// did not arrive within the wait limit.  stall: the test hook -- no copy is
// issued and the wait on its barrier runs out
__device__ __forceinline__ bool mlp_tile_setup(MlpTile &t, const unsigned char *blob,
                                               bool stall = false) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(smem_u32(&t.mbar_w), 1);
        mbar_init(smem_u32(&t.mbar_mma), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((tid >> 5) == 0) tmem_alloc(smem_u32(&t.taddr), MLP_TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (stall) {
        const bool none = mbar_poll(smem_u32(&t.mbar_w), 0, MLP_STALL_POLLS);
        return !__syncthreads_or(!none);
    }
    if (tid == 0) {
        mbar_expect_tx(smem_u32(&t.mbar_w), MLP_BLOB);
        bulk_g2s(smem_u32(t.wb), blob, MLP_BLOB, smem_u32(&t.mbar_w));
    }
    bool ok = mbar_wait(smem_u32(&t.mbar_w), 0, MLP_WAIT_SPINS);
    if (!ok) ok = mbar_wait(smem_u32(&t.mbar_w), 0, MLP_WAIT_SPINS);   // copy still in flight?
    return !__syncthreads_or(!ok);
}

// row r of A1 from standardised features (all 12; the K padding is zero)
__device__ __forceinline__ void mlp_put_row(MlpTile &t, int r, const float xs[MLP_NF]) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = xs[k];
    store_bf16x8(t.a1 + kmajor_off(r, 0, 2), v);
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = k < MLP_NF - 8 ? xs[8 + k] : 0.f;
    store_bf16x8(t.a1 + kmajor_off(r, 8, 2), v);
}

// every thread of the CTA; returns this thread's row output.  `phase` is
// each thread's copy of the MMA barrier parity (0 before the first call).
// On a wait that gives up, *ok becomes false (for every thread), y is 0 and
// the tile must not be evaluated again.
__device__ __forceinline__ float mlp_tile_eval(MlpTile &t, uint32_t &phase, bool *ok) {
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t tbase = t.taddr;
    const uint32_t tlane = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
    const uint32_t idesc = umma_idesc_bf16(128, 64);
    const uint32_t mbar = smem_u32(&t.mbar_mma);
    const float *F = mlp_f(t);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        tc_fence_after();
        umma_bf16(tbase, umma_desc(smem_u32(t.a1), 128, 256),
                  umma_desc(smem_u32(t.wb + MLP_W1_OFF), 128, 256), idesc, 0u);
        umma_commit(mbar);
    }
    bool w = mbar_wait(mbar, phase, MLP_WAIT_SPINS);
    if (!w) w = mbar_wait(mbar, phase, MLP_WAIT_SPINS);
    phase ^= 1u;
    if (__syncthreads_or(!w)) {
        *ok = false;
        return 0.f;
    }
    tc_fence_after();
#pragma unroll
    for (int c0 = 0; c0 < MLP_NH; c0 += 16) {
        float v[16];
        tmem_ld16(tlane + (uint32_t)c0, v);
#pragma unroll
        for (int c = 0; c < 16; c++) v[c] = fmaxf(v[c] + F[MLP_FB1 + c0 + c], 0.f);
        store_bf16x8(t.a2 + kmajor_off(tid, c0, 8), v);
        store_bf16x8(t.a2 + kmajor_off(tid, c0 + 8, 8), v + 8);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int k = 0; k < 4; k++)
            umma_bf16(tbase, umma_desc(smem_u32(t.a2) + 256 * k, 128, 1024),
                      umma_desc(smem_u32(t.wb + MLP_W2_OFF) + 256 * k, 128, 1024), idesc,
                      k > 0 ? 1u : 0u);
        umma_commit(mbar);
    }
    w = mbar_wait(mbar, phase, MLP_WAIT_SPINS);
    if (!w) w = mbar_wait(mbar, phase, MLP_WAIT_SPINS);
    phase ^= 1u;
    if (__syncthreads_or(!w)) {
        *ok = false;
        return 0.f;
    }
    tc_fence_after();
    float z = F[MLP_FB3];
#pragma unroll
    for (int c0 = 0; c0 < MLP_NH; c0 += 16) {
        float v[16];
        tmem_ld16(tlane + (uint32_t)c0, v);
#pragma unroll
        for (int c = 0; c < 16; c++) z = fmaf(fmaxf(v[c] + F[MLP_FB2 + c0 + c], 0.f), F[MLP_FW3 + c0 + c], z);
    }
    tc_fence_before();
    return fmaf(F[MLP_FTSCALE], z, F[MLP_FTMEAN]);
}

// all threads: release the TMEM columns (also after a failed setup or wait)
__device__ __forceinline__ void mlp_tile_teardown(MlpTile &t) {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(t.taddr, MLP_TMEM_COLS);
}

// The learned starting pressure p_TS exp(y) (p_TS = p_a exp(lts), the
// two-shock feature before standardisation), or -1 when out of range: a
// feature outside the box of the training data, or a correction |y| > 2
// (or not finite).
__device__ __forceinline__ float mlp_guess(bool in, float pa, float lts, float y) {
    return (in && fabsf(y) <= 2.f) ? pa * __expf(lts + y) : -1.f;
}

// standardised features of one row; false when a feature lies outside the
// box [xmin, xmax] of the training data (out of range) or is not finite
__device__ __forceinline__ bool mlp_standardise(const MlpTile &t, float x[MLP_NF]) {
    const float *F = mlp_f(t);
    bool in = true;
#pragma unroll
    for (int k = 0; k < MLP_NF; k++) {
        in = in && x[k] >= F[MLP_FXMIN + k] && x[k] <= F[MLP_FXMAX + k];
        x[k] = __fdividef(x[k] - F[MLP_FMEAN + k], F[MLP_FSCALE + k]);
    }
    return in;
}

}  // namespace hyd
