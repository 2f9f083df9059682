// Morton ordering of the particles (the GPU form of the tree-ordered particle
// array of §2.2.1: spatially close particles become contiguous so that a
// bucket of 32 is a compact region, §2.2.3), a stable LSD radix sort, and the
// gathers/scatters between the caller's order and the sorted order.
#include "hydro_internal.cuh"

namespace hyd {

namespace {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ROUNDS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ROUNDS;   // keys per CTA
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 2;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t to_fixed(double x, double L) {
    double t = x / L * 4294967296.0;
    if (t >= 4294967296.0) t -= 4294967296.0;
    if (t < 0.0) t = 0.0;
    return (uint32_t)t;
}

__device__ __forceinline__ int box_of(const int64_t *box_off, int64_t nbox, int64_t i) {
    int64_t lo = 0, hi = nbox;   // box_off[lo] <= i < box_off[hi]
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (box_off[mid] <= i) lo = mid; else hi = mid;
    }
    return (int)lo;
}

__global__ void k_morton(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                         const double *__restrict__ z, const int64_t *__restrict__ box_off,
                         int64_t nbox, const Box *__restrict__ boxes,
                         unsigned long long *__restrict__ keys, int32_t *__restrict__ vals) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int b = nbox > 1 ? box_of(box_off, nbox, i) : 0;
    const Box bx = boxes[b];
    // cubic cells of side Lmax / 1024 on every axis, so that a run of
    // consecutive keys is a compact region also in elongated boxes
    const double Lmax = fmax(bx.L[0], fmax(bx.L[1], bx.L[2]));
    uint32_t qx = min((uint32_t)(x[i] / Lmax * 1024.0), 1023u);
    uint32_t qy = min((uint32_t)(y[i] / Lmax * 1024.0), 1023u);
    uint32_t qz = min((uint32_t)(z[i] / Lmax * 1024.0), 1023u);
    uint32_t m = (spread10(qx) << 2) | (spread10(qy) << 1) | spread10(qz);
    keys[i] = ((unsigned long long)b << 30) | m;
    vals[i] = (int32_t)i;
}

// per-tile digit histogram, digit-major: hist[d * ntiles + tile]
__global__ void k_radix_hist(int64_t n, const unsigned long long *__restrict__ keys, int shift,
                             int64_t ntiles, int64_t *__restrict__ hist) {
    __shared__ int h[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0;
    __syncthreads();
    int64_t base = blockIdx.x * (int64_t)SORT_TILE;
    for (int r = 0; r < SORT_ROUNDS; r++) {
        int64_t i = base + r * SORT_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += blockDim.x) hist[(int64_t)t * ntiles + blockIdx.x] = h[t];
}

// stable scatter: within a tile, elements keep their order per digit
__global__ void k_radix_scatter(int64_t n, const unsigned long long *__restrict__ keys,
                                const int32_t *__restrict__ vals, int shift, int64_t ntiles,
                                const int64_t *__restrict__ offs,
                                unsigned long long *__restrict__ okeys,
                                int32_t *__restrict__ ovals) {
    constexpr int W = SORT_THREADS / 32;
    __shared__ int cnt[W][256];
    __shared__ int base[256];
    __shared__ long long goff[256];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = threadIdx.x; t < 256; t += blockDim.x) {
        base[t] = 0;
        goff[t] = offs[(int64_t)t * ntiles + blockIdx.x];
    }
    unsigned lt = (1u << lane) - 1u;
    int64_t tile0 = blockIdx.x * (int64_t)SORT_TILE;
    for (int r = 0; r < SORT_ROUNDS; r++) {
        for (int t = threadIdx.x; t < W * 256; t += blockDim.x) (&cnt[0][0])[t] = 0;
        __syncthreads();
        int64_t i = tile0 + r * SORT_THREADS + threadIdx.x;
        bool valid = i < n;
        unsigned long long k = valid ? keys[i] : 0ull;
        int32_t v = valid ? vals[i] : 0;
        int d = valid ? (int)((k >> shift) & 255u) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int leader = __ffs(peers) - 1;
        int rank = __popc(peers & lt);
        if (valid && lane == leader) cnt[warp][d] = __popc(peers);
        __syncthreads();
        if (threadIdx.x < 256) {
            int dd = threadIdx.x;
            int run = base[dd];
            for (int w = 0; w < W; w++) {
                int c = cnt[w][dd];
                cnt[w][dd] = run;
                run += c;
            }
            base[dd] = run;
        }
        __syncthreads();
        if (valid) {
            long long pos = goff[d] + cnt[warp][d] + rank;
            okeys[pos] = k;
            ovals[pos] = v;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    int lane = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive scan of one tile; block total to sums[blockIdx.x]
__global__ void k_scan_tile(const int64_t *__restrict__ in, int64_t *__restrict__ out, int64_t n,
                            int64_t *__restrict__ sums) {
    __shared__ int64_t wsum[SCAN_THREADS / 32];
    int64_t base = blockIdx.x * (int64_t)SCAN_TILE + threadIdx.x * (int64_t)SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t tot = 0;
    for (int k = 0; k < SCAN_ITEMS; k++) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        tot += v[k];
    }
    int64_t incl = warp_incl_scan(tot);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < SCAN_THREADS / 32 ? wsum[lane] : 0;
        int64_t wi = warp_incl_scan(w);
        if (lane < SCAN_THREADS / 32) wsum[lane] = wi - w;
        if (lane == SCAN_THREADS / 32 - 1 && sums) sums[blockIdx.x] = wi;
    }
    __syncthreads();
    int64_t run = wsum[warp] + incl - tot;
    for (int k = 0; k < SCAN_ITEMS; k++) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

__global__ void k_scan_add(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ add) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] += add[i / SCAN_TILE];
}

template <typename R>
__global__ void k_gather_state(int64_t n, const int32_t *__restrict__ perm,
                               const int64_t *__restrict__ box_off, int64_t nbox,
                               const Box *__restrict__ boxes, const double *__restrict__ x,
                               const double *__restrict__ y, const double *__restrict__ z,
                               const double *__restrict__ h_in, const double *__restrict__ h_search,
                               double margin, double *__restrict__ xs, double *__restrict__ ys,
                               double *__restrict__ zs, uint32_t *__restrict__ qx,
                               uint32_t *__restrict__ qy, uint32_t *__restrict__ qz,
                               double *__restrict__ hsorted, double *__restrict__ hs,
                               int32_t *__restrict__ pbox, R *__restrict__ rec) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    int o = perm[s];
    int b = nbox > 1 ? box_of(box_off, nbox, o) : 0;
    const Box bx = boxes[b];
    double px = x[o], py = y[o], pz = z[o];
    xs[s] = px; ys[s] = py; zs[s] = pz;
    uint32_t ux = to_fixed(px, bx.L[0]), uy = to_fixed(py, bx.L[1]), uz = to_fixed(pz, bx.L[2]);
    qx[s] = ux; qy[s] = uy; qz[s] = uz;
    double h = h_in[o];
    hsorted[s] = h;
    double r = h_search ? h_search[o] : margin * h;
    hs[s] = r;
    pbox[s] = b;
    R *rr = rec + (int64_t)s * REC;
    if (sizeof(R) == 8) {
        rr[R_X] = (R)px; rr[R_Y] = (R)py; rr[R_Z] = (R)pz;
    } else {
        rr[R_X] = __uint_as_float(ux); rr[R_Y] = __uint_as_float(uy); rr[R_Z] = __uint_as_float(uz);
    }
    rr[R_H] = (R)h;
}

__global__ void k_gather6(int64_t n, const int32_t *__restrict__ perm, const double *a0,
                          const double *a1, const double *a2, const double *a3, const double *a4,
                          const double *a5, double *__restrict__ Q) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    int o = perm[s];
    Q[s] = a0[o];
    Q[n + s] = a1[o];
    Q[2 * n + s] = a2[o];
    Q[3 * n + s] = a3[o];
    Q[4 * n + s] = a4[o];
    Q[5 * n + s] = a5[o];
}

// dst[perm[s] * ncomp + k] = src[k * stride + s]
__global__ void k_scatter_caller(int64_t n, int ncomp, const int32_t *__restrict__ perm,
                                 const double *__restrict__ src, int64_t stride,
                                 double *__restrict__ dst) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    int64_t o = perm[s];
    for (int k = 0; k < ncomp; k++) dst[o * ncomp + k] = src[k * stride + s];
}

// dst[k * stride + s] = src[perm[s] * ncomp + k]
__global__ void k_gather_caller(int64_t n, int ncomp, const int32_t *__restrict__ perm,
                                const double *__restrict__ src, double *__restrict__ dst,
                                int64_t stride) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    int64_t o = perm[s];
    for (int k = 0; k < ncomp; k++) dst[k * stride + s] = src[o * ncomp + k];
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp,
                               stream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        k_scan_tile<<<1, SCAN_THREADS, 0, st>>>(in, out, n, nullptr);
        return launch_check();
    }
    int64_t *sums = tmp;
    int64_t *rest = tmp + nb;
    k_scan_tile<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, out, n, sums);
    HYD_CUDA(launch_check());
    HYD_CUDA(exclusive_scan_i64(sums, sums, nb, rest, st));
    k_scan_add<<<grid_for(n, 256), 256, 0, st>>>(out, n, sums);
    return launch_check();
}

static int64_t scan_tmp_size(int64_t n) {
    int64_t t = 0;
    while (n > SCAN_TILE) {
        n = (n + SCAN_TILE - 1) / SCAN_TILE;
        t += n;
    }
    return t + 16;
}

cudaError_t sort_particles(hydro_ctx *c, const hydro_particles *p, stream_t st) {
    const int64_t n = p->n;
    c->have_order = false;   // (hydro_step sets it once its step is done)
    HYD_CUDA(c->d_keys.ensure(n));
    HYD_CUDA(c->d_keys_alt.ensure(n));
    HYD_CUDA(c->d_perm.ensure(n));
    HYD_CUDA(c->d_perm_alt.ensure(n));
    int64_t ntiles = (n + SORT_TILE - 1) / SORT_TILE;
    int64_t nh = 256 * ntiles;
    HYD_CUDA(c->d_scan_tmp.ensure(2 * nh + scan_tmp_size(nh)));
    k_morton<<<grid_for(n, 256), 256, 0, st>>>(n, p->x, p->y, p->z, c->d_box_off.get(),
                                                 c->plan.nbox, c->d_boxes.get(), c->d_keys.get(),
                                                 c->d_perm.get());
    HYD_CUDA(launch_check());
    int bits = 30;
    while ((1ll << (bits - 30)) < c->plan.nbox) bits++;
    int64_t *hist = c->d_scan_tmp.get();
    int64_t *offs = hist + nh;
    int64_t *tmp = offs + nh;
    unsigned long long *ka = c->d_keys.get(), *kb = c->d_keys_alt.get();
    int32_t *va = c->d_perm.get(), *vb = c->d_perm_alt.get();
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<(unsigned)ntiles, SORT_THREADS, 0, st>>>(n, ka, shift, ntiles, hist);
        HYD_CUDA(launch_check());
        HYD_CUDA(exclusive_scan_i64(hist, offs, nh, tmp, st));
        k_radix_scatter<<<(unsigned)ntiles, SORT_THREADS, 0, st>>>(n, ka, va, shift, ntiles, offs,
                                                                   kb, vb);
        HYD_CUDA(launch_check());
        unsigned long long *tk = ka; ka = kb; kb = tk;
        int32_t *tv = va; va = vb; vb = tv;
    }
    if (va != c->d_perm.get())
        HYD_CUDA(cudaMemcpyAsync(c->d_perm.get(), va, n * sizeof(int32_t),
                                 cudaMemcpyDeviceToDevice, st));
    return cudaSuccess;
}

cudaError_t gather_state(hydro_ctx *c, const hydro_particles *p, const double *h_in,
                         const double *h_search, double margin, bool want_Q, stream_t st) {
    const int64_t n = p->n;
    HYD_CUDA(c->d_xs.ensure(n)); HYD_CUDA(c->d_ys.ensure(n)); HYD_CUDA(c->d_zs.ensure(n));
    HYD_CUDA(c->d_qx.ensure(n)); HYD_CUDA(c->d_qy.ensure(n)); HYD_CUDA(c->d_qz.ensure(n));
    HYD_CUDA(c->d_hs.ensure(n)); HYD_CUDA(c->d_hsorted.ensure(n)); HYD_CUDA(c->d_omsorted.ensure(n));
    HYD_CUDA(c->d_pbox.ensure(n));
    const bool mixed = c->cfg.precision == HYDRO_MIXED;
    if (mixed) {
        HYD_CUDA(c->d_recf.ensure((size_t)n * REC));
        k_gather_state<float><<<grid_for(n, 256), 256, 0, st>>>(
            n, c->d_perm.get(), c->d_box_off.get(), c->plan.nbox, c->d_boxes.get(), p->x, p->y,
            p->z, h_in, h_search, margin, c->d_xs.get(), c->d_ys.get(), c->d_zs.get(),
            c->d_qx.get(), c->d_qy.get(), c->d_qz.get(), c->d_hsorted.get(), c->d_hs.get(),
            c->d_pbox.get(), c->d_recf.get());
    } else {
        HYD_CUDA(c->d_recd.ensure((size_t)n * REC));
        k_gather_state<double><<<grid_for(n, 256), 256, 0, st>>>(
            n, c->d_perm.get(), c->d_box_off.get(), c->plan.nbox, c->d_boxes.get(), p->x, p->y,
            p->z, h_in, h_search, margin, c->d_xs.get(), c->d_ys.get(), c->d_zs.get(),
            c->d_qx.get(), c->d_qy.get(), c->d_qz.get(), c->d_hsorted.get(), c->d_hs.get(),
            c->d_pbox.get(), c->d_recd.get());
    }
    HYD_CUDA(launch_check());
    if (want_Q) {
        HYD_CUDA(c->d_Q.ensure((size_t)6 * n));
        k_gather6<<<grid_for(n, 256), 256, 0, st>>>(n, c->d_perm.get(), p->mass, p->px, p->py,
                                                     p->pz, p->etot, p->eint, c->d_Q.get());
        HYD_CUDA(launch_check());
    }
    return cudaSuccess;
}

cudaError_t scatter_to_caller(const int32_t *perm, const double *src, int64_t n, int ncomp,
                              int64_t src_stride, double *dst, stream_t st) {
    if (!dst || n <= 0) return cudaSuccess;
    k_scatter_caller<<<grid_for(n, 256), 256, 0, st>>>(n, ncomp, perm, src, src_stride, dst);
    return launch_check();
}

cudaError_t gather_from_caller(const int32_t *perm, const double *src, int64_t n, int ncomp,
                               double *dst, int64_t dst_stride, stream_t st) {
    if (!src || n <= 0) return cudaSuccess;
    k_gather_caller<<<grid_for(n, 256), 256, 0, st>>>(n, ncomp, perm, src, dst, dst_stride);
    return launch_check();
}

}  // namespace hyd
