// Bucketed neighbour search (§2.2.3).  The Morton-sorted particles are cut
// into buckets of 32 (one warp each); buckets are grouped 32 at a time into
// a fixed-arity bounding-box tree per periodic box.  One warp walks the tree
// once for its whole bucket (the paper's single search per bucket), tests
// every candidate particle against each of its 32 particles, and appends
// the matches to per-lane lists in shared memory before one bulk write.
//
// Membership r_ij < h_search,i is decided exactly as the definition states
// in double precision: a float test on the fixed-point separation settles
// every candidate farther than 1e-4 (relative, on r^2) from the boundary,
// and the rest are re-tested with the double-precision minimum image.
#include "hydro_internal.cuh"

namespace hyd {

namespace {

constexpr int LIST_WARPS = 4;
constexpr int STACK = 256;

__device__ __forceinline__ uint32_t wmin(uint32_t v) {
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ uint32_t wmax(uint32_t v) {
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float wmaxf(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// level 0: bucket boxes from the particles
__global__ void k_aabb_leaf(int64_t nbucket, const int32_t *__restrict__ first,
                            const int32_t *__restrict__ cnt, const uint32_t *__restrict__ qx,
                            const uint32_t *__restrict__ qy, const uint32_t *__restrict__ qz,
                            const double *__restrict__ hs, uint4 *__restrict__ lo,
                            uint4 *__restrict__ hi) {
    int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (b >= nbucket) return;
    int f = first[b], c = cnt[b];
    uint32_t x0 = 0xffffffffu, y0 = 0xffffffffu, z0 = 0xffffffffu, x1 = 0, y1 = 0, z1 = 0;
    float h = 0.f;
    if (lane < c) {
        int s = f + lane;
        x0 = x1 = qx[s];
        y0 = y1 = qy[s];
        z0 = z1 = qz[s];
        h = __double2float_ru(hs[s]);
    }
    x0 = wmin(x0); y0 = wmin(y0); z0 = wmin(z0);
    x1 = wmax(x1); y1 = wmax(y1); z1 = wmax(z1);
    h = wmaxf(h);
    if (lane == 0) {
        lo[b] = make_uint4(x0, y0, z0, __float_as_uint(h));
        hi[b] = make_uint4(x1, y1, z1, 0u);
    }
}

// level >= 1: union of the children's boxes
__global__ void k_aabb_node(int64_t node0, int64_t nnode, const int32_t *__restrict__ first,
                            const int32_t *__restrict__ cnt, uint4 *__restrict__ lo,
                            uint4 *__restrict__ hi) {
    int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (k >= nnode) return;
    int64_t node = node0 + k;
    int f = first[node], c = cnt[node];
    uint32_t x0 = 0xffffffffu, y0 = 0xffffffffu, z0 = 0xffffffffu, x1 = 0, y1 = 0, z1 = 0;
    float h = 0.f;
    if (lane < c) {
        uint4 a = lo[f + lane], b = hi[f + lane];
        x0 = a.x; y0 = a.y; z0 = a.z; h = __uint_as_float(a.w);
        x1 = b.x; y1 = b.y; z1 = b.z;
    }
    x0 = wmin(x0); y0 = wmin(y0); z0 = wmin(z0);
    x1 = wmax(x1); y1 = wmax(y1); z1 = wmax(z1);
    h = wmaxf(h);
    if (lane == 0) {
        lo[node] = make_uint4(x0, y0, z0, __float_as_uint(h));
        hi[node] = make_uint4(x1, y1, z1, 0u);
    }
}

// smallest periodic gap (fixed-point units) between [a0,a1] and [b0,b1]
__device__ __forceinline__ float axis_gap(uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1) {
    const long long P = 1ll << 32;
    long long d1 = (long long)b0 - (long long)a1;
    long long d2 = (long long)a0 - (long long)b1;
    long long g0 = max(0ll, max(d1, d2));
    long long g1 = max(0ll, max(d1 + P, d2 - P));
    long long g2 = max(0ll, max(d1 - P, d2 + P));
    return (float)min(g0, min(g1, g2));
}

__device__ __forceinline__ bool boxes_near(uint4 alo, uint4 ahi, uint4 blo, uint4 bhi,
                                           const Box &bx, float rad2) {
    float gx = axis_gap(alo.x, ahi.x, blo.x, bhi.x) * bx.s[0];
    float gy = axis_gap(alo.y, ahi.y, blo.y, bhi.y) * bx.s[1];
    float gz = axis_gap(alo.z, ahi.z, blo.z, bhi.z) * bx.s[2];
    return gx * gx + gy * gy + gz * gz <= rad2;
}

struct ListArgs {
    int64_t nbucket;
    const int32_t *node_first, *node_cnt, *node_box, *box_root;
    int64_t nbucket_total;   // node ids below this are buckets
    const uint4 *lo, *hi;
    const uint32_t *qx, *qy, *qz;
    const double *xs, *ys, *zs, *hs;
    const Box *boxes;
    int32_t *nbr_idx;
    int64_t *nbr_off;
    int32_t *nbr_cnt;
    int64_t capacity;
    DevCounters *cnt;
    int cap;   // per-lane staging entries
    int mode;  // 0: stage in shared memory, one bulk write; 1: count only;
               // 2: write at nbr_off (from a scan of the counts)
};

// stage a candidate bucket in shared memory and test it against all lanes
__device__ __forceinline__ void test_bucket(const ListArgs &a, int cb, int lane, bool own,
                                            int s_own, uint32_t qxi, uint32_t qyi, uint32_t qzi, double xi,
                                            double yi, double zi, double hsi, float lo2,
                                            float hi2, bool always_exact, const Box &bx,
                                            double *sx, double *sy, double *sz, uint32_t *sq,
                                            int32_t *list, int &count) {
    int f = a.node_first[cb], c = a.node_cnt[cb];
    __syncwarp();
    if (lane < c) {
        int j = f + lane;
        sx[lane] = a.xs[j];
        sy[lane] = a.ys[j];
        sz[lane] = a.zs[j];
        sq[lane] = a.qx[j];
        sq[32 + lane] = a.qy[j];
        sq[64 + lane] = a.qz[j];
    }
    __syncwarp();
    if (!own) return;
    double h2 = __dmul_rn(hsi, hsi);
    for (int k = 0; k < c; k++) {
        bool in;
        if (!always_exact) {
            float dx = qdiff(qxi, sq[k], bx.s[0]);
            float dy = qdiff(qyi, sq[32 + k], bx.s[1]);
            float dz = qdiff(qzi, sq[64 + k], bx.s[2]);
            float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < lo2) in = true;
            else if (r2 > hi2) in = false;
            else {
                double ex = fold64(__dsub_rn(sx[k], xi), bx.L[0]);
                double ey = fold64(__dsub_rn(sy[k], yi), bx.L[1]);
                double ez = fold64(__dsub_rn(sz[k], zi), bx.L[2]);
                in = r2_exact(ex, ey, ez) < h2;
            }
        } else {
            double ex = fold64(__dsub_rn(sx[k], xi), bx.L[0]);
            double ey = fold64(__dsub_rn(sy[k], yi), bx.L[1]);
            double ez = fold64(__dsub_rn(sz[k], zi), bx.L[2]);
            in = r2_exact(ex, ey, ez) < h2;
        }
        if (in) {
            if (a.mode == 0) {
                if (count < a.cap) list[count * 32 + lane] = f + k;
            } else if (a.mode == 2) {
                a.nbr_idx[a.nbr_off[s_own] + count] = f + k;
            }
            count++;
        }
    }
}

__global__ void k_build_lists(ListArgs a) {
    extern __shared__ unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b = blockIdx.x * (int64_t)LIST_WARPS + warp;
    // per-warp shared memory: list[cap][32] | stack[STACK] | sx sy sz [32] | sq[96]
    size_t per_warp = (size_t)a.cap * 32 * 4 + STACK * 4 + 3 * 32 * 8 + 96 * 4;
    unsigned char *base = smem_raw + per_warp * warp;   // cap = 0 in modes 1, 2
    int32_t *list = (int32_t *)base;
    int32_t *stack = (int32_t *)(base + (size_t)a.cap * 32 * 4);
    double *sx = (double *)(base + (size_t)a.cap * 32 * 4 + STACK * 4);
    double *sy = sx + 32;
    double *sz = sy + 32;
    uint32_t *sq = (uint32_t *)(sz + 32);
    if (b >= a.nbucket) return;

    const int f = a.node_first[b], c = a.node_cnt[b];
    const Box bx = a.boxes[a.node_box[b]];
    const bool own = lane < c;
    const int s = f + (own ? lane : 0);
    uint32_t qxi = a.qx[s], qyi = a.qy[s], qzi = a.qz[s];
    double xi = a.xs[s], yi = a.ys[s], zi = a.zs[s], hsi = a.hs[s];
    float hf = (float)hsi;
    float lo2 = hf * hf * (1.0f - 1e-4f), hi2 = hf * hf * (1.0f + 1e-4f);
    const double Lmin = fmin(bx.L[0], fmin(bx.L[1], bx.L[2]));
    bool always_exact = hsi < Lmin * (1.0 / 4096.0);
    const uint4 qlo = a.lo[b], qhi = a.hi[b];
    const float qh = __uint_as_float(qlo.w) * 1.00001f;
    const float rad2 = qh * qh;
    int count = 0;

    int sp = 0;
    int root = a.box_root[a.node_box[b]];
    if (root < a.nbucket_total) {
        test_bucket(a, root, lane, own, s, qxi, qyi, qzi, xi, yi, zi, hsi, lo2, hi2, always_exact,
                    bx, sx, sy, sz, sq, list, count);
    } else {
        if (lane == 0) stack[0] = root;
        sp = 1;
    }
    __syncwarp();
    while (sp > 0) {
        sp--;
        int node = stack[sp];
        __syncwarp();
        int nf = a.node_first[node], nc = a.node_cnt[node];
        bool hit = false;
        int child = nf + lane;
        if (lane < nc) hit = boxes_near(qlo, qhi, a.lo[child], a.hi[child], bx, rad2);
        unsigned m = __ballot_sync(0xffffffffu, hit);
        if (nf < a.nbucket_total) {
            // children are buckets
            while (m) {
                int k = __ffs(m) - 1;
                m &= m - 1;
                test_bucket(a, nf + k, lane, own, s, qxi, qyi, qzi, xi, yi, zi, hsi, lo2, hi2,
                            always_exact, bx, sx, sy, sz, sq, list, count);
            }
        } else {
            int np = __popc(m);
            if (sp + np > STACK) {
                if (lane == 0) set_flag(a.cnt, ST_STACK);
                break;
            }
            if (hit) stack[sp + __popc(m & ((1u << lane) - 1u))] = child;
            sp += np;
            __syncwarp();
        }
    }

    if (a.mode == 1) {
        if (own) a.nbr_cnt[s] = count;
        return;
    }
    if (a.mode == 2) {
        return;
    }
    // write the lists out
    if (own && count > a.cap) set_flag(a.cnt, ST_LIST_OVERFLOW);
    int mine = own ? min(count, a.cap) : 0;
    int incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    int total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long gbase = 0;
    if (lane == 0) gbase = atomicAdd(&a.cnt->list_cursor, (unsigned long long)total);
    gbase = __shfl_sync(0xffffffffu, gbase, 0);
    int64_t start = (int64_t)gbase + (incl - mine);
    if (own) {
        a.nbr_off[s] = start;
        a.nbr_cnt[s] = mine;
    }
    if ((int64_t)gbase + total > a.capacity) {
        if (lane == 0) set_flag(a.cnt, ST_LIST_CAPACITY);
        return;
    }
    __syncwarp();
    for (int k = 0; k < mine; k++) a.nbr_idx[start + k] = list[k * 32 + lane];
}

__global__ void k_widen(int64_t n, const int32_t *__restrict__ cnt, int64_t *__restrict__ out) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s < n) out[s] = cnt[s];
    if (s == n) out[n] = 0;
}

__global__ void k_export_count(int64_t n, const int32_t *__restrict__ perm,
                               const int32_t *__restrict__ cnt, int64_t *__restrict__ rowlen) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s < n) rowlen[perm[s]] = cnt[s];
    if (s == n) rowlen[n] = 0;
}

__global__ void k_export_fill(int64_t n, const int32_t *__restrict__ perm,
                              const int64_t *__restrict__ off_in, const int32_t *__restrict__ cnt,
                              const int32_t *__restrict__ idx_in, const int64_t *__restrict__ off_out,
                              int32_t *__restrict__ idx_out) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    int64_t o = perm[s];
    int32_t *dst = idx_out + off_out[o];
    const int32_t *src = idx_in + off_in[s];
    int c = cnt[s];
    for (int k = 0; k < c; k++) {
        int32_t v = perm[src[k]];
        int m = k;
        while (m > 0 && dst[m - 1] > v) { dst[m] = dst[m - 1]; m--; }
        dst[m] = v;
    }
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

static cudaError_t widen_counts(const int32_t *cnt, int64_t n, int64_t *out, stream_t st) {
    k_widen<<<grid_for(n + 1, 256), 256, 0, st>>>(n, cnt, out);
    return launch_check();
}

cudaError_t build_tree(hydro_ctx *c, stream_t st) {
    const Plan &P = c->plan;
    k_aabb_leaf<<<grid_for(P.nbucket * 32, 256), 256, 0, st>>>(
        P.nbucket, c->d_node_first.get(), c->d_node_cnt.get(), c->d_qx.get(), c->d_qy.get(),
        c->d_qz.get(), c->d_hs.get(), c->d_node_aabb.get(), c->d_node_aabb_hi.get());
    HYD_CUDA(launch_check());
    for (int l = 1; l < P.nlevels; l++) {
        int64_t n0 = P.level_off[l], nn = P.level_off[l + 1] - P.level_off[l];
        k_aabb_node<<<grid_for(nn * 32, 256), 256, 0, st>>>(n0, nn, c->d_node_first.get(),
                                                            c->d_node_cnt.get(),
                                                            c->d_node_aabb.get(),
                                                            c->d_node_aabb_hi.get());
        HYD_CUDA(launch_check());
    }
    return cudaSuccess;
}

static ListArgs list_args(hydro_ctx *c, int cap, int mode) {
    const Plan &P = c->plan;
    ListArgs a;
    a.nbucket = P.nbucket;
    a.node_first = c->d_node_first.get();
    a.node_cnt = c->d_node_cnt.get();
    a.node_box = c->d_node_box.get();
    a.box_root = c->d_box_root.get();
    a.nbucket_total = P.nbucket;
    a.lo = c->d_node_aabb.get();
    a.hi = c->d_node_aabb_hi.get();
    a.qx = c->d_qx.get(); a.qy = c->d_qy.get(); a.qz = c->d_qz.get();
    a.xs = c->d_xs.get(); a.ys = c->d_ys.get(); a.zs = c->d_zs.get();
    a.hs = c->d_hs.get();
    a.boxes = c->d_boxes.get();
    a.nbr_idx = c->d_nbr_idx.get();
    a.nbr_off = c->d_nbr_off.get();
    a.nbr_cnt = c->d_nbr_cnt.get();
    a.capacity = (int64_t)c->d_nbr_idx.cap;
    a.cnt = c->d_cnt;
    a.cap = cap;
    a.mode = mode;
    return a;
}

static cudaError_t launch_lists(const ListArgs &a, int64_t nbucket, stream_t st) {
    size_t per_warp = (size_t)a.cap * 32 * 4 + STACK * 4 + 3 * 32 * 8 + 96 * 4;
    size_t smem = per_warp * LIST_WARPS;
    static size_t configured = 48 * 1024;
    if (configured < smem) {
        HYD_CUDA(cudaFuncSetAttribute(k_build_lists, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        configured = smem;
    }
    k_build_lists<<<grid_for(nbucket, LIST_WARPS), LIST_WARPS * 32, smem, st>>>(a);
    return launch_check();
}

// one pass: lists staged per lane in shared memory (cap entries), bulk write
cudaError_t build_lists(hydro_ctx *c, int cap, stream_t st) {
    const int64_t n = c->plan.n;
    HYD_CUDA(c->d_nbr_off.ensure(n + 1));
    HYD_CUDA(c->d_nbr_cnt.ensure(n));
    HYD_CUDA(c->d_nbr_idx.ensure((size_t)n * c->nbr_per_particle));
    HYD_CUDA(cudaMemsetAsync(&c->d_cnt->list_cursor, 0, sizeof(unsigned long long), st));
    return launch_lists(list_args(c, cap, 0), c->plan.nbucket, st);
}

// two passes for particles with more candidates than the staging holds:
// count, exclusive scan into nbr_off, then write in place (synchronous)
cudaError_t build_lists_twopass(hydro_ctx *c, stream_t st) {
    const int64_t n = c->plan.n;
    HYD_CUDA(c->d_nbr_off.ensure(n + 1));
    HYD_CUDA(c->d_nbr_cnt.ensure(n));
    HYD_CUDA(launch_lists(list_args(c, 0, 1), c->plan.nbucket, st));
    HYD_CUDA(c->d_scan_tmp.ensure((size_t)(n + 1) + (n + 1) / 2048 + 64));
    int64_t *cnt64 = c->d_scan_tmp.get();
    int64_t *tmp = cnt64 + (n + 1);
    HYD_CUDA(widen_counts(c->d_nbr_cnt.get(), n, cnt64, st));
    HYD_CUDA(exclusive_scan_i64(cnt64, c->d_nbr_off.get(), n + 1, tmp, st));
    int64_t total = 0;
    HYD_CUDA(cudaMemcpyAsync(&total, c->d_nbr_off.get() + n, sizeof(int64_t),
                             cudaMemcpyDeviceToHost, st));
    HYD_CUDA(cudaStreamSynchronize(st));
    if ((size_t)total > c->d_nbr_idx.cap) {
        HYD_CUDA(c->d_nbr_idx.ensure((size_t)total + (size_t)n * 4));
        c->nbr_per_particle = (int)(c->d_nbr_idx.cap / (size_t)n) + 1;
    }
    return launch_lists(list_args(c, 0, 2), c->plan.nbucket, st);
}

cudaError_t export_lists(hydro_ctx *c, hydro_nbrlist *out, stream_t st) {
    const int64_t n = c->plan.n;
    HYD_CUDA(c->d_scan_tmp.ensure((size_t)(n + 1) + (n + 1) / 2048 + 64));
    int64_t *rowlen = c->d_scan_tmp.get();
    int64_t *tmp = rowlen + (n + 1);
    k_export_count<<<grid_for(n + 1, 256), 256, 0, st>>>(n, c->d_perm.get(), c->d_nbr_cnt.get(),
                                                         rowlen);
    HYD_CUDA(launch_check());
    HYD_CUDA(exclusive_scan_i64(rowlen, out->off, n + 1, tmp, st));
    int64_t total = 0;
    HYD_CUDA(cudaMemcpyAsync(&total, out->off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    HYD_CUDA(cudaStreamSynchronize(st));
    out->needed = total;
    if (total > out->capacity || !out->idx) return cudaSuccess;
    k_export_fill<<<grid_for(n, 128), 128, 0, st>>>(n, c->d_perm.get(), c->d_nbr_off.get(),
                                                   c->d_nbr_cnt.get(), c->d_nbr_idx.get(),
                                                   out->off, out->idx);
    return launch_check();
}

}  // namespace hyd
