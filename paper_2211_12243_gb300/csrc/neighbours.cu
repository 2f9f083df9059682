// Bucketed neighbour search (§2.2.3).  The Morton-sorted particles are cut
// into buckets of 32 (one warp each); buckets are grouped 32 at a time into
// a fixed-arity bounding-box tree per periodic box.  One warp walks the tree
// once for its whole bucket (the paper's single search per bucket).  Each
// candidate bucket is staged in shared memory -- only its particles within
// the search radius of the warp's bucket box, compacted -- and every lane
// tests the staged particles against its own, appending matches to its
// fixed-stride row of the list (or, for long lists, the overflow region).
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

// level 0: bucket boxes from the particles; lo.w the largest search
// radius hs, hi.w the largest smoothing length h (both rounded up)
__global__ void k_aabb_leaf(int64_t nbucket, const int32_t *__restrict__ first,
                            const int32_t *__restrict__ cnt, const uint32_t *__restrict__ qx,
                            const uint32_t *__restrict__ qy, const uint32_t *__restrict__ qz,
                            const double *__restrict__ hs, const double *__restrict__ hh,
                            uint4 *__restrict__ lo, uint4 *__restrict__ hi) {
    int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (b >= nbucket) return;
    int f = first[b], c = cnt[b];
    uint32_t x0 = 0xffffffffu, y0 = 0xffffffffu, z0 = 0xffffffffu, x1 = 0, y1 = 0, z1 = 0;
    float h = 0.f, hm = 0.f;
    if (lane < c) {
        int s = f + lane;
        x0 = x1 = qx[s];
        y0 = y1 = qy[s];
        z0 = z1 = qz[s];
        h = __double2float_ru(hs[s]);
        hm = __double2float_ru(hh[s]);
    }
    x0 = wmin(x0); y0 = wmin(y0); z0 = wmin(z0);
    x1 = wmax(x1); y1 = wmax(y1); z1 = wmax(z1);
    h = wmaxf(h);
    hm = wmaxf(hm);
    if (lane == 0) {
        lo[b] = make_uint4(x0, y0, z0, __float_as_uint(h));
        hi[b] = make_uint4(x1, y1, z1, __float_as_uint(hm));
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
    float h = 0.f, hm = 0.f;
    if (lane < c) {
        uint4 a = lo[f + lane], b = hi[f + lane];
        x0 = a.x; y0 = a.y; z0 = a.z; h = __uint_as_float(a.w);
        x1 = b.x; y1 = b.y; z1 = b.z; hm = __uint_as_float(b.w);
    }
    x0 = wmin(x0); y0 = wmin(y0); z0 = wmin(z0);
    x1 = wmax(x1); y1 = wmax(y1); z1 = wmax(z1);
    h = wmaxf(h);
    hm = wmaxf(hm);
    if (lane == 0) {
        lo[node] = make_uint4(x0, y0, z0, __float_as_uint(h));
        hi[node] = make_uint4(x1, y1, z1, __float_as_uint(hm));
    }
}

// Raise the bounds of the buckets holding the particles idx[0 .. *nidx):
// lo.w to at least their search radius hs, hi.w to at least their h.  In a
// guard round only those particles' radii move, so the tree built before
// the rounds stays exact in its boxes and an upper bound in .w (a bound
// that stays above a radius that shrank only prunes less); the node levels
// are then recomputed from the buckets.  Positive floats order like their
// bit patterns, so the maximum is an integer atomic.  A particle's bucket is
// the last one whose first particle is at or before it (buckets are
// consecutive and non-empty).
__global__ void k_aabb_raise(const int32_t *__restrict__ idx, const int *__restrict__ nidx,
                             const int32_t *__restrict__ first, int64_t nbucket,
                             const double *__restrict__ hs, const double *__restrict__ hh,
                             uint4 *__restrict__ lo, uint4 *__restrict__ hi) {
    const int ni = *nidx;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ni; t += gridDim.x * blockDim.x) {
        const int s = idx[t];
        int64_t a = 0, b = nbucket - 1;
        while (a < b) {
            const int64_t m = (a + b + 1) >> 1;
            if (first[m] <= s) a = m; else b = m - 1;
        }
        atomicMax(&lo[a].w, __float_as_uint(__double2float_ru(hs[s])));
        atomicMax(&hi[a].w, __float_as_uint(__double2float_ru(hh[s])));
    }
}

// Lower bound of the periodic distance (fixed-point units) between the
// intervals [a0,a1] and [b0,b1] on the circle of 2^32 units: the circular
// distance of the centres minus both half-widths (rounded up), in 32-bit
// integers only (64-bit conversions would run on the FP64 pipe).
__device__ __forceinline__ uint32_t axis_gap(uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1) {
    uint32_t wa = (a1 - a0 + 1u) >> 1, wb = (b1 - b0 + 1u) >> 1;
    uint32_t ca = a0 + ((a1 - a0) >> 1), cb = b0 + ((b1 - b0) >> 1);
    int32_t dc = (int32_t)(cb - ca);
    uint32_t d = dc < 0 ? (uint32_t)(-(int64_t)dc) : (uint32_t)dc;
    uint32_t w = wa + wb + 2u;
    return d > w ? d - w : 0u;
}

__device__ __forceinline__ bool boxes_near(uint4 alo, uint4 ahi, uint4 blo, uint4 bhi,
                                           const Box &bx, float rad2) {
    float gx = (float)axis_gap(alo.x, ahi.x, blo.x, bhi.x) * bx.s[0];
    float gy = (float)axis_gap(alo.y, ahi.y, blo.y, bhi.y) * bx.s[1];
    float gz = (float)axis_gap(alo.z, ahi.z, blo.z, bhi.z) * bx.s[2];
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
    int cap;   // fixed slots per particle (row s at s cap)
    int mode;  // 0: write the fixed-stride rows (buckets with a row longer
               //    than cap are queued in ovf_list);
               // 1: count and reserve storage (queued buckets);
               // 2: write at nbr_off (queued buckets)
    int32_t *ovf_list;      // queued bucket ids
    int *ovf_count;
    bool nq_dev;            // modes 1, 2: warps past *ovf_count have no bucket
};

__device__ __forceinline__ float u2f(uint32_t v) {
    return fmaf(i2f_small((int32_t)(v >> 11)), 2048.0f, i2f_small((int32_t)(v & 0x7FFu)));
}

// Per-lane state of the walk: the owner particle, its position relative to
// the bucket's corner (float), and the exact-test data.
struct Lane {
    bool own;
    int s;
    uint32_t qx, qy, qz;
    float rx, ry, rz;        // relative to the warp's origin
    double x, y, z, hs, h2;
    float lo2, hi2;          // float band around hs^2 (lo2 < 0 < hi2 = inf: always exact)
    bool rel_ok;             // bucket extent + radius < L/4: relative coordinates are exact images
};

// circular gap (fixed-point units) between a point and an interval
__device__ __forceinline__ uint32_t point_gap(uint32_t p, uint32_t b0, uint32_t b1) {
    uint32_t w = (b1 - b0 + 1u) >> 1, c = b0 + ((b1 - b0) >> 1);
    int32_t d = (int32_t)(c - p);
    uint32_t e = d < 0 ? 0u - (uint32_t)d : (uint32_t)d;
    return e > w + 2u ? e - w - 2u : 0u;
}

// does the lane's sphere reach the box?
__device__ __forceinline__ bool sphere_near(const Lane &L, uint4 blo, uint4 bhi, const Box &bx) {
    float gx = u2f(point_gap(L.qx, blo.x, bhi.x)) * bx.s[0];
    float gy = u2f(point_gap(L.qy, blo.y, bhi.y)) * bx.s[1];
    float gz = u2f(point_gap(L.qz, blo.z, bhi.z)) * bx.s[2];
    return L.own && gx * gx + gy * gy + gz * gz <= L.hi2;
}

// one staged candidate particle (registers of the lane that loads it)
struct Cand {
    double x, y, z;
    uint32_t qx, qy, qz;
};

__device__ __forceinline__ void cand_load(const ListArgs &a, int j, Cand &c) {
    c.x = a.xs[j]; c.y = a.ys[j]; c.z = a.zs[j];
    c.qx = a.qx[j]; c.qy = a.qy[j]; c.qz = a.qz[j];
}

struct Stage {
    double *sx, *sy, *sz;
    float4 *sr;              // position relative to the warp's origin; .w = index bits
    uint32_t *sq;
};

// per-stage bytes: sr[32] float4 | sx sy sz [32] double | sq[96]
constexpr size_t STAGE_BYTES = 32 * 16 + 3 * 32 * 8 + 96 * 4;

// Stage this lane's candidate (keep = it can lie within the search radius
// of some particle of the warp's bucket): the kept candidates are compacted
// to the front in their original order; returns their number.
__device__ __forceinline__ int cand_stage(const Stage &S, bool keep, int lane, const Cand &c, int j,
                                          uint32_t ox, uint32_t oy, uint32_t oz, const Box &bx) {
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) {
        const int pos = __popc(m & ((1u << lane) - 1u));
        S.sx[pos] = c.x; S.sy[pos] = c.y; S.sz[pos] = c.z;
        S.sq[pos] = c.qx; S.sq[32 + pos] = c.qy; S.sq[64 + pos] = c.qz;
        S.sr[pos] = make_float4(qdiff(ox, c.qx, bx.s[0]), qdiff(oy, c.qy, bx.s[1]),
                                qdiff(oz, c.qz, bx.s[2]), __int_as_float(j));
    }
    return __popc(m);
}

// can candidate c lie within rad2 of a point of the bucket box [lo, hi]?
// (a lower bound of the periodic distance, as in sphere_near)
__device__ __forceinline__ bool cand_near(const Cand &c, uint4 lo, uint4 hi, const Box &bx,
                                          float rad2) {
    float gx = u2f(point_gap(c.qx, lo.x, hi.x)) * bx.s[0];
    float gy = u2f(point_gap(c.qy, lo.y, hi.y)) * bx.s[1];
    float gz = u2f(point_gap(c.qz, lo.z, hi.z)) * bx.s[2];
    return gx * gx + gy * gy + gz * gz <= rad2;
}

// Output row of a lane: where its matches go and how many fit.
struct Row {
    int32_t *out;
    int lim;
};

// decide staged candidate k for this lane
__device__ __forceinline__ void decide(const Lane &L, const Row &R, const Stage &S, const Box &bx,
                                       int k, float r2, int &count) {
    bool in = r2 < L.lo2;
    if (!in && r2 <= L.hi2) {   // within the float band: decide in double
        double ex = fold64(__dsub_rn(S.sx[k], L.x), bx.L[0]);
        double ey = fold64(__dsub_rn(S.sy[k], L.y), bx.L[1]);
        double ez = fold64(__dsub_rn(S.sz[k], L.z), bx.L[2]);
        in = r2_exact(ex, ey, ez) < L.h2;
    }
    if (in) {
        if (count < R.lim) R.out[count] = __float_as_int(S.sr[k].w);
        count++;
    }
}

// every lane scans the c staged candidates (four at a time for overlap)
__device__ __forceinline__ void scan_stage(const Lane &L, const Row &R, const Stage &S,
                                           const Box &bx, int c, int &count) {
    if (!L.own) return;
    if (L.rel_ok) {
        for (int k = 0; k < c; k += 4) {
            float r2[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                float4 r = S.sr[k + u];
                float dx = r.x - L.rx, dy = r.y - L.ry, dz = r.z - L.rz;
                r2[u] = dx * dx + dy * dy + dz * dz;
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (k + u < c) decide(L, R, S, bx, k + u, r2[u], count);
        }
    } else {
        for (int k = 0; k < c; k++) {
            float dx = qdiff(L.qx, S.sq[k], bx.s[0]);
            float dy = qdiff(L.qy, S.sq[32 + k], bx.s[1]);
            float dz = qdiff(L.qz, S.sq[64 + k], bx.s[2]);
            decide(L, R, S, bx, k, dx * dx + dy * dy + dz * dz, count);
        }
    }
}

__global__ void __launch_bounds__(LIST_WARPS * 32, 5) k_build_lists(ListArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t b = blockIdx.x * (int64_t)LIST_WARPS + warp;
    // per-warp shared memory: stack[STACK] | 2 stages
    size_t per_warp = STACK * 4 + 2 * STAGE_BYTES;
    unsigned char *base = smem_raw + per_warp * warp;
    int32_t *stack = (int32_t *)base;
    // the two staging buffers, addressed arithmetically (no local array)
    auto stage = [&](int t) {
        unsigned char *p = base + STACK * 4 + t * STAGE_BYTES;
        Stage st;
        st.sr = (float4 *)p;
        st.sx = (double *)(p + 32 * 16);
        st.sy = st.sx + 32;
        st.sz = st.sy + 32;
        st.sq = (uint32_t *)(st.sz + 32);
        return st;
    };
    if (b >= a.nbucket) return;
    if (a.mode != 0) {
        if (a.nq_dev && b >= *a.ovf_count) return;
        b = a.ovf_list[b];
    }

    const int f = a.node_first[b], c = a.node_cnt[b];
    const Box bx = a.boxes[a.node_box[b]];
    const uint4 qlo = a.lo[b], qhi = a.hi[b];
    const uint32_t ox = qlo.x, oy = qlo.y, oz = qlo.z;   // the warp's origin
    Lane L;
    L.own = lane < c;
    L.s = f + (L.own ? lane : 0);
    L.qx = a.qx[L.s]; L.qy = a.qy[L.s]; L.qz = a.qz[L.s];
    L.rx = qdiff(ox, L.qx, bx.s[0]);
    L.ry = qdiff(oy, L.qy, bx.s[1]);
    L.rz = qdiff(oz, L.qz, bx.s[2]);
    L.x = a.xs[L.s]; L.y = a.ys[L.s]; L.z = a.zs[L.s]; L.hs = a.hs[L.s];
    L.h2 = __dmul_rn(L.hs, L.hs);
    {
        float hf = (float)L.hs;
        L.lo2 = hf * hf * (1.0f - 1e-4f);
        L.hi2 = hf * hf * (1.0f + 1e-4f);
        const double Lmin = fmin(bx.L[0], fmin(bx.L[1], bx.L[2]));
        if (L.hs < Lmin * (1.0 / 4096.0)) { L.lo2 = -1.0f; L.hi2 = 3.0e38f; }
    }
    const float qh = __uint_as_float(qlo.w) * 1.00001f;
    const float rad2 = qh * qh;
    {
        // relative coordinates from the bucket corner give exact minimum
        // images while every candidate that can be inside lies within L/4
        float ex = u2f(qhi.x - qlo.x) * bx.s[0], ey = u2f(qhi.y - qlo.y) * bx.s[1],
              ez = u2f(qhi.z - qlo.z) * bx.s[2];
        L.rel_ok = ex + 2.f * qh < 0.25f * (float)bx.L[0] && ey + 2.f * qh < 0.25f * (float)bx.L[1] &&
                   ez + 2.f * qh < 0.25f * (float)bx.L[2];
    }
    int count = 0;
    Row R;
    R.out = nullptr;
    R.lim = 0;
    if (a.mode == 0) {
        R.out = a.nbr_idx + (int64_t)L.s * a.cap;
        R.lim = a.cap;
    } else if (a.mode == 2) {
        // storage was reserved in mode 1; a reservation that did not fit
        // (the capacity flag is set and the host rebuilds) must not write
        // past the buffer
        const int64_t o = a.nbr_off[L.s];
        R.out = a.nbr_idx + o;
        R.lim = (int)max((int64_t)0, min(a.capacity - o, (int64_t)0x7fffffff));
    }

    int sp = 0;
    int root = a.box_root[a.node_box[b]];
    if (root < a.nbucket_total) {
        // the whole box is one bucket
        Cand cd;
        const int rf = a.node_first[root], rc = a.node_cnt[root];
        if (lane < rc) cand_load(a, rf + lane, cd);
        __syncwarp();
        const int kc = cand_stage(stage(0), lane < rc && cand_near(cd, qlo, qhi, bx, rad2), lane, cd,
                                  rf + lane, ox, oy, oz, bx);
        __syncwarp();
        scan_stage(L, R, stage(0), bx, kc, count);
    } else {
        if (lane == 0) stack[0] = root;
        sp = 1;
    }
    __syncwarp();
    while (sp > 0) {
        sp--;
        int node = stack[sp];
        __syncwarp();
        const int nf = a.node_first[node], nc = a.node_cnt[node];
        bool hit = false;
        const int child = nf + lane;
        uint4 clo = make_uint4(0, 0, 0, 0), chi = make_uint4(0, 0, 0, 0);
        int cfirst = 0, ccnt = 0;
        if (lane < nc) {
            clo = a.lo[child];
            chi = a.hi[child];
            hit = boxes_near(qlo, qhi, clo, chi, bx, rad2);
        }
        unsigned m = __ballot_sync(0xffffffffu, hit);
        if (nf < a.nbucket_total) {
            // children are buckets: keep the ones some lane's sphere reaches,
            // then stage bucket k+1 (global loads in flight) while scanning k
            if (hit) { cfirst = a.node_first[child]; ccnt = a.node_cnt[child]; }
            unsigned keep = 0;
            unsigned mm = m;
            while (mm) {
                int k = __ffs(mm) - 1;
                mm &= mm - 1;
                uint4 blo, bhi;
                blo.x = __shfl_sync(0xffffffffu, clo.x, k); blo.y = __shfl_sync(0xffffffffu, clo.y, k);
                blo.z = __shfl_sync(0xffffffffu, clo.z, k);
                bhi.x = __shfl_sync(0xffffffffu, chi.x, k); bhi.y = __shfl_sync(0xffffffffu, chi.y, k);
                bhi.z = __shfl_sync(0xffffffffu, chi.z, k);
                if (__any_sync(0xffffffffu, sphere_near(L, blo, bhi, bx))) keep |= 1u << k;
            }
            if (!keep) continue;
            int k = __ffs(keep) - 1;
            keep &= keep - 1;
            int cf = __shfl_sync(0xffffffffu, cfirst, k), cc = __shfl_sync(0xffffffffu, ccnt, k);
            Cand cd;
            if (lane < cc) cand_load(a, cf + lane, cd);
            int buf = 0;
            int kc = cand_stage(stage(buf), lane < cc && cand_near(cd, qlo, qhi, bx, rad2), lane, cd,
                                cf + lane, ox, oy, oz, bx);
            __syncwarp();
            for (;;) {
                int nk = keep ? __ffs(keep) - 1 : -1;
                int nfst = 0, ncc = 0;
                if (nk >= 0) {
                    keep &= keep - 1;
                    nfst = __shfl_sync(0xffffffffu, cfirst, nk);
                    ncc = __shfl_sync(0xffffffffu, ccnt, nk);
                    if (lane < ncc) cand_load(a, nfst + lane, cd);
                }
                scan_stage(L, R, stage(buf), bx, kc, count);
                if (nk < 0) break;
                kc = cand_stage(stage(buf ^ 1), lane < ncc && cand_near(cd, qlo, qhi, bx, rad2), lane,
                                cd, nfst + lane, ox, oy, oz, bx);
                __syncwarp();
                buf ^= 1;
            }
            __syncwarp();
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
    const bool own = L.own;
    const int s = L.s;

    if (a.mode == 2) return;
    if (a.mode == 0) {
        // each particle owns cap slots at s * cap; a longer list sends the
        // whole bucket to the count-then-fill passes (overflow region)
        unsigned over = __ballot_sync(0xffffffffu, own && count > a.cap);
        if (over) {
            if (lane == 0) a.ovf_list[atomicAdd(a.ovf_count, 1)] = (int32_t)b;
            return;
        }
        if (own) {
            a.nbr_off[s] = (int64_t)s * a.cap;
            a.nbr_cnt[s] = count;
        }
        return;
    }
    // mode 1: reserve storage in the overflow region for the warp's lists
    int mine = own ? count : 0;
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
        if (own) a.nbr_cnt[s] = 0;   // nothing stored for these lists
    }
}

// Lists of single particles (the N_cond guard's grown particles, whose
// search radii rose): one warp per particle walks the tree with that
// particle's own sphere -- the lanes test a node's children at once, then a
// bucket's particles at once -- instead of rebuilding the lists of the
// particle's whole bucket at its largest radius.  The walk takes the
// children in the order of k_build_lists's walk (internal nodes last pushed
// first, buckets in ascending order), so a list holds the same entries in
// the same order as a bucket rebuild would give it.  mode 1 counts and
// reserves storage in the overflow region (flagging ST_LIST_CAPACITY when it
// does not fit), mode 2 writes.  Warps stride over the *npidx particles of
// pidx (the count is read on the device); with `active` set, only those
// with an ACT_SOLVE flag (a guard round's re-search: the guard particles
// whose root left their radius), and mode 1 clears the search-failure flag
// that the new lists answer.
struct PartListArgs {
    const int32_t *pidx;
    const int *npidx;
    const uint8_t *active;
    const int32_t *node_first, *node_cnt, *box_root, *pbox;
    int64_t nbucket_total;
    const uint4 *lo, *hi;
    const uint32_t *qx, *qy, *qz;
    const double *xs, *ys, *zs, *hs;
    const Box *boxes;
    int32_t *nbr_idx;
    int64_t *nbr_off;
    int32_t *nbr_cnt;
    int64_t capacity;
    DevCounters *cnt;
    int mode;
};

constexpr int PL_WARPS = 4;

__global__ void __launch_bounds__(PL_WARPS * 32) k_particle_lists(PartListArgs a) {
    __shared__ int32_t stack_all[PL_WARPS][STACK];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t *stack = stack_all[warp];
    const int np = *a.npidx;
    const int nwarps = gridDim.x * PL_WARPS;
    if (a.active && a.mode == 1 && blockIdx.x == 0 && threadIdx.x == 0)
        atomicAnd(&a.cnt->flags, ~ST_SEARCH);
    for (int g = blockIdx.x * PL_WARPS + warp; g < np; g += nwarps) {
        const int s = a.pidx[g];
        if (a.active && !(a.active[s] & ACT_SOLVE)) continue;   // (warp-uniform: one particle)
        const Box bx = a.boxes[a.pbox[s]];
        const uint32_t px = a.qx[s], py = a.qy[s], pz = a.qz[s];
        const double x = a.xs[s], y = a.ys[s], z = a.zs[s], hs = a.hs[s];
        const double h2 = __dmul_rn(hs, hs);
        float lo2, hi2;
        {
            const float hf = (float)hs;
            lo2 = hf * hf * (1.0f - 1e-4f);
            hi2 = hf * hf * (1.0f + 1e-4f);
            const double Lmin = fmin(bx.L[0], fmin(bx.L[1], bx.L[2]));
            if (hs < Lmin * (1.0 / 4096.0)) { lo2 = -1.0f; hi2 = 3.0e38f; }
        }
        int32_t *out = nullptr;
        int64_t lim = 0;
        if (a.mode == 2) {
            const int64_t o = a.nbr_off[s];
            out = a.nbr_idx + o;
            lim = max((int64_t)0, a.capacity - o);
        }
        int count = 0;
        // the particles of bucket b within the sphere, appended in order
        auto scan_bucket = [&](int b) {
            const int f = a.node_first[b], c = a.node_cnt[b];
            bool in = false;
            int j = f + lane;
            if (lane < c) {
                const float dx = qdiff(px, a.qx[j], bx.s[0]);
                const float dy = qdiff(py, a.qy[j], bx.s[1]);
                const float dz = qdiff(pz, a.qz[j], bx.s[2]);
                const float r2 = dx * dx + dy * dy + dz * dz;
                in = r2 < lo2;
                if (!in && r2 <= hi2) {   // within the float band: decide in double
                    const double ex = fold64(__dsub_rn(a.xs[j], x), bx.L[0]);
                    const double ey = fold64(__dsub_rn(a.ys[j], y), bx.L[1]);
                    const double ez = fold64(__dsub_rn(a.zs[j], z), bx.L[2]);
                    in = r2_exact(ex, ey, ez) < h2;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, in);
            if (in && a.mode == 2) {
                const int pos = count + __popc(m & ((1u << lane) - 1u));
                if (pos < lim) out[pos] = j;
            }
            count += __popc(m);
        };
        const int root = a.box_root[a.pbox[s]];
        int sp = 0;
        if (root < a.nbucket_total) {
            scan_bucket(root);
        } else {
            if (lane == 0) stack[0] = root;
            sp = 1;
        }
        __syncwarp();
        bool stack_ovf = false;
        while (sp > 0) {
            sp--;
            const int node = stack[sp];
            __syncwarp();
            const int nf = a.node_first[node], nc = a.node_cnt[node];
            bool hit = false;
            if (lane < nc) {
                const uint4 l = a.lo[nf + lane], u = a.hi[nf + lane];
                const float gx = u2f(point_gap(px, l.x, u.x)) * bx.s[0];
                const float gy = u2f(point_gap(py, l.y, u.y)) * bx.s[1];
                const float gz = u2f(point_gap(pz, l.z, u.z)) * bx.s[2];
                hit = gx * gx + gy * gy + gz * gz <= hi2;
            }
            unsigned m = __ballot_sync(0xffffffffu, hit);
            if (nf < a.nbucket_total) {
                while (m) {
                    const int k = __ffs(m) - 1;
                    m &= m - 1;
                    scan_bucket(nf + k);
                }
                __syncwarp();
            } else {
                const int nh = __popc(m);
                if (sp + nh > STACK) {   // (cannot happen for trees of MAX_LEVELS levels)
                    stack_ovf = true;
                    break;
                }
                if (hit) stack[sp + __popc(m & ((1u << lane) - 1u))] = nf + lane;
                sp += nh;
                __syncwarp();
            }
        }
        if (stack_ovf) {
            if (lane == 0) set_flag(a.cnt, ST_STACK);
            continue;
        }
        if (a.mode == 1 && lane == 0) {
            const unsigned long long base =
                atomicAdd(&a.cnt->list_cursor, (unsigned long long)count);
            a.nbr_off[s] = (int64_t)base;
            a.nbr_cnt[s] = count;
            if ((int64_t)base + count > a.capacity) {
                set_flag(a.cnt, ST_LIST_CAPACITY);
                a.nbr_cnt[s] = 0;   // nothing stored for this list
            }
        }
        __syncwarp();
    }
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

// queue the buckets holding a particle with one of the bits set (bit 0: to
// search again, and then clear the search-failure flag that the rebuild
// answers)
__global__ void k_queue_active(int64_t nbucket, const int32_t *__restrict__ first,
                               const int32_t *__restrict__ cnt, const uint8_t *__restrict__ active,
                               int32_t *__restrict__ queue, int *__restrict__ nqueue,
                               DevCounters *counters, uint8_t bits = 1) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (bits == 1 && w0 == 0 && lane == 0) atomicAnd(&counters->flags, ~ST_SEARCH);
    // (warps stride over the buckets: a small grid covers every bucket)
    for (int64_t b = w0; b < nbucket; b += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        bool act = lane < cnt[b] && (active[first[b] + lane] & bits);
        if (__any_sync(0xffffffffu, act) && lane == 0) queue[atomicAdd(nqueue, 1)] = (int32_t)b;
    }
}

// The particles that hold a guard particle a in their list, i.e. r_ia < h_i
// (the list's own radius: the reverse of a's list), by one walk of the
// bucket tree per guard particle and warp.  The lanes test the children of
// a node at once: a child is entered when the lower bound of its periodic
// distance from a is within the largest search radius of its particles
// (hs >= h), or (use_h) within their largest h when the tree was built --
// the tighter bound for a guard round, where only the guard particles' h
// moved since, and each of those marks itself; the particles of an entered
// bucket are tested exactly, one per lane (the double-precision membership
// of the lists).  Marks ACT_REDO on them and on a itself.  Warps stride
// over the guard particles, whose count is read on the device.
// a guard round marks by scanning every list when it grew more than
// n / MARK_SCAN_RATIO particles (k_mark_by_lists), else by tree walks
constexpr int MARK_SCAN_RATIO = 1024;

__device__ __forceinline__ bool mark_by_scan(int nguard, int64_t n) {
    return (int64_t)nguard * MARK_SCAN_RATIO > n;
}

constexpr int RSTACK = 320;   // 32-ary tree of at most MAX_LEVELS levels
constexpr int RWARPS = 4;

__global__ void __launch_bounds__(RWARPS * 32)
k_mark_reverse(const int32_t *__restrict__ guard_idx, const int *__restrict__ nguard,
               const int32_t *__restrict__ node_first, const int32_t *__restrict__ node_cnt,
               const int32_t *__restrict__ box_root, int64_t nbucket,
               const uint4 *__restrict__ lo, const uint4 *__restrict__ hi,
               const uint32_t *__restrict__ qx, const uint32_t *__restrict__ qy,
               const uint32_t *__restrict__ qz, const double *__restrict__ xs,
               const double *__restrict__ ys, const double *__restrict__ zs,
               const double *__restrict__ h, const int32_t *__restrict__ pbox,
               const Box *__restrict__ boxes, uint8_t *__restrict__ active, DevCounters *cnt,
               bool use_h, int64_t nparticles) {
    __shared__ int stack_all[RWARPS][RSTACK];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *stack = stack_all[warp];
    const int ng = *nguard;
    // (a guard round with many grown particles marks by the list scan below)
    if (use_h && mark_by_scan(ng, nparticles)) return;
    const int nwarps = gridDim.x * RWARPS;
    for (int g = blockIdx.x * RWARPS + warp; g < ng; g += nwarps) {
        const int a = guard_idx[g];
        const Box bx = boxes[pbox[a]];
        const uint32_t pax = qx[a], pay = qy[a], paz = qz[a];
        const double xa = xs[a], ya = ys[a], za = zs[a];
        if (lane == 0) {
            active[a] |= ACT_REDO;
            stack[0] = box_root[pbox[a]];
        }
        int sp = 1;
        __syncwarp();
        while (sp > 0) {
            const int node = stack[--sp];
            __syncwarp();
            const int f = node_first[node], c = node_cnt[node];
            if (node < nbucket) {
                // a bucket: lane k tests its particle f + k
                const int i = f + lane;
                if (lane < c && i != a) {
                    const double ex = fold64(__dsub_rn(xa, xs[i]), bx.L[0]);
                    const double ey = fold64(__dsub_rn(ya, ys[i]), bx.L[1]);
                    const double ez = fold64(__dsub_rn(za, zs[i]), bx.L[2]);
                    const double hi_ = h[i];
                    if (r2_exact(ex, ey, ez) < __dmul_rn(hi_, hi_)) active[i] |= ACT_REDO;
                }
                continue;
            }
            bool hit = false;
            if (lane < c) {
                const uint4 l = lo[f + lane], u = hi[f + lane];
                const float rmax = __uint_as_float(use_h ? u.w : l.w) * 1.0001f;
                const float gx = u2f(point_gap(pax, l.x, u.x)) * bx.s[0];
                const float gy = u2f(point_gap(pay, l.y, u.y)) * bx.s[1];
                const float gz = u2f(point_gap(paz, l.z, u.z)) * bx.s[2];
                hit = gx * gx + gy * gy + gz * gz <= rmax * rmax;
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            const int np = __popc(m);
            if (sp + np > RSTACK) {   // (cannot happen for trees of MAX_LEVELS levels)
                if (lane == 0) set_flag(cnt, ST_STACK);
                break;
            }
            if (hit) stack[sp + __popc(m & ((1u << lane) - 1u))] = f + lane;
            sp += np;
            __syncwarp();
        }
        __syncwarp();
    }
}

// The same marks from the lists: particle i holds a guard particle a in its
// list iff r_ia < h_i falls within the list's radius, and every list is
// complete for r < h_i (after the density stage it holds its members and a
// few entries just beyond), so scanning each particle's own list for a
// guard flag marks every particle the walk would, plus a few whose
// recomputation gives back their unchanged values.  One pass over all lists
// costs about as much as the walks of n / MARK_SCAN_RATIO guard particles:
// each kernel reads the round's guard count on the device and only one of
// them works (the first round grows many particles, the later ones few).
// Eight lanes read a list together, eight consecutive entries (one 32-byte
// sector) at a time, so a warp scans four lists at once with whole-sector
// reads rather than one scattered entry per lane.
constexpr int MARK_GROUP = 8;

__global__ void __launch_bounds__(256)
k_mark_by_lists(int64_t n, const int *__restrict__ nguard, const int64_t *__restrict__ nbr_off,
                const int32_t *__restrict__ nbr_cnt, const int32_t *__restrict__ nbr_idx,
                const uint32_t *__restrict__ gbits, uint8_t *__restrict__ active) {
    if (!mark_by_scan(*nguard, n)) return;
    constexpr int PER_WARP = 32 / MARK_GROUP;
    const int lane = threadIdx.x & 31, sub = lane & (MARK_GROUP - 1);
    const unsigned gmask = ((1u << MARK_GROUP) - 1u) << (lane & ~(MARK_GROUP - 1));
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s0 = w * PER_WARP; s0 < n; s0 += nw * PER_WARP) {
        const int64_t s = s0 + lane / MARK_GROUP;
        int64_t o = 0;
        int c = 0;
        bool hit = false;
        if (s < n) {
            o = nbr_off[s];
            c = nbr_cnt[s];
            hit = (gbits[s >> 5] >> (s & 31)) & 1u;   // (a guard particle marks itself)
        }
        const int cmax = __reduce_max_sync(0xffffffffu, hit ? 0 : c);
        for (int k0 = 0; k0 < cmax; k0 += MARK_GROUP) {
            bool h = false;
            if (!hit && k0 + sub < c) {
                const int j = nbr_idx[o + k0 + sub];
                h = (gbits[j >> 5] >> (j & 31)) & 1u;
            }
            hit |= (__ballot_sync(0xffffffffu, h) & gmask) != 0u;
            if (__all_sync(0xffffffffu, hit || k0 + MARK_GROUP >= c)) break;
        }
        if (hit && sub == 0) active[s] |= ACT_REDO;
    }
}

// the guard round's particles as a bitmap (one bit per particle, a 32nd of
// the flag bytes: the scan's lookups stay in L1 and L2)
__global__ void k_guard_bits(const int32_t *__restrict__ guard_idx, const int *__restrict__ nguard,
                             uint32_t *__restrict__ gbits) {
    const int ng = *nguard;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ng; t += gridDim.x * blockDim.x) {
        const int s = guard_idx[t];
        atomicOr(&gbits[s >> 5], 1u << (s & 31));
    }
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t mark_guard_reverse(hydro_ctx *c, stream_t st) {
    HYD_CUDA(mark_reverse(c, st, true));
    const int64_t nw = (c->plan.n + 31) / 32;
    HYD_CUDA(c->d_guard_bits.ensure(nw));
    HYD_CUDA(cudaMemsetAsync(c->d_guard_bits.get(), 0, nw * sizeof(uint32_t), st));
    k_guard_bits<<<152 * 4, 256, 0, st>>>(c->d_guard_idx.get(), &c->d_cnt->nguard,
                                          c->d_guard_bits.get());
    HYD_CUDA(launch_check());
    k_mark_by_lists<<<SWEEP_GRID, 256, 0, st>>>(c->plan.n, &c->d_cnt->nguard, c->d_nbr_off.get(),
                                                c->d_nbr_cnt.get(), c->d_nbr_idx.get(),
                                                c->d_guard_bits.get(), c->d_active.get());
    return launch_check();
}

cudaError_t mark_reverse(hydro_ctx *c, stream_t st, bool use_h) {
    const Plan &P = c->plan;
    // (a latency-bound walk per guard particle: as many resident warps as
    // its 40 registers allow, 12 CTAs of 4 warps per SM)
    k_mark_reverse<<<152 * 12, RWARPS * 32, 0, st>>>(
        c->d_guard_idx.get(), &c->d_cnt->nguard, c->d_node_first.get(), c->d_node_cnt.get(),
        c->d_box_root.get(), P.nbucket, c->d_node_aabb.get(), c->d_node_aabb_hi.get(),
        c->d_qx.get(), c->d_qy.get(), c->d_qz.get(), c->d_xs.get(), c->d_ys.get(), c->d_zs.get(),
        c->d_hsorted.get(), c->d_pbox.get(), c->d_boxes.get(), c->d_active.get(), c->d_cnt,
        use_h, P.n);
    return launch_check();
}

cudaError_t build_tree(hydro_ctx *c, stream_t st) {
    const Plan &P = c->plan;
    k_aabb_leaf<<<grid_for(P.nbucket * 32, 256), 256, 0, st>>>(
        P.nbucket, c->d_node_first.get(), c->d_node_cnt.get(), c->d_qx.get(), c->d_qy.get(),
        c->d_qz.get(), c->d_hs.get(), c->d_hsorted.get(), c->d_node_aabb.get(),
        c->d_node_aabb_hi.get());
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

// the tree's radius bounds raised for the guard round's particles
// (guard_idx, count nguard on the device), the node levels recomputed
cudaError_t raise_tree(hydro_ctx *c, stream_t st) {
    const Plan &P = c->plan;
    k_aabb_raise<<<152 * 4, 256, 0, st>>>(c->d_guard_idx.get(), &c->d_cnt->nguard,
                                          c->d_node_first.get(), P.nbucket, c->d_hs.get(),
                                          c->d_hsorted.get(), c->d_node_aabb.get(),
                                          c->d_node_aabb_hi.get());
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
    // cap: slots per particle in the fixed-stride part of nbr_idx
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
    a.ovf_list = c->d_ovf.get();
    a.ovf_count = &c->d_cnt->ovf_buckets;
    a.nq_dev = false;
    return a;
}

static cudaError_t launch_lists(const ListArgs &a, int64_t nbucket, stream_t st) {
    size_t per_warp = STACK * 4 + 2 * STAGE_BYTES;
    size_t smem = per_warp * LIST_WARPS;
    k_build_lists<<<grid_for(nbucket, LIST_WARPS), LIST_WARPS * 32, smem, st>>>(a);
    return launch_check();
}

// one pass over all buckets; buckets with a row longer than cap are queued
// for build_lists_queued().  Layout of nbr_idx: particle s owns the slots [s cap, s cap + cap); lists
// longer than cap live in the overflow region that follows (n cap onwards),
// reserved by build_lists_queued.
cudaError_t build_lists(hydro_ctx *c, int cap, stream_t st) {
    const int64_t n = c->plan.n;
    HYD_CUDA(c->d_nbr_off.ensure(n + 1));
    HYD_CUDA(c->d_nbr_cnt.ensure(n));
    size_t need = (size_t)n * cap + (size_t)c->ovf_reserve;
    if (c->d_nbr_idx.cap < need) HYD_CUDA(c->d_nbr_idx.ensure(need + need / 8));
    HYD_CUDA(c->d_ovf.ensure(c->plan.nbucket));
    c->list_cap = cap;
    HYD_CUDA(set_u64(&c->d_cnt->list_cursor, (unsigned long long)n * cap, st));
    HYD_CUDA(cudaMemsetAsync(&c->d_cnt->ovf_buckets, 0, sizeof(int), st));
    return launch_lists(list_args(c, cap, 0), c->plan.nbucket, st);
}

// the queued buckets: count and reserve in the overflow region, then fill
cudaError_t build_lists_queued(hydro_ctx *c, int nq, stream_t st) {
    ListArgs a = list_args(c, c->list_cap, 1);
    a.nbucket = nq;   // warps index the queue
    HYD_CUDA(launch_lists(a, nq, st));
    a.mode = 2;
    return launch_lists(a, nq, st);
}

// the queued passes over as many warps as there are buckets; the count of
// queued buckets is read by the warps themselves
cudaError_t build_lists_queued_dev(hydro_ctx *c, stream_t st) {
    ListArgs a = list_args(c, c->list_cap, 1);
    a.nq_dev = true;
    HYD_CUDA(launch_lists(a, c->plan.nbucket, st));
    a.mode = 2;
    return launch_lists(a, c->plan.nbucket, st);
}

cudaError_t rebuild_active_lists_dev(hydro_ctx *c, stream_t st, bool guard) {
    // (in a guard round only guard particles can have left their radius)
    if (guard) return guard_particle_lists(c, st, true);
    const Plan &P = c->plan;
    HYD_CUDA(cudaMemsetAsync(&c->d_cnt->ovf_buckets, 0, sizeof(int), st));
    k_queue_active<<<std::min(grid_for(P.nbucket * 32, 256), SWEEP_GRID), 256, 0, st>>>(
        P.nbucket, c->d_node_first.get(), c->d_node_cnt.get(), c->d_active.get(), c->d_ovf.get(),
        &c->d_cnt->ovf_buckets, c->d_cnt);
    HYD_CUDA(launch_check());
    // (in a guard round only the guard particles' radii grew)
    HYD_CUDA(guard ? raise_tree(c, st) : build_tree(c, st));
    return build_lists_queued_dev(c, st);
}

// new lists (in the overflow region) for the buckets that hold a particle
// whose search radius grew; every other list stays as it is.  *nq receives
// the number of buckets rebuilt (the host waits for it).
cudaError_t rebuild_active_lists(hydro_ctx *c, int *nq, stream_t st, bool guard) {
    if (guard) {
        *nq = 0;   // (no bucket rebuilt: the re-searched particles' own lists)
        return guard_particle_lists(c, st, true);
    }
    const Plan &P = c->plan;
    HYD_CUDA(c->d_ovf.ensure(P.nbucket));
    HYD_CUDA(cudaMemsetAsync(&c->d_cnt->ovf_buckets, 0, sizeof(int), st));
    k_queue_active<<<std::min(grid_for(P.nbucket * 32, 256), SWEEP_GRID), 256, 0, st>>>(
        P.nbucket, c->d_node_first.get(), c->d_node_cnt.get(), c->d_active.get(), c->d_ovf.get(),
        &c->d_cnt->ovf_buckets, c->d_cnt);
    HYD_CUDA(launch_check());
    HYD_CUDA(cudaMemcpyAsync(nq, &c->d_cnt->ovf_buckets, sizeof(int), cudaMemcpyDeviceToHost, st));
    HYD_CUDA(cudaStreamSynchronize(st));
    if (*nq == 0) return cudaSuccess;
    // the buckets' search radii changed
    HYD_CUDA(build_tree(c, st));
    return build_lists_queued(c, *nq, st);
}

// new lists, in the overflow region, for the particles of guard_idx (the
// guard round's grown particles, count nguard on the device; only_search:
// only those flagged ACT_SOLVE by the re-search); the tree must hold the
// current positions (its search radii are not used).  Every other list
// stays as it is, compacted or not: a bucket rebuild would give the
// re-searched particles the same lists.
cudaError_t guard_particle_lists(hydro_ctx *c, stream_t st, bool only_search) {
    const Plan &P = c->plan;
    PartListArgs a;
    a.pidx = c->d_guard_idx.get();
    a.npidx = &c->d_cnt->nguard;
    a.active = only_search ? c->d_active.get() : nullptr;
    a.node_first = c->d_node_first.get();
    a.node_cnt = c->d_node_cnt.get();
    a.box_root = c->d_box_root.get();
    a.pbox = c->d_pbox.get();
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
    const unsigned grid = 152 * 8;
    for (int mode = 1; mode <= 2; mode++) {
        a.mode = mode;
        k_particle_lists<<<grid, PL_WARPS * 32, 0, st>>>(a);
        HYD_CUDA(launch_check());
    }
    return cudaSuccess;
}

cudaError_t queue_flagged(hydro_ctx *c, uint8_t bits, stream_t st) {
    const Plan &P = c->plan;
    HYD_CUDA(c->d_ovf.ensure(P.nbucket));
    HYD_CUDA(cudaMemsetAsync(&c->d_cnt->ovf_buckets, 0, sizeof(int), st));
    k_queue_active<<<std::min(grid_for(P.nbucket * 32, 256), SWEEP_GRID), 256, 0, st>>>(
        P.nbucket, c->d_node_first.get(), c->d_node_cnt.get(), c->d_active.get(), c->d_ovf.get(),
        &c->d_cnt->ovf_buckets, c->d_cnt, bits);
    return launch_check();
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
