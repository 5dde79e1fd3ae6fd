// Core quantities from a sample's nearest neighbours (Sec. 4: a random sample
// of min(N, sqrt(5000 N)) particles, a brute-force search for each sampled
// particle's 6 nearest neighbours, and the density estimator and
// density-weighted averages of Casertano & Hut, which the paper cites).
//
// Search (p3t_sample_knn6): one thread per sampled particle walks the built
// tree (one cluster) depth first.  It opens a node unless the FP32 distance from
// the particle to the node's box exceeds the filter threshold below, and tests
// the particles of the opened leaves.  A node whose box lies beyond an upper
// bound of the 6th distance holds no candidate, so the result is that of the
// brute-force search, which p3t_sample_knn6_brute performs as the paper does:
// every sampled particle against every particle, blocks pairing 128 sampled
// particles with one chunk of candidates in key order (staged through shared
// memory), a second kernel merging the chunks' lists.
//
// Both test each candidate first in FP32 on double-single coordinates relative
// to the frame centre (the hi parts of the tree's splits; the brute-force scan
// takes two candidates per packed FP32x2 instruction): a candidate whose FP32
// squared distance exceeds an upper bound of the current 6th distance, widened
// by the filter's error, cannot enter the list.  The others are decided with the
// exact FP64 distance (dx*dx + dy*dy) + dz*dz and inserted by (distance,
// original index).  The result is unique, so it equals the oracle's bit for bit.
#include <cstdint>
#include <cmath>

#include "p3t_internal.cuh"

namespace p3t {

constexpr int kKnn = 6;
constexpr int kKnnThreads = 128;
constexpr int kKnnTile = 256;

struct KnnArgs {
    Tree T;
    int n, s;
    const int32_t *sample;
    int chunk;             // candidates per chunk
    int n_chunks;
    double *part_d2;       // [s][n_chunks][6]
    int32_t *part_idx;
};

// (d, i) < (e, j) in the order of the lists: distance, then original index
__device__ __forceinline__ bool knn_less(double d, int i, double e, int j)
{
    return d < e || (d == e && i < j);
}

__device__ __forceinline__ void knn_insert(double (&bd)[kKnn], int (&bi)[kKnn], double d, int i)
{
    if (!knn_less(d, i, bd[kKnn - 1], bi[kKnn - 1])) return;
    bd[kKnn - 1] = d, bi[kKnn - 1] = i;
#pragma unroll
    for (int q = kKnn - 1; q > 0; q--) {
        if (knn_less(bd[q], bi[q], bd[q - 1], bi[q - 1])) {
            const double td = bd[q];
            const int ti = bi[q];
            bd[q] = bd[q - 1], bi[q] = bi[q - 1];
            bd[q - 1] = td, bi[q - 1] = ti;
        }
    }
}

// FP32 filter threshold for candidates that may enter a list whose 6th squared
// distance is at most lim.  The test uses only the hi parts of the splits: every
// coordinate difference is then within 2u R (both roundings to FP32, u = 2^-24,
// R the frame's half-size) plus u of itself of the exact one, so a candidate at
// exact distance r has an FP32 squared distance of at most
// ((1 + u) r + sqrt(3) 2u R)^2 (1 + 3u) (triangle inequality over the three
// coordinates); thr covers that with sqrt(lim) (1 + 8u) + 4u R and (1 + 32u).
__device__ __forceinline__ float knn_threshold(double lim, float eR)
{
    if (!(lim < INFINITY)) return INFINITY;
    const float s = sqrtf((float)lim) * (1.f + 8.f * kFp32U) + eR;
    return s * s * (1.f + 32.f * kFp32U);
}

__global__ void __launch_bounds__(kKnnThreads) knn_chunk_kernel(KnnArgs a)
{
    // candidates in pairs (hi parts relative to the frame centre): {x0 x1 y0 y1}, {z0 z1}
    __shared__ float4 sxy[kKnnTile / 2];
    __shared__ float2 sz[kKnnTile / 2];
    const Tree &T = a.T;
    const int t = blockIdx.x * kKnnThreads + threadIdx.x;
    const int c = blockIdx.y;
    bool active = t < a.s;
    int me = -1, km = 0;
    float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
    double4_32a p = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    if (active) {
        me = a.sample[t];
        if ((unsigned)me >= (unsigned)a.n) {  // not a particle: no list
            if (c == 0) latch_error(T.meta, P3T_ERR_INVALID_INPUT);
            active = false;
            me = -1;
        } else {
            km = T.inv[me];
            h = T.ph[km];
            p = T.sp[km];
        }
    }
    const float eR = 4.f * kFp32U * (float)T.cl[0].frame[3];
    double bd[kKnn];
    int bi[kKnn];
    // upper bound of the 6th distance: the 6th nearest among the 32 particles next
    // to this one in key order (spatial neighbours); no nearer-than-true neighbour
    // is lost, since the true 6th distance is at most this one
    double bound = INFINITY;
    if (active) {
#pragma unroll
        for (int q = 0; q < kKnn; q++) bd[q] = INFINITY, bi[q] = 0x7fffffff;
        const int lo = max(0, km - 16), hi = min(a.n, km + 17);
        for (int kj = lo; kj < hi; kj++) {
            if (kj == km) continue;
            const double4_32a pj = T.sp[kj];
            const double ex = dsub(pj.x, p.x), ey = dsub(pj.y, p.y), ez = dsub(pj.z, p.z);
            knn_insert(bd, bi, dadd(dadd(dmul(ex, ex), dmul(ey, ey)), dmul(ez, ez)), kj);
        }
        bound = bd[kKnn - 1];
    }
#pragma unroll
    for (int q = 0; q < kKnn; q++) bd[q] = INFINITY, bi[q] = 0x7fffffff;
    // FP32 squared distances above this cannot enter the list
    float thr = knn_threshold(bound, eR);
    const float2 NX = make_float2(-h.x, -h.x), NY = make_float2(-h.y, -h.y), NZ = make_float2(-h.z, -h.z);
    const int k0 = c * a.chunk, k1 = min(a.n, k0 + a.chunk);
    for (int base = k0; base < k1; base += kKnnTile) {
        const int nt = min(kKnnTile, k1 - base);
        const int np = (nt + 1) >> 1;
        __syncthreads();
        for (int q = threadIdx.x; q < np; q += kKnnThreads) {
            const float4 a0 = T.ph[base + 2 * q];
            // an odd tail's partner sits far away: never within any threshold
            const float4 a1 = 2 * q + 1 < nt ? T.ph[base + 2 * q + 1] : make_float4(1e30f, 1e30f, 1e30f, 0.f);
            sxy[q] = make_float4(a0.x, a1.x, a0.y, a1.y);
            sz[q] = make_float2(a0.z, a1.z);
        }
        __syncthreads();
        if (!active) continue;
#pragma unroll 4
        for (int q = 0; q < np; q++) {
            const float4 xy = sxy[q];
            const float2 dx = __fadd2_rn(make_float2(xy.x, xy.y), NX);
            const float2 dy = __fadd2_rn(make_float2(xy.z, xy.w), NY);
            const float2 dz = __fadd2_rn(sz[q], NZ);
            float2 r2 = __fmul2_rn(dx, dx);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            if (fminf(r2.x, r2.y) <= thr) {  // one of the two may enter the list: decide exactly
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    const int kj = base + 2 * q + e;
                    if ((e ? r2.y : r2.x) <= thr && 2 * q + e < nt) {
                        const int oj = T.perm[kj];
                        if (oj != me) {
                            const double4_32a pj = T.sp[kj];
                            const double ex = dsub(pj.x, p.x), ey = dsub(pj.y, p.y), ez = dsub(pj.z, p.z);
                            const double d2 = dadd(dadd(dmul(ex, ex), dmul(ey, ey)), dmul(ez, ez));
                            knn_insert(bd, bi, d2, oj);
                            thr = knn_threshold(fmin(bd[kKnn - 1], bound), eR);
                        }
                    }
                }
            }
        }
    }
    if (active) {
        const size_t o = ((size_t)t * a.n_chunks + c) * kKnn;
#pragma unroll
        for (int q = 0; q < kKnn; q++) a.part_d2[o + q] = bd[q], a.part_idx[o + q] = bi[q];
    }
}

__global__ void knn_merge_kernel(KnnArgs a, int32_t *nn_idx, double *nn_d2)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < a.s; t += gridDim.x * blockDim.x) {
        double bd[kKnn];
        int bi[kKnn];
#pragma unroll
        for (int q = 0; q < kKnn; q++) bd[q] = INFINITY, bi[q] = 0x7fffffff;
        for (int c = 0; c < a.n_chunks; c++) {
            const size_t o = ((size_t)t * a.n_chunks + c) * kKnn;
            for (int q = 0; q < kKnn; q++) knn_insert(bd, bi, a.part_d2[o + q], a.part_idx[o + q]);
        }
#pragma unroll
        for (int q = 0; q < kKnn; q++) {
            const bool found = bd[q] < INFINITY;
            nn_idx[(size_t)t * kKnn + q] = found ? bi[q] : -1;
            nn_d2[(size_t)t * kKnn + q] = bd[q];
        }
    }
}

// The 6 nearest neighbours of sampled particle t by a depth-first walk of the
// tree.  A point-box test in FP32 on the walk record's box (relative to the
// frame centre) and the hi part of the particle's split has the same error as
// the candidates' filter (each coordinate difference within 2u R + u of itself
// of the exact one; max(., 0) adds none), so a node whose FP32 box distance
// exceeds the threshold holds no particle within the bound.
constexpr int kKnnStack = 192;  // 7 open siblings a level over 22 levels, and the root
__global__ void __launch_bounds__(kKnnThreads) knn_tree_kernel(Tree T, int n, int s,
                                                               const int32_t *sample,
                                                               int32_t *nn_idx, double *nn_d2)
{
    const int t = blockIdx.x * kKnnThreads + threadIdx.x;
    if (t >= s) return;
    const int me = sample[t];
    if ((unsigned)me >= (unsigned)n) {  // not a particle: no list
        latch_error(T.meta, P3T_ERR_INVALID_INPUT);
        return;
    }
    const int km = T.inv[me];
    const float4 h = T.ph[km];
    const double4_32a p = T.sp[km];
    const float eR = 4.f * kFp32U * (float)T.cl[0].frame[3];
    double bd[kKnn];
    int bi[kKnn];
    // upper bound of the 6th distance from the 32 particles next in key order
#pragma unroll
    for (int q = 0; q < kKnn; q++) bd[q] = INFINITY, bi[q] = 0x7fffffff;
    {
        const int lo = max(0, km - 16), hi = min(n, km + 17);
        for (int kj = lo; kj < hi; kj++) {
            if (kj == km) continue;
            const double4_32a pj = T.sp[kj];
            const double ex = dsub(pj.x, p.x), ey = dsub(pj.y, p.y), ez = dsub(pj.z, p.z);
            knn_insert(bd, bi, dadd(dadd(dmul(ex, ex), dmul(ey, ey)), dmul(ez, ez)), kj);
        }
    }
    const double bound = bd[kKnn - 1];
#pragma unroll
    for (int q = 0; q < kKnn; q++) bd[q] = INFINITY, bi[q] = 0x7fffffff;
    float thr = knn_threshold(bound, eR);
    int stk[kKnnStack];
    int sp = 0;
    stk[sp++] = 0;  // the root of the one cluster
    const int nn = T.meta->n_nodes;
    while (sp > 0) {
        const int node = stk[--sp];
        const auto w = wrec_at(T.wn, node);
        const float4 b = w[1], c = w[2];  // box lo - O and child / particle start; box hi - O and count
        const float tx = fmaxf(fmaxf(b.x - h.x, h.x - c.x), 0.f);
        const float ty = fmaxf(fmaxf(b.y - h.y, h.y - c.y), 0.f);
        const float tz = fmaxf(fmaxf(b.z - h.z, h.z - c.z), 0.f);
        if (tx * tx + ty * ty + tz * tz > thr) continue;
        const int info = __float_as_int(b.w), cnt = __float_as_int(c.w);
        if (info < 0) {  // leaf: particles [-1 - info, + cnt) in key order
            const int k0 = -1 - info;
            if (cnt < 1 || k0 + cnt > n) {
                latch_error(T.meta, P3T_ERR_INTERNAL);
                break;
            }
            for (int kj = k0; kj < k0 + cnt; kj++) {
                const float4 hj = T.ph[kj];
                const float dx = hj.x - h.x, dy = hj.y - h.y, dz = hj.z - h.z;
                if (dx * dx + dy * dy + dz * dz > thr) continue;
                const int oj = T.perm[kj];
                if (oj == me) continue;
                const double4_32a pj = T.sp[kj];
                const double ex = dsub(pj.x, p.x), ey = dsub(pj.y, p.y), ez = dsub(pj.z, p.z);
                knn_insert(bd, bi, dadd(dadd(dmul(ex, ex), dmul(ey, ey)), dmul(ez, ez)), oj);
                thr = knn_threshold(fmin(bd[kKnn - 1], bound), eR);
            }
        } else {
            if (cnt < 1 || cnt > 8 || info + cnt > nn || sp + cnt > kKnnStack) {
                latch_error(T.meta, P3T_ERR_INTERNAL);
                break;
            }
            for (int q = cnt - 1; q >= 0; q--) stk[sp++] = info + q;  // octant 0 on top
        }
    }
#pragma unroll
    for (int q = 0; q < kKnn; q++) {
        const bool found = bd[q] < INFINITY;
        nn_idx[(size_t)t * kKnn + q] = found ? bi[q] : -1;
        nn_d2[(size_t)t * kKnn + q] = bd[q];
    }
}

// ---- core quantities (one block, fixed reduction order) ---------------------
constexpr int kCoreThreads = 1024;

__device__ double block_sum_d(double v, double *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sh[32] = s;
    }
    __syncthreads();
    return sh[32];
}

struct CoreArgs {
    int n, s;
    const double *x, *y, *z, *m;
    const int32_t *sample, *idx6;
    const double *d26;
    double *rho, *out;
    unsigned long long *count;
    Meta *meta;
};

__global__ void __launch_bounds__(kCoreThreads) core_sums_kernel(CoreArgs a)
{
    __shared__ double sh[33];
    const double four_pi_3 = 4.0 * 3.14159265358979323846 / 3.0;
    double w = 0.0, w2 = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
    bool bad = false;
    for (int t = threadIdx.x; t < a.s; t += blockDim.x) {
        double mass = 0.0;
        for (int q = 0; q < 5; q++) {
            const int j = a.idx6[6 * t + q];
            if (j == -1) continue;  // fewer than 6 neighbours: d2 = inf, rho = 0
            if ((unsigned)j >= (unsigned)a.n) {
                bad = true;
                continue;
            }
            mass = dadd(mass, a.m[j]);
        }
        const double r6 = dsqrt(a.d26[6 * t + 5]);
        const double r = ddiv(mass, dmul(four_pi_3, dmul(dmul(r6, r6), r6)));
        const int i = a.sample[t];
        if ((unsigned)i >= (unsigned)a.n) {  // not a particle: weight 0
            bad = true;
            a.rho[t] = 0.0;
            continue;
        }
        a.rho[t] = r;
        w = dadd(w, r), w2 = dadd(w2, dmul(r, r));
        cx = dadd(cx, dmul(r, a.x[i])), cy = dadd(cy, dmul(r, a.y[i])), cz = dadd(cz, dmul(r, a.z[i]));
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) latch_error(a.meta, P3T_ERR_INVALID_INPUT);
    w = block_sum_d(w, sh);
    w2 = block_sum_d(w2, sh);
    cx = ddiv(block_sum_d(cx, sh), w);
    cy = ddiv(block_sum_d(cy, sh), w);
    cz = ddiv(block_sum_d(cz, sh), w);
    double acc = 0.0;
    for (int t = threadIdx.x; t < a.s; t += blockDim.x) {
        const int i = a.sample[t];
        if ((unsigned)i >= (unsigned)a.n) continue;
        const double dx = dsub(a.x[i], cx), dy = dsub(a.y[i], cy), dz = dsub(a.z[i], cz);
        const double r = a.rho[t];
        acc = dadd(acc, dmul(dmul(r, r), dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz))));
    }
    acc = block_sum_d(acc, sh);
    if (threadIdx.x == 0) {
        a.out[0] = cx, a.out[1] = cy, a.out[2] = cz;
        a.out[3] = dsqrt(ddiv(acc, w2));
        a.out[4] = ddiv(w2, w);
        *a.count = 0ULL;
    }
}

__global__ void core_count_kernel(CoreArgs a)
{
    const double cx = a.out[0], cy = a.out[1], cz = a.out[2], rc = a.out[3];
    const double rc2 = dmul(rc, rc);
    unsigned int cnt = 0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.n; j += gridDim.x * blockDim.x) {
        const double dx = dsub(a.x[j], cx), dy = dsub(a.y[j], cy), dz = dsub(a.z[j], cz);
        cnt += dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz)) < rc2;
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(a.count, (unsigned long long)cnt);
}

__global__ void core_finish_kernel(CoreArgs a)
{
    a.out[5] = (double)*a.count;
}

}  // namespace p3t

using namespace p3t;

extern "C" {

int p3t_sample_knn6(p3t_ctx *c, int64_t n, int64_t s, const int32_t *sample, int32_t *nn_idx,
                    double *nn_d2)
{
    if (!c || !sample || !nn_idx || !nn_d2 || n <= 0 || s <= 0 || s > n) return P3T_ERR_INVALID_ARG;
    if (!c->built || c->n != n || c->tree.n_clusters != 1) return P3T_ERR_ORDER;
    knn_tree_kernel<<<(int)((s + kKnnThreads - 1) / kKnnThreads), kKnnThreads, 0, c->stream>>>(
        c->tree, (int)n, (int)s, sample, nn_idx, nn_d2);
    return check_launch(c);
}

int p3t_sample_knn6_brute(p3t_ctx *c, int64_t n, int64_t s, const int32_t *sample, int32_t *nn_idx,
                          double *nn_d2)
{
    if (!c || !sample || !nn_idx || !nn_d2 || n <= 0 || s <= 0 || s > n) return P3T_ERR_INVALID_ARG;
    if (!c->built || c->n != n || c->tree.n_clusters != 1) return P3T_ERR_ORDER;
    // chunks so that the grid covers the GPU about four times over
    const int sblocks = (int)((s + kKnnThreads - 1) / kKnnThreads);
    int chunks = (4 * 4 * c->sm_count + sblocks - 1) / sblocks;
    if (chunks < 1) chunks = 1;
    if (chunks > 64) chunks = 64;
    const size_t need = (size_t)s * chunks * kKnn * (sizeof(double) + sizeof(int32_t));
    if (c->knn_bytes < need) {
        if (c->knn_buf) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->knn_buf);
            c->knn_buf = nullptr;
            c->knn_bytes = 0;
        }
        if (cudaMalloc(&c->knn_buf, need) != cudaSuccess) {
            cudaGetLastError();
            return P3T_ERR_OOM;
        }
        c->knn_bytes = need;
    }
    KnnArgs a;
    a.T = c->tree;
    a.n = (int)n;
    a.s = (int)s;
    a.sample = sample;
    a.n_chunks = chunks;
    a.chunk = (int)((n + chunks - 1) / chunks);
    a.part_d2 = (double *)c->knn_buf;
    a.part_idx = (int32_t *)((char *)c->knn_buf + (size_t)s * chunks * kKnn * sizeof(double));
    dim3 grid(sblocks, chunks);
    knn_chunk_kernel<<<grid, kKnnThreads, 0, c->stream>>>(a);
    knn_merge_kernel<<<(int)((s + 255) / 256), 256, 0, c->stream>>>(a, nn_idx, nn_d2);
    return check_launch(c);
}

int p3t_core_quantities(p3t_ctx *c, int64_t n, const double *x, const double *y, const double *z,
                        const double *m, int64_t s, const int32_t *sample, const int32_t *nn_idx,
                        const double *nn_d2, double *rho, double *out)
{
    if (!c || !x || !y || !z || !m || !sample || !nn_idx || !nn_d2 || !rho || !out || n <= 0 ||
        s <= 0 || n >= (1LL << 31) - 1 || s >= (1LL << 31) - 1)
        return P3T_ERR_INVALID_ARG;
    if (!c->meta) return P3T_ERR_ORDER;
    CoreArgs a;
    a.n = (int)n, a.s = (int)s;
    a.x = x, a.y = y, a.z = z, a.m = m;
    a.sample = sample, a.idx6 = nn_idx, a.d26 = nn_d2;
    a.rho = rho, a.out = out;
    a.count = &c->meta->core_count;
    a.meta = c->meta;
    core_sums_kernel<<<1, kCoreThreads, 0, c->stream>>>(a);
    const long long want = (n + 255) / 256;
    core_count_kernel<<<(int)(want < 8LL * c->sm_count ? want : 8LL * c->sm_count), 256, 0, c->stream>>>(a);
    core_finish_kernel<<<1, 1, 0, c->stream>>>(a);
    return check_launch(c);
}

}  // extern "C"
