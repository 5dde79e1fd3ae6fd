// Tree build of the distant-force path (Sec. 2.4: Barnes-Hut tree).
//
// Steps (all on the context's stream, no host synchronisation):
//   bbox      FP64 min/max over x, y, z (order-preserving integer atomics),
//             input validation (finite x, y, z, m; m >= 0)
//   keys      q_d = floor((x_d - min_d) * 2^21/side), clamped, interleaved
//             into a 63-bit Morton key (bit 3k+2 <- q_x, 3k+1 <- q_y, 3k <- q_z)
//   sort      stable LSD radix sort of (key, index), 8 passes of 8 bits
//   gather    particles in key order as double4_32a {x, y, z, m}
//   topology  canonical octree (a node at level l is split iff it holds more
//             than leaf_cap particles and l < 21; children are the non-empty
//             octants, numbered breadth first): from each particle's first and
//             last levels and one scan of per-tile node counts, or level by level
//             with a look-back scan per level for a rank's range build; walk-group
//             starts are flagged on the way
//   groups    flags -> scan -> ranges, tight FP64 boxes
//   moments   bottom-up: each leaf sums its particles in key order, the last
//             child to finish combines its parent's children in octant order
//             (mass, COM, traceless quadrupole, box, opening radius)
// Every FP64 operation that feeds a decision uses round-to-nearest intrinsics
// with no contraction, so keys, topology, COMs, boxes and opening radii are
// reproducible bit for bit.
#include <cstdint>

#include "build_common.cuh"

namespace p3t {

constexpr int kBuildThreads = 256;
constexpr int kSortTile = kSortTileItems;
constexpr int kSortItems = kSortTile / kBuildThreads;

int topo_status_stride(long long n);

// ---------------------------------------------------------------------------
// metadata reset
__global__ void init_meta_kernel(Meta *m)
{
    int t = threadIdx.x;
    if (t < kMaxLevelSlots) {
        m->level_start[t] = 0;
        m->level_count[t] = 0;
    }
    if (t < 32) m->tickets[t] = 0;
    if (t == 0) {
        m->n_nodes = 0;
        m->n_groups = 0;
        m->n_leaves = 0;
        m->depth = 0;
        m->fallback_tests = 0;
        m->uncounted = 0;
    }
}

__global__ void init_clusters_kernel(Cluster *cl, int C)
{
    pdl_wait();
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x)
        for (int d = 0; d < 3; d++) {
            cl[c].minmax[d] = ~0ULL;   // running minimum
            cl[c].minmax[3 + d] = 0;   // running maximum
        }
}

// physics of every cluster: the batch's table {theta, r_in, r_out, r_list} or the
// context's values, with the derived constants the walk and neighbour kernels use
__global__ void cluster_params_kernel(Cluster *cl, int C, const double *__restrict__ prm,
                                      double theta, double r_in, double r_out, double r_list,
                                      Meta *meta)
{
    pdl_wait();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    double th = theta, ri = r_in, ro = r_out, rl = r_list;
    if (prm) {
        th = prm[4 * c], ri = prm[4 * c + 1], ro = prm[4 * c + 2], rl = prm[4 * c + 3];
        const bool ok = th >= 0.0 && isfinite(th) && ri >= 0.0 && ro > ri && isfinite(ro) &&
                        rl >= 0.0 && isfinite(rl);
        if (!ok) {
            latch_error(meta, P3T_ERR_INVALID_INPUT);
            th = theta, ri = r_in, ro = r_out, rl = r_list;
        }
    }
    Cluster &K = cl[c];
    K.theta = th;
    K.r_in = ri;
    K.r_out = ro;
    K.r_list = rl;
    K.inv_dr_d = ddiv(1.0, dsub(ro, ri));
    K.rout2_d = dmul(ro, ro);
    K.rl2_d = dmul(rl, rl);
    K.inv_dr_f = (float)K.inv_dr_d;
    K.rin_dr_f = (float)dmul(ri, K.inv_dr_d);
    K.rout2_f = (float)K.rout2_d;
    K.rl2_f = (float)K.rl2_d;
    K.rl_f = (float)rl;
    K.counted = rl > 0.0;  // the mixed walk counts every list radius (shell ranges beyond r_out)
    if (!K.counted) atomicAdd(&meta->uncounted, 1);
}

// cluster of every particle from the offsets (validated: 0 = seg[0] < ... < seg[C] = n)
__global__ void __launch_bounds__(kBuildThreads)
    cid_kernel(int n, int C, const int64_t *__restrict__ seg, int32_t *__restrict__ cid, Meta *meta)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= C && i < C + 1) {
        const long long v = seg[i];
        const bool ok = (i == 0 ? v == 0 : v > seg[i - 1]) && (i < C || v == n);
        if (!ok) latch_error(meta, P3T_ERR_INVALID_INPUT);
    }
    if (i >= n) return;
    int lo = 0, hi = C;  // last c with seg[c] <= i
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (seg[mid] <= i)
            lo = mid;
        else
            hi = mid;
    }
    cid[i] = lo;
}

// isfinite(v) and (for a finite v) v >= 0, tested on the bits (no FP64 instruction)
__device__ __forceinline__ bool finite_bits(double v)
{
    return ((unsigned long long)__double_as_longlong(v) & 0x7ff0000000000000ULL) != 0x7ff0000000000000ULL;
}
__device__ __forceinline__ bool nonneg_bits(double v)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) == 0 || u == 0x8000000000000000ULL;  // -0 >= 0
}

// Per-cluster bounding box (exact, order-preserving integer min/max) and input
// validation.  Each warp keeps running minima and maxima for its current cluster
// in registers across its grid-stride iterations and reduces them into the
// cluster table (warp shuffle + 6 atomics) only when the cluster changes and at
// the end; a warp whose 32 particles straddle a cluster boundary updates the
// table per lane for that iteration.
__global__ void __launch_bounds__(kBuildThreads)
    bbox_kernel(int n, const double *__restrict__ x, const double *__restrict__ y,
                const double *__restrict__ z, const double *__restrict__ m,
                const int32_t *__restrict__ cid, Cluster *cl, Meta *meta)
{
    pdl_wait();
    const int lane = threadIdx.x & 31;
    bool bad = false;
    int cur = -1;  // cluster of the running extrema (warp-uniform)
    unsigned long long mn[3] = {~0ULL, ~0ULL, ~0ULL}, mx[3] = {0, 0, 0};
    auto flush = [&]() {
        if (cur < 0) return;
#pragma unroll
        for (int d = 0; d < 3; d++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long a = __shfl_xor_sync(0xffffffffu, mn[d], o);
                const unsigned long long bb = __shfl_xor_sync(0xffffffffu, mx[d], o);
                mn[d] = a < mn[d] ? a : mn[d];
                mx[d] = bb > mx[d] ? bb : mx[d];
            }
        }
        if (lane == 0)
#pragma unroll
            for (int d = 0; d < 3; d++) {
                atomicMin(&cl[cur].minmax[d], mn[d]);
                atomicMax(&cl[cur].minmax[3 + d], mx[d]);
            }
#pragma unroll
        for (int d = 0; d < 3; d++) mn[d] = ~0ULL, mx[d] = 0;
        cur = -1;
    };
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += (long long)gridDim.x * blockDim.x) {
        const long long i = base + lane;
        unsigned long long e[3] = {~0ULL, ~0ULL, ~0ULL};
        bool ok = false;
        int c = -1;
        if (i < n) {
            const double p[3] = {x[i], y[i], z[i]};
            const double mi = m[i];
            ok = finite_bits(p[0]) && finite_bits(p[1]) && finite_bits(p[2]) && finite_bits(mi) &&
                 nonneg_bits(mi);
            bad |= !ok;
            c = cid ? cid[i] : 0;
            if (ok)
#pragma unroll
                for (int d = 0; d < 3; d++) e[d] = enc_double(p[d]);
        }
        const int c0 = __shfl_sync(0xffffffffu, c, 0);
        if (__all_sync(0xffffffffu, c < 0 || c == c0)) {
            if (c0 != cur) {
                flush();
                cur = c0;
            }
            if (ok)
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    mn[d] = e[d] < mn[d] ? e[d] : mn[d];
                    mx[d] = e[d] > mx[d] ? e[d] : mx[d];
                }
        } else if (ok) {  // a cluster boundary inside this warp's 32 particles
#pragma unroll
            for (int d = 0; d < 3; d++) {
                atomicMin(&cl[c].minmax[d], e[d]);
                atomicMax(&cl[c].minmax[3 + d], e[d]);
            }
        }
    }
    flush();
    if (__any_sync(0xffffffffu, bad) && lane == 0) latch_error(meta, P3T_ERR_INVALID_INPUT);
}

// rule 1 per cluster: the bounding cube, and the frame of the FP32 walk filter
__global__ void cube_kernel(Cluster *cl, int C)
{
    pdl_wait();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    Cluster &K = cl[c];
    double lo[3], hi[3], side = 0.0;
    for (int d = 0; d < 3; d++) {
        lo[d] = dec_double(K.minmax[d]);
        hi[d] = dec_double(K.minmax[3 + d]);
        if (K.minmax[d] == ~0ULL) lo[d] = hi[d] = 0.0;  // no valid particle
        double ext = dsub(hi[d], lo[d]);
        if (ext > side) side = ext;
    }
    if (side == 0.0) side = 1.0;
    double R = 0.0;
    for (int d = 0; d < 3; d++) {
        K.cube[d] = lo[d];
        double o = dmul(0.5, dadd(lo[d], hi[d]));
        K.frame[d] = o;
        R = dmax(R, dmax(dsub(hi[d], o), dsub(o, lo[d])));
    }
    K.cube[3] = side;
    K.scale = ddiv(2097152.0, side);
    // |x - O| <= R for every particle; pad for the rounding of O
    K.frame[3] = R * (1.0 + 1e-9) + 1e-300;
}

__global__ void __launch_bounds__(kBuildThreads)
    keys_kernel(int n, const double *__restrict__ x, const double *__restrict__ y,
                const double *__restrict__ z, const int32_t *__restrict__ cid,
                const Cluster *__restrict__ cl, uint64_t *__restrict__ keys,
                int32_t *__restrict__ perm)
{
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Cluster &K = cl[cid ? cid[i] : 0];
    const double s = K.scale;  // 2^21 / side
    unsigned long long qx = quantise(x[i], K.cube[0], s);
    unsigned long long qy = quantise(y[i], K.cube[1], s);
    unsigned long long qz = quantise(z[i], K.cube[2], s);
    keys[i] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
    perm[i] = i;
}

// ---------------------------------------------------------------------------
// radix sort: per-block digit histograms, a scan, then a stable scatter
// digit of an item: bits [shift, shift+8) of the key, or of the cluster id of its
// payload (the stable passes that group a batched build by cluster)
__device__ __forceinline__ int sort_digit(uint64_t key, int32_t val, int shift,
                                          const int32_t *__restrict__ cid)
{
    return cid ? (cid[val] >> shift) & 255 : (int)((key >> shift) & 255);
}

__global__ void __launch_bounds__(kBuildThreads)
    sort_hist_kernel(int n, const uint64_t *__restrict__ keys, const int32_t *__restrict__ vals,
                     const int32_t *__restrict__ cid, int shift, int nblocks,
                     int32_t *__restrict__ hist, unsigned long long *scan_status, int scan_words,
                     unsigned int *scan_ticket)
{
    pdl_wait();
    __shared__ int cnt[256];
    if (blockIdx.x == 0) clear_scan_state(scan_status, scan_words, scan_ticket);  // the digit scan's
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int k = 0; k < kSortItems; k++) {
        long long i = base + k * kBuildThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[sort_digit(keys[i], vals[i], shift, cid)], 1);
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kBuildThreads)
    sort_scatter_kernel(int n, const uint64_t *__restrict__ kin, const int32_t *__restrict__ vin,
                        uint64_t *__restrict__ kout, int32_t *__restrict__ vout,
                        const int32_t *__restrict__ cid, int shift, int nblocks,
                        const int32_t *__restrict__ hist_off)
{
    pdl_wait();
    constexpr int W = kBuildThreads / 32;
    __shared__ int gofs[256];
    __shared__ int wcnt[W][256];
    __shared__ int pofs[W][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    gofs[tid] = hist_off[tid * nblocks + blockIdx.x];
#pragma unroll
    for (int w = 0; w < W; w++) wcnt[w][tid] = 0;
    // every item of the tile is loaded before the ranking rounds
    const long long base = (long long)blockIdx.x * kSortTile;
    uint64_t key[kSortItems];
    int32_t val[kSortItems];
    int dig[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        const long long i = base + r * kBuildThreads + tid;
        const bool valid = i < n;
        key[r] = valid ? kin[i] : 0;
        val[r] = valid ? vin[i] : 0;
    }
#pragma unroll
    for (int r = 0; r < kSortItems; r++)
        dig[r] = base + r * kBuildThreads + tid < n ? sort_digit(key[r], val[r], shift, cid) : 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        const bool valid = base + r * kBuildThreads + tid < n;
        const int d = dig[r];
        // lanes of this warp holding the same digit: one ballot per digit bit
        unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int b = 0; b < 8; b++) {
            const bool bit = (d >> b) & 1;
            const unsigned bal = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bal : ~bal;
        }
        const int wrank = __popc(peers & lt);
        if (valid && wrank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            int s = gofs[tid];
#pragma unroll
            for (int w = 0; w < W; w++) {
                int c = wcnt[w][tid];
                pofs[w][tid] = s;
                wcnt[w][tid] = 0;
                s += c;
            }
            gofs[tid] = s;
        }
        __syncthreads();
        if (valid) {
            const int pos = pofs[warp][d] + wrank;
            kout[pos] = key[r];
            vout[pos] = val[r];
        }
    }
}

// ---------------------------------------------------------------------------
// particles in key order, FP64 and as a double-single split relative to O
__global__ void __launch_bounds__(kBuildThreads)
    gather_kernel(int n, const double *__restrict__ x, const double *__restrict__ y,
                  const double *__restrict__ z, const double *__restrict__ m,
                  const int32_t *__restrict__ perm, const int32_t *__restrict__ cid,
                  const Cluster *__restrict__ cl, double4_32a *__restrict__ sp,
                  float4 *__restrict__ ph, float4 *__restrict__ pl, int32_t *__restrict__ inv,
                  int32_t *__restrict__ cid_s, const int64_t *__restrict__ gid, int32_t *__restrict__ rid)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int i = perm[s];
    inv[i] = s;
    if (gid) rid[s] = (int32_t)gid[i];
    const int c = cid ? cid[i] : 0;
    cid_s[s] = c;
    const double *O = cl[c].frame;
    double px = x[i], py = y[i], pz = z[i], pm = m[i];
    sp[s] = make_double4_32a(px, py, pz, pm);
    float hx, hy, hz, lx, ly, lz;
    ds_split(dsub(px, O[0]), hx, lx);
    ds_split(dsub(py, O[1]), hy, ly);
    ds_split(dsub(pz, O[2]), hz, lz);
    ph[s] = make_float4(hx, hy, hz, __double2float_rn(pm));
    pl[s] = make_float4(lx, ly, lz, 0.f);
}

// ---------------------------------------------------------------------------
// topology

// Walk groups: with B = 16 G, a node holding <= B particles whose parent holds
// more than B (or the root if n <= B), and a leaf holding more than B, are cut
// into consecutive chunks of G particles; flag the first particle of each chunk.
constexpr int kGroupNodeFactor = 16;

__device__ __forceinline__ void flag_groups(unsigned char *gflag, int first, int count,
                                            bool parent_big, bool is_leaf, int G)
{
    if (!parent_big) return;
    if (count <= kGroupNodeFactor * G || is_leaf)
        for (int f = 0; f < count; f += G) gflag[first + f] = 1;
}

// one root per cluster at level 0 (node c covers cluster c in key order)
__global__ void topo_root_kernel(Tree T, int n, int leaf_cap, int G)
{
    const int C = T.n_clusters;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) {
        T.meta->level_start[0] = 0;
        T.meta->level_count[0] = C;
    }
    if (c >= C) return;
    long long first = T.seg ? T.seg[c] : 0, end = T.seg ? T.seg[c + 1] : n;
    if (!(first >= 0 && end > first && end <= n)) {  // invalid offsets: empty, safe root
        latch_error(T.meta, P3T_ERR_INVALID_INPUT);
        first = 0;
        end = 0;
    }
    const int cnt = (int)(end - first);
    T.topo[c] = make_int4((int)first, cnt, -1, 0);
    T.level[c] = 0;
    T.parent[c] = -1;
    const bool top = T.n_top > 0 && is_top_cell(T, 0, 0ULL);  // a decomposed cluster's root
    if (cnt <= leaf_cap && !top) T.leaves[atomicAdd(&T.meta->n_leaves, 1)] = c;
    if (!top) flag_groups(T.gflag, (int)first, cnt, true, cnt <= leaf_cap, G);
}

// A level with at most kTopoWideNodes nodes splits one node per warp with a 32-way
// search: a node of 10^6 keys takes 4 dependent load steps instead of the 20 of a
// binary search.  status holds status_cap lookback flags (one per tile).
__global__ void __launch_bounds__(kBuildThreads)
    topo_level_kernel(Tree T, int l, int leaf_cap, int G, unsigned long long *status,
                      int status_cap, unsigned int *ticket)
{
    __shared__ unsigned int sh_t;
    __shared__ long long sh_scan[32];
    __shared__ long long sh_pre;
    Meta *M = T.meta;
    const int nl = M->level_count[l];
    const int base = M->level_start[l];
    const bool wide = nl <= kTopoWideNodes;  // uniform over the launch
    const int per_tile = wide ? kBuildThreads / 32 : kBuildThreads;
    const int ntiles = (nl + per_tile - 1) / per_tile;
    const int shift = 63 - 3 * (l + 1);
    const int lane = threadIdx.x & 31;
    if (ntiles > status_cap) {  // more tiles than flags (cannot happen for nl <= n)
        if (threadIdx.x == 0) latch_error(M, P3T_ERR_INTERNAL);
        return;
    }
    while (true) {
        if (threadIdx.x == 0) sh_t = atomicAdd(ticket, 1u);
        __syncthreads();
        const int t = (int)sh_t;
        __syncthreads();
        if (t >= ntiles) break;
        // wide: warp w of the block holds node t * 8 + w (every lane), else one node a thread
        const int node = base + t * per_tile + (wide ? (int)(threadIdx.x >> 5) : (int)threadIdx.x);
        const bool mine = node < base + nl;
        int bnd[9];
        int nch = 0;
        int4 tp = make_int4(0, 0, -1, 0);
        if (mine) tp = T.topo[node];
        // a top cell of a decomposed cluster splits whatever its local count
        const bool top = mine && T.n_top > 0 && tp.y > 0 && is_top_cell(T, l, T.keys[tp.x] >> (63 - 3 * l));
        const bool split = mine && (tp.y > leaf_cap || top) && l < kLevels;
        if (split) {
            const int b = tp.x, e = tp.x + tp.y;
            const uint64_t pfx = T.keys[b] >> (shift + 3);
            bnd[0] = b;
            bnd[8] = e;
            // the 7 octant boundaries: lower bounds of ((pfx << 3) | o) << shift in
            // keys[b, e), searched in lockstep (the 7 loads of a step are independent)
            uint64_t tgt[8];
#pragma unroll
            for (int o = 1; o < 8; o++) tgt[o] = ((pfx << 3) | (uint64_t)o) << shift;
            if (wide) {
                // the lower bound lies in [lo, hi] (keys[lo - 1] < tgt <= keys[hi]);
                // lane j probes lo + j * stride, the probes below tgt are a prefix of
                // the lanes (keys ascending), and the range shrinks to one stride
                int lo[8], hi[8];
#pragma unroll
                for (int o = 1; o < 8; o++) lo[o] = b, hi[o] = e;
                while (true) {
                    bool any = false;
                    uint64_t kv[8];
                    int st[8];
#pragma unroll
                    for (int o = 1; o < 8; o++) {
                        const int len = hi[o] - lo[o];
                        st[o] = (len + 31) >> 5;
                        const int pj = lo[o] + lane * st[o];
                        kv[o] = len > 0 && pj < hi[o] ? T.keys[pj] : ~0ull;
                        any |= len > 0;
                    }
                    if (!any) break;
#pragma unroll
                    for (int o = 1; o < 8; o++) {
                        const int k = __popc(__ballot_sync(0xffffffffu, kv[o] < tgt[o]));
                        const int l0 = lo[o];
                        if (hi[o] > l0) {
                            if (k > 0) lo[o] = l0 + (k - 1) * st[o] + 1;
                            if (l0 + k * st[o] < hi[o]) hi[o] = l0 + k * st[o];
                        }
                    }
                }
#pragma unroll
                for (int o = 1; o < 8; o++) bnd[o] = lo[o];
            } else {
                // branchless halving with a common length
                int at[8];
#pragma unroll
                for (int o = 1; o < 8; o++) at[o] = b;
                for (int len = e - b; len > 1;) {
                    const int half = len >> 1;
#pragma unroll
                    for (int o = 1; o < 8; o++)
                        at[o] = T.keys[at[o] + half] < tgt[o] ? at[o] + half : at[o];
                    len -= half;
                }
#pragma unroll
                for (int o = 1; o < 8; o++) bnd[o] = at[o] + (T.keys[at[o]] < tgt[o] ? 1 : 0);
            }
#pragma unroll
            for (int o = 0; o < 8; o++) nch += bnd[o + 1] > bnd[o];
        }
        const bool owner = !wide || lane == 0;  // writes the node's children
        long long tot;
        long long ex = block_excl_scan<long long>(owner ? (long long)nch : 0LL, &tot, sh_scan);
        long long pre = lookback_prefix(status, t, tot, M, &sh_pre);
        const int child_base = base + nl + (int)(pre + ex);
        const bool fits = child_base + nch <= T.cap_nodes;
        if (split && owner && !fits) latch_error(M, P3T_ERR_CAPACITY);
        const bool write = split && owner && fits;
        // leaves appended with one atomic per warp
        int nlf = 0;
        if (write) {
#pragma unroll
            for (int o = 0; o < 8; o++) {
                const int cnt = bnd[o + 1] - bnd[o];
                const bool ctop = T.n_top > 0 && cnt > 0 &&
                                  is_top_cell(T, l + 1, T.keys[bnd[o]] >> (63 - 3 * (l + 1)));
                nlf += cnt > 0 && (cnt <= leaf_cap || l + 1 >= kLevels) && !ctop;
            }
        }
        const int inc = warp_incl_scan(nlf);
        int lf = 0;
        if (lane == 31 && inc > 0) lf = atomicAdd(&M->n_leaves, inc);
        lf = __shfl_sync(0xffffffffu, lf, 31) + inc - nlf;
        if (write) {
            // a top cell holds more than 16 G particles over all ranks
            const bool big = tp.y > kGroupNodeFactor * G || top;
            int k = 0;
#pragma unroll
            for (int o = 0; o < 8; o++) {
                int cnt = bnd[o + 1] - bnd[o];
                if (cnt > 0) {
                    int c = child_base + k++;
                    T.topo[c] = make_int4(bnd[o], cnt, -1, 0);
                    T.level[c] = l + 1;
                    T.parent[c] = node;
                    const bool ctop = T.n_top > 0 && is_top_cell(T, l + 1, T.keys[bnd[o]] >> (63 - 3 * (l + 1)));
                    bool leaf = (cnt <= leaf_cap || l + 1 >= kLevels) && !ctop;
                    if (leaf) T.leaves[lf++] = c;
                    if (!ctop) flag_groups(T.gflag, bnd[o], cnt, big, leaf, G);
                }
            }
            T.topo[node] = make_int4(tp.x, tp.y, child_base, nch);
        }
        if (t == ntiles - 1 && threadIdx.x == 0) {
            M->level_start[l + 1] = base + nl;
            M->level_count[l + 1] = (int)(pre + tot);
        }
    }
}

// ---- the same topology without a launch per level (one cluster or a batch; not a
// rank's range build, whose top cells split whatever their count) ----------------------
// Particle i starts the cells of every level above the levels its key shares with
// particle i - 1 (all of them when i starts its cluster).  A level-l cell holds more
// than L particles iff some L + 1 consecutive particles inside it share the cell's
// prefix, and every cell containing i holds such a window containing i, so with
// M(i) = the largest number of levels shared by keys j and j + L over the windows
// [j, j + L] of i's cluster that contain i, the cells containing i down to level
// lam(i) = min(M(i) + 1, 21) exist (their ancestors are split) and the one at lam(i)
// is a leaf.  So i starts the nodes of levels shared(i) + 1 .. lam(i), a node is
// split iff its level is below lam of its first particle, and breadth-first order is
// (level, first particle): a count of each level's nodes per tile of particles and one
// scan give every node its index.
constexpr int kFlatLevels = kLevels + 1;  // levels 0 .. 21

__device__ __forceinline__ int shared_levels(uint64_t a, uint64_t b)
{
    const uint64_t x = a ^ b;
    if (x == 0) return kLevels;
    const int eq = __clzll((long long)x) - 1;  // equal key bits below the unused bit 63
    return eq / 3 < kLevels ? eq / 3 : kLevels;
}

// cluster bounds [cs, ce) of particle i (key order; batched clusters are contiguous)
__device__ __forceinline__ void cluster_bounds(const Tree &T, int n, int i, int &cs, int &ce)
{
    if (!T.seg) {
        cs = 0;
        ce = n;
        return;
    }
    int lo = 0, hi = T.n_clusters;  // the last c with seg[c] <= i
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (T.seg[mid] <= i)
            lo = mid;
        else
            hi = mid;
    }
    // (clamped so that invalid offsets, latched by the cluster-id pass, stay in bounds)
    const long long a = T.seg[lo], b = T.seg[lo + 1];
    cs = (int)(a < 0 ? 0 : (a > i ? i : a));
    ce = (int)(b > n ? n : (b <= i ? i + 1 : b));
}

// per particle: packed (shared + 1) | lam << 8; per tile of kBuildThreads particles and
// level: the nodes the tile's particles start (cnt[l * ntiles + tile])
constexpr int kFlatMaxLeaf = 128;  // leaf capacities above this take the level launches
__global__ void __launch_bounds__(kBuildThreads)
    topo_flat_count_kernel(Tree T, int n, int leaf_cap, int ntiles, int32_t *__restrict__ packed,
                           int32_t *__restrict__ cnt, unsigned long long *scan_status, int scan_words,
                           unsigned int *scan_ticket)
{
    pdl_wait();
    if (blockIdx.x == 0) clear_scan_state(scan_status, scan_words, scan_ticket);  // the count scan's
    __shared__ uint64_t sk[kBuildThreads + 2 * kFlatMaxLeaf];
    __shared__ int sw[kBuildThreads + kFlatMaxLeaf];
    __shared__ int lc[kFlatLevels];
    const int tid = threadIdx.x, lane = tid & 31;
    const int t0 = blockIdx.x * kBuildThreads;
    const int L = leaf_cap;
    if (tid < kFlatLevels) lc[tid] = 0;
    // keys [t0 - L, t0 + kBuildThreads + L)
    for (int q = tid; q < kBuildThreads + 2 * L; q += kBuildThreads) {
        const int j = t0 - L + q;
        sk[q] = j >= 0 && j < n ? T.keys[j] : 0ULL;
    }
    __syncthreads();
    // w(j) for the window starts j in [t0 - L, t0 + kBuildThreads): the levels keys j
    // and j + L share (the windows that cross a cluster's bounds are skipped below)
    for (int q = tid; q < kBuildThreads + L; q += kBuildThreads) {
        const int j = t0 - L + q;
        sw[q] = j >= 0 && j + L < n ? shared_levels(sk[q], sk[q + L]) : -1;
    }
    __syncthreads();
    const int i = t0 + tid;
    if (i < n) T.gflag[i] = 0;  // (the finish pass flags the walk groups)
    int sh = 0, lam = -1;
    if (i < n) {
        int cs, ce;
        cluster_bounds(T, n, i, cs, ce);
        sh = i == cs ? -1 : shared_levels(sk[tid + L - 1], sk[tid + L]);
        const int j0 = i - L > cs ? i - L : cs, j1 = i < ce - 1 - L ? i : ce - 1 - L;
        int m = -1;
        for (int j = j0; j <= j1; j++) {
            const int w = sw[j - t0 + L];
            m = w > m ? w : m;
        }
        lam = m + 1 < kLevels ? m + 1 : kLevels;
        packed[i] = (sh + 1) | (lam << 8);
    }
#pragma unroll 1
    for (int l = 0; l < kFlatLevels; l++) {
        const unsigned b = __ballot_sync(0xffffffffu, i < n && sh < l && l <= lam);
        if (lane == 0 && b) atomicAdd(&lc[l], __popc(b));
    }
    __syncthreads();
    if (tid < kFlatLevels) cnt[tid * ntiles + blockIdx.x] = lc[tid];
    if (blockIdx.x == 0 && tid == 0) cnt[kFlatLevels * ntiles] = 0;  // the scan's total
}

// every node's index from the scanned counts (level, then first particle): node
// (l, i) gets first i, its level, and its first child (l + 1, i) when it is split;
// leaves join the moments' work list
__global__ void __launch_bounds__(kBuildThreads)
    topo_flat_emit_kernel(Tree T, int n, int ntiles, const int32_t *__restrict__ packed,
                          const int32_t *__restrict__ base)
{
    pdl_wait();
    constexpr int W = kBuildThreads / 32;
    __shared__ int wc[kFlatLevels][W];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int i = blockIdx.x * kBuildThreads + tid;
    int sh = 0, lam = -1;
    if (i < n) {
        const int pk = packed[i];
        sh = (pk & 0xff) - 1;
        lam = pk >> 8;
    }
#pragma unroll 1
    for (int l = 0; l < kFlatLevels; l++) {
        const unsigned b = __ballot_sync(0xffffffffu, i < n && sh < l && l <= lam);
        if (lane == 0) wc[l][warp] = __popc(b);
    }
    __syncthreads();
    const int cap = T.cap_nodes;
    int next = -1, leaf_id = -1;  // node (l + 1, i); node (lam, i) if i starts it
#pragma unroll 1
    for (int l = kFlatLevels - 1; l >= 0; l--) {  // deepest first: the child is known
        const bool mine = i < n && sh < l && l <= lam;
        const unsigned b = __ballot_sync(0xffffffffu, mine);
        if (!mine) continue;
        int id = base[l * ntiles + blockIdx.x] + __popc(b & lt);
        for (int w = 0; w < warp; w++) id += wc[l][w];
        if (id < cap) {  // (more nodes than the capacity are latched by the meta pass)
            T.topo[id] = make_int4(i, 0, l < lam ? next : -1, 0);
            T.level[id] = l;
        }
        if (l == lam) leaf_id = id;
        next = id;
    }
    const bool leaf = leaf_id >= 0 && leaf_id < cap;
    const unsigned lb = __ballot_sync(0xffffffffu, leaf);
    if (lb) {
        const int lead = __ffs(lb) - 1;
        int at = 0;
        if (lane == lead) at = atomicAdd(&T.meta->n_leaves, __popc(lb));
        at = __shfl_sync(0xffffffffu, at, lead);
        if (leaf) T.leaves[at + __popc(lb & lt)] = leaf_id;
    }
}

// per node: its particle count (the end of its cell: an exponential then a binary
// search over the keys for the first key outside the cell's prefix, within the
// cluster), its children (the next nodes of level l + 1 whose first particles lie in
// the cell, at most 8), the children's parent, and the walk-group starts of the
// children (whose counts are the gaps between their first particles) and of the roots
__global__ void __launch_bounds__(kBuildThreads) topo_flat_finish_kernel(Tree T, int n, int G)
{
    pdl_wait();
    const Meta *M = T.meta;
    const int nn = M->n_nodes < T.cap_nodes ? M->n_nodes : T.cap_nodes;
    int *tpw = reinterpret_cast<int *>(T.topo);  // the emit pass wrote x (first) and z (child)
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += gridDim.x * blockDim.x) {
        const int i = tpw[4 * (size_t)k], child = tpw[4 * (size_t)k + 2];
        const int l = T.level[k];
        int cs, ce;
        cluster_bounds(T, n, i, cs, ce);
        int end = ce;
        if (l > 0) {
            // first j in (i, ce) whose key leaves the level-l cell of key i, else ce
            const uint64_t ki = T.keys[i];
            const int sft = 63 - 3 * l;
            const uint64_t pfx = ki >> sft;
            int lo = i, step = 1;  // keys[lo] inside; probe lo + step
            while (lo + step < ce && (T.keys[lo + step] >> sft) == pfx) {
                lo += step;
                step <<= 1;
            }
            int hi = lo + step < ce ? lo + step : ce;  // keys[hi] outside, or hi == ce
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if ((T.keys[mid] >> sft) == pfx)
                    lo = mid;
                else
                    hi = mid;
            }
            end = hi;
        }
        const int count = end - i;
        tpw[4 * (size_t)k + 1] = count;
        if (l == 0) {
            T.parent[k] = -1;
            flag_groups(T.gflag, i, count, true, child < 0, G);
        }
        int nch = 0;
        if (child >= 0) {
            const int lend = M->level_start[l + 1] + M->level_count[l + 1];
            const int cend = lend < T.cap_nodes ? lend : T.cap_nodes;
            const bool big = count > kGroupNodeFactor * G;
            // the level's first particles ascend, so the children are the run of nodes
            // from child on whose first particles lie below end
            int f[8];
#pragma unroll
            for (int o = 0; o < 8; o++) {
                f[o] = child + o < cend ? tpw[4 * (size_t)(child + o)] : end;
                nch += f[o] < end;
            }
#pragma unroll
            for (int o = 0; o < 8; o++) {
                if (o < nch) {
                    const int c = child + o;
                    const int cnt = (o < 7 && o + 1 < nch ? f[o < 7 ? o + 1 : 7] : end) - f[o];
                    T.parent[c] = k;
                    flag_groups(T.gflag, f[o], cnt, big, tpw[4 * (size_t)c + 2] < 0, G);
                }
            }
        }
        tpw[4 * (size_t)k + 3] = nch;
    }
}

// the level starts and counts and the node total from the scanned counts
__global__ void topo_flat_meta_kernel(Meta *M, const int32_t *__restrict__ base, int ntiles, int cap_nodes)
{
    pdl_wait();
    const int total = base[kFlatLevels * ntiles];
    int depth = 0;
    for (int l = 0; l < kFlatLevels; l++) {
        const int b = base[l * ntiles];
        const int e = l + 1 < kFlatLevels ? base[(l + 1) * ntiles] : total;
        M->level_start[l] = b;
        M->level_count[l] = e - b;
        if (e > b) depth = l;
    }
    if (total > cap_nodes) latch_error(M, P3T_ERR_CAPACITY);
    M->n_nodes = total;
    M->depth = depth;
}

__global__ void topo_finish_kernel(Meta *M, int cap_nodes)
{
    int total = 0, depth = 0;
    for (int l = 0; l <= kLevels; l++) {
        total += M->level_count[l];
        if (M->level_count[l] > 0) depth = l;
    }
    if (total > cap_nodes) latch_error(M, P3T_ERR_CAPACITY);
    M->n_nodes = total;
    M->depth = depth;
}

// ---------------------------------------------------------------------------
// groups
__global__ void __launch_bounds__(kBuildThreads)
    group_first_kernel(int n, const unsigned char *__restrict__ gflag,
                       const int32_t *__restrict__ gidx, int2 *__restrict__ grp)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && gflag[i]) grp[gidx[i]].x = i;
}

// one warp per group: count and tight box (exact min/max, order-free)
__global__ void __launch_bounds__(kBuildThreads) group_finish_kernel(Tree T, int n)
{
    const int ng = T.meta->n_groups;
    const int lane = threadIdx.x & 31;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ng;
         g += (gridDim.x * blockDim.x) >> 5) {
        const int first = T.grp[g].x;
        const int end = g + 1 < ng ? T.grp[g + 1].x : n;
        // min/max of the order-preserving encodings on the integer pipes (the FP64
        // pipe is slow); equal to the FP64 min/max up to the sign of a zero
        EncBox box;
        box.reset();
        for (int i = first + lane; i < end; i += 32) {
            const double4_32a p = T.sp[i];
            box.add(p.x, p.y, p.z);
        }
#pragma unroll
        for (int d = 0; d < 3; d++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long a = __shfl_xor_sync(0xffffffffu, box.lo[d], o);
                const unsigned long long b = __shfl_xor_sync(0xffffffffu, box.hi[d], o);
                box.lo[d] = a < box.lo[d] ? a : box.lo[d];
                box.hi[d] = b > box.hi[d] ? b : box.hi[d];
            }
        }
        if (lane == 0) {
            double lo[3], hi[3];
            box.get(lo, hi);
            T.grp[g].y = end - first;
            T.glo[g] = make_double4_32a(lo[0], lo[1], lo[2], 0.0);
            T.ghi[g] = make_double4_32a(hi[0], hi[1], hi[2], 0.0);
        }
    }
}

// the FP32 frame quantities of every group, one thread per group: the mixed walks
// and the neighbour passes load them instead of deriving them on the FP64 pipe
// per warp (same operations as those walks used: c_g = (lo + hi) / 2, its
// double-single split relative to the cluster's frame centre O, the box - O)
__global__ void __launch_bounds__(kBuildThreads) group_frames_kernel(Tree T)
{
    const int ng = T.meta->n_groups;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        const double4_32a glo = T.glo[g], ghi = T.ghi[g];
        const double *O = T.cl[T.cid_s[T.grp[g].x]].frame;
        float hx, hy, hz, lx, ly, lz;
        ds_split(dsub(dmul(0.5, dadd(glo.x, ghi.x)), O[0]), hx, lx);
        ds_split(dsub(dmul(0.5, dadd(glo.y, ghi.y)), O[1]), hy, ly);
        ds_split(dsub(dmul(0.5, dadd(glo.z, ghi.z)), O[2]), hz, lz);
        T.gfr[3 * (size_t)g] = make_float4(hx, hy, hz, lx);
        T.gfr[3 * (size_t)g + 1] = make_float4(ly, lz, __double2float_rn(dsub(glo.x, O[0])),
                                               __double2float_rn(dsub(glo.y, O[1])));
        T.gfr[3 * (size_t)g + 2] =
            make_float4(__double2float_rn(dsub(glo.z, O[2])), __double2float_rn(dsub(ghi.x, O[0])),
                        __double2float_rn(dsub(ghi.y, O[1])), __double2float_rn(dsub(ghi.z, O[2])));
    }
}

// The order in which the walks take the groups: by the size of the group box
// (the FP32 exponent and two mantissa bits of its longest side), smallest first.
// Small boxes hold the densest groups, which carry the most particle terms, so
// the persistent walk starts them first and its tail holds light groups.  Inside
// a bin the groups keep their key order (a stable counting sort over chunks of
// kOrderChunk groups), so that the groups walked at the same time lie close
// together and share node records and sources in L2.  No result depends on the
// order (groups are independent).
constexpr int kGroupBins = 256;
constexpr int kOrderChunk = 1024;  // groups of one block's chunk, 4 per thread
__device__ __forceinline__ int group_bin(const Tree &T, int g)
{
    const float4 g1 = T.gfr[3 * (size_t)g + 1], g2 = T.gfr[3 * (size_t)g + 2];
    const float side = fmaxf(fmaxf(fmaxf(g2.y - g1.z, g2.z - g1.w), g2.w - g2.x), 0.f);
    const int b = (int)(__float_as_uint(side) >> 21) - (int)(__float_as_uint(1e-12f) >> 21);
    return min(max(b, 0), kGroupBins - 1);
}

// bin counts of every chunk: hist[bin * nchunks + chunk] (one block per chunk; chunks
// past the groups count nothing)
__global__ void __launch_bounds__(kBuildThreads) group_bins_kernel(Tree T, int32_t *hist, int nchunks)
{
    static_assert(kBuildThreads == kGroupBins, "one thread per bin");
    __shared__ int cnt[kGroupBins];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int ng = T.meta->n_groups;
    const int g0 = blockIdx.x * kOrderChunk;
    for (int g = g0 + threadIdx.x; g < min(ng, g0 + kOrderChunk); g += kBuildThreads)
        atomicAdd(&cnt[group_bin(T, g)], 1);
    __syncthreads();
    hist[threadIdx.x * nchunks + blockIdx.x] = cnt[threadIdx.x];
}

// stable placement: a chunk's groups of one bin go to that bin's offset for the chunk
// (hist, scanned bin-major), in the order of their index
__global__ void __launch_bounds__(kBuildThreads)
    group_order_kernel(Tree T, const int32_t *__restrict__ hist, int nchunks)
{
    constexpr int W = kBuildThreads / 32;
    __shared__ int base[kGroupBins];
    __shared__ int wcnt[W][kGroupBins];
    __shared__ int pofs[W][kGroupBins];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int ng = T.meta->n_groups;
    base[tid] = hist[tid * nchunks + blockIdx.x];
#pragma unroll
    for (int w = 0; w < W; w++) wcnt[w][tid] = 0;
    __syncthreads();
#pragma unroll 1
    for (int r = 0; r < kOrderChunk / kBuildThreads; r++) {
        const int g = blockIdx.x * kOrderChunk + r * kBuildThreads + tid;
        const bool valid = g < ng;
        const int bin = valid ? group_bin(T, g) : kGroupBins;  // (kGroupBins: no group)
        const unsigned peers = __match_any_sync(0xffffffffu, bin);
        const int wrank = __popc(peers & lt);
        if (valid && wrank == 0) wcnt[warp][bin] = __popc(peers);
        __syncthreads();
        {
            int s = base[tid];
#pragma unroll
            for (int w = 0; w < W; w++) {
                pofs[w][tid] = s;
                s += wcnt[w][tid];
                wcnt[w][tid] = 0;
            }
            base[tid] = s;
        }
        __syncthreads();
        if (valid) T.gorder[pofs[warp][bin] + wrank] = g;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// moments (rule 6) and the opening radius (rule 8)

template <bool Q64>
__device__ void leaf_moments(Tree &T, int k, int4 tp, double theta)
{
    const int b = tp.x, e = tp.x + tp.y;
    double M = 0.0, S[3] = {0, 0, 0}, lo[3], hi[3], com[3];
    EncBox box;
    box.reset();
    // chunks of 8 particles: the loads of a chunk are issued before its
    // (sequential, fixed-order) sums
    for (int i0 = b; i0 < e; i0 += 8) {
        double4_32a pc[8];
#pragma unroll
        for (int u = 0; u < 8; u++)
            if (i0 + u < e) pc[u] = T.sp[i0 + u];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            if (i0 + u < e) {
                const double4_32a &p = pc[u];
                M = dadd(M, p.w);
                S[0] = dadd(S[0], dmul(p.w, p.x));
                S[1] = dadd(S[1], dmul(p.w, p.y));
                S[2] = dadd(S[2], dmul(p.w, p.z));
                box.add(p.x, p.y, p.z);
            }
        }
    }
    box.get(lo, hi);
    for (int d = 0; d < 3; d++) com[d] = M > 0.0 ? ddiv(S[d], M) : dmul(0.5, dadd(lo[d], hi[d]));
    double q[6];
    if (Q64) {
        double Q[6] = {0, 0, 0, 0, 0, 0};
        for (int i = b; i < e; i++) {
            double4_32a p = T.sp[i];
            double m = p.w;
            double dx = dsub(p.x, com[0]), dy = dsub(p.y, com[1]), dz = dsub(p.z, com[2]);
            double r2 = dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz));
            Q[0] = dadd(Q[0], dmul(m, dsub(dmul(dmul(3.0, dx), dx), r2)));
            Q[1] = dadd(Q[1], dmul(m, dmul(dmul(3.0, dx), dy)));
            Q[2] = dadd(Q[2], dmul(m, dmul(dmul(3.0, dx), dz)));
            Q[3] = dadd(Q[3], dmul(m, dsub(dmul(dmul(3.0, dy), dy), r2)));
            Q[4] = dadd(Q[4], dmul(m, dmul(dmul(3.0, dy), dz)));
            Q[5] = dadd(Q[5], dmul(m, dsub(dmul(dmul(3.0, dz), dz), r2)));
        }
        for (int a = 0; a < 6; a++) q[a] = Q[a];
    } else {
        // FP32 quadrupole on offsets from the double-single splits (x - O) - (com - O)
        const double *O = T.cl[T.cid_s[b < T.n ? b : 0]].frame;
        float chx, chy, chz, clx, cly, clz;
        ds_split(dsub(com[0], O[0]), chx, clx);
        ds_split(dsub(com[1], O[1]), chy, cly);
        ds_split(dsub(com[2], O[2]), chz, clz);
        float Q[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll 8
        for (int i = b; i < e; i++) {
            const float4 h = T.ph[i], l = T.pl[i];
            const float m = h.w;
            const float dx = (h.x - chx) + (l.x - clx);
            const float dy = (h.y - chy) + (l.y - cly);
            const float dz = (h.z - chz) + (l.z - clz);
            float r2 = dx * dx + dy * dy + dz * dz;
            Q[0] += m * (3.f * dx * dx - r2);
            Q[1] += m * (3.f * dx * dy);
            Q[2] += m * (3.f * dx * dz);
            Q[3] += m * (3.f * dy * dy - r2);
            Q[4] += m * (3.f * dy * dz);
            Q[5] += m * (3.f * dz * dz - r2);
        }
        for (int a = 0; a < 6; a++) q[a] = Q[a];
    }
    write_node<Q64>(T, k, M, com, lo, hi, q, theta, tp);
}

// A mixed-form leaf's records from its sums: the steps of write_node<false> with the
// FP32 quadrupole and the double-single COM (relative to the frame O) passed in
__device__ __forceinline__ void write_leaf_mixed(Tree &T, int k, int4 tp, double M, const double com[3],
                                                 const double lo[3], const double hi[3], const float Q[6],
                                                 const float ch[3], const float cl[3], const float blo[3],
                                                 const float bhi[3], const Cluster &K)
{
    const double theta = K.theta;
    double l = dsub(hi[0], lo[0]);
    if (dsub(hi[1], lo[1]) > l) l = dsub(hi[1], lo[1]);
    if (dsub(hi[2], lo[2]) > l) l = dsub(hi[2], lo[2]);
    const double cx = dsub(dmul(0.5, dadd(lo[0], hi[0])), com[0]);
    const double cy = dsub(dmul(0.5, dadd(lo[1], hi[1])), com[1]);
    const double cz = dsub(dmul(0.5, dadd(lo[2], hi[2])), com[2]);
    const double delta = dsqrt(dadd(dadd(dmul(cx, cx), dmul(cy, cy)), dmul(cz, cz)));
    double ro2 = INFINITY;
    if (theta > 0.0) {
        const double ro = dadd(ddiv(l, theta), delta);
        ro2 = dmul(ro, ro);
    }
    T.comM[k] = make_double4_32a(com[0], com[1], com[2], M);
    T.lo[k] = make_double4_32a(lo[0], lo[1], lo[2], ro2);
    T.hi[k] = make_double4_32a(hi[0], hi[1], hi[2], 0.0);
    float2 *q2 = reinterpret_cast<float2 *>(T.q32 + 6 * (size_t)k);
    q2[0] = make_float2(Q[0], Q[1]);
    q2[1] = make_float2(Q[2], Q[3]);
    q2[2] = make_float2(Q[4], Q[5]);
    const auto w = wrec_at(T.wn, k);
    w[0] = make_float4(ch[0], ch[1], ch[2], __double2float_rn(ro2));
    w[1] = make_float4(blo[0], blo[1], blo[2], __int_as_float(-1 - tp.x));
    w[2] = make_float4(bhi[0], bhi[1], bhi[2], __int_as_float(tp.y));
    w[3] = make_float4(cl[0], cl[1], cl[2], __double2float_rn(M));
    w[4] = make_float4(Q[0], Q[1], Q[2], Q[3]);
    w[5] = make_float4(Q[4], Q[5], 0.f, 0.f);
}

// A mixed-form leaf (k >= 0) from its FP64 sums: COM, FP32 quadrupole on offsets from
// the double-single splits (x - O) - (com - O), records
__device__ __forceinline__ void leaf_finish_mixed(Tree &T, int k, int4 tp, double M, const double S[3],
                                                  const EncBox &box)
{
    if (k < 0) return;
    double lo[3], hi[3], com[3];
    box.get(lo, hi);
    for (int d = 0; d < 3; d++) com[d] = M > 0.0 ? ddiv(S[d], M) : dmul(0.5, dadd(lo[d], hi[d]));
    const Cluster &K = T.cl[T.cid_s[tp.x < T.n ? tp.x : 0]];
    float ch[3], cl[3];
    for (int d = 0; d < 3; d++) ds_split(dsub(com[d], K.frame[d]), ch[d], cl[d]);
    // the FP32 box relative to O: RN(RN(x - O)) rises with x, so the min and max of the
    // particles' high parts are the rounded min and max of x - O (the box the FP64 path
    // would round), without the FP64 steps
    float Q[6] = {0, 0, 0, 0, 0, 0}, blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll 4
    for (int i = tp.x; i < tp.x + tp.y; i++) {
        const float4 h = T.ph[i], l = T.pl[i];
        blo[0] = fminf(blo[0], h.x), blo[1] = fminf(blo[1], h.y), blo[2] = fminf(blo[2], h.z);
        bhi[0] = fmaxf(bhi[0], h.x), bhi[1] = fmaxf(bhi[1], h.y), bhi[2] = fmaxf(bhi[2], h.z);
        const float m = h.w;
        const float dx = (h.x - ch[0]) + (l.x - cl[0]);
        const float dy = (h.y - ch[1]) + (l.y - cl[1]);
        const float dz = (h.z - ch[2]) + (l.z - cl[2]);
        const float r2 = dx * dx + dy * dy + dz * dz;
        Q[0] += m * (3.f * dx * dx - r2);
        Q[1] += m * (3.f * dx * dy);
        Q[2] += m * (3.f * dx * dz);
        Q[3] += m * (3.f * dy * dy - r2);
        Q[4] += m * (3.f * dy * dz);
        Q[5] += m * (3.f * dz * dz - r2);
    }
    write_leaf_mixed(T, k, tp, M, com, lo, hi, Q, ch, cl, blo, bhi, K);
}

// Two mixed-form leaves on one lane (ka, kb; -1: none), their particles taken as one
// stream for the FP64 sums: the sums of each leaf stay sequential in key order (the
// same operations as leaf_moments<false>), and a lane's FP64 steps are the two
// leaves' total
__device__ __forceinline__ void leaf_pair_mixed(Tree &T, int ka, int kb)
{
    const int4 ta = ka >= 0 ? T.topo[ka] : make_int4(0, 0, -1, 0);
    const int4 tb = kb >= 0 ? T.topo[kb] : make_int4(0, 0, -1, 0);
    const int na = ta.y, tot = ta.y + tb.y;
    double M = 0.0, S[3] = {0, 0, 0}, Ma = 0.0, Sa[3] = {0, 0, 0};
    EncBox box, boxa;
    box.reset();
    boxa.reset();
    for (int p0 = 0; p0 < tot; p0 += 4) {
        double4_32a pc[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int p = p0 + u;
            if (p < tot) pc[u] = T.sp[p < na ? ta.x + p : tb.x + (p - na)];
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int p = p0 + u;
            if (p < tot) {
                if (p == na) {  // leaf a done: its sums aside, b starts from zero
                    Ma = M;
                    Sa[0] = S[0], Sa[1] = S[1], Sa[2] = S[2];
                    boxa = box;
                    M = 0.0;
                    S[0] = S[1] = S[2] = 0.0;
                    box.reset();
                }
                const double4_32a &q = pc[u];
                M = dadd(M, q.w);
                S[0] = dadd(S[0], dmul(q.w, q.x));
                S[1] = dadd(S[1], dmul(q.w, q.y));
                S[2] = dadd(S[2], dmul(q.w, q.z));
                box.add(q.x, q.y, q.z);
            }
        }
    }
    if (tot == na) {  // no particles of b: the running sums are a's
        Ma = M;
        Sa[0] = S[0], Sa[1] = S[1], Sa[2] = S[2];
        boxa = box;
    }
    leaf_finish_mixed(T, ka, ta, Ma, Sa, boxa);
    leaf_finish_mixed(T, kb, tb, M, S, box);
}

// The mixed-form leaves, 64 a warp: sorted by particle count (a counting sort over
// the warp) and paired smallest with largest, so that the warp's FP64 steps follow
// its largest pair rather than its largest leaf twice
constexpr int kLeafClasses = 18;  // counts 0 .. 16, and 17 for every larger count
__global__ void __launch_bounds__(kBuildThreads) moments_leaf_pair_kernel(Tree T)
{
    pdl_wait();
    __shared__ int sl[kBuildThreads / 32][64];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int nl = T.meta->n_leaves;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int l0 = 64 * gw; l0 < nl; l0 += 64 * nw) {
        const int ka = l0 + lane < nl ? T.leaves[l0 + lane] : -1;
        const int kb = l0 + 32 + lane < nl ? T.leaves[l0 + 32 + lane] : -1;
        const int na = ka >= 0 ? T.topo[ka].y : 0, nb = kb >= 0 ? T.topo[kb].y : 0;
        const int va = na < kLeafClasses - 1 ? na : kLeafClasses - 1;
        const int vb = nb < kLeafClasses - 1 ? nb : kLeafClasses - 1;
        int base = 0, ra = 0, rb = 0;
#pragma unroll 1
        for (int v = 0; v < kLeafClasses; v++) {
            const unsigned ba = __ballot_sync(0xffffffffu, va == v), bb = __ballot_sync(0xffffffffu, vb == v);
            if (va == v) ra = base + __popc(ba & lt);
            if (vb == v) rb = base + __popc(ba) + __popc(bb & lt);
            base += __popc(ba) + __popc(bb);
        }
        sl[warp][ra] = ka;
        sl[warp][rb] = kb;
        __syncwarp();
        const int k0 = sl[warp][lane], k1 = sl[warp][63 - lane];
        __syncwarp();
        leaf_pair_mixed(T, k0, k1);
    }
}

// The internal node k of the mixed form on three lanes, lane d doing dimension
// d of every FP64 step (the same operations in the same order as
// internal_moments<false> + write_node<false>; M and the steps after the box are
// repeated on the three lanes, and lane d sums quadrupole components 2d and 2d + 1).
// A warp issues about a third of the FP64 instructions of one node per lane for the
// same 32 / 3 nodes' worth of work.  Every load comes first, so that a node's
// latency is one round of loads and its chain of FP64 steps (65 to 670 cycles each
// on this part), which sets the time of the levels with few nodes.  Every lane of
// the warp calls this (the shuffles); act: the lane holds dimension d of node k.
__device__ __forceinline__ void internal_moments3(Tree &T, int k, int4 tp, bool act, int d, int lane0)
{
    auto sh = [&](double v, int j) { return __shfl_sync(0xffffffffu, v, lane0 + j); };
    auto shf = [&](float v, int j) { return __shfl_sync(0xffffffffu, v, lane0 + j); };
    const int c0 = tp.z, nc = act ? tp.w : 0;
    const Cluster &K = T.cl[T.cid_s[act && tp.x < T.n ? tp.x : 0]];
    // the children's mass, COM, box and double-single COM in dimension d, FP32 mass
    // and quadrupole components 2d, 2d + 1
    double cw[8], cc[8], cl0[8], ch0[8];
    float wh[8], wl[8], wm[8], qa[8], qb[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        if (i < nc) {
            const int c = c0 + i;
            const double *cm = reinterpret_cast<const double *>(&T.comM[c]);
            cw[i] = __ldcg(cm + 3);
            cc[i] = __ldcg(cm + d);
            cl0[i] = __ldcg(reinterpret_cast<const double *>(&T.lo[c]) + d);
            ch0[i] = __ldcg(reinterpret_cast<const double *>(&T.hi[c]) + d);
            const float *w0 = reinterpret_cast<const float *>(&T.wn[wrec(c, 0)]);
            const float *w3 = reinterpret_cast<const float *>(&T.wn[wrec(c, 3)]);
            wh[i] = __ldcg(w0 + d);
            wl[i] = __ldcg(w3 + d);
            wm[i] = __ldcg(w3 + 3);
            const float *Qc = T.q32 + 6 * (size_t)c + 2 * d;
            qa[i] = __ldcg(Qc);
            qb[i] = __ldcg(Qc + 1);
        }
    }
    const double O = K.frame[d], theta = K.theta;
    double M = 0.0, S = 0.0;
    unsigned long long elo = ~0ULL, ehi = 0ULL;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        if (i < nc) {
            M = dadd(M, cw[i]);
            S = dadd(S, dmul(cw[i], cc[i]));
            const unsigned long long a = enc_double(cl0[i]), b = enc_double(ch0[i]);
            elo = a < elo ? a : elo;
            ehi = b > ehi ? b : ehi;
        }
    }
    const double lo = dec_double(elo), hi = dec_double(ehi);
    const double com = M > 0.0 ? ddiv(S, M) : dmul(0.5, dadd(lo, hi));
    // relative to the cluster's frame O: the double-single COM
    float ch, cl;
    ds_split(dsub(com, O), ch, cl);
    // quadrupole from the children (FP32): each lane's offsets from the double-single
    // COMs of its dimension, then all three
    float Qa = 0.f, Qb = 0.f;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const float dd = i < nc ? (wh[i] - ch) + (wl[i] - cl) : 0.f;
        const float dx = shf(dd, 0), dy = shf(dd, 1), dz = shf(dd, 2);
        if (i < nc) {
            const float Mc = wm[i];
            const float d2 = dx * dx + dy * dy + dz * dz;
            if (d == 0) {
                Qa += qa[i] + Mc * (3.f * dx * dx - d2);
                Qb += qb[i] + Mc * (3.f * dx * dy);
            } else if (d == 1) {
                Qa += qa[i] + Mc * (3.f * dx * dz);
                Qb += qb[i] + Mc * (3.f * dy * dy - d2);
            } else {
                Qa += qa[i] + Mc * (3.f * dy * dz);
                Qb += qb[i] + Mc * (3.f * dz * dz - d2);
            }
        }
    }
    // opening radius l/theta + delta (rule 8)
    const double side = dsub(hi, lo);
    const double sx = sh(side, 0), sy = sh(side, 1), sz = sh(side, 2);
    double l = sx;
    if (sy > l) l = sy;
    if (sz > l) l = sz;
    const double c = dsub(dmul(0.5, dadd(lo, hi)), com);
    const double c2 = dmul(c, c);
    const double cx2 = sh(c2, 0), cy2 = sh(c2, 1), cz2 = sh(c2, 2);
    double ro2 = INFINITY;
    if (act) {
        const double delta = dsqrt(dadd(dadd(cx2, cy2), cz2));
        if (theta > 0.0) {
            const double ro = dadd(ddiv(l, theta), delta);
            ro2 = dmul(ro, ro);
        }
    }
    // records: lane d writes its dimension (and its quadrupole components), lane 0
    // the rest; the FP32 box relative to O
    if (act) {
        double *cm = reinterpret_cast<double *>(&T.comM[k]);
        double *bl = reinterpret_cast<double *>(&T.lo[k]);
        double *bh = reinterpret_cast<double *>(&T.hi[k]);
        cm[d] = com;
        bl[d] = lo;
        bh[d] = hi;
        reinterpret_cast<float2 *>(T.q32 + 6 * (size_t)k)[d] = make_float2(Qa, Qb);
        float *w0 = reinterpret_cast<float *>(&T.wn[wrec(k, 0)]);
        float *w1 = reinterpret_cast<float *>(&T.wn[wrec(k, 1)]);
        float *w2 = reinterpret_cast<float *>(&T.wn[wrec(k, 2)]);
        float *w3 = reinterpret_cast<float *>(&T.wn[wrec(k, 3)]);
        float *w4 = reinterpret_cast<float *>(&T.wn[wrec(k, 4)]);  // w4, w5: Q0 .. Q5, 0, 0
        w0[d] = ch;
        w1[d] = __double2float_rn(dsub(lo, O));
        w2[d] = __double2float_rn(dsub(hi, O));
        w3[d] = cl;
        if (d < 2) {
            reinterpret_cast<float2 *>(w4)[d] = make_float2(Qa, Qb);
        } else {
            float *w5 = reinterpret_cast<float *>(&T.wn[wrec(k, 5)]);
            *reinterpret_cast<float4 *>(w5) = make_float4(Qa, Qb, 0.f, 0.f);
        }
        if (d == 0) {
            cm[3] = M;
            bl[3] = ro2;
            bh[3] = 0.0;
            w0[3] = __double2float_rn(ro2);
            w1[3] = __int_as_float(tp.z);
            w2[3] = __int_as_float(tp.w);
            w3[3] = __double2float_rn(M);
        }
    }
}

// internal nodes of level l in the mixed form, ten nodes a warp (three lanes each)
__global__ void __launch_bounds__(kBuildThreads) moments_level3_kernel(Tree T, int l)
{
    pdl_wait();
    const int b = T.meta->level_start[l], e = b + T.meta->level_count[l];
    const int lane = threadIdx.x & 31;
    const int slot = lane / 3, d = lane - 3 * slot;  // lanes 30, 31: slot 10, idle
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int k0 = b + 10 * warp; k0 < e; k0 += 10 * nwarps) {
        const int k = k0 + slot;
        const bool in = slot < 10 && k < e;
        const int4 tp = in ? T.topo[k] : make_int4(0, 0, -1, 0);
        internal_moments3(T, k, tp, in && tp.z >= 0, slot < 10 ? d : 0, slot < 10 ? 3 * slot : 0);
    }
}

// leaves first (one thread per leaf), then the internal nodes level by level,
// deepest first, each from its children in octant order; every pass keeps
// whole warps busy (FP64 instructions cost the same for one lane as for 32)
template <bool Q64>
__global__ void __launch_bounds__(kBuildThreads) moments_leaf_kernel(Tree T, double theta)
{
    const int nl = T.meta->n_leaves;
    for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < nl; li += gridDim.x * blockDim.x) {
        const int k = T.leaves[li];
        leaf_moments<Q64>(T, k, T.topo[k], theta);
    }
}

template <bool Q64>
__global__ void __launch_bounds__(kBuildThreads) moments_level_kernel(Tree T, int l, double theta)
{
    const int b = T.meta->level_start[l], e = b + T.meta->level_count[l];
    for (int k = b + blockIdx.x * blockDim.x + threadIdx.x; k < e; k += gridDim.x * blockDim.x) {
        const int4 tp = T.topo[k];
        if (tp.z >= 0) internal_moments<Q64>(T, k, tp, theta);
    }
}

// ---------------------------------------------------------------------------
// global indices (< 2^31) as int32 digits for the range build's first sort passes
__global__ void __launch_bounds__(kBuildThreads)
    gid32_kernel(int n, const int64_t *__restrict__ gid, int32_t *__restrict__ g32, Meta *meta)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t v = gid[i];
    if (v < 0 || v >= (1LL << 31)) latch_error(meta, P3T_ERR_INVALID_INPUT);
    g32[i] = (int32_t)v;
}

// the global bounding box of a decomposed cluster in place of the rank's own (the
// rank's particles, already validated by bbox_kernel, must lie inside it)
__global__ void set_bbox_kernel(Cluster *cl, double lx, double ly, double lz, double hx, double hy,
                                double hz, Meta *meta)
{
    Cluster &K = cl[0];
    const double lo[3] = {lx, ly, lz}, hi[3] = {hx, hy, hz};
    for (int d = 0; d < 3; d++) {
        const unsigned long long a = enc_double(lo[d]), b = enc_double(hi[d]);
        const bool empty = K.minmax[d] == ~0ULL;
        if (!empty && (K.minmax[d] < a || K.minmax[3 + d] > b)) latch_error(meta, P3T_ERR_INVALID_INPUT);
        K.minmax[d] = a;
        K.minmax[3 + d] = b;
    }
}

// The cube and frame of a decomposed cluster's global bounding box into the device
// cluster record *cl (rule 1, as a build computes them), for the key counts and the
// partition of particles among ranks.
int global_frame(cudaStream_t s, const double box[6], Cluster *cl, Meta *meta)
{
    init_clusters_kernel<<<1, 32, 0, s>>>(cl, 1);
    set_bbox_kernel<<<1, 1, 0, s>>>(cl, box[0], box[1], box[2], box[3], box[4], box[5], meta);
    cube_kernel<<<1, 32, 0, s>>>(cl, 1);
    return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

int build_tree(p3t_ctx *c, int n, int n_clusters, const int64_t *seg, const double *cprm,
               const double *x, const double *y, const double *z, const double *m,
               const RangeSpec *range)
{
    cudaStream_t s = c->stream;
    Tree &T = c->tree;
    Meta *M = c->meta;
    const p3t_params &P = c->prm;
    T.n = n;
    T.n_src = n;
    T.n_clusters = n_clusters;
    T.seg = seg;
    T.n_top = range ? range->n_top : 0;
    T.top_key = c->top_buf;
    T.top_level = reinterpret_cast<const int32_t *>(c->top_buf + kMaxTopCells);
    const int32_t *cid = seg ? T.cid : nullptr;  // null: a single cluster
    const int grid_n = (n + kBuildThreads - 1) / kBuildThreads;
    const int grid_c = (n_clusters + 127) / 128;
    const int persistent = 4 * c->sm_count;

    init_meta_kernel<<<1, 64, 0, s>>>(M);
    // the kernels of one build follow one another on the stream with programmatic
    // dependent launches (each waits for the one before it; their launches overlap)
    bool ok = launch_pdl(init_clusters_kernel, dim3(grid_c), dim3(128), s, T.cl, n_clusters) == cudaSuccess &&
              launch_pdl(cluster_params_kernel, dim3(grid_c), dim3(128), s, T.cl, n_clusters, cprm, P.theta,
                         P.r_in, P.r_out, P.r_list, M) == cudaSuccess;
    if (seg) cid_kernel<<<(n > n_clusters ? grid_n : grid_c + 1), kBuildThreads, 0, s>>>(n, n_clusters, seg, T.cid, M);
    ok = ok && launch_pdl(bbox_kernel, dim3(persistent), dim3(kBuildThreads), s, n, x, y, z, m, cid, T.cl, M) ==
                   cudaSuccess;
    if (range)
        set_bbox_kernel<<<1, 1, 0, s>>>(T.cl, range->box[0], range->box[1], range->box[2], range->box[3],
                                        range->box[4], range->box[5], M);
    ok = ok &&
         launch_pdl(cube_kernel, dim3(grid_c), dim3(128), s, T.cl, n_clusters) == cudaSuccess &&
         launch_pdl(keys_kernel, dim3(grid_n), dim3(kBuildThreads), s, n, x, y, z, cid, (const Cluster *)T.cl,
                    c->keys_buf[0], c->perm_buf[0]) == cudaSuccess;
    if (!ok || check_launch(c)) return P3T_ERR_CUDA;

    // 8 passes of 8 bits over the key, then (batched builds) stable passes over the
    // cluster id, so the order is (cluster, key, original index).  A rank's part of
    // a decomposed cluster sorts by the global index first (4 passes over its low 32
    // bits), so that its order is (key, global index), as in one build of the whole.
    const int nb = (n + kSortTile - 1) / kSortTile;
    const int cid_passes = seg ? (n_clusters <= 256 ? 1 : (n_clusters <= 65536 ? 2 : 3)) : 0;
    const int gid_passes = range && range->gid ? 4 : 0;
    if (gid_passes) gid32_kernel<<<grid_n, kBuildThreads, 0, s>>>(n, range->gid, c->rid_buf, M);
    const int passes = gid_passes + 8 + cid_passes;
    for (int pass = 0; pass < passes; pass++) {
        const bool by_gid = pass < gid_passes;
        const bool by_cid = pass >= gid_passes + 8;
        const int shift = by_gid ? 8 * pass : (by_cid ? 8 * (pass - gid_passes - 8) : 8 * (pass - gid_passes));
        uint64_t *kin = c->keys_buf[pass & 1], *kout = c->keys_buf[(pass + 1) & 1];
        int32_t *vin = c->perm_buf[pass & 1], *vout = c->perm_buf[(pass + 1) & 1];
        const int32_t *dcid = by_cid ? T.cid : (by_gid ? c->rid_buf : nullptr);
        if (launch_pdl(sort_hist_kernel, dim3(nb), dim3(kBuildThreads), s, n, (const uint64_t *)kin,
                       (const int32_t *)vin, dcid, shift, nb, c->sort_hist, c->scan_status,
                       scan_status_words(256 * nb), &M->tickets[31]) != cudaSuccess)
            return P3T_ERR_CUDA;
        int e = scan_excl_i32_to_i32_cleared(c->sort_hist, c->sort_hist, 256 * nb, c->scan_status,
                                             &M->tickets[31], M, s);
        if (e) return e;
        if (launch_pdl(sort_scatter_kernel, dim3(nb), dim3(kBuildThreads), s, n, (const uint64_t *)kin,
                       (const int32_t *)vin, kout, vout, dcid, shift, nb, (const int32_t *)c->sort_hist) !=
            cudaSuccess)
            return P3T_ERR_CUDA;
    }
    T.keys = c->keys_buf[passes & 1];
    T.perm = c->perm_buf[passes & 1];
    const int64_t *gid = range ? range->gid : nullptr;
    T.rid = gid ? c->rid_buf : T.perm;
    // the gather on the side stream beside the topology, which reads only the keys (the
    // moments and the groups wait for it)
    const bool gfork = c->side_stream != nullptr && c->join_ev2 != nullptr;
    const cudaStream_t gts = gfork ? c->side_stream : s;
    if (gfork && (cudaEventRecord(c->fork_ev, s) != cudaSuccess || cudaStreamWaitEvent(gts, c->fork_ev, 0) != cudaSuccess))
        return P3T_ERR_CUDA;
    gather_kernel<<<grid_n, kBuildThreads, 0, gts>>>(n, x, y, z, m, T.perm, cid, T.cl, T.sp, T.ph, T.pl,
                                                      T.inv, T.cid_s, gid, T.rid);
    if (gfork && cudaEventRecord(c->join_ev2, gts) != cudaSuccess) return P3T_ERR_CUDA;

    // topology: in one flat pass over the particles (per-particle levels, a scan of
    // the per-tile node counts, the nodes, their counts and children), or level by
    // level for a rank's range build (its top cells split whatever their count) and
    // for leaf capacities past the flat pass's window
    const bool flat = !range && P.leaf_cap <= kFlatMaxLeaf;
    if (!flat && cudaMemsetAsync(T.gflag, 0, n, s) != cudaSuccess) return P3T_ERR_CUDA;
    if (flat) {
        // per-particle levels in the group index buffer and per-tile counts in the sort
        // histogram (both free until the groups): 22 ceil(n / 256) + 1 <= 256 ceil(n / 1024)
        const int ntiles = grid_n;
        const int ncnt = kFlatLevels * ntiles + 1;
        if (launch_pdl(topo_flat_count_kernel, dim3(ntiles), dim3(kBuildThreads), s, T, n, P.leaf_cap, ntiles,
                       T.gidx, c->sort_hist, c->scan_status, scan_status_words(ncnt), &M->tickets[31]) !=
            cudaSuccess)
            return P3T_ERR_CUDA;
        int e = scan_excl_i32_to_i32_cleared(c->sort_hist, c->sort_hist, ncnt, c->scan_status,
                                             &M->tickets[31], M, s);
        if (e) return e;
        if (launch_pdl(topo_flat_meta_kernel, dim3(1), dim3(1), s, M, (const int32_t *)c->sort_hist, ntiles,
                       T.cap_nodes) != cudaSuccess ||
            launch_pdl(topo_flat_emit_kernel, dim3(ntiles), dim3(kBuildThreads), s, T, n, ntiles,
                       (const int32_t *)T.gidx, (const int32_t *)c->sort_hist) != cudaSuccess ||
            launch_pdl(topo_flat_finish_kernel, dim3(persistent), dim3(kBuildThreads), s, T, n, P.group_size) !=
                cudaSuccess)
            return P3T_ERR_CUDA;
    } else {
        unsigned long long *topo_status = c->scan_status + (n / 256 + 64 + 256 * nb / 256);
        const int stride = topo_status_stride(n);
        if (cudaMemsetAsync(topo_status, 0, sizeof(unsigned long long) * stride * kMaxLevelSlots, s) !=
            cudaSuccess)
            return P3T_ERR_CUDA;
        topo_root_kernel<<<grid_c, 128, 0, s>>>(T, n, P.leaf_cap, P.group_size);
        const int topo_grid = 2 * c->sm_count;
        for (int l = 0; l < kLevels; l++)
            topo_level_kernel<<<topo_grid, kBuildThreads, 0, s>>>(
                T, l, P.leaf_cap, P.group_size, topo_status + (size_t)l * stride, stride, &M->tickets[l]);
        topo_finish_kernel<<<1, 1, 0, s>>>(M, T.cap_nodes);
    }
    if (check_launch(c)) return P3T_ERR_CUDA;
    if (gfork && cudaStreamWaitEvent(s, c->join_ev2, 0) != cudaSuccess) return P3T_ERR_CUDA;  // the gather

    // groups, on the side stream beside the moments: both only read the topology
    // (the stream joins again before the build returns)
    const bool fork = c->side_stream != nullptr;
    const cudaStream_t gs = fork ? c->side_stream : s;
    if (fork && (cudaEventRecord(c->fork_ev, s) != cudaSuccess || cudaStreamWaitEvent(gs, c->fork_ev, 0) != cudaSuccess))
        return P3T_ERR_CUDA;
    int e = scan_excl_u8_to_i32(T.gflag, T.gidx, n, &M->n_groups, c->scan_status, &M->tickets[30],
                                M, gs);
    if (e) return e;
    group_first_kernel<<<grid_n, kBuildThreads, 0, gs>>>(n, T.gflag, T.gidx, T.grp);
    group_finish_kernel<<<persistent, kBuildThreads, 0, gs>>>(T, n);
    group_frames_kernel<<<persistent, kBuildThreads, 0, gs>>>(T);
    // the walk order: a stable counting sort of the groups by box size (chunks sized
    // for the largest group count, n; the sort's histogram and scan buffers, free now)
    const int nchunks = (n + kOrderChunk - 1) / kOrderChunk;
    group_bins_kernel<<<nchunks, kBuildThreads, 0, gs>>>(T, c->sort_hist, nchunks);
    if ((e = scan_excl_i32_to_i32(c->sort_hist, c->sort_hist, kGroupBins * nchunks, c->scan_status,
                                  &M->tickets[31], M, gs)))
        return e;
    group_order_kernel<<<nchunks, kBuildThreads, 0, gs>>>(T, c->sort_hist, nchunks);
    if (fork && cudaEventRecord(c->join_ev, gs) != cudaSuccess) return P3T_ERR_CUDA;

    // moments: leaves, then levels 20 .. 0 (a level without internal nodes exits at once)
    const bool q64 = P.precision == P3T_FP64;
    if (q64)
        moments_leaf_kernel<true><<<persistent, kBuildThreads, 0, s>>>(T, P.theta);
    else {
        int leaf_blocks = 0;  // one resident wave (a grid-stride loop over the leaves)
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&leaf_blocks, moments_leaf_pair_kernel, kBuildThreads, 0) !=
                cudaSuccess ||
            leaf_blocks < 1 ||
            launch_pdl(moments_leaf_pair_kernel, dim3(leaf_blocks * c->sm_count), dim3(kBuildThreads), s, T) !=
                cudaSuccess)
            return P3T_ERR_CUDA;
    }
    // the mixed form's level passes: blocks of 128 threads, as many as fit on the SMs at
    // once (a level's nodes are taken ten a warp in one sweep of the resident grid; a
    // level without internal nodes costs the launch of that grid alone)
    int lvl_blocks = 0;
    if (!q64 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&lvl_blocks, moments_level3_kernel,
                                                               kBuildThreads / 2, 0) != cudaSuccess ||
                 lvl_blocks < 1))
        return P3T_ERR_CUDA;
    for (int l = kLevels - 1; l >= 0; l--) {
        if (q64)
            moments_level_kernel<true><<<persistent, kBuildThreads, 0, s>>>(T, l, P.theta);
        else if (launch_pdl(moments_level3_kernel, dim3(lvl_blocks * c->sm_count), dim3(kBuildThreads / 2), s, T,
                            l) != cudaSuccess)
            return P3T_ERR_CUDA;
    }
    if (fork && cudaStreamWaitEvent(s, c->join_ev, 0) != cudaSuccess) return P3T_ERR_CUDA;
    return check_launch(c);
}

// ---------------------------------------------------------------------------
// export (inspection)
__global__ void export_nodes_kernel(Tree T, bool q64, int32_t *level, int32_t *first,
                                    int32_t *count, int32_t *child, int32_t *nchild, double *M,
                                    double *com, double *Q, double *lo, double *hi, double *ropen2)
{
    const int nn = T.meta->n_nodes;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += gridDim.x * blockDim.x) {
        int4 tp = T.topo[k];
        if (level) level[k] = T.level[k];
        if (first) first[k] = tp.x;
        if (count) count[k] = tp.y;
        if (child) child[k] = tp.z;
        if (nchild) nchild[k] = tp.w;
        double4_32a cm = T.comM[k], l = T.lo[k], h = T.hi[k];
        if (M) M[k] = cm.w;
        if (com) com[3 * k] = cm.x, com[3 * k + 1] = cm.y, com[3 * k + 2] = cm.z;
        if (lo) lo[3 * k] = l.x, lo[3 * k + 1] = l.y, lo[3 * k + 2] = l.z;
        if (hi) hi[3 * k] = h.x, hi[3 * k + 1] = h.y, hi[3 * k + 2] = h.z;
        if (ropen2) ropen2[k] = l.w;
        if (Q)
            for (int a = 0; a < 6; a++)
                Q[6 * k + a] = q64 ? T.q64[6 * (size_t)k + a] : (double)T.q32[6 * (size_t)k + a];
    }
}

__global__ void export_groups_kernel(Tree T, int32_t *g_first, int32_t *g_count)
{
    const int ng = T.meta->n_groups;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        if (g_first) g_first[g] = T.grp[g].x;
        if (g_count) g_count[g] = T.grp[g].y;
    }
}

int export_tree(p3t_ctx *c, uint64_t *keys, int32_t *perm, int32_t *level, int32_t *first,
                int32_t *count, int32_t *child, int32_t *nchild, double *M, double *com,
                double *Q, double *lo, double *hi, double *ropen2, int32_t *g_first,
                int32_t *g_count)
{
    cudaStream_t s = c->stream;
    const Tree &T = c->tree;
    if (keys && cudaMemcpyAsync(keys, T.keys, 8 * (size_t)c->n, cudaMemcpyDeviceToDevice, s))
        return P3T_ERR_CUDA;
    if (perm && cudaMemcpyAsync(perm, T.perm, 4 * (size_t)c->n, cudaMemcpyDeviceToDevice, s))
        return P3T_ERR_CUDA;
    export_nodes_kernel<<<4 * c->sm_count, kBuildThreads, 0, s>>>(
        T, c->built_precision == P3T_FP64, level, first, count, child, nchild, M, com, Q, lo, hi,
        ropen2);
    export_groups_kernel<<<4 * c->sm_count, kBuildThreads, 0, s>>>(T, g_first, g_count);
    return check_launch(c);
}

}  // namespace p3t
