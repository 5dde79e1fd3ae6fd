// Internal declarations of the P3T distant-force library (sm_103a).
//
// Device layout of one built tree (all in the context's scratch, see ctx.cu):
//   particles, Morton order:  keys u64[n], perm i32[n] (sorted -> original),
//                             sp double4_32a[n] = {x, y, z, m}
//   nodes, breadth-first:     topo int4 = {first, count, child (-1 = leaf), nchild},
//                             level i32, parent i32,
//                             comM double4_32a = {com.xyz, M}, lo double4_32a = {lo.xyz, r_open^2},
//                             hi double4_32a = {hi.xyz, 0}, Q (FP64: double[6] | FP32: float[6]),
//                             walk record wn float4[6] per node (96 bytes, one load batch):
//                               [0] {hi part of com-O, r_open^2}  [1] {lo-O, child | -1-first}
//                               [2] {hi-O, nchild | count}        [3] {lo part of com-O, M}
//                               [4] {Qxx, Qxy, Qxz, Qyy}          [5] {Qyz, Qzz, 0, 0}
//                             (O = centre of the bounding cube; FP32 values)
//   groups, particle order:   grp int2 = {first, count}, glo/ghi double4_32a (tight box)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/p3t.h"

namespace p3t {

constexpr int kLevels = 21;          // key bits per axis = tree depth
constexpr int kMaxLevelSlots = 24;   // per-level bookkeeping arrays
// Bounded waits: polls before a wait gives up and latches P3T_ERR_TIMEOUT (a
// context may set its own limit, Meta::spin_limit).  The first 64 polls sleep
// 32 ns, the rest 256 ns, so 2^22 polls take about 1.1 s.
constexpr long long kSpinLimit = 1LL << 22;
constexpr int kWalkRecord = 6;               // float4 per node in Tree::wn
// Node k's walk record, field f (0 .. kWalkRecord - 1): blocks of 32 nodes stored field
// by field, so that a warp reading one field of consecutive nodes (the children of the
// ranges it popped) reads consecutive 16-byte words.  Buffers hold whole blocks.
__host__ __device__ __forceinline__ size_t wrec(int k, int f)
{
    return ((size_t)(k >> 5) * kWalkRecord + f) * 32 + (k & 31);
}
__host__ __device__ __forceinline__ size_t wrec_words(long long nodes)  // float4 of a buffer
{
    return (size_t)((nodes + 31) / 32) * 32 * kWalkRecord;
}
template <typename V>
struct WRecRef {
    V *base;
    int k;
    __host__ __device__ __forceinline__ V &operator[](int f) const { return base[wrec(k, f)]; }
};
template <typename V>
__host__ __device__ __forceinline__ WRecRef<V> wrec_at(V *base, int k)
{
    return WRecRef<V>{base, k};
}
constexpr float kFp32U = 5.9604644775390625e-8f;  // 2^-24, FP32 unit round-off

// Error band of an FP32 squared-distance test d2 < r2 in a cluster frame of half
// size R (coordinates relative to the frame centre carry <= 2^-24 R rounding):
// |d2_fp32 - d2_exact| <= k_rel (d2 + r2) + k_abs |t|_1 + k_sq, with about twice
// the derived bound in each constant.  With |t|_1 <= sqrt(3 d2) <= sqrt(3)
// (d2 / 2r + r / 2) this is at most A d2 + B, a band linear in d2 whose two
// coefficients depend only on the threshold r and R; A and B come rounded up.
// Tight near d2 = r2 and for r of the order of the distances tested, so it
// serves the box tests against the cluster radii (r_out, r_list); the opening
// angle's radius can be arbitrarily small (single-particle nodes), where A
// would swamp every test, so that test keeps the |t|_1 form.
struct Band {
    float a, b;
};
__host__ __device__ inline Band fp32_band(float R, float r2)
{
    const float k_rel = 8.f * kFp32U, k_abs = 8.f * kFp32U * R, k_sq = 16.f * kFp32U * kFp32U * R * R;
    if (!(r2 > 0.f) || r2 > 3e38f) return Band{0.f, 0.f};  // r = 0 or infinite: d2 < r2 is fixed
    const float r = sqrtf(r2) * 1.0001f;
    return Band{(k_rel + 0.8661f * k_abs / r) * 1.001f,
                (k_rel * r2 * 1.0001f + 0.8661f * k_abs * r + k_sq) * 1.001f};
}

// ---- key sort: items per block of the radix-sort passes (256 threads x 4) -----
constexpr int kSortTileItems = 1024;
// A tree level with at most this many nodes (the top of the tree: few nodes of
// many particles) is split one node per warp, tiles of 8 nodes; deeper levels
// one node per thread, tiles of 256.
constexpr int kTopoWideNodes = 4096;

// ---- device metadata block (one per context) -------------------------------
struct Meta {
    int err;                       // first latched error code (0 = none)
    int n_nodes;
    int n_groups;
    int depth;
    int n_leaves;
    int level_start[kMaxLevelSlots];
    int level_count[kMaxLevelSlots];
    unsigned int tickets[32];      // work-distribution counters (reset per launch)
    long long nbr_total;
    long long fallback_tests;      // FP64 decisions taken after an undecided FP32 filter
    unsigned long long core_count; // particles within the core radius (core quantities)
    int row_class[20];             // neighbour rows by length class: counts, fill cursors
    int uncounted;                 // clusters whose neighbours the mixed walk does not count
    int row_over;                  // row mode: a row outgrew its room since the rows were laid out
    long long spin_limit;          // polls of a bounded wait (0: kSpinLimit)
    int cell_forms[2];             // clusters whose groups take the r^-5 / the r^-3 cell term
};

// ---- one cluster of a (possibly batched) build -----------------------------------
struct Cluster {
    double cube[4];                // min.xyz, side (rule 1)
    double scale;                  // 2^21 / side
    double frame[4];               // O.xyz (box centre), R (bound on |x - O| per axis)
    unsigned long long minmax[6];  // order-preserving encodings for the bbox reduction
    // physics of this cluster (the context's parameters, or the batch's table)
    double theta, r_in, r_out, r_list;
    double rout2_d, rl2_d, inv_dr_d;        // r_out^2, r_list^2, 1/(r_out - r_in)
    float rout2_f, rl2_f, rl_f, inv_dr_f, rin_dr_f;
    int counted;                   // 1: the mixed far-force walk counts its neighbours
    int fast_cells;                // 1: the r^-5 cell term stays in the FP32 range (walk)
};

// ---- tree view passed by value to kernels ------------------------------------
struct Tree {
    int n;
    int cap_nodes;
    int n_clusters;        // independent clusters; cluster c's root is node c
    const int64_t *seg;    // device cluster offsets [n_clusters + 1] (null: one cluster)
    int32_t *cid;          // cluster of each particle, original order (null: one cluster)
    int32_t *cid_s;        // cluster of each particle, key order
    Cluster *cl;
    uint64_t *keys;
    int32_t *perm;
    double4_32a *sp;
    float4 *ph, *pl;
    int4 *topo;
    int32_t *level;
    int32_t *parent;
    double4_32a *comM;
    double4_32a *lo;
    double4_32a *hi;
    double *q64;   // 6 per node (FP64 form)
    float *q32;    // 6 per node (mixed form)
    float4 *wn;    // kWalkRecord float4 per node (layout: wrec)
    int2 *grp;
    double4_32a *glo, *ghi;
    // per group, three float4 made once per build (mixed walks): the double-single
    // split of c_g - O {hx hy hz lx} {ly lz, box lo - O: x y} {z, box hi - O: x y z}
    float4 *gfr;
    int32_t *gorder;       // the walks' order of the groups (smallest boxes first)
    unsigned char *gflag;  // group-start flags, particle order
    int32_t *gidx;         // scan of gflag
    int32_t *leaves;       // leaf node indices, in creation order (moments work list)
    int32_t *inv;          // original index -> position in key order
    Meta *meta;
    // the ids neighbour rows hold, key order: perm (the caller's original index) or,
    // for a rank of a decomposed cluster, the particle's global index
    int32_t *rid;
    int n_src;             // particles in the source arrays (sp, ph, pl, rid): n, or more
                           // once remote particles are joined to a rank's tree
    // a rank's part of a decomposed cluster: cells split whatever their count (they
    // hold particles of other ranks too) and never cut into walk groups
    int n_top;
    const unsigned long long *top_key;  // first key of each such cell
    const int32_t *top_level;
};

// Row mode: target s (key order) owns scratch entries [row_off[s], row_off[s + 1])
// clipped to the scratch; a row with more neighbours comes from the fill pass.
__device__ __forceinline__ void row_span(const int64_t *row_off, long long entries, int s, long long &lo, int &cap)
{
    lo = row_off[s];
    const long long hi = row_off[s + 1] < entries ? row_off[s + 1] : entries;
    cap = hi > lo ? (int)(hi - lo) : 0;
}

constexpr int kMaxTopCells = 256;  // top cells of a decomposed cluster (about 21 per splitter)

// node k of a range build is a top cell: level l, prefix = its first key >> (63 - 3 l)
__device__ __forceinline__ bool is_top_cell(const Tree &T, int l, unsigned long long prefix)
{
    for (int i = 0; i < T.n_top; i++)
        if (T.top_level[i] == l && (T.top_key[i] >> (63 - 3 * l)) == prefix) return true;
    return false;
}

// ---- error latch ---------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with launch_pdl may be scheduled
// while the kernel before it on the stream drains; it calls pdl_wait() before its
// first memory access, which returns once that kernel has completed and its writes
// are visible (a no-op for a kernel launched the ordinary way).  What overlaps is
// the launch latency alone.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl_smem(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                          cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s,
                                     Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

__device__ __forceinline__ void latch_error(Meta *m, int code)
{
    atomicCAS(&m->err, 0, code);
}

// ---- exact FP64 arithmetic (never contracted into FMA) -------------------------
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double dsqrt(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ double dmax(double a, double b) { return a > b ? a : b; }
__device__ __forceinline__ double dmin(double a, double b) { return a < b ? a : b; }

// Squared distance from point p to box [lo, hi]: per axis max(0, lo-p, p-hi),
// summed as (tx*tx + ty*ty) + tz*tz.  Same operation order as the oracle.
__device__ __forceinline__ double dist2_point_box(double px, double py, double pz, double4_32a lo,
                                                  double4_32a hi)
{
    double tx = dmax(dmax(dsub(lo.x, px), dsub(px, hi.x)), 0.0);
    double ty = dmax(dmax(dsub(lo.y, py), dsub(py, hi.y)), 0.0);
    double tz = dmax(dmax(dsub(lo.z, pz), dsub(pz, hi.z)), 0.0);
    return dadd(dadd(dmul(tx, tx), dmul(ty, ty)), dmul(tz, tz));
}

// Squared distance between group box g and cell box c: per axis
// max(0, clo - ghi, glo - chi).
__device__ __forceinline__ double dist2_box_box(double4_32a glo, double4_32a ghi, double4_32a clo, double4_32a chi)
{
    double tx = dmax(dmax(dsub(clo.x, ghi.x), dsub(glo.x, chi.x)), 0.0);
    double ty = dmax(dmax(dsub(clo.y, ghi.y), dsub(glo.y, chi.y)), 0.0);
    double tz = dmax(dmax(dsub(clo.z, ghi.z), dsub(glo.z, chi.z)), 0.0);
    return dadd(dadd(dmul(tx, tx), dmul(ty, ty)), dmul(tz, tz));
}

// Double-single split of an FP64 value: v ~ hi + lo with |v - hi - lo| <= 2^-48 |v|.
__device__ __forceinline__ void ds_split(double v, float &hi, float &lo)
{
    hi = __double2float_rn(v);
    lo = __double2float_rn(dsub(v, (double)hi));
}

// ---- relaxed device-scope loads/stores for cross-block flags ---------------------
__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// ---- warp traversal stack of node ranges -------------------------------------------
// Entries pack (first node << 3) | (count - 1), count 1..8 (the children of one
// node).  pop_batch takes up to 32 nodes from the top entries, one per lane,
// and returns this lane's node (-1 if none); a partly taken entry is advanced
// in place.  The prefix sum of the entry sizes is formed from four ballots of
// the size bits, and the lane -> entry map from the mask of entry starts.
__device__ __forceinline__ int pack_range(int first, int count) { return (first << 3) | (count - 1); }

__device__ __forceinline__ int pop_batch(int *stk, int &sp)
{
    const unsigned full_mask = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int e = lane < sp ? stk[sp - 1 - lane] : 0;
    const int cnt = lane < sp ? (e & 7) + 1 : 0;
    const unsigned b0 = __ballot_sync(full_mask, cnt & 1), b1 = __ballot_sync(full_mask, cnt & 2),
                   b2 = __ballot_sync(full_mask, cnt & 4), b3 = __ballot_sync(full_mask, cnt & 8);
    const int excl = __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt) + 8 * __popc(b3 & lt);
    const int total = __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2) + 8 * __popc(b3);
    const int take = total < 32 ? total : 32;
    const bool starts = cnt > 0 && excl < take;
    const unsigned smask = __reduce_or_sync(full_mask, starts ? (1u << excl) : 0u);
    const unsigned consumed = __ballot_sync(full_mask, cnt > 0 && excl + cnt <= take);
    if (starts && excl + cnt > take) stk[sp - 1 - lane] = pack_range((e >> 3) + (take - excl), cnt - (take - excl));
    const unsigned le = lane == 31 ? full_mask : ((2u << lane) - 1u);
    const int k = (__popc(smask & le) - 1) & 31;
    const int kfirst = __shfl_sync(full_mask, e >> 3, k);
    const int kexcl = __shfl_sync(full_mask, excl, k);
    sp -= __popc(consumed);
    __syncwarp();
    return lane < take ? kfirst + (lane - kexcl) : -1;
}

// The far-force walk's stack entries may carry a flag in bit 31 (ranges visited
// only for the neighbour count); node indices then stay below 2^28.
constexpr unsigned kRangeFlag = 0x80000000u;
// leaf-queue entries: bit 30 marks a leaf whose box lies r_out or more from the
// group's box (particle indices stay below the node capacity bound 2^28)
constexpr unsigned kFarLeaf = 0x40000000u;
__device__ __forceinline__ int pack_range_f(int first, int count, bool flag)
{
    return (int)(((unsigned)first << 3) | (unsigned)(count - 1) | (flag ? kRangeFlag : 0u));
}

// pop_batch for flagged entries: also returns this lane's entry flag.
__device__ __forceinline__ int pop_batch_f(int *stk, int &sp, bool &flag)
{
    const unsigned full_mask = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int e = lane < sp ? stk[sp - 1 - lane] : 0;
    const int first_e = (int)(((unsigned)e >> 3) & 0x0fffffffu);
    const int cnt = lane < sp ? (e & 7) + 1 : 0;
    const unsigned b0 = __ballot_sync(full_mask, cnt & 1), b1 = __ballot_sync(full_mask, cnt & 2),
                   b2 = __ballot_sync(full_mask, cnt & 4), b3 = __ballot_sync(full_mask, cnt & 8);
    const int excl = __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt) + 8 * __popc(b3 & lt);
    const int total = __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2) + 8 * __popc(b3);
    const int take = total < 32 ? total : 32;
    const bool starts = cnt > 0 && excl < take;
    const unsigned smask = __reduce_or_sync(full_mask, starts ? (1u << excl) : 0u);
    const unsigned consumed = __ballot_sync(full_mask, cnt > 0 && excl + cnt <= take);
    if (starts && excl + cnt > take)
        stk[sp - 1 - lane] = pack_range_f(first_e + (take - excl), cnt - (take - excl), e < 0);
    const unsigned le = lane == 31 ? full_mask : ((2u << lane) - 1u);
    const int k = (__popc(smask & le) - 1) & 31;
    const int kraw = __shfl_sync(full_mask, e, k);
    const int kexcl = __shfl_sync(full_mask, excl, k);
    sp -= __popc(consumed);
    __syncwarp();
    flag = lane < take && kraw < 0;
    return lane < take ? (int)(((unsigned)kraw >> 3) & 0x0fffffffu) + (lane - kexcl) : -1;
}

// ---- block-wide exclusive scan (blockDim.x a multiple of 32, <= 1024) --------------
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Returns the exclusive prefix of v within the block; *total gets the block sum.
// `sh` must hold 32 elements of T.  Contains __syncthreads.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T *total, T *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T s = lane < nw ? sh[lane] : T(0);
        s = warp_incl_scan(s);
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    T base = wid > 0 ? sh[wid - 1] : T(0);
    *total = sh[nw - 1];
    __syncthreads();
    return base + inc - v;
}

// ---- decoupled look-back across blocks -----------------------------------------
// status[t]: bits 62-63 = flag (0 none, 1 aggregate, 2 inclusive prefix), bits
// 0-61 = value.  Called by ALL threads of the block holding ticket t with the
// block aggregate; returns the exclusive prefix of the block.  The wait on a
// predecessor is bounded: after Meta::spin_limit polls the error is latched and the
// partial prefix is used, so the kernel always terminates.
constexpr unsigned long long kFlagAgg = 1ULL << 62, kFlagPre = 2ULL << 62,
                             kValMask = (1ULL << 62) - 1;

__device__ __forceinline__ long long lookback_prefix(unsigned long long *status, int t,
                                                      long long aggregate, Meta *meta,
                                                      long long *sh_out)
{
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        long long excl = 0;
        if (t == 0) {
            if (lane == 0) st_relaxed(&status[0], kFlagPre | (unsigned long long)aggregate);
        } else {
            if (lane == 0) st_relaxed(&status[t], kFlagAgg | (unsigned long long)aggregate);
            int j = t - 1;  // this lane inspects j - lane
            const long long limit = meta->spin_limit > 0 ? meta->spin_limit : kSpinLimit;
            long long spins = 0;
            while (true) {
                int idx = j - lane;
                unsigned long long s = idx >= 0 ? ld_relaxed(&status[idx]) : kFlagPre;
                unsigned long long flag = s & ~kValMask;
                // wait until every inspected predecessor published something
                if (__any_sync(0xffffffffu, flag == 0)) {
                    if (++spins > limit) {
                        if (lane == 0) latch_error(meta, P3T_ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(spins < 64 ? 32 : 256);
                    continue;
                }
                unsigned pre = __ballot_sync(0xffffffffu, flag == kFlagPre);
                long long val = (long long)(s & kValMask);
                if (idx < 0) val = 0;
                if (pre) {
                    int first_pre = __ffs(pre) - 1;  // nearest predecessor with a prefix
                    long long mine = lane <= first_pre ? val : 0;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
                    excl += mine;
                    break;
                }
                long long mine = val;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
                excl += mine;
                j -= 32;
            }
            if (lane == 0)
                st_relaxed(&status[t], kFlagPre | (unsigned long long)(excl + aggregate));
        }
        if (lane == 0) *sh_out = excl;
    }
    __syncthreads();
    long long r = *sh_out;
    __syncthreads();
    return r;
}

// ---- host helpers ----------------------------------------------------------------
int scan_excl_u8_to_i32(const unsigned char *in, int32_t *out, int n, int32_t *total_dev,
                        unsigned long long *status, unsigned int *ticket, Meta *meta,
                        cudaStream_t s);
int scan_excl_i32_to_i64(const int32_t *in, int64_t *out, int n, int64_t *total_dev,
                         unsigned long long *status, unsigned int *ticket, Meta *meta,
                         cudaStream_t s);
int scan_excl_i32_to_i32(const int32_t *in, int32_t *out, int n, unsigned long long *status,
                         unsigned int *ticket, Meta *meta, cudaStream_t s);
int scan_status_words(int n);  // status array length for an n-element scan
int scan_excl_i32_to_i32_cleared(const int32_t *in, int32_t *out, int n, unsigned long long *status,
                                 unsigned int *ticket, Meta *meta, cudaStream_t s);
int scan_excl_i32_to_i64_cleared(const int32_t *in, int64_t *out, int n, int64_t *total_dev,
                                 unsigned long long *status, unsigned int *ticket, Meta *meta, cudaStream_t s);
// clears a scan's status words and ticket (one block of a kernel that runs before it)
__device__ __forceinline__ void clear_scan_state(unsigned long long *status, int nwords, unsigned int *ticket)
{
    for (int t = threadIdx.x; t < nwords; t += blockDim.x) status[t] = 0ULL;
    if (threadIdx.x == 0) *ticket = 0u;
}

}  // namespace p3t

// ---- context ---------------------------------------------------------------------------
struct p3t_ctx {
    p3t_params prm;
    cudaStream_t stream;
    int device;
    int debug;
    int sm_count;
    // capacities of the current allocation
    long long cap_n;
    long long cap_nodes;
    int cap_leaf;
    int has_q64;
    // state
    int n;
    int built;
    int built_precision;
    int counts_valid;  // neighbour counts of the current tree already in nbr_count
    int rows_valid;    // the walk wrote the rows of the current tree into row_scratch
    int walk_counted;  // the far-force walk counted the neighbours of clusters with `counted`
    int uniform_params;  // every cluster uses the context's parameters
    int cap_clusters;
    p3t::Cluster *clusters;  // per-cluster table (separate allocation)
    int pending_err;  // host-side latched error
    long long spin_limit;  // polls of a bounded device wait (0: the default)
    // device memory
    p3t::Meta *meta;
    p3t::Tree tree;
    uint64_t *keys_buf[2];
    int32_t *perm_buf[2];
    int32_t *sort_hist;               // 256 * sort blocks
    unsigned long long *scan_status;  // look-back status words
    int32_t *nbr_count;               // per particle (original order)
    int32_t *row_list;                // neighbour rows binned by length class
    int32_t *rid_buf;                 // global row ids of a range build (key order)
    unsigned long long *top_buf;      // top cells of a range build: keys, then levels
    int32_t *row_scratch;             // row mode: neighbour rows written by the far-force walk
    size_t row_scratch_entries;       // (rows in key order, laid out by row_off)
    int row_cap;                      // > 0: row mode on (the scratch's mean entries per particle)
    int rows_cap_used;                // row_off lays out the rows of the current tree
    int64_t *row_off;                 // row mode: first scratch entry of each row, key order (n + 1)
    long long counts_n;               // nbr_count holds every particle's count for these n particles
    int64_t *grp_cells, *grp_parts;   // per group debug counts
    void *blob;                       // single allocation backing everything above
    size_t blob_bytes;
    void *host_stage;                 // device staging of p3t_step_host
    size_t host_stage_bytes;
    cudaStream_t side_stream;         // the build's groups, beside its moments (null: in line)
    cudaEvent_t fork_ev, join_ev;
    cudaStream_t side_stream2;        // the row sort's third branch (null: on side_stream)
    cudaEvent_t join_ev2;
    cudaStream_t copy_stream;         // p3t_step_host: velocity upload and neighbour-list
    cudaEvent_t lists_ready;          // copy beside the build and the far force
    cudaEvent_t v_ready;
    unsigned long long gen;           // bumped whenever blob or clusters move
    void *irr_buf;                    // double-single states of p3t_irregular (mixed)
    size_t irr_bytes;
    void *knn_buf;                    // per-chunk lists of p3t_sample_knn6
    size_t knn_bytes;
    // a rank's part of a decomposed cluster (decomp.cu)
    int range_built;                  // the current tree came from p3t_build_tree_range
    int joined;                       // ... and has been joined with remote trees
    int n_top;                        // its top cells (host copy)
    unsigned long long top_key[p3t::kMaxTopCells];
    int32_t top_level[p3t::kMaxTopCells];
    double gbox[6];                   // the global bounding box
    void *dec_buf;                    // working memory of the decomposition calls
    size_t dec_bytes;
    void *join_buf;                   // the joined tree's node and particle arrays
    size_t join_bytes;
};

namespace p3t {
// Host-side state that the entry points update as they enqueue work; a CUDA
// graph restores the state of its captured step when it is launched.
struct HostState {
    int n, built, built_precision, counts_valid, walk_counted, uniform_params;
    int rows_valid, rows_cap_used;
    Tree tree;
};
inline HostState save_state(const p3t_ctx *c)
{
    return HostState{c->n,           c->built,          c->built_precision,
                     c->counts_valid, c->walk_counted,  c->uniform_params,
                     c->rows_valid,  c->rows_cap_used, c->tree};
}
inline void restore_state(p3t_ctx *c, const HostState &h)
{
    c->n = h.n, c->built = h.built, c->built_precision = h.built_precision;
    c->counts_valid = h.counts_valid, c->walk_counted = h.walk_counted;
    c->uniform_params = h.uniform_params, c->tree = h.tree;
    c->rows_valid = h.rows_valid, c->rows_cap_used = h.rows_cap_used;
}
}  // namespace p3t

namespace p3t {
int ensure_capacity(p3t_ctx *c, long long n);
int irregular(p3t_ctx *c, int n, const int64_t *offs, const int32_t *idx, const double *x,
              const double *y, const double *z, const double *m, const double *vx,
              const double *vy, const double *vz, double *fx, double *fy, double *fz, double *jx,
              double *jy, double *jz);
int reserve(p3t_ctx *c, long long n, int n_clusters);
int scan_stalled(int n, const int32_t *in, int32_t *out, unsigned long long *status,
                 unsigned int *ticket, Meta *meta, cudaStream_t s);
int check_launch(p3t_ctx *c);
int prepare_rows(p3t_ctx *c);
// A rank's part of a decomposed cluster (p3t_build_tree_range): the global bounding
// box (min xyz, max xyz), the ranks' top cells and the particles' global indices.
struct RangeSpec {
    double box[6];
    int n_top;
    const int64_t *gid;  // device, the caller's order (null: rows hold local indices)
};
int build_tree(p3t_ctx *c, int n, int n_clusters, const int64_t *seg, const double *cprm,
               const double *x, const double *y, const double *z, const double *m,
               const RangeSpec *range = nullptr);
void reset_tree_views(p3t_ctx *c);
int global_frame(cudaStream_t s, const double box[6], Cluster *cl, Meta *meta);
int far_force(p3t_ctx *c, void *ax, void *ay, void *az, double *pot, int64_t *nc, int64_t *np);
int neighbours(p3t_ctx *c, int64_t *offsets, int32_t *idx, long long capacity, int64_t *total_dev,
               bool sync, int64_t *total_host);
int kick(p3t_ctx *c, double dt, const void *ax, const void *ay, const void *az, double *vx,
         double *vy, double *vz);
int drift(p3t_ctx *c, int n, double dt, double *x, double *y, double *z, const double *vx,
          const double *vy, const double *vz);
int export_tree(p3t_ctx *c, uint64_t *keys, int32_t *perm, int32_t *level, int32_t *first,
                int32_t *count, int32_t *child, int32_t *nchild, double *M, double *com,
                double *Q, double *lo, double *hi, double *ropen2, int32_t *g_first,
                int32_t *g_count);
}  // namespace p3t
