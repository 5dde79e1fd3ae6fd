// One cluster decomposed over several ranks (the multi-GPU force calculator the
// paper names as future work, Sec. 4).  Rank r holds the particles whose Morton
// keys lie in [b_r, b_r+1), splitters chosen at cell boundaries of the global octree
// so that every cell straddling a splitter ("top cell") holds more than
// max(16 G, leaf_cap) particles: then the global tree is the top cells plus, below
// them, complete subtrees that each belong to one rank, and the global walk groups
// lie inside single ranks.
//
// Per step, with every call here on one rank's context:
//   p3t_local_bbox        the rank's bounding box (the caller reduces them: rule 1's box)
//   p3t_key_range_counts  particles per key interval, for choosing the splitters and
//                         the top cells (the caller sums them over ranks)
//   p3t_partition         the particles packed by destination rank
//   p3t_build_tree_range  (ctx.cu) the rank's tree: top cells split whatever their
//                         count, sorted by (key, global index)
//   p3t_subtree_boxes     the boxes of the rank's subtree roots (every group lies in one)
//   p3t_let_export        the locally essential tree for another rank: the rank's
//                         subtrees as the receiver's subtree boxes see them (rule 8 with
//                         the receiver's radius), nodes and the particles of opened leaves
//   p3t_tree_join         the rank's tree joined with the top tree and the remote
//                         subtrees: its groups then walk the global tree, so their
//                         interaction lists, forces and neighbour rows are those of a
//                         single build of the whole cluster
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "build_common.cuh"

namespace p3t {

constexpr int kDecThreads = 256;
constexpr int kMaxRanges = 1024;  // key intervals of one p3t_key_range_counts call
constexpr int kMaxDomainBoxes = 4096;  // a rank's subtree roots (the receiver's boxes of a LET)

// Morton key of a point in the cube of K (rules 2-3, as keys_kernel computes it)
__device__ __forceinline__ unsigned long long key_of(double x, double y, double z, const Cluster &K)
{
    const double s = K.scale;
    return (spread3(quantise(x, K.cube[0], s)) << 2) | (spread3(quantise(y, K.cube[1], s)) << 1) |
           spread3(quantise(z, K.cube[2], s));
}

// ---- one node of a locally essential tree, as shipped between ranks ---------------
// The records a walk reads (relative to the frame centre O, which every rank shares),
// the FP64 data of its exact decisions and moments, and the node's links in the
// sender's LET numbering.
struct LetNode {
    float4 wn[kWalkRecord];
    double4_32a comM, lo, hi;
    double q64[6];
    float q32[6];
    int32_t link;   // opened internal: first child (LET index); opened leaf: -1 - first particle
    int32_t cnt;    // children or particles
    uint64_t key;   // first key of the node's cell
    int32_t level;
    int32_t kind;   // 0 opened internal node, 1 opened leaf, 2 accepted (no children shipped)
};
struct LetPart {
    double4_32a sp;
    float4 ph, pl;
    int32_t rid;
    int32_t pad[7];
};
static_assert(sizeof(LetNode) == P3T_LET_NODE_BYTES, "LET node size");
static_assert(sizeof(LetPart) == P3T_LET_PART_BYTES, "LET particle size");

// working memory of the decomposition calls (grown on demand, never shrunk)
static int dec_reserve(p3t_ctx *c, size_t bytes)
{
    if (bytes <= c->dec_bytes) return P3T_OK;
    cudaStreamSynchronize(c->stream);
    if (c->dec_buf) cudaFree(c->dec_buf);
    c->dec_buf = nullptr;
    c->dec_bytes = 0;
    if (cudaMalloc(&c->dec_buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return P3T_ERR_OOM;
    }
    c->dec_bytes = bytes;
    return P3T_OK;
}

static size_t al(size_t v) { return (v + 255) / 256 * 256; }

// ---- bounding box ----------------------------------------------------------------
__global__ void __launch_bounds__(kDecThreads)
    box_kernel(int n, const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
               unsigned long long *enc, Meta *meta)
{
    unsigned long long mn[3] = {~0ULL, ~0ULL, ~0ULL}, mx[3] = {0, 0, 0};
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double p[3] = {x[i], y[i], z[i]};
#pragma unroll
        for (int d = 0; d < 3; d++) {
            bad |= !isfinite(p[d]);
            const unsigned long long e = enc_double(p[d]);
            mn[d] = e < mn[d] ? e : mn[d];
            mx[d] = e > mx[d] ? e : mx[d];
        }
    }
#pragma unroll
    for (int d = 0; d < 3; d++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long a = __shfl_xor_sync(0xffffffffu, mn[d], o);
            const unsigned long long b = __shfl_xor_sync(0xffffffffu, mx[d], o);
            mn[d] = a < mn[d] ? a : mn[d];
            mx[d] = b > mx[d] ? b : mx[d];
        }
    }
    if ((threadIdx.x & 31) == 0)
        for (int d = 0; d < 3; d++) {
            atomicMin(&enc[d], mn[d]);
            atomicMax(&enc[3 + d], mx[d]);
        }
    if (bad) latch_error(meta, P3T_ERR_INVALID_INPUT);
}

__global__ void box_init_kernel(unsigned long long *enc)
{
    for (int d = 0; d < 3; d++) enc[d] = ~0ULL, enc[3 + d] = 0ULL;
}

__global__ void box_decode_kernel(const unsigned long long *enc, double *out)
{
    for (int d = 0; d < 6; d++) out[d] = dec_double(enc[d]);
}

// ---- particles per key interval ----------------------------------------------------
__global__ void __launch_bounds__(kDecThreads)
    range_count_kernel(int n, const double *__restrict__ x, const double *__restrict__ y,
                       const double *__restrict__ z, const Cluster *cl, int nr,
                       const unsigned long long *__restrict__ rlo, const unsigned long long *__restrict__ rhi,
                       unsigned long long *counts)
{
    __shared__ unsigned int sh[kMaxRanges];
    for (int r = threadIdx.x; r < nr; r += blockDim.x) sh[r] = 0;
    __syncthreads();
    const Cluster K = cl[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned long long k = key_of(x[i], y[i], z[i], K);
        for (int r = 0; r < nr; r++)
            if (k >= rlo[r] && k < rhi[r]) atomicAdd(&sh[r], 1u);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nr; r += blockDim.x)
        if (sh[r]) atomicAdd(&counts[r], (unsigned long long)sh[r]);
}

// ---- packing by destination rank -----------------------------------------------------
__global__ void __launch_bounds__(kDecThreads)
    dest_kernel(int n, const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                const Cluster *cl, int nb, const unsigned long long *__restrict__ bounds, int32_t *__restrict__ dest)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long k = key_of(x[i], y[i], z[i], cl[0]);
    int lo = 0, hi = nb;  // last r with bounds[r] <= k
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (bounds[mid] <= k)
            lo = mid;
        else
            hi = mid;
    }
    dest[i] = lo;
}

__global__ void __launch_bounds__(kDecThreads)
    dest_flag_kernel(int n, const int32_t *__restrict__ dest, int d, unsigned char *__restrict__ flag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = dest[i] == d;
}

struct PackArrays {
    const unsigned long long *src[8];
    unsigned long long *dst[8];
    int n;
};

__global__ void __launch_bounds__(kDecThreads)
    pack_kernel(int n, const int32_t *__restrict__ dest, int d, const int32_t *__restrict__ pos, long long base,
                PackArrays A)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || dest[i] != d) return;
    const long long o = base + pos[i];
#pragma unroll
    for (int a = 0; a < 8; a++)
        if (a < A.n) A.dst[a][o] = A.src[a][i];
}

// ---- locally essential tree ------------------------------------------------------------
// The rank's subtree roots: nodes outside the top cells whose parent is a top cell
// (node order, i.e. breadth first).
__global__ void __launch_bounds__(kDecThreads) root_flag_kernel(Tree T, int nn, unsigned char *flag)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nn) return;
    const int4 tp = T.topo[k];
    const int l = T.level[k];
    const bool top = tp.y > 0 && is_top_cell(T, l, T.keys[tp.x] >> (63 - 3 * l));
    bool root = false;
    if (!top && T.parent[k] >= 0) {
        const int p = T.parent[k];
        const int4 pp = T.topo[p];
        root = pp.y > 0 && is_top_cell(T, l - 1, T.keys[pp.x] >> (63 - 3 * (l - 1)));
    }
    flag[k] = root;
}

__global__ void __launch_bounds__(kDecThreads)
    compact_kernel(int nn, const unsigned char *__restrict__ flag, const int32_t *__restrict__ pos,
                   int32_t *__restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nn && flag[k]) out[pos[k]] = k;
}

// One level of the LET: frontier node f (local id front[f], LET index base + f) is
// opened iff the receiver's domain box B would open it (rule 8 with the receiver's
// radius, exact FP64); opened internal nodes contribute their children to the next
// frontier, opened leaves their particles.  Pass 0 counts them (nch, npt); pass 1
// forms the next frontier and, when `write`, the LET records and particles.
__global__ void __launch_bounds__(kDecThreads)
    let_level_kernel(Tree T, int nf, const int32_t *__restrict__ front, int nbox, const double4_32a *__restrict__ boxes,
                     double r2, int pass, int32_t *__restrict__ nch, int32_t *__restrict__ npt,
                     const int64_t *__restrict__ ch_off, const int64_t *__restrict__ pt_off, long long next_base,
                     long long part_base, int32_t *__restrict__ next, bool write, LetNode *out_nodes,
                     long long node_base, LetPart *out_parts, bool q64)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int u = front[f];
    const int4 tp = T.topo[u];
    const double4_32a cm = T.comM[u], cl = T.lo[u], ch = T.hi[u];
    // opened iff one of the receiver's boxes opens it (each of its groups lies in one)
    bool open = false;
    for (int i = 0; i < nbox && !open; i++) {
        const double4_32a blo = boxes[2 * i], bhi = boxes[2 * i + 1];
        open = dist2_point_box(cm.x, cm.y, cm.z, blo, bhi) < cl.w || dist2_box_box(blo, bhi, cl, ch) < r2;
    }
    const bool leaf = tp.z < 0;
    if (pass == 0) {
        nch[f] = open && !leaf ? tp.w : 0;
        npt[f] = open && leaf ? tp.y : 0;
        return;
    }
    if (open && !leaf)
        for (int j = 0; j < tp.w; j++) next[ch_off[f] + j] = tp.z + j;
    if (!write) return;
    LetNode &o = out_nodes[node_base + f];
    const auto w = wrec_at(T.wn, u);
#pragma unroll
    for (int j = 0; j < kWalkRecord; j++) o.wn[j] = w[j];
    o.comM = cm, o.lo = cl, o.hi = ch;
    for (int a = 0; a < 6; a++) {
        o.q64[a] = q64 ? T.q64[6 * (size_t)u + a] : 0.0;
        o.q32[a] = q64 ? 0.f : T.q32[6 * (size_t)u + a];
    }
    o.key = T.keys[tp.x];
    o.level = T.level[u];
    if (open && !leaf) {
        o.kind = 0;
        o.link = (int32_t)(next_base + ch_off[f]);
        o.cnt = tp.w;
    } else if (open) {
        o.kind = 1;
        o.link = (int32_t)(-1 - (part_base + pt_off[f]));
        o.cnt = tp.y;
        for (int j = 0; j < tp.y; j++) {
            LetPart &p = out_parts[part_base + pt_off[f] + j];
            const int s = tp.x + j;
            p.sp = T.sp[s];
            p.ph = T.ph[s];
            p.pl = T.pl[s];
            p.rid = T.rid[s];
        }
    } else {
        o.kind = 2;  // accepted by every group of the receiver: never opened there
        o.link = 0;
        o.cnt = 0;
    }
}

// level and first key of the listed nodes (the skeleton of a join)
__global__ void node_keys_kernel(Tree T, int n, const int32_t *__restrict__ ids, int32_t *__restrict__ level,
                                 unsigned long long *__restrict__ key)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = ids[i];
    level[i] = T.level[k];
    key[i] = T.keys[T.topo[k].x];
}

// the exact boxes (min xyz, max xyz) of the listed nodes
__global__ void node_boxes_kernel(Tree T, int n, const int32_t *__restrict__ ids, double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4_32a l = T.lo[ids[i]], h = T.hi[ids[i]];
    double *o = out + 6 * (size_t)i;
    o[0] = l.x, o[1] = l.y, o[2] = l.z, o[3] = h.x, o[4] = h.y, o[5] = h.z;
}

__global__ void __launch_bounds__(kDecThreads) top_flag_kernel(Tree T, int nn, unsigned char *flag)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nn) return;
    const int4 tp = T.topo[k];
    const int l = T.level[k];
    flag[k] = tp.y > 0 && is_top_cell(T, l, T.keys[tp.x] >> (63 - 3 * l));
}

// ---- joining ---------------------------------------------------------------------------
// New index of every local node: skeleton nodes (top cells and roots) from the
// host's table, the others in order after the skeleton.
__global__ void __launch_bounds__(kDecThreads)
    interior_flag_kernel(Tree T, int nn, const unsigned char *__restrict__ root, unsigned char *__restrict__ flag)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nn) return;
    const int4 tp = T.topo[k];
    const int l = T.level[k];
    const bool top = tp.y > 0 && is_top_cell(T, l, T.keys[tp.x] >> (63 - 3 * l));
    flag[k] = !top && !root[k];
}

__global__ void __launch_bounds__(kDecThreads)
    local_map_kernel(int nn, const unsigned char *__restrict__ interior, const int32_t *__restrict__ pos, int base,
                     int32_t *__restrict__ map)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nn) map[k] = interior[k] ? base + pos[k] : -1;
}

__global__ void skel_map_kernel(int ns, const int32_t *__restrict__ node, const int32_t *__restrict__ idx,
                                int32_t *__restrict__ map)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ns) map[node[i]] = idx[i];
}

// the arrays of the joined tree
struct Joined {
    int4 *topo;
    double4_32a *comM, *lo, *hi;
    double *q64;
    float *q32;
    float4 *wn;
    double4_32a *sp;
    float4 *ph, *pl;
    int32_t *rid, *cid_s;
};

__device__ __forceinline__ void put_links(const Joined &J, int k, int4 tp)
{
    J.topo[k] = tp;
    const auto w = wrec_at(J.wn, k);
    const bool leaf = tp.z < 0;
    w[1].w = __int_as_float(leaf ? -1 - tp.x : tp.z);
    w[2].w = __int_as_float(leaf ? tp.y : tp.w);
}

// local nodes that are not top cells: records copied, child links renumbered
__global__ void __launch_bounds__(kDecThreads)
    copy_local_kernel(Tree T, int nn, const int32_t *__restrict__ map, Joined J, bool q64)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nn) return;
    const int d = map[k];
    if (d < 0) return;  // a top cell: its record is made from the joined children
    int4 tp = T.topo[k];
    if (tp.z >= 0) tp.z = map[tp.z];
    J.comM[d] = T.comM[k];
    J.lo[d] = T.lo[k];
    J.hi[d] = T.hi[k];
    for (int a = 0; a < 6; a++) {
        if (q64)
            J.q64[6 * (size_t)d + a] = T.q64[6 * (size_t)k + a];
        else
            J.q32[6 * (size_t)d + a] = T.q32[6 * (size_t)k + a];
    }
    const auto w = wrec_at(T.wn, k);
    const auto o = wrec_at(J.wn, d);
    for (int j = 0; j < kWalkRecord; j++) o[j] = w[j];
    put_links(J, d, tp);
}

// one remote LET: its roots to their skeleton slots, the other nodes after base
__global__ void __launch_bounds__(kDecThreads)
    copy_let_kernel(const LetNode *__restrict__ L, int nl, int nroots, const int32_t *__restrict__ root_idx,
                    int base, long long part_base, int n_parts, Joined J, bool q64, Meta *meta)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nl) return;
    const LetNode &o = L[k];
    const int d = k < nroots ? root_idx[k] : base + (k - nroots);
    int4 tp;
    if (o.kind == 0) {
        const bool ok = o.link >= nroots && o.link + o.cnt <= nl && o.cnt >= 1 && o.cnt <= 8;
        if (!ok) latch_error(meta, P3T_ERR_INVALID_INPUT);
        tp = make_int4(0, 0, ok ? base + (o.link - nroots) : 0, ok ? o.cnt : 0);
    } else if (o.kind == 1) {
        const long long f = -1LL - o.link;
        const bool ok = f >= 0 && f + o.cnt <= n_parts && o.cnt >= 1;
        if (!ok) latch_error(meta, P3T_ERR_INVALID_INPUT);
        tp = make_int4(ok ? (int)(part_base + f) : 0, ok ? o.cnt : 0, -1, 0);
    } else {
        tp = make_int4(0, 0, 0, 0);  // no children: a walk that opened it would latch an error
    }
    J.comM[d] = o.comM;
    J.lo[d] = o.lo;
    J.hi[d] = o.hi;
    for (int a = 0; a < 6; a++) {
        if (q64)
            J.q64[6 * (size_t)d + a] = o.q64[a];
        else
            J.q32[6 * (size_t)d + a] = o.q32[a];
    }
    const auto w = wrec_at(J.wn, d);
    for (int j = 0; j < kWalkRecord; j++) w[j] = o.wn[j];
    put_links(J, d, tp);
}

__global__ void __launch_bounds__(kDecThreads) copy_local_parts_kernel(Tree T, int n, Joined J)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    J.sp[s] = T.sp[s];
    J.ph[s] = T.ph[s];
    J.pl[s] = T.pl[s];
    J.rid[s] = T.rid[s];
    J.cid_s[s] = T.cid_s[s];
}

__global__ void __launch_bounds__(kDecThreads)
    copy_let_parts_kernel(const LetPart *__restrict__ P, int np, long long base, Joined J)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= np) return;
    const LetPart &p = P[s];
    J.sp[base + s] = p.sp;
    J.ph[base + s] = p.ph;
    J.pl[base + s] = p.pl;
    J.rid[base + s] = p.rid;
    J.cid_s[base + s] = 0;
}

// the top cells, deepest first (children before parents), from their joined children
// in octant order (rule 6) with their records (rule 8): one thread, a few dozen nodes
template <bool Q64>
__global__ void top_moments_kernel(Tree T, int ntop, const int32_t *__restrict__ top_idx,
                                   const int32_t *__restrict__ child0, const int32_t *__restrict__ nchild,
                                   double theta)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int i = ntop - 1; i >= 0; i--) {
        const int k = top_idx[i];
        const int4 tp = make_int4(0, 0, child0[i], nchild[i]);
        T.topo[k] = tp;
        internal_moments<Q64>(T, k, tp, theta);
    }
}

__global__ void set_nodes_kernel(Meta *M, int nn) { M->n_nodes = nn; }

}  // namespace p3t

using namespace p3t;

static int sync_status(p3t_ctx *c)
{
    if (cudaGetLastError() != cudaSuccess) return P3T_ERR_CUDA;
    return p3t_status(c);
}

extern "C" {

int p3t_local_bbox(p3t_ctx *c, int64_t n, const double *x, const double *y, const double *z, double *box)
{
    if (!c || !x || !y || !z || !box || n <= 0 || n >= (1LL << 31) - 1) return P3T_ERR_INVALID_ARG;
    int e = reserve(c, 1, 1);  // the metadata block (errors)
    if (e) return e;
    e = dec_reserve(c, 256);
    if (e) return e;
    unsigned long long *enc = (unsigned long long *)c->dec_buf;
    double *out = (double *)(enc + 8);
    box_init_kernel<<<1, 1, 0, c->stream>>>(enc);
    box_kernel<<<2 * c->sm_count, kDecThreads, 0, c->stream>>>((int)n, x, y, z, enc, c->meta);
    box_decode_kernel<<<1, 1, 0, c->stream>>>(enc, out);
    if (cudaMemcpyAsync(box, out, 6 * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return P3T_ERR_CUDA;
    return sync_status(c);
}

int p3t_key_range_counts(p3t_ctx *c, int64_t n, const double *x, const double *y, const double *z,
                         const double *global_box, int32_t n_ranges, const uint64_t *lo, const uint64_t *hi,
                         int64_t *counts)
{
    if (!c || !global_box || !lo || !hi || !counts || n < 0 || n >= (1LL << 31) - 1 || n_ranges < 1 ||
        n_ranges > kMaxRanges || (n > 0 && (!x || !y || !z)))
        return P3T_ERR_INVALID_ARG;
    int e = reserve(c, 1, 1);
    if (e) return e;
    const size_t off_k = al(sizeof(Cluster)), off_c = off_k + al(16 * (size_t)n_ranges);
    e = dec_reserve(c, off_c + al(8 * (size_t)n_ranges));
    if (e) return e;
    char *b = (char *)c->dec_buf;
    Cluster *cl = (Cluster *)b;
    unsigned long long *rk = (unsigned long long *)(b + off_k);
    unsigned long long *cnt = (unsigned long long *)(b + off_c);
    std::vector<unsigned long long> h(2 * (size_t)n_ranges);
    for (int r = 0; r < n_ranges; r++) h[r] = lo[r], h[n_ranges + r] = hi[r];
    e = global_frame(c->stream, global_box, cl, c->meta);
    if (e) return e;
    if (cudaMemcpyAsync(rk, h.data(), 16 * (size_t)n_ranges, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemsetAsync(cnt, 0, 8 * (size_t)n_ranges, c->stream) != cudaSuccess)
        return P3T_ERR_CUDA;
    if (n > 0)
        range_count_kernel<<<2 * c->sm_count, kDecThreads, 0, c->stream>>>((int)n, x, y, z, cl, n_ranges, rk,
                                                                           rk + n_ranges, cnt);
    if (cudaMemcpyAsync(counts, cnt, 8 * (size_t)n_ranges, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return P3T_ERR_CUDA;
    return sync_status(c);
}

int p3t_partition(p3t_ctx *c, int64_t n, const double *x, const double *y, const double *z,
                  const double *global_box, int32_t n_ranks, const uint64_t *bounds, int32_t n_arrays,
                  const void *const *src, void *const *dst, int64_t *counts)
{
    if (!c || !global_box || !bounds || !counts || n < 0 || n >= (1LL << 31) - 1 || n_ranks < 1 ||
        n_ranks > 4096 || n_arrays < 0 || n_arrays > 8 || (n > 0 && (!x || !y || !z)) ||
        (n_arrays > 0 && (!src || !dst)))
        return P3T_ERR_INVALID_ARG;
    if (bounds[0] != 0 || bounds[n_ranks] != (1ULL << 63)) return P3T_ERR_INVALID_ARG;
    for (int r = 0; r < n_ranks; r++)
        if (bounds[r] > bounds[r + 1]) return P3T_ERR_INVALID_ARG;
    PackArrays A;
    A.n = n_arrays;
    for (int a = 0; a < 8; a++) {
        A.src[a] = a < n_arrays ? (const unsigned long long *)src[a] : nullptr;
        A.dst[a] = a < n_arrays ? (unsigned long long *)dst[a] : nullptr;
        if (a < n_arrays && (!A.src[a] || !A.dst[a])) return P3T_ERR_INVALID_ARG;
    }
    for (int r = 0; r < n_ranks; r++) counts[r] = 0;
    if (n == 0) return P3T_OK;
    int e = reserve(c, n, 1);  // scan status words and the metadata block
    if (e) return e;
    const size_t off_b = al(sizeof(Cluster)), off_d = off_b + al(8 * (size_t)(n_ranks + 1)),
                 off_f = off_d + al(4 * (size_t)n), off_p = off_f + al((size_t)n + 16),
                 off_t = off_p + al(4 * (size_t)n);
    e = dec_reserve(c, off_t + 256);
    if (e) return e;
    char *b = (char *)c->dec_buf;
    Cluster *cl = (Cluster *)b;
    unsigned long long *db = (unsigned long long *)(b + off_b);
    int32_t *dest = (int32_t *)(b + off_d);
    unsigned char *flag = (unsigned char *)(b + off_f);
    int32_t *pos = (int32_t *)(b + off_p);
    int32_t *tot = (int32_t *)(b + off_t);
    e = global_frame(c->stream, global_box, cl, c->meta);
    if (e) return e;
    if (cudaMemcpyAsync(db, bounds, 8 * (size_t)(n_ranks + 1), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return P3T_ERR_CUDA;
    const int grid = (int)((n + kDecThreads - 1) / kDecThreads);
    dest_kernel<<<grid, kDecThreads, 0, c->stream>>>((int)n, x, y, z, cl, n_ranks, db, dest);
    long long base = 0;
    for (int d = 0; d < n_ranks; d++) {
        dest_flag_kernel<<<grid, kDecThreads, 0, c->stream>>>((int)n, dest, d, flag);
        e = scan_excl_u8_to_i32(flag, pos, (int)n, tot, c->scan_status, &c->meta->tickets[28], c->meta,
                                c->stream);
        if (e) return e;
        pack_kernel<<<grid, kDecThreads, 0, c->stream>>>((int)n, dest, d, pos, base, A);
        int32_t cnt = 0;
        if (cudaMemcpyAsync(&cnt, tot, 4, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return P3T_ERR_CUDA;
        counts[d] = cnt;
        base += cnt;
    }
    return sync_status(c);
}

// device list of the nodes with flag[k] set, in node order; returns their count
static int flagged_list(p3t_ctx *c, int nn, const unsigned char *flag, int32_t *pos, int32_t *out, int32_t *tot,
                        int *count)
{
    int e = scan_excl_u8_to_i32(flag, pos, nn, tot, c->scan_status, &c->meta->tickets[28], c->meta, c->stream);
    if (e) return e;
    compact_kernel<<<(nn + kDecThreads - 1) / kDecThreads, kDecThreads, 0, c->stream>>>(nn, flag, pos, out);
    if (cudaMemcpyAsync(count, tot, 4, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return P3T_ERR_CUDA;
    return P3T_OK;
}

int p3t_let_export(p3t_ctx *c, int32_t n_boxes, const double *boxes, double r_halo, int64_t cap_nodes, void *nodes,
                   int64_t cap_parts, void *parts, int64_t *n_nodes, int64_t *n_parts, int32_t *n_roots)
{
    if (!c || n_boxes < 1 || n_boxes > kMaxDomainBoxes || !boxes || !n_nodes || !n_parts || !n_roots ||
        !(r_halo >= 0.0) || !std::isfinite(r_halo) || cap_nodes < 0 || cap_parts < 0 || (cap_nodes > 0 && !nodes) ||
        (cap_parts > 0 && !parts))
        return P3T_ERR_INVALID_ARG;
    if (!c->built || !c->range_built || c->joined || c->n_top < 1) return P3T_ERR_ORDER;
    int e = p3t_status(c);
    if (e) return e;
    int nn = 0;
    if (cudaMemcpy(&nn, &c->meta->n_nodes, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return P3T_ERR_CUDA;
    const Tree &T = c->tree;
    const size_t off_p = al((size_t)nn + 16), off_a = off_p + al(4 * (size_t)nn),
                 off_b = off_a + al(4 * (size_t)nn), off_c = off_b + al(4 * (size_t)nn),
                 off_d = off_c + al(4 * (size_t)nn), off_e = off_d + al(4 * (size_t)nn),
                 off_g = off_e + al(8 * (size_t)nn), off_t = off_g + al(8 * (size_t)nn),
                 off_x = off_t + 256;
    e = dec_reserve(c, off_x + al(64 * (size_t)n_boxes));
    if (e) return e;
    char *b = (char *)c->dec_buf;
    double4_32a *dbox = (double4_32a *)(b + off_x);
    {
        std::vector<double4_32a> hb(2 * (size_t)n_boxes);
        for (int i = 0; i < n_boxes; i++) {
            const double *q = boxes + 6 * (size_t)i;
            hb[2 * i] = make_double4_32a(q[0], q[1], q[2], 0.0);
            hb[2 * i + 1] = make_double4_32a(q[3], q[4], q[5], 0.0);
        }
        if (cudaMemcpyAsync(dbox, hb.data(), 64 * (size_t)n_boxes, cudaMemcpyHostToDevice, c->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return P3T_ERR_CUDA;
    }
    unsigned char *flag = (unsigned char *)b;
    int32_t *pos = (int32_t *)(b + off_p);
    int32_t *front = (int32_t *)(b + off_a), *next = (int32_t *)(b + off_b);
    int32_t *nch = (int32_t *)(b + off_c), *npt = (int32_t *)(b + off_d);
    int64_t *cho = (int64_t *)(b + off_e), *pto = (int64_t *)(b + off_g);
    int32_t *tot = (int32_t *)(b + off_t);
    int64_t *tot64 = (int64_t *)(b + off_t + 64);
    cudaStream_t s = c->stream;
    const int gnn = (nn + kDecThreads - 1) / kDecThreads;
    root_flag_kernel<<<gnn, kDecThreads, 0, s>>>(T, nn, flag);
    int nf = 0;
    e = flagged_list(c, nn, flag, pos, front, tot, &nf);
    if (e) return e;
    *n_roots = nf;
    const double r2 = r_halo * r_halo;
    const bool q64 = c->built_precision == P3T_FP64;
    long long node_base = 0, part_base = 0;
    bool fits = cap_nodes > 0;
    while (nf > 0) {
        const int gf = (nf + kDecThreads - 1) / kDecThreads;
        let_level_kernel<<<gf, kDecThreads, 0, s>>>(T, nf, front, n_boxes, dbox, r2, 0, nch, npt, nullptr, nullptr, 0, 0,
                                                    nullptr, false, nullptr, 0, nullptr, q64);
        e = scan_excl_i32_to_i64(nch, cho, nf, tot64, c->scan_status, &c->meta->tickets[28], c->meta, s);
        if (e) return e;
        e = scan_excl_i32_to_i64(npt, pto, nf, tot64 + 1, c->scan_status, &c->meta->tickets[27], c->meta, s);
        if (e) return e;
        int64_t t2[2] = {0, 0};
        if (cudaMemcpyAsync(t2, tot64, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return P3T_ERR_CUDA;
        if (t2[0] > nn) return P3T_ERR_INTERNAL;  // a frontier holds distinct nodes
        fits = fits && node_base + nf <= cap_nodes && part_base + t2[1] <= cap_parts;
        let_level_kernel<<<gf, kDecThreads, 0, s>>>(T, nf, front, n_boxes, dbox, r2, 1, nullptr, nullptr, cho, pto,
                                                    node_base + nf, part_base, next, fits, (LetNode *)nodes,
                                                    node_base, (LetPart *)parts, q64);
        node_base += nf;
        part_base += t2[1];
        std::swap(front, next);
        nf = (int)t2[0];
    }
    *n_nodes = node_base;
    *n_parts = part_base;
    e = sync_status(c);
    if (e) return e;
    return fits ? P3T_OK : P3T_ERR_CAPACITY;
}

int p3t_subtree_boxes(p3t_ctx *c, int32_t cap, double *boxes, int32_t *n_boxes)
{
    if (!c || !n_boxes || cap < 0 || (cap > 0 && !boxes)) return P3T_ERR_INVALID_ARG;
    if (!c->built || !c->range_built || c->joined || c->n_top < 1) return P3T_ERR_ORDER;
    int e = p3t_status(c);
    if (e) return e;
    int nn = 0;
    if (cudaMemcpy(&nn, &c->meta->n_nodes, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return P3T_ERR_CUDA;
    const size_t off_p = al((size_t)nn + 16), off_r = off_p + al(4 * (size_t)nn), off_t = off_r + al(4 * (size_t)nn),
                 off_o = off_t + 256;
    e = dec_reserve(c, off_o + al(64 * (size_t)kMaxDomainBoxes));
    if (e) return e;
    char *b = (char *)c->dec_buf;
    unsigned char *flag = (unsigned char *)b;
    int32_t *pos = (int32_t *)(b + off_p), *ids = (int32_t *)(b + off_r), *tot = (int32_t *)(b + off_t);
    double *out = (double *)(b + off_o);
    root_flag_kernel<<<(nn + kDecThreads - 1) / kDecThreads, kDecThreads, 0, c->stream>>>(c->tree, nn, flag);
    int cnt = 0;
    e = flagged_list(c, nn, flag, pos, ids, tot, &cnt);
    if (e) return e;
    *n_boxes = cnt;
    if (cnt > cap) return P3T_ERR_CAPACITY;
    if (cnt > kMaxDomainBoxes) return P3T_ERR_INTERNAL;
    if (cnt > 0) {
        node_boxes_kernel<<<(cnt + 255) / 256, 256, 0, c->stream>>>(c->tree, cnt, ids, out);
        if (cudaMemcpyAsync(boxes, out, 48 * (size_t)cnt, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
            return P3T_ERR_CUDA;
    }
    return sync_status(c);
}

int p3t_tree_join(p3t_ctx *c, int32_t n_let, const void *const *let_nodes, const int64_t *let_n_nodes,
                  const int32_t *let_n_roots, const void *const *let_parts, const int64_t *let_n_parts)
{
    if (!c || n_let < 0 || (n_let > 0 && (!let_nodes || !let_n_nodes || !let_n_roots || !let_parts || !let_n_parts)))
        return P3T_ERR_INVALID_ARG;
    for (int r = 0; r < n_let; r++)
        if (let_n_nodes[r] < let_n_roots[r] || let_n_roots[r] < 0 || let_n_parts[r] < 0 ||
            (let_n_nodes[r] > 0 && !let_nodes[r]) || (let_n_parts[r] > 0 && !let_parts[r]))
            return P3T_ERR_INVALID_ARG;
    if (!c->built || !c->range_built || c->joined || c->n_top < 1) return P3T_ERR_ORDER;
    int e = p3t_status(c);
    if (e) return e;
    cudaStream_t s = c->stream;
    int nn = 0;
    if (cudaMemcpy(&nn, &c->meta->n_nodes, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return P3T_ERR_CUDA;
    Tree &T = c->tree;
    const int n_loc = c->n;
    // ---- the skeleton: every top cell and every rank's subtree roots, breadth first
    const size_t off_p = al((size_t)nn + 16), off_q = off_p + al(4 * (size_t)nn), off_r = off_q + al((size_t)nn + 16),
                 off_m = off_r + al(4 * (size_t)nn), off_l = off_m + al(4 * (size_t)nn),
                 off_k = off_l + al(4 * (size_t)nn), off_t = off_k + al(8 * (size_t)nn);
    const size_t off_x = off_t + 256;  // small tables of the skeleton
    const size_t tbl = 4 * (size_t)(kMaxTopCells * 9 + 8 * 4096);
    e = dec_reserve(c, off_x + al(tbl));
    if (e) return e;
    char *b = (char *)c->dec_buf;
    unsigned char *rflag = (unsigned char *)b, *iflag = (unsigned char *)(b + off_q);
    int32_t *pos = (int32_t *)(b + off_p), *ids = (int32_t *)(b + off_r), *map = (int32_t *)(b + off_m);
    int32_t *lev = (int32_t *)(b + off_l);
    unsigned long long *key = (unsigned long long *)(b + off_k);
    int32_t *tot = (int32_t *)(b + off_t);
    int32_t *dtab = (int32_t *)(b + off_x);
    const int gnn = (nn + kDecThreads - 1) / kDecThreads;
    struct Entry {
        int level;
        unsigned long long key;
        int kind;   // 0 top cell, 1 local root, 2 remote root
        int src;    // local node id (kinds 0 with a local node, 1) or LET index (2)
        int let;    // LET of a remote root
    };
    std::vector<Entry> sk;
    for (int i = 0; i < c->n_top; i++) sk.push_back({c->top_level[i], c->top_key[i], 0, -1, -1});
    // local top nodes (their ids, to skip them) and local roots
    std::vector<int> lroot_id, ltop_id;
    std::vector<int> hl;
    std::vector<unsigned long long> hk;
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 0)
            root_flag_kernel<<<gnn, kDecThreads, 0, s>>>(T, nn, rflag);
        else
            top_flag_kernel<<<gnn, kDecThreads, 0, s>>>(T, nn, iflag);
        int cnt = 0;
        e = flagged_list(c, nn, pass == 0 ? rflag : iflag, pos, ids, tot, &cnt);
        if (e) return e;
        std::vector<int> hid(cnt);
        hl.assign(cnt, 0);
        hk.assign(cnt, 0);
        if (cnt > 0) {
            node_keys_kernel<<<(cnt + 255) / 256, 256, 0, s>>>(T, cnt, ids, lev, key);
            if (cudaMemcpyAsync(hid.data(), ids, 4 * (size_t)cnt, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaMemcpyAsync(hl.data(), lev, 4 * (size_t)cnt, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaMemcpyAsync(hk.data(), key, 8 * (size_t)cnt, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return P3T_ERR_CUDA;
        }
        for (int i = 0; i < cnt; i++) {
            if (pass == 0) {
                sk.push_back({hl[i], hk[i], 1, hid[i], -1});
                lroot_id.push_back(hid[i]);
            } else {
                ltop_id.push_back(hid[i]);
            }
        }
    }
    // remote roots: the first n_roots nodes of every LET
    for (int r = 0; r < n_let; r++) {
        const int nr = let_n_roots[r];
        std::vector<LetNode> h(nr);
        if (nr > 0 && (cudaMemcpyAsync(h.data(), let_nodes[r], sizeof(LetNode) * (size_t)nr, cudaMemcpyDeviceToHost,
                                       s) != cudaSuccess ||
                       cudaStreamSynchronize(s) != cudaSuccess))
            return P3T_ERR_CUDA;
        for (int k = 0; k < nr; k++) sk.push_back({h[k].level, h[k].key, 2, k, r});
    }
    std::stable_sort(sk.begin(), sk.end(), [](const Entry &a, const Entry &b2) {
        return a.level != b2.level ? a.level < b2.level : a.key < b2.key;
    });
    const int S = (int)sk.size();
    // a node appears once; the root is a top cell; every other entry's parent is a top cell
    std::vector<int> top_idx, child0, nchild;
    for (int i = 0; i < S; i++) {
        if (i > 0 && sk[i].level == sk[i - 1].level && sk[i].key == sk[i - 1].key) return P3T_ERR_INVALID_INPUT;
        if (i == 0 && !(sk[0].level == 0 && sk[0].kind == 0)) return P3T_ERR_INVALID_INPUT;
    }
    for (int i = 0; i < S; i++) {
        if (sk[i].kind != 0) continue;
        const int l = sk[i].level;
        const unsigned long long pfx = sk[i].key >> (63 - 3 * l);
        int first = -1, cnt = 0;
        for (int j = i + 1; j < S; j++) {
            if (sk[j].level != l + 1) continue;
            if ((sk[j].key >> (63 - 3 * l)) == pfx) {
                if (first < 0) first = j;
                if (j != first + cnt) return P3T_ERR_INVALID_INPUT;  // children not contiguous
                cnt++;
            }
        }
        if (cnt < 1 || cnt > 8) return P3T_ERR_INVALID_INPUT;
        top_idx.push_back(i);
        child0.push_back(first);
        nchild.push_back(cnt);
    }
    for (int i = 1; i < S; i++) {  // every entry below the root hangs from a top cell
        const int l = sk[i].level;
        bool found = false;
        for (size_t t = 0; t < top_idx.size() && !found; t++) {
            const Entry &p = sk[top_idx[t]];
            found = p.level == l - 1 && (p.key >> (63 - 3 * (l - 1))) == (sk[i].key >> (63 - 3 * (l - 1)));
        }
        if (!found) return P3T_ERR_INVALID_INPUT;
    }
    // ---- sizes of the joined tree
    const long long n_int = (long long)nn - (long long)lroot_id.size() - (long long)ltop_id.size();
    long long nodes_tot = S + n_int, parts_tot = n_loc;
    std::vector<long long> let_base(n_let), part_base(n_let);
    for (int r = 0; r < n_let; r++) {
        let_base[r] = nodes_tot;
        nodes_tot += let_n_nodes[r] - let_n_roots[r];
        part_base[r] = parts_tot;
        parts_tot += let_n_parts[r];
    }
    if (nodes_tot >= (1LL << 28) || parts_tot >= (1LL << 31) - 1) return P3T_ERR_CAPACITY;
    // ---- the joined arrays
    const size_t NN = (size_t)nodes_tot, NP = (size_t)parts_tot;
    size_t jo = 0;
    auto slot = [&](size_t bytes) {
        const size_t o = jo;
        jo += al(bytes);
        return o;
    };
    const size_t o_topo = slot(16 * NN), o_comM = slot(32 * NN), o_lo = slot(32 * NN), o_hi = slot(32 * NN),
                 o_q64 = slot(48 * NN), o_q32 = slot(24 * NN), o_wn = slot(16 * wrec_words((long long)NN)),
                 o_sp = slot(32 * NP), o_ph = slot(16 * NP), o_pl = slot(16 * NP), o_rid = slot(4 * NP),
                 o_cid = slot(4 * NP);
    if (jo > c->join_bytes) {
        cudaStreamSynchronize(s);
        if (c->join_buf) cudaFree(c->join_buf);
        c->join_buf = nullptr;
        c->join_bytes = 0;
        if (cudaMalloc(&c->join_buf, jo) != cudaSuccess) {
            cudaGetLastError();
            return P3T_ERR_OOM;
        }
        c->join_bytes = jo;
    }
    char *jb = (char *)c->join_buf;
    Joined J;
    J.topo = (int4 *)(jb + o_topo);
    J.comM = (double4_32a *)(jb + o_comM);
    J.lo = (double4_32a *)(jb + o_lo);
    J.hi = (double4_32a *)(jb + o_hi);
    J.q64 = (double *)(jb + o_q64);
    J.q32 = (float *)(jb + o_q32);
    J.wn = (float4 *)(jb + o_wn);
    J.sp = (double4_32a *)(jb + o_sp);
    J.ph = (float4 *)(jb + o_ph);
    J.pl = (float4 *)(jb + o_pl);
    J.rid = (int32_t *)(jb + o_rid);
    J.cid_s = (int32_t *)(jb + o_cid);
    // ---- local nodes: interior ones after the skeleton, roots to their skeleton slots
    interior_flag_kernel<<<gnn, kDecThreads, 0, s>>>(T, nn, rflag, iflag);
    e = scan_excl_u8_to_i32(iflag, pos, nn, tot, c->scan_status, &c->meta->tickets[28], c->meta, s);
    if (e) return e;
    local_map_kernel<<<gnn, kDecThreads, 0, s>>>(nn, iflag, pos, S, map);
    std::vector<int32_t> hnode, hidx;
    for (int i = 0; i < S; i++)
        if (sk[i].kind == 1) hnode.push_back(sk[i].src), hidx.push_back(i);
    const int nlr = (int)hnode.size();
    if (nlr > 4096) return P3T_ERR_CAPACITY;
    // device tables: local root ids + slots, then per LET its roots' slots, then the top cells
    std::vector<int32_t> h(2 * (size_t)nlr);
    for (int i = 0; i < nlr; i++) h[i] = hnode[i], h[nlr + i] = hidx[i];
    std::vector<std::vector<int32_t>> rslot(n_let);
    for (int i = 0; i < S; i++)
        if (sk[i].kind == 2) {
            auto &v = rslot[sk[i].let];
            if ((int)v.size() < let_n_roots[sk[i].let]) v.resize(let_n_roots[sk[i].let], -1);
            v[sk[i].src] = i;
        }
    size_t need = h.size() + 3 * top_idx.size();
    for (int r = 0; r < n_let; r++) need += let_n_roots[r];
    if (4 * need > tbl) return P3T_ERR_CAPACITY;
    std::vector<int32_t> all(h);
    std::vector<size_t> roff(n_let);
    for (int r = 0; r < n_let; r++) {
        roff[r] = all.size();
        all.insert(all.end(), rslot[r].begin(), rslot[r].end());
    }
    const size_t toff = all.size();
    all.insert(all.end(), top_idx.begin(), top_idx.end());
    all.insert(all.end(), child0.begin(), child0.end());
    all.insert(all.end(), nchild.begin(), nchild.end());
    if (!all.empty() &&
        (cudaMemcpyAsync(dtab, all.data(), 4 * all.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess))
        return P3T_ERR_CUDA;
    if (nlr > 0) skel_map_kernel<<<(nlr + 255) / 256, 256, 0, s>>>(nlr, dtab, dtab + nlr, map);
    const bool q64 = c->built_precision == P3T_FP64;
    copy_local_kernel<<<gnn, kDecThreads, 0, s>>>(T, nn, map, J, q64);
    copy_local_parts_kernel<<<(n_loc + kDecThreads - 1) / kDecThreads, kDecThreads, 0, s>>>(T, n_loc, J);
    for (int r = 0; r < n_let; r++) {
        const int nl = (int)let_n_nodes[r];
        if (nl > 0)
            copy_let_kernel<<<(nl + kDecThreads - 1) / kDecThreads, kDecThreads, 0, s>>>(
                (const LetNode *)let_nodes[r], nl, let_n_roots[r], dtab + roff[r], (int)let_base[r], part_base[r],
                (int)let_n_parts[r], J, q64, c->meta);
        const int np = (int)let_n_parts[r];
        if (np > 0)
            copy_let_parts_kernel<<<(np + kDecThreads - 1) / kDecThreads, kDecThreads, 0, s>>>(
                (const LetPart *)let_parts[r], np, part_base[r], J);
    }
    // ---- the joined tree becomes the context's tree; then the top cells' moments
    T.topo = J.topo, T.comM = J.comM, T.lo = J.lo, T.hi = J.hi, T.q64 = J.q64, T.q32 = J.q32, T.wn = J.wn;
    T.sp = J.sp, T.ph = J.ph, T.pl = J.pl, T.rid = J.rid, T.cid_s = J.cid_s;
    T.n_src = (int)parts_tot;
    T.cap_nodes = (int)nodes_tot;
    const int nt = (int)top_idx.size();
    const int32_t *dt = dtab + toff;
    if (q64)
        top_moments_kernel<true><<<1, 1, 0, s>>>(T, nt, dt, dt + nt, dt + 2 * nt, c->prm.theta);
    else
        top_moments_kernel<false><<<1, 1, 0, s>>>(T, nt, dt, dt + nt, dt + 2 * nt, c->prm.theta);
    set_nodes_kernel<<<1, 1, 0, s>>>(c->meta, (int)nodes_tot);
    c->joined = 1;
    c->counts_valid = 0;
    c->walk_counted = 0;
    c->rows_valid = 0;
    return sync_status(c);
}

}  // extern "C"
