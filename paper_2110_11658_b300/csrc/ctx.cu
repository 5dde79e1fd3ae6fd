// Context management and the exported C ABI of the P3T distant-force library.
// Each entry point validates its arguments, enqueues kernels on the context's
// stream (build_tree.cu, walk.cu, neighbours.cu, kick.cu) and maps CUDA
// failures to P3T_ERR_CUDA.  Nothing here throws.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "p3t_internal.cuh"

namespace p3t {

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

long long node_capacity(long long n, int leaf_cap)
{
    // leaves are disjoint and non-empty (<= n); internal nodes hold more than
    // leaf_cap particles and are disjoint within a level (<= n/(leaf_cap+1) per
    // level, levels 0..20)
    return n + (long long)kLevels * (n / (leaf_cap + 1)) + 1;
}

// lookback flags per tree level: one per tile of the level's nodes (a level holds
// at most n nodes; tiles of 256 nodes, or of 8 on levels of at most
// kTopoWideNodes nodes)
int topo_status_stride(long long n)
{
    const long long wide = (n < kTopoWideNodes ? n : kTopoWideNodes) / 8 + 4;
    const long long narrow = n / 256 + 4;
    return (int)(wide > narrow ? wide : narrow);
}

// The scratch layout of a context for n particles: every buffer, in order, each
// 256-byte aligned.  With base == nullptr only the total is computed.
static size_t scratch_plan(p3t_ctx *c, long long N, int L, char *base)
{
    const long long NN = node_capacity(N, L);
    const long long sort_blocks = (N + kSortTileItems - 1) / kSortTileItems;
    const long long scan_words = N / 256 + 64 + 256 * sort_blocks / 256;
    const long long topo_words = (long long)kMaxLevelSlots * topo_status_stride(N);
    Tree &T = c->tree;
    size_t off = 0;
    auto put = [&](void *slot, size_t bytes) {
        if (base) *(void **)slot = base + off;
        off += align_up(bytes, 256);
    };
    put(&c->meta, sizeof(Meta));
    put(&c->keys_buf[0], 8 * (size_t)N);
    put(&c->keys_buf[1], 8 * (size_t)N);
    put(&c->perm_buf[0], 4 * (size_t)N);
    put(&c->perm_buf[1], 4 * (size_t)N);
    put(&T.sp, 32 * (size_t)N);
    put(&T.ph, 16 * (size_t)N);
    put(&T.pl, 16 * (size_t)N);
    put(&T.gflag, (size_t)N + 16);
    put(&T.gidx, 4 * (size_t)N);
    put(&T.leaves, 4 * (size_t)N);
    put(&T.cid, 4 * (size_t)N);
    put(&T.cid_s, 4 * (size_t)N);
    put(&T.inv, 4 * (size_t)N);
    put(&T.grp, 8 * (size_t)N);
    put(&T.glo, 32 * (size_t)N);
    put(&T.ghi, 32 * (size_t)N);
    put(&T.gfr, 48 * (size_t)N);
    put(&T.gorder, 4 * (size_t)N);
    put(&c->nbr_count, 4 * (size_t)N);
    put(&c->row_list, 4 * (size_t)N);
    put(&c->rid_buf, 4 * (size_t)N);
    put(&c->row_off, 8 * ((size_t)N + 1));
    put(&c->top_buf, 12 * (size_t)kMaxTopCells);
    put(&c->grp_cells, 8 * (size_t)N);
    put(&c->grp_parts, 8 * (size_t)N);
    put(&c->sort_hist, 4 * 256 * (size_t)sort_blocks);
    put(&c->scan_status, 8 * (size_t)(scan_words + topo_words));
    put(&T.topo, 16 * (size_t)NN);
    put(&T.level, 4 * (size_t)NN);
    put(&T.parent, 4 * (size_t)NN);
    put(&T.comM, 32 * (size_t)NN);
    put(&T.lo, 32 * (size_t)NN);
    put(&T.hi, 32 * (size_t)NN);
    put(&T.q32, 24 * (size_t)NN);
    put(&T.q64, 48 * (size_t)NN);
    put(&T.wn, 16 * wrec_words(NN));
    return off;
}

size_t scratch_bytes(long long n, int leaf_cap, int n_clusters)
{
    p3t_ctx dummy;
    memset((void *)&dummy, 0, sizeof(dummy));
    const int cap = n_clusters < 256 ? 256 : n_clusters;
    return scratch_plan(&dummy, n, leaf_cap, nullptr) + sizeof(Cluster) * (size_t)cap;
}

int ensure_capacity(p3t_ctx *c, long long n)
{
    const int L = c->prm.leaf_cap;
    const long long need_nodes = node_capacity(n, L);
    if (c->blob && n <= c->cap_n && need_nodes <= c->cap_nodes) return P3T_OK;
    if (c->blob) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->blob);
        c->blob = nullptr;
    }
    const size_t total = scratch_plan(c, n, L, nullptr);
    void *blob = nullptr;
    if (cudaMalloc(&blob, total) != cudaSuccess) {
        cudaGetLastError();
        c->cap_n = 0;
        c->cap_nodes = 0;
        return P3T_ERR_OOM;
    }
    scratch_plan(c, n, L, (char *)blob);
    c->blob = blob;
    c->blob_bytes = total;
    c->gen++;
    c->cap_n = n;
    c->cap_nodes = need_nodes;
    c->counts_n = 0;  // the neighbour counts went with the old scratch
    c->cap_leaf = L;
    c->tree.meta = c->meta;
    c->tree.cap_nodes = (int)need_nodes;
    if (cudaMemsetAsync(c->meta, 0, sizeof(Meta), c->stream) != cudaSuccess) return P3T_ERR_CUDA;
    if (c->spin_limit &&
        cudaMemcpyAsync(&c->meta->spin_limit, &c->spin_limit, sizeof(long long),
                        cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return P3T_ERR_CUDA;
    return P3T_OK;
}

// Point the tree views back at the context's own scratch (a rank's tree may
// have been joined with remote nodes and particles in other buffers).
void reset_tree_views(p3t_ctx *c)
{
    if (c->blob) scratch_plan(c, c->cap_n, c->cap_leaf, (char *)c->blob);
    c->tree.meta = c->meta;
    c->tree.cap_nodes = (int)c->cap_nodes;
}

// Scratch for n particles in n_clusters clusters (no work is enqueued unless
// memory is (re)allocated).
int reserve(p3t_ctx *c, long long n, int n_clusters)
{
    int e = ensure_capacity(c, n);
    if (e) return e;
    if (n_clusters > c->cap_clusters) {
        if (c->clusters) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->clusters);
            c->clusters = nullptr;
        }
        int cap = n_clusters < 256 ? 256 : n_clusters;
        if (cudaMalloc(&c->clusters, sizeof(Cluster) * (size_t)cap) != cudaSuccess) {
            cudaGetLastError();
            c->cap_clusters = 0;
            return P3T_ERR_OOM;
        }
        c->cap_clusters = cap;
        c->gen++;
    }
    c->tree.cl = c->clusters;
    return P3T_OK;
}

int check_launch(p3t_ctx *c)
{
    (void)c;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "p3t: CUDA error %s\n", cudaGetErrorString(e));
        return P3T_ERR_CUDA;
    }
    return P3T_OK;
}

static int validate_params(const p3t_params *p)
{
    if (!p) return P3T_ERR_INVALID_ARG;
    if (!(p->theta >= 0.0) || !std::isfinite(p->theta)) return P3T_ERR_INVALID_ARG;
    if (!(p->r_in >= 0.0) || !(p->r_out > p->r_in) || !std::isfinite(p->r_out))
        return P3T_ERR_INVALID_ARG;
    if (!(p->r_list >= 0.0) || !std::isfinite(p->r_list)) return P3T_ERR_INVALID_ARG;
    if (p->leaf_cap < 1 || p->leaf_cap > (1 << 20)) return P3T_ERR_INVALID_ARG;
    if (p->group_size < 1 || p->group_size > 128) return P3T_ERR_INVALID_ARG;
    if (p->tile < 32 || p->tile > 256 || p->tile % 32) return P3T_ERR_INVALID_ARG;
    if (p->threads_per_group != 32 && p->threads_per_group != 64 && p->threads_per_group != 128)
        return P3T_ERR_INVALID_ARG;
    if (p->threads_per_group > 32 && p->group_size > p->threads_per_group) return P3T_ERR_INVALID_ARG;
    if (p->precision != P3T_FP32_MIXED && p->precision != P3T_FP64) return P3T_ERR_INVALID_ARG;
    if (p->quadrupole != 0 && p->quadrupole != 1) return P3T_ERR_INVALID_ARG;
    return P3T_OK;
}

}  // namespace p3t

using namespace p3t;

extern "C" {

int p3t_default_params(p3t_params *p)
{
    if (!p) return P3T_ERR_INVALID_ARG;
    p->theta = 0.5;
    p->r_in = 0.005;
    p->r_out = 0.05;
    p->r_list = 0.05;
    p->leaf_cap = 16;
    p->group_size = 32;
    p->tile = 64;
    p->threads_per_group = 32;
    p->precision = P3T_FP32_MIXED;
    p->quadrupole = 1;
    return P3T_OK;
}

int p3t_create(p3t_ctx **out, const p3t_params *p, void *cuda_stream)
{
    if (!out) return P3T_ERR_INVALID_ARG;
    *out = nullptr;
    int e = validate_params(p);
    if (e) return e;
    p3t_ctx *c = new (std::nothrow) p3t_ctx();
    if (!c) return P3T_ERR_OOM;
    memset((void *)c, 0, sizeof(*c));
    c->prm = *p;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) !=
            cudaSuccess) {
        cudaGetLastError();
        delete c;
        return P3T_ERR_CUDA;
    }
    // a second stream for the build's group pass (without it the pass runs in line)
    if (cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (c->side_stream) cudaStreamDestroy(c->side_stream);
        if (c->fork_ev) cudaEventDestroy(c->fork_ev);
        c->side_stream = nullptr, c->fork_ev = c->join_ev = nullptr;
    }
    if (c->side_stream && (cudaStreamCreateWithFlags(&c->side_stream2, cudaStreamNonBlocking) != cudaSuccess ||
                           cudaEventCreateWithFlags(&c->join_ev2, cudaEventDisableTiming) != cudaSuccess)) {
        cudaGetLastError();
        if (c->side_stream2) cudaStreamDestroy(c->side_stream2);
        c->side_stream2 = nullptr, c->join_ev2 = nullptr;
    }
    *out = c;
    return P3T_OK;
}

int p3t_destroy(p3t_ctx *c)
{
    if (!c) return P3T_ERR_INVALID_ARG;
    cudaStreamSynchronize(c->stream);
    if (c->blob) cudaFree(c->blob);
    if (c->host_stage) cudaFree(c->host_stage);
    if (c->row_scratch) cudaFree(c->row_scratch);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    if (c->lists_ready) cudaEventDestroy(c->lists_ready);
    if (c->v_ready) cudaEventDestroy(c->v_ready);
    if (c->side_stream) {
        cudaStreamSynchronize(c->side_stream);
        cudaStreamDestroy(c->side_stream);
    }
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->join_ev) cudaEventDestroy(c->join_ev);
    if (c->side_stream2) {
        cudaStreamSynchronize(c->side_stream2);
        cudaStreamDestroy(c->side_stream2);
    }
    if (c->join_ev2) cudaEventDestroy(c->join_ev2);
    if (c->clusters) cudaFree(c->clusters);
    if (c->irr_buf) cudaFree(c->irr_buf);
    if (c->knn_buf) cudaFree(c->knn_buf);
    if (c->dec_buf) cudaFree(c->dec_buf);
    if (c->join_buf) cudaFree(c->join_buf);
    delete c;
    return P3T_OK;
}

int p3t_set_params(p3t_ctx *c, const p3t_params *p)
{
    if (!c) return P3T_ERR_INVALID_ARG;
    int e = validate_params(p);
    if (e) return e;
    c->prm = *p;
    c->built = 0;
    return P3T_OK;
}

int p3t_reserve(p3t_ctx *c, int64_t n, int32_t n_clusters)
{
    if (!c || n <= 0 || n >= (1LL << 31) - 1 || n_clusters < 1 || n_clusters > n)
        return P3T_ERR_INVALID_ARG;
    if (node_capacity(n, c->prm.leaf_cap) >= (1LL << 28)) return P3T_ERR_INVALID_ARG;
    return reserve(c, n, n_clusters);
}

int p3t_scratch_bytes(const p3t_params *p, int64_t n, int32_t n_clusters, int64_t *bytes)
{
    if (!bytes) return P3T_ERR_INVALID_ARG;
    int e = validate_params(p);
    if (e) return e;
    if (n <= 0 || n >= (1LL << 31) - 1 || n_clusters < 1 || n_clusters > n) return P3T_ERR_INVALID_ARG;
    *bytes = (int64_t)scratch_bytes(n, p->leaf_cap, n_clusters);
    return P3T_OK;
}

static int build_common(p3t_ctx *c, int64_t n, int n_clusters, const int64_t *seg,
                        const double *cprm, const double *x, const double *y, const double *z,
                        const double *m, const RangeSpec *range = nullptr)
{
    if (!c || !x || !y || !z || !m) return P3T_ERR_INVALID_ARG;
    if (n <= 0 || n >= (1LL << 31) - 1) return P3T_ERR_INVALID_ARG;
    if (n_clusters < 1 || n_clusters > n) return P3T_ERR_INVALID_ARG;
    if (node_capacity(n, c->prm.leaf_cap) >= (1LL << 28)) return P3T_ERR_INVALID_ARG;
    int e = reserve(c, n, n_clusters);
    if (e) return e;
    reset_tree_views(c);  // a joined tree's views point elsewhere
    c->built = 0;
    c->counts_valid = 0;
    c->walk_counted = 0;
    c->rows_valid = 0;
    c->range_built = range != nullptr;
    c->joined = 0;
    c->uniform_params = cprm == nullptr;
    e = build_tree(c, (int)n, n_clusters, seg, cprm, x, y, z, m, range);
    if (e) return e;
    c->n = (int)n;
    c->built = 1;
    c->built_precision = c->prm.precision;
    return P3T_OK;
}

int p3t_build_tree(p3t_ctx *c, int64_t n, const double *x, const double *y, const double *z,
                   const double *m)
{
    return build_common(c, n, 1, nullptr, nullptr, x, y, z, m);
}

int p3t_build_tree_range(p3t_ctx *c, int64_t n, const double *x, const double *y, const double *z,
                         const double *m, const int64_t *gid, const double *global_box, int32_t n_top,
                         const uint64_t *top_key, const int32_t *top_level)
{
    if (!c || !global_box || n_top < 0 || n_top > kMaxTopCells || (n_top > 0 && (!top_key || !top_level)))
        return P3T_ERR_INVALID_ARG;
    for (int d = 0; d < 3; d++)
        if (!(global_box[d] <= global_box[3 + d]) || !std::isfinite(global_box[d]) ||
            !std::isfinite(global_box[3 + d]))
            return P3T_ERR_INVALID_ARG;
    for (int i = 0; i < n_top; i++) {
        const int l = top_level[i];
        // a top cell splits: level < 21, its key the first of a level-l cell
        if (l < 0 || l >= kLevels || (l > 0 && (top_key[i] & ((1ULL << (63 - 3 * l)) - 1))) ||
            (l == 0 && top_key[i] != 0) || top_key[i] >= (1ULL << 63))
            return P3T_ERR_INVALID_ARG;
    }
    if (!x || n <= 0 || n >= (1LL << 31) - 1) return P3T_ERR_INVALID_ARG;
    if (node_capacity(n, c->prm.leaf_cap) >= (1LL << 28)) return P3T_ERR_INVALID_ARG;
    int e = reserve(c, n, 1);  // the scratch the top-cell table lives in (the build reserves no more)
    if (e) return e;
    c->n_top = n_top;
    memcpy(c->gbox, global_box, sizeof(c->gbox));
    for (int i = 0; i < n_top; i++) c->top_key[i] = top_key[i], c->top_level[i] = top_level[i];
    unsigned long long hbuf[kMaxTopCells + kMaxTopCells / 2];
    memcpy(hbuf, top_key, sizeof(uint64_t) * n_top);
    memcpy(reinterpret_cast<char *>(hbuf) + 8 * kMaxTopCells, top_level, sizeof(int32_t) * n_top);
    if (n_top > 0 &&
        (cudaMemcpyAsync(c->top_buf, hbuf, 8 * n_top, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
         cudaMemcpyAsync(reinterpret_cast<char *>(c->top_buf) + 8 * kMaxTopCells,
                         reinterpret_cast<char *>(hbuf) + 8 * kMaxTopCells, 4 * n_top,
                         cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
         cudaStreamSynchronize(c->stream) != cudaSuccess))
        return P3T_ERR_CUDA;
    RangeSpec r;
    memcpy(r.box, global_box, sizeof(r.box));
    r.n_top = n_top;
    r.gid = gid;
    return build_common(c, n, 1, nullptr, nullptr, x, y, z, m, &r);
}

int p3t_build_tree_batch(p3t_ctx *c, int32_t n_clusters, int64_t n, const int64_t *seg_offsets,
                         const double *cluster_params, const double *x, const double *y,
                         const double *z, const double *m)
{
    if (!seg_offsets) return P3T_ERR_INVALID_ARG;
    return build_common(c, n, n_clusters, seg_offsets, cluster_params, x, y, z, m);
}

int p3t_far_force(p3t_ctx *c, void *ax, void *ay, void *az, double *pot, int64_t *n_cell_inter,
                  int64_t *n_part_inter)
{
    if (!c || !ax || !ay || !az) return P3T_ERR_INVALID_ARG;
    if (!c->built) return P3T_ERR_ORDER;
    return far_force(c, ax, ay, az, pot, n_cell_inter, n_part_inter);
}

int p3t_neighbours(p3t_ctx *c, int64_t *offsets, int32_t *idx, int64_t capacity, int64_t *total)
{
    if (!c || !offsets || !total || capacity < 0 || (capacity > 0 && !idx))
        return P3T_ERR_INVALID_ARG;
    if (!c->built) return P3T_ERR_ORDER;
    return neighbours(c, offsets, idx, capacity, nullptr, true, total);
}

int p3t_neighbours_async(p3t_ctx *c, int64_t *offsets, int32_t *idx, int64_t capacity,
                         int64_t *total_dev)
{
    if (!c || !offsets || !total_dev || capacity < 0 || (capacity > 0 && !idx))
        return P3T_ERR_INVALID_ARG;
    if (!c->built) return P3T_ERR_ORDER;
    return neighbours(c, offsets, idx, capacity, total_dev, false, nullptr);
}

int p3t_kick(p3t_ctx *c, double dt, const void *ax, const void *ay, const void *az, double *vx,
             double *vy, double *vz)
{
    if (!c || !ax || !ay || !az || !vx || !vy || !vz || !std::isfinite(dt))
        return P3T_ERR_INVALID_ARG;
    if (!c->built) return P3T_ERR_ORDER;
    return kick(c, dt, ax, ay, az, vx, vy, vz);
}

int p3t_drift(p3t_ctx *c, int64_t n, double dt, double *x, double *y, double *z, const double *vx,
              const double *vy, const double *vz)
{
    if (!c || !x || !y || !z || !vx || !vy || !vz || n <= 0 || n >= (1LL << 31) ||
        !std::isfinite(dt))
        return P3T_ERR_INVALID_ARG;
    return drift(c, (int)n, dt, x, y, z, vx, vy, vz);
}

int p3t_status(p3t_ctx *c)
{
    if (!c) return P3T_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return P3T_ERR_CUDA;
    }
    if (c->pending_err) {
        int e = c->pending_err;
        c->pending_err = 0;
        return e;
    }
    if (!c->meta) return P3T_OK;
    int err = 0;
    if (cudaMemcpy(&err, &c->meta->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return P3T_ERR_CUDA;
    if (err) {
        int zero = 0;
        cudaMemcpy(&c->meta->err, &zero, sizeof(int), cudaMemcpyHostToDevice);
    }
    return err;
}

int p3t_tree_info(p3t_ctx *c, int64_t *n, int64_t *n_nodes, int64_t *n_groups, int32_t *depth)
{
    if (!c) return P3T_ERR_INVALID_ARG;
    if (!c->built) return P3T_ERR_ORDER;
    int e = p3t_status(c);
    if (e) return e;
    Meta h;
    if (cudaMemcpy(&h, c->meta, sizeof(Meta), cudaMemcpyDeviceToHost) != cudaSuccess)
        return P3T_ERR_CUDA;
    if (n) *n = c->n;
    if (n_nodes) *n_nodes = h.n_nodes;
    if (n_groups) *n_groups = h.n_groups;
    if (depth) *depth = h.depth;
    return P3T_OK;
}

int p3t_export_tree(p3t_ctx *c, uint64_t *keys, int32_t *perm, int32_t *level, int32_t *first,
                    int32_t *count, int32_t *child, int32_t *nchild, double *M, double *com,
                    double *Q, double *lo, double *hi, double *ropen2, int32_t *g_first,
                    int32_t *g_count)
{
    if (!c) return P3T_ERR_INVALID_ARG;
    if (!c->built) return P3T_ERR_ORDER;
    return export_tree(c, keys, perm, level, first, count, child, nchild, M, com, Q, lo, hi,
                       ropen2, g_first, g_count);
}

int p3t_group_counts(p3t_ctx *c, int64_t *n_cell, int64_t *n_part)
{
    if (!c || !n_cell || !n_part) return P3T_ERR_INVALID_ARG;
    if (!c->built) return P3T_ERR_ORDER;
    int64_t ng = 0;
    int e = p3t_tree_info(c, nullptr, nullptr, &ng, nullptr);
    if (e) return e;
    if (cudaMemcpyAsync(n_cell, c->grp_cells, 8 * ng, cudaMemcpyDeviceToDevice, c->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(n_part, c->grp_parts, 8 * ng, cudaMemcpyDeviceToDevice, c->stream) !=
            cudaSuccess)
        return P3T_ERR_CUDA;
    return P3T_OK;
}

int p3t_irregular(p3t_ctx *c, int64_t n, const int64_t *offsets, const int32_t *idx,
                  const double *x, const double *y, const double *z, const double *m,
                  const double *vx, const double *vy, const double *vz, double *fx, double *fy,
                  double *fz, double *jx, double *jy, double *jz)
{
    if (!c || !offsets || !idx || !x || !y || !z || !m || !vx || !vy || !vz || !fx || !fy || !fz ||
        !jx || !jy || !jz || n <= 0 || n >= (1LL << 31) - 1)
        return P3T_ERR_INVALID_ARG;
    if (!c->built || !c->meta || c->n != n) return P3T_ERR_ORDER;  // a tree of these n particles
    return irregular(c, (int)n, offsets, idx, x, y, z, m, vx, vy, vz, fx, fy, fz, jx, jy, jz);
}

int p3t_row_mode(p3t_ctx *c, int32_t *row_cap, int32_t *rows_valid)
{
    if (!c) return P3T_ERR_INVALID_ARG;
    if (row_cap) *row_cap = c->row_cap;
    if (rows_valid) *rows_valid = c->rows_valid;
    return P3T_OK;
}

int p3t_filter_fallbacks(p3t_ctx *c, int64_t *count)
{
    if (!c || !count) return P3T_ERR_INVALID_ARG;
    if (!c->built) return P3T_ERR_ORDER;
    int e = p3t_status(c);
    if (e) return e;
    long long v = 0;
    if (cudaMemcpy(&v, &c->meta->fallback_tests, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess)
        return P3T_ERR_CUDA;
    *count = v;
    return P3T_OK;
}

int p3t_set_debug(p3t_ctx *c, int on)
{
    if (!c) return P3T_ERR_INVALID_ARG;
    c->debug = on ? 1 : 0;
    return P3T_OK;
}

int p3t_set_spin_limit(p3t_ctx *c, int64_t polls)
{
    if (!c || polls < 0) return P3T_ERR_INVALID_ARG;
    c->spin_limit = polls;
    if (!c->meta) return P3T_OK;  // written into the device block when it is allocated
    if (cudaMemcpyAsync(&c->meta->spin_limit, &c->spin_limit, sizeof(long long),
                        cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return P3T_ERR_CUDA;
    }
    return P3T_OK;
}

int p3t_debug_stalled_scan(p3t_ctx *c, int64_t n)
{
    if (!c || n <= 0) return P3T_ERR_INVALID_ARG;
    if (!c->meta || n > c->cap_n) return P3T_ERR_ORDER;
    c->counts_valid = 0;  // the scan runs over the neighbour-count buffer
    int e = scan_stalled((int)n, c->nbr_count, c->row_list, c->scan_status, &c->meta->tickets[30],
                         c->meta, c->stream);
    if (e) return e;
    return p3t_status(c);
}

const char *p3t_error_string(int code)
{
    switch (code) {
    case P3T_OK: return "ok";
    case P3T_ERR_INVALID_ARG: return "invalid argument";
    case P3T_ERR_INVALID_INPUT: return "invalid input (non-finite position or mass, or negative mass)";
    case P3T_ERR_OOM: return "device allocation failed";
    case P3T_ERR_CAPACITY: return "output capacity too small";
    case P3T_ERR_ORDER: return "no tree built: call p3t_build_tree first";
    case P3T_ERR_TIMEOUT: return "a bounded device-side wait ran out";
    case P3T_ERR_CUDA: return "CUDA runtime error";
    case P3T_ERR_INTERNAL: return "device-side consistency check failed";
    default: return "unknown error";
    }
}

}  // extern "C"
