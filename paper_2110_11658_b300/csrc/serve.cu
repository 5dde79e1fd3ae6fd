// Serving support: move the clusters of one batch between a resident arena and
// a contiguous staging area, so that a batch of arbitrary resident clusters
// can go through one batched step (p3t_build_tree_batch ... p3t_kick).
//
// A batch of n_seg clusters is described by
//   batch_off[n_seg + 1]  segment offsets in the staging area (its seg_offsets)
//   arena_off[n_seg]      first particle of each cluster in the arena
// (both device int64).  Particle i of the staging area belongs to the segment
// k with batch_off[k] <= i < batch_off[k + 1] (binary search) and maps to
// arena element arena_off[k] + (i - batch_off[k]).
#include <cstdint>

#include "p3t_internal.cuh"

namespace p3t {

constexpr int kMoveArrays = 10;

struct MoveArgs {
    int n_seg;
    const int64_t *batch_off;
    const int64_t *arena_off;
    int n_arrays;
    char *arena[kMoveArrays];
    char *batch[kMoveArrays];
    int elem[kMoveArrays];
    int to_batch;
};

// last k with off[k] <= i (off ascending, off[0] <= i < off[n])
__device__ __forceinline__ int segment_of(const int64_t *off, int n, long long i)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= i)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__global__ void batch_move_kernel(MoveArgs a)
{
    const long long total = a.batch_off[a.n_seg];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = segment_of(a.batch_off, a.n_seg, i);
        const long long j = a.arena_off[k] + (i - a.batch_off[k]);
        for (int q = 0; q < a.n_arrays; q++) {
            if (a.elem[q] == 8) {
                double *b = (double *)a.batch[q] + i, *r = (double *)a.arena[q] + j;
                if (a.to_batch)
                    *b = *r;
                else
                    *r = *b;
            } else {
                float *b = (float *)a.batch[q] + i, *r = (float *)a.arena[q] + j;
                if (a.to_batch)
                    *b = *r;
                else
                    *r = *b;
            }
        }
    }
}

struct NbrMoveArgs {
    int n_seg;
    const int64_t *batch_off;
    const int64_t *row_arena_off;   // [n_seg] first row-offset slot of each cluster
    const int64_t *ent_arena_off;   // [n_seg] first entry slot of each cluster
    const int64_t *ent_arena_cap;   // [n_seg] entry capacity of each cluster
    const int64_t *offsets;         // batch row offsets [batch_off[n_seg] + 1]
    const int32_t *idx;             // batch entries (batch indices)
    int64_t *arena_offsets;
    int32_t *arena_idx;
    int32_t *status;
    long long max_entries;          // capacity of the batch's idx
};

// rows: cluster-local offsets (N_k + 1 per cluster)
__global__ void nbr_rows_kernel(NbrMoveArgs a)
{
    const long long total = a.batch_off[a.n_seg];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = segment_of(a.batch_off, a.n_seg, i);
        const long long s0 = a.batch_off[k], s1 = a.batch_off[k + 1];
        const long long base = a.offsets[s0];
        const long long count = a.offsets[s1] - base;
        if (count > a.ent_arena_cap[k]) {
            if (i == s0) atomicCAS(a.status, 0, P3T_ERR_CAPACITY);
            continue;
        }
        int64_t *ro = a.arena_offsets + a.row_arena_off[k];
        ro[i - s0] = a.offsets[i] - base;
        if (i == s1 - 1) ro[s1 - s0] = count;
    }
}

// entries: batch index -> cluster-local index
__global__ void nbr_entries_kernel(NbrMoveArgs a)
{
    const long long np = a.batch_off[a.n_seg];
    const long long total = a.offsets[np];
    if (total > a.max_entries) {  // the batch's own fill overflowed: its entries are not valid
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(a.status, 0, P3T_ERR_CAPACITY);
        return;
    }
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        // segment k with offsets[batch_off[k]] <= e < offsets[batch_off[k + 1]]
        int lo = 0, hi = a.n_seg;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.offsets[a.batch_off[mid]] <= e)
                lo = mid;
            else
                hi = mid;
        }
        // empty clusters share their start with the next one: take the last such k
        const long long s0 = a.batch_off[lo], s1 = a.batch_off[lo + 1];
        const long long base = a.offsets[s0];
        if (a.offsets[s1] - base > a.ent_arena_cap[lo]) continue;
        a.arena_idx[a.ent_arena_off[lo] + (e - base)] = a.idx[e] - (int32_t)s0;
    }
}

}  // namespace p3t

using namespace p3t;

extern "C" {

int p3t_batch_move(void *cuda_stream, int32_t n_seg, int64_t n_batch, const int64_t *batch_off,
                   const int64_t *arena_off, int32_t n_arrays, const p3t_seg_array *arrays,
                   int32_t to_batch)
{
    if (n_seg < 1 || n_batch < 0 || !batch_off || !arena_off || n_arrays < 1 ||
        n_arrays > kMoveArrays || !arrays)
        return P3T_ERR_INVALID_ARG;
    MoveArgs a;
    a.n_seg = n_seg;
    a.batch_off = batch_off;
    a.arena_off = arena_off;
    a.n_arrays = n_arrays;
    a.to_batch = to_batch ? 1 : 0;
    for (int q = 0; q < n_arrays; q++) {
        if (!arrays[q].arena || !arrays[q].batch ||
            (arrays[q].elem_bytes != 4 && arrays[q].elem_bytes != 8))
            return P3T_ERR_INVALID_ARG;
        a.arena[q] = (char *)arrays[q].arena;
        a.batch[q] = (char *)arrays[q].batch;
        a.elem[q] = arrays[q].elem_bytes;
    }
    if (n_batch == 0) return P3T_OK;
    int dev = 0, sm = 148;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return P3T_ERR_CUDA;
    }
    const long long want = (n_batch + 255) / 256;
    const int grid = (int)(want < 8LL * sm ? want : 8LL * sm);
    batch_move_kernel<<<grid, 256, 0, (cudaStream_t)cuda_stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

int p3t_batch_scatter_neighbours(void *cuda_stream, int32_t n_seg, int64_t n_batch,
                                 int64_t max_entries, const int64_t *batch_off,
                                 const int64_t *row_arena_off, const int64_t *ent_arena_off,
                                 const int64_t *ent_arena_cap, const int64_t *offsets,
                                 const int32_t *idx, int64_t *arena_offsets, int32_t *arena_idx,
                                 int32_t *status)
{
    if (n_seg < 1 || n_batch < 0 || max_entries < 0 || !batch_off || !row_arena_off ||
        !ent_arena_off || !ent_arena_cap || !offsets || !arena_offsets || !status ||
        (max_entries > 0 && (!idx || !arena_idx)))
        return P3T_ERR_INVALID_ARG;
    NbrMoveArgs a{n_seg,   batch_off,     row_arena_off, ent_arena_off, ent_arena_cap, offsets,
                  idx,     arena_offsets, arena_idx,     status,        max_entries};
    if (n_batch == 0) return P3T_OK;
    int dev = 0, sm = 148;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return P3T_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const long long want = (n_batch + 255) / 256;
    const int grid = (int)(want < 8LL * sm ? want : 8LL * sm);
    nbr_rows_kernel<<<grid, 256, 0, s>>>(a);
    {
        const long long want_e = (max_entries + 255) / 256;
        const int grid_e = (int)(want_e < 1 ? 1 : (want_e < 8LL * sm ? want_e : 8LL * sm));
        nbr_entries_kernel<<<grid_e, 256, 0, s>>>(a);
    }
    return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

}  // extern "C"
