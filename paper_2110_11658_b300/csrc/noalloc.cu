// Morton order without any device allocation.
//
// Some callers cannot call cudaMalloc at the point where they need this
// library: a host that hands the library only buffers it allocated itself
// (for example an application whose memory pool already owns the GPU's
// memory), or a loop that must never allocate once it runs, because an
// allocation can synchronise the device and stall work on other streams.
// For them this file offers the key-and-sort part of the tree build (bounding
// cube, 63-bit Morton keys, stable radix sort by (key, index)) with all of its
// scratch memory -- the second sort buffer, the digit histograms, the scan
// status words and the metadata block -- in one file-scope static device
// array.  The caller still passes its inputs and the two output arrays.
//
// The array is sized for P3T_NOALLOC_MAX_N particles (about 0.8 MB) and every
// GPU that loads the library holds it until the process exits.  Every call
// shares it: calls whose work overlaps on a GPU (different streams or host
// threads at the same time) race on it.  Each call clears the parts that must
// start at zero.
#include <cstring>
#include <mutex>

#include "p3t_internal.cuh"

namespace p3t {

// kernels of build_tree.cu (same launch sequence as the tree build's first steps)
__global__ void init_meta_kernel(Meta *m);
__global__ void init_clusters_kernel(Cluster *cl, int C);
__global__ void bbox_kernel(int n, const double *__restrict__ x, const double *__restrict__ y,
                            const double *__restrict__ z, const double *__restrict__ m,
                            const int32_t *__restrict__ cid, Cluster *cl, Meta *meta);
__global__ void cube_kernel(Cluster *cl, int C);
__global__ void keys_kernel(int n, const double *__restrict__ x, const double *__restrict__ y,
                            const double *__restrict__ z, const int32_t *__restrict__ cid,
                            const Cluster *__restrict__ cl, uint64_t *__restrict__ keys,
                            int32_t *__restrict__ perm);
__global__ void sort_hist_kernel(int n, const uint64_t *__restrict__ keys,
                                 const int32_t *__restrict__ vals, const int32_t *__restrict__ cid,
                                 int shift, int nblocks, int32_t *__restrict__ hist,
                                 unsigned long long *scan_status, int scan_words, unsigned int *scan_ticket);
__global__ void sort_scatter_kernel(int n, const uint64_t *__restrict__ kin,
                                    const int32_t *__restrict__ vin, uint64_t *__restrict__ kout,
                                    int32_t *__restrict__ vout, const int32_t *__restrict__ cid,
                                    int shift, int nblocks, const int32_t *__restrict__ hist_off);

namespace {

constexpr int kMaxN = P3T_NOALLOC_MAX_N;
constexpr int kTile = kSortTileItems;             // items per sort block
constexpr int kMaxBlocks = (kMaxN + kTile - 1) / kTile;
constexpr size_t kClusterOff = (sizeof(Meta) + 15) / 16 * 16;                     // Cluster after Meta
constexpr size_t kMetaBytes = (kClusterOff + sizeof(Cluster) + 255) / 256 * 256;
constexpr size_t kKeysBytes = 8 * (size_t)kMaxN;
constexpr size_t kPermBytes = 4 * (size_t)kMaxN;
constexpr size_t kHistBytes = 4 * 256 * (size_t)kMaxBlocks;
constexpr size_t kStatusWords = 64;               // >= scan tiles of 256 * kMaxBlocks + 2
constexpr size_t kScratchBytes = kMetaBytes + kKeysBytes + kPermBytes + kHistBytes + 8 * kStatusWords;

static_assert(256 * kMaxBlocks / 2048 + 2 <= (int)kStatusWords, "scan status words");

__device__ __align__(256) static unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[256];  // device address of g_scratch, per device ordinal

// Looks up the device address of g_scratch once per device (the device must
// be current); host code cannot use the symbol itself as a device pointer.
int scratch_address(void **out, int *device)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return P3T_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return P3T_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    *device = dev;
    return P3T_OK;
}

}  // namespace
}  // namespace p3t

using namespace p3t;

extern "C" int p3t_morton_order_noalloc(int64_t n, const double *x, const double *y,
                                        const double *z, const double *m, uint64_t *keys,
                                        int32_t *perm, void *cuda_stream)
{
    if (!x || !y || !z || !m || !keys || !perm || n <= 0) return P3T_ERR_INVALID_ARG;
    if (n > kMaxN) return P3T_ERR_CAPACITY;
    void *base = nullptr;
    int dev = 0;
    int e = scratch_address(&base, &dev);
    if (e) return e;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    char *p = (char *)base;
    Meta *meta = (Meta *)p;
    Cluster *cl = (Cluster *)(p + kClusterOff);
    uint64_t *keys_alt = (uint64_t *)(p + kMetaBytes);
    int32_t *perm_alt = (int32_t *)(p + kMetaBytes + kKeysBytes);
    int32_t *hist = (int32_t *)(p + kMetaBytes + kKeysBytes + kPermBytes);
    unsigned long long *status =
        (unsigned long long *)(p + kMetaBytes + kKeysBytes + kPermBytes + kHistBytes);
    int sm = 0;
    if (cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sm = 148;
    const int N = (int)n;
    const int grid_n = (N + 255) / 256;
    // the previous call's latched error and counters must not leak into this one
    if (cudaMemsetAsync(meta, 0, sizeof(Meta), s) != cudaSuccess) return P3T_ERR_CUDA;
    init_meta_kernel<<<1, 64, 0, s>>>(meta);
    init_clusters_kernel<<<1, 32, 0, s>>>(cl, 1);
    bbox_kernel<<<2 * sm, 256, 0, s>>>(N, x, y, z, m, nullptr, cl, meta);
    cube_kernel<<<1, 32, 0, s>>>(cl, 1);
    keys_kernel<<<grid_n, 256, 0, s>>>(N, x, y, z, nullptr, cl, keys, perm);
    if (cudaGetLastError() != cudaSuccess) return P3T_ERR_CUDA;
    // 8 passes of 8 bits between the caller's arrays and the scratch copy;
    // after an even number of passes the result is back in the caller's arrays
    const int nb = (N + kTile - 1) / kTile;
    uint64_t *kb[2] = {keys, keys_alt};
    int32_t *pb[2] = {perm, perm_alt};
    for (int pass = 0; pass < 8; pass++) {
        const int shift = 8 * pass;
        sort_hist_kernel<<<nb, 256, 0, s>>>(N, kb[pass & 1], pb[pass & 1], nullptr, shift, nb, hist, status,
                                            scan_status_words(256 * nb), &meta->tickets[31]);
        e = scan_excl_i32_to_i32_cleared(hist, hist, 256 * nb, status, &meta->tickets[31], meta, s);
        if (e) return e;
        sort_scatter_kernel<<<nb, 256, 0, s>>>(N, kb[pass & 1], pb[pass & 1], kb[(pass + 1) & 1],
                                               pb[(pass + 1) & 1], nullptr, shift, nb, hist);
        if (cudaGetLastError() != cudaSuccess) return P3T_ERR_CUDA;
    }
    int err = 0;
    if (cudaMemcpyAsync(&err, &meta->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return P3T_ERR_CUDA;
    }
    return err;
}
