// Device-wide exclusive prefix sums in one pass (decoupled look-back).
// Used for group numbering (flags -> indices), neighbour-row offsets and the
// radix-sort digit offsets.  Blocks take tiles in ticket order, so a block
// only ever waits on tiles already owned by running blocks; each wait is
// bounded (p3t_internal.cuh).
#include "p3t_internal.cuh"

namespace p3t {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

int scan_status_words(int n) { return (n + kScanTile - 1) / kScanTile + 2; }

template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kScanThreads)
    scan_kernel(const TIn *in, TOut *out, int n, TOut *total_dev,
                unsigned long long *status, unsigned int *ticket, Meta *meta)
{
    __shared__ unsigned int sh_t;
    __shared__ long long sh_scan[32];
    __shared__ long long sh_pre;
    pdl_wait();
    if (threadIdx.x == 0) sh_t = atomicAdd(ticket, 1u);
    __syncthreads();
    const int t = (int)sh_t;
    const long long base = (long long)t * kScanTile + (long long)threadIdx.x * kScanItems;
    long long v[kScanItems];
    long long sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        long long i = base + k;
        v[k] = i < n ? (long long)in[i] : 0;
        sum += v[k];
    }
    long long tot;
    long long ex = block_excl_scan<long long>(sum, &tot, sh_scan);
    long long pre = lookback_prefix(status, t, tot, meta, &sh_pre);
    long long run = pre + ex;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        long long i = base + k;
        if (i < n) out[i] = (TOut)run;
        run += v[k];
    }
    const int ntiles = (n + kScanTile - 1) / kScanTile;
    if (t == ntiles - 1 && threadIdx.x == 0 && total_dev) *total_dev = (TOut)(pre + tot);
}

template <typename TIn, typename TOut>
static int run_scan(const TIn *in, TOut *out, int n, TOut *total_dev, unsigned long long *status,
                    unsigned int *ticket, Meta *meta, cudaStream_t s)
{
    if (n <= 0) {
        if (total_dev && cudaMemsetAsync(total_dev, 0, sizeof(TOut), s) != cudaSuccess)
            return P3T_ERR_CUDA;
        return P3T_OK;
    }
    int ntiles = (n + kScanTile - 1) / kScanTile;
    if (cudaMemsetAsync(status, 0, sizeof(unsigned long long) * ntiles, s) != cudaSuccess ||
        cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s) != cudaSuccess)
        return P3T_ERR_CUDA;
    scan_kernel<TIn, TOut><<<ntiles, kScanThreads, 0, s>>>(in, out, n, total_dev, status, ticket,
                                                            meta);
    return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

int scan_excl_u8_to_i32(const unsigned char *in, int32_t *out, int n, int32_t *total_dev,
                        unsigned long long *status, unsigned int *ticket, Meta *meta,
                        cudaStream_t s)
{
    return run_scan<unsigned char, int32_t>(in, out, n, total_dev, status, ticket, meta, s);
}

int scan_excl_i32_to_i64(const int32_t *in, int64_t *out, int n, int64_t *total_dev,
                         unsigned long long *status, unsigned int *ticket, Meta *meta,
                         cudaStream_t s)
{
    return run_scan<int32_t, int64_t>(in, out, n, total_dev, status, ticket, meta, s);
}

int scan_excl_i32_to_i32(const int32_t *in, int32_t *out, int n, unsigned long long *status,
                         unsigned int *ticket, Meta *meta, cudaStream_t s)
{
    return run_scan<int32_t, int32_t>(in, out, n, (int32_t *)nullptr, status, ticket, meta, s);
}

// The same scan with its status words and ticket already cleared by the kernel
// before it on the stream (scan_status_words(n) words and the ticket), which saves
// the two clearing steps between them
int scan_excl_i32_to_i32_cleared(const int32_t *in, int32_t *out, int n, unsigned long long *status,
                                 unsigned int *ticket, Meta *meta, cudaStream_t s)
{
    if (n <= 0) return P3T_OK;
    const int ntiles = (n + kScanTile - 1) / kScanTile;
    return launch_pdl(scan_kernel<int32_t, int32_t>, dim3(ntiles), dim3(kScanThreads), s, in, out, n,
                      (int32_t *)nullptr, status, ticket, meta) == cudaSuccess
               ? P3T_OK
               : P3T_ERR_CUDA;
}

int scan_excl_i32_to_i64_cleared(const int32_t *in, int64_t *out, int n, int64_t *total_dev,
                                 unsigned long long *status, unsigned int *ticket, Meta *meta, cudaStream_t s)
{
    if (n <= 0) return P3T_ERR_INVALID_ARG;
    const int ntiles = (n + kScanTile - 1) / kScanTile;
    return launch_pdl(scan_kernel<int32_t, int64_t>, dim3(ntiles), dim3(kScanThreads), s, in, out, n, total_dev,
                      status, ticket, meta) == cudaSuccess
               ? P3T_OK
               : P3T_ERR_CUDA;
}

__global__ void set_ticket_kernel(unsigned int *ticket, unsigned int v) { *ticket = v; }

// The scan above with tile 0's ticket never handed out: the block holding tile
// 1 (and every tile whose look-back window of 32 reaches tile 0) waits on a
// predecessor that never publishes, so its bounded wait runs out, latches
// P3T_ERR_TIMEOUT and goes on with a partial prefix; later tiles find those
// published prefixes and finish.  The last of the ntiles blocks takes ticket
// ntiles, past the last tile: it reads nothing, writes no output and publishes
// status word ntiles (the status array holds ntiles + 2 words).
int scan_stalled(int n, const int32_t *in, int32_t *out, unsigned long long *status,
                 unsigned int *ticket, Meta *meta, cudaStream_t s)
{
    if (n <= 0) return P3T_ERR_INVALID_ARG;
    const int ntiles = (n + kScanTile - 1) / kScanTile;
    if (cudaMemsetAsync(status, 0, sizeof(unsigned long long) * (ntiles + 1), s) != cudaSuccess)
        return P3T_ERR_CUDA;
    set_ticket_kernel<<<1, 1, 0, s>>>(ticket, 1u);
    scan_kernel<int32_t, int32_t><<<ntiles, kScanThreads, 0, s>>>(in, out, n, (int32_t *)nullptr,
                                                                   status, ticket, meta);
    return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

}  // namespace p3t
