// p3t_step_host: one regular step from and to host memory -- the boundary of
// the paper's REGF (host arrays in; regular force and neighbour lists out,
// Sec. 2.4) followed by RKICK (Eq. 12).  Device staging buffers are owned by
// the context and grow on demand.  A second stream of the context uploads the
// velocities during the build and copies the neighbour lists (built before the
// far force) back during the walk.
#include <cstring>

#include "p3t_internal.cuh"

using namespace p3t;

extern "C" int p3t_step_host(p3t_ctx *c, int64_t n, double dt, const double *x, const double *y,
                             const double *z, const double *m, double *vx, double *vy, double *vz,
                             void *ax, void *ay, void *az, int64_t *offsets, int32_t *idx,
                             int64_t capacity, int64_t *total)
{
    if (!c || !x || !y || !z || !m || !vx || !vy || !vz || !ax || !ay || !az || !offsets || !total ||
        capacity < 0 || (capacity > 0 && !idx) || n <= 0 || n >= (1LL << 31) - 1)
        return P3T_ERR_INVALID_ARG;
    cudaStream_t s = c->stream;
    const size_t asz = c->prm.precision == P3T_FP64 ? 8 : 4;
    const size_t need = 7 * 8 * (size_t)n + 3 * asz * (size_t)n + 8 * ((size_t)n + 1) +
                        4 * (size_t)capacity + 8 * 256;
    if (need > c->host_stage_bytes) {
        if (c->host_stage) {
            cudaStreamSynchronize(s);
            cudaFree(c->host_stage);
            c->host_stage = nullptr;
            c->host_stage_bytes = 0;
        }
        if (cudaMalloc(&c->host_stage, need) != cudaSuccess) {
            cudaGetLastError();
            return P3T_ERR_OOM;
        }
        c->host_stage_bytes = need;
    }
    char *p = (char *)c->host_stage;
    auto take = [&](size_t bytes) {
        char *q = p;
        p += (bytes + 255) / 256 * 256;
        return q;
    };
    double *dx = (double *)take(8 * n), *dy = (double *)take(8 * n), *dz = (double *)take(8 * n);
    double *dm = (double *)take(8 * n);
    double *dvx = (double *)take(8 * n), *dvy = (double *)take(8 * n), *dvz = (double *)take(8 * n);
    void *dax = take(asz * n), *day = take(asz * n), *daz = take(asz * n);
    int64_t *doffs = (int64_t *)take(8 * (n + 1));
    int32_t *didx = capacity > 0 ? (int32_t *)take(4 * capacity) : nullptr;
    if (!c->copy_stream) {
        if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            c->copy_stream = nullptr;
            return P3T_ERR_CUDA;
        }
        if (cudaEventCreateWithFlags(&c->lists_ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->v_ready, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return P3T_ERR_CUDA;
        }
    }
    cudaStream_t cs = c->copy_stream;
    // positions and masses on the compute stream; the velocities, which only the
    // kick reads, on the copy stream while the tree is built
    const double *hin[7] = {x, y, z, m, vx, vy, vz};
    double *din[7] = {dx, dy, dz, dm, dvx, dvy, dvz};
    for (int k = 0; k < 7; k++)
        if (cudaMemcpyAsync(din[k], hin[k], 8 * n, cudaMemcpyHostToDevice, k < 4 ? s : cs) !=
            cudaSuccess) {
            cudaStreamSynchronize(cs);
            return P3T_ERR_CUDA;
        }
    if (cudaEventRecord(c->v_ready, cs) != cudaSuccess) {
        cudaStreamSynchronize(cs);
        return P3T_ERR_CUDA;
    }
    // neighbour lists first (their count pass replaces the count inside the
    // walk), so that their copy to the host runs on a second stream while the
    // far-force walk computes
    int e = p3t_build_tree(c, n, dx, dy, dz, dm);
    if (e) {
        cudaStreamSynchronize(cs);
        return e;
    }
    int ne = p3t_neighbours(c, doffs, didx, capacity, total);
    if (ne && ne != P3T_ERR_CAPACITY) {
        cudaStreamSynchronize(cs);
        return ne;
    }
    if (cudaEventRecord(c->lists_ready, s) != cudaSuccess ||
        cudaStreamWaitEvent(cs, c->lists_ready, 0) != cudaSuccess ||
        cudaMemcpyAsync(offsets, doffs, 8 * (n + 1), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
        (!ne && *total > 0 &&
         cudaMemcpyAsync(idx, didx, 4 * (size_t)*total, cudaMemcpyDeviceToHost, cs) != cudaSuccess)) {
        cudaStreamSynchronize(cs);
        return P3T_ERR_CUDA;
    }
    e = p3t_far_force(c, dax, day, daz, nullptr, nullptr, nullptr);
    if (e == P3T_OK && cudaStreamWaitEvent(s, c->v_ready, 0) != cudaSuccess) e = P3T_ERR_CUDA;
    if (e == P3T_OK) e = p3t_kick(c, dt, dax, day, daz, dvx, dvy, dvz);
    if (e) {
        cudaStreamSynchronize(cs);
        return e;
    }
    void *hout[6] = {ax, ay, az, vx, vy, vz};
    const void *dout[6] = {dax, day, daz, dvx, dvy, dvz};
    const size_t osz[6] = {asz, asz, asz, 8, 8, 8};
    for (int k = 0; k < 6; k++)
        if (cudaMemcpyAsync(hout[k], dout[k], osz[k] * n, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            cudaStreamSynchronize(cs);
            return P3T_ERR_CUDA;
        }
    if (cudaStreamSynchronize(cs) != cudaSuccess) return P3T_ERR_CUDA;
    e = p3t_status(c);
    if (e) return e;
    return ne;
}
