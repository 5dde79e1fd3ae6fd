// Leapfrog kick of Eq. 12 (v += (dt_reg/2) F_R) and the benchmark drift.
#include "p3t_internal.cuh"

namespace p3t {

template <typename A>
__global__ void __launch_bounds__(256)
    kick_kernel(int n, double h, const A *__restrict__ ax, const A *__restrict__ ay,
                const A *__restrict__ az, double *__restrict__ vx, double *__restrict__ vy,
                double *__restrict__ vz)
{
    pdl_wait();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        // v + h*a with the product and the sum each rounded (no contraction)
        vx[i] = dadd(vx[i], dmul(h, (double)ax[i]));
        vy[i] = dadd(vy[i], dmul(h, (double)ay[i]));
        vz[i] = dadd(vz[i], dmul(h, (double)az[i]));
    }
}

__global__ void __launch_bounds__(256)
    drift_kernel(int n, double dt, double *__restrict__ x, double *__restrict__ y,
                 double *__restrict__ z, const double *__restrict__ vx,
                 const double *__restrict__ vy, const double *__restrict__ vz)
{
    pdl_wait();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = dadd(x[i], dmul(dt, vx[i]));
        y[i] = dadd(y[i], dmul(dt, vy[i]));
        z[i] = dadd(z[i], dmul(dt, vz[i]));
    }
}

int kick(p3t_ctx *c, double dt, const void *ax, const void *ay, const void *az, double *vx,
         double *vy, double *vz)
{
    const double h = 0.5 * dt;
    const int n = c->n;
    const int grid = (n + 255) / 256 < 8 * c->sm_count ? (n + 255) / 256 : 8 * c->sm_count;
    const cudaError_t r =
        c->built_precision == P3T_FP64
            ? launch_pdl(kick_kernel<double>, dim3(grid), dim3(256), c->stream, n, h, (const double *)ax,
                         (const double *)ay, (const double *)az, vx, vy, vz)
            : launch_pdl(kick_kernel<float>, dim3(grid), dim3(256), c->stream, n, h, (const float *)ax,
                         (const float *)ay, (const float *)az, vx, vy, vz);
    if (r != cudaSuccess) return P3T_ERR_CUDA;
    return check_launch(c);
}

int drift(p3t_ctx *c, int n, double dt, double *x, double *y, double *z, const double *vx,
          const double *vy, const double *vz)
{
    const int grid = (n + 255) / 256 < 8 * c->sm_count ? (n + 255) / 256 : 8 * c->sm_count;
    if (launch_pdl(drift_kernel, dim3(grid), dim3(256), c->stream, n, dt, x, y, z, vx, vy, vz) != cudaSuccess)
        return P3T_ERR_CUDA;
    return check_launch(c);
}

}  // namespace p3t
