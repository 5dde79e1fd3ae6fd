// Irregular (neighbour) force and its time derivative over the neighbour rows
// (Sec. 2.1, Eqs. 1, 2, 6-10): the other side of the changeover, which the
// Hermite integrator of the P3T scheme needs at every irregular step:
//   F_I,i    = sum_j K m_j d / r^3
//   dF_I,i/dt = sum_j m_j [K (u / r^3 - 3 (d.u) d / r^5) + Kdot d / r^3]
// with d = x_j - x_i, u = v_j - v_i, K = 1 - W, and Kdot = dK/dt =
// -dW/dx (d.u) / (r (r_out - r_in)) (the exact derivative of Eq. 1: Eq. 2 as
// printed drops m_j and K from its middle term and Eq. 7 prints K' with the
// opposite sign).  Pairs at r = 0 (singular) and at r >= r_out (K = 0)
// contribute nothing.
//
// One warp per target row; lanes take every 32nd entry and their partial sums
// are reduced by shuffles (in FP64 for the FP64 form, in FP32 for the mixed
// one).  Targets are visited in key order (the built tree's), so warps running
// together share their neighbours in the caches.  The FP64 form repeats the
// oracle's operations per pair (no contraction).  The mixed form first splits
// every position (relative to its cluster's frame centre O) and velocity into
// double-single FP32 pairs (hi + lo, made in FP64 once per particle and stored
// in original order, so that a row's entries index them directly), then forms
// each difference as (hi_j - hi_i) + (lo_j - lo_i) and evaluates the pair in
// FP32, with the changeover's FP32 constants from the cluster table: no FP64
// instruction per pair, and each difference within 2^-23 of its own size plus
// 2^-46 of the cluster size (the relative error of a term is ~1e-7).
#include <cstdint>

#include "p3t_internal.cuh"

namespace p3t {

constexpr int kIrrWarps = 8;

// double-single state of one particle (mixed form)
struct DsState {
    float4 ph;  // {hi of x - O, m}
    float4 pl;  // {lo of x - O, 0}
    float4 vh;  // {hi of v, 0}
    float4 vl;  // {lo of v, 0}
};

struct IrrArgs {
    int n;
    const int64_t *offs;
    const int32_t *idx;
    const double *x, *y, *z, *m, *vx, *vy, *vz;
    double *fx, *fy, *fz, *jx, *jy, *jz;
    const int32_t *order;   // targets in this order (key order) or null
    const int32_t *inv;     // original -> key order (FP64 form's per-cluster radii)
    const int32_t *cid_s;   // cluster of each particle, key order
    const Cluster *cl;      // per-cluster radii (null: r_in, r_out below)
    const Cluster *cl_frame;  // cluster table (frame centres of the split)
    double r_in, r_out;
    Meta *meta;
    DsState *ds;            // mixed form: per-particle splits, original order
};

// mixed form: split position (relative to the cluster's frame centre) and
// velocity of every particle into hi + lo FP32 pairs, stored in original order
__global__ void __launch_bounds__(256) irregular_split_kernel(IrrArgs a)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n; k += gridDim.x * blockDim.x) {
        const int i = a.order[k];
        const double *O = a.cl_frame[a.cid_s[k]].frame;
        DsState s;
        ds_split(dsub(a.x[i], O[0]), s.ph.x, s.pl.x);
        ds_split(dsub(a.y[i], O[1]), s.ph.y, s.pl.y);
        ds_split(dsub(a.z[i], O[2]), s.ph.z, s.pl.z);
        ds_split(a.vx[i], s.vh.x, s.vl.x);
        ds_split(a.vy[i], s.vh.y, s.vl.y);
        ds_split(a.vz[i], s.vh.z, s.vl.z);
        s.ph.w = (float)a.m[i];
        s.pl.w = s.vh.w = s.vl.w = 0.f;
        a.ds[i] = s;  // original order: a row's entries index it directly
    }
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <bool MIXED>
__global__ void __launch_bounds__(kIrrWarps * 32) irregular_kernel(IrrArgs a)
{
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * kIrrWarps;
    bool bad = false;
    for (int k = blockIdx.x * kIrrWarps + (threadIdx.x >> 5); k < a.n; k += nw) {
        const int i = a.order ? a.order[k] : k;
        double r_in = a.r_in, r_out = a.r_out;
        if (!MIXED && a.cl) {
            const Cluster &K = a.cl[a.cid_s[a.inv[i]]];
            r_in = K.r_in, r_out = K.r_out;
        }
        const double dr = MIXED ? 0.0 : dsub(r_out, r_in);
        double xi = 0.0, yi = 0.0, zi = 0.0, uxi = 0.0, uyi = 0.0, uzi = 0.0;
        DsState si;
        float inv_dr_f = 0.f, rin_dr_f = 0.f;
        if (MIXED) {
            // target k of key order: its split state and its cluster's FP32 constants of
            // the changeover, 1/(r_out - r_in) and r_in/(r_out - r_in) (no FP64 per row)
            si = a.ds[i];
            const Cluster &K = a.cl_frame[a.cid_s[k]];
            inv_dr_f = K.inv_dr_f, rin_dr_f = K.rin_dr_f;
        } else {
            xi = a.x[i], yi = a.y[i], zi = a.z[i];
            uxi = a.vx[i], uyi = a.vy[i], uzi = a.vz[i];
        }
        const long long o0 = a.offs[i], o1 = a.offs[i + 1];
        double F[3] = {0.0, 0.0, 0.0}, J[3] = {0.0, 0.0, 0.0};
        float Ff[3] = {0.f, 0.f, 0.f}, Jf[3] = {0.f, 0.f, 0.f};
        for (long long e = o0 + lane; e < o1; e += 32) {
            const int j = a.idx[e];
            if ((unsigned)j >= (unsigned)a.n) {
                bad = true;
                continue;
            }
            if (MIXED) {
                const DsState sj = a.ds[j];
                const float dx = (sj.ph.x - si.ph.x) + (sj.pl.x - si.pl.x);
                const float dy = (sj.ph.y - si.ph.y) + (sj.pl.y - si.pl.y);
                const float dz = (sj.ph.z - si.ph.z) + (sj.pl.z - si.pl.z);
                const float ux = (sj.vh.x - si.vh.x) + (sj.vl.x - si.vl.x);
                const float uy = (sj.vh.y - si.vh.y) + (sj.vl.y - si.vl.y);
                const float uz = (sj.vh.z - si.vh.z) + (sj.vl.z - si.vl.z);
                const float mj = sj.ph.w;
                const float r2 = dx * dx + dy * dy + dz * dz;
                const float ri = rsqrtf(fmaxf(r2, 4e-26f));
                const float r = r2 * ri;
                const float xx = __saturatef(fmaf(r, inv_dr_f, -rin_dr_f));
                // K = 1 - W(x) = W(1 - x) (the changeover is symmetric), evaluated as
                // y^4 (35 - 84 y + 70 y^2 - 20 y^3) with y = 1 - x: no cancellation as
                // x -> 1, so K keeps FP32's relative accuracy; dW/dx = 140 x^3 y^3
                const float yy = 1.f - xx;
                const float y2 = yy * yy;
                const float Kw = (y2 * y2) * (35.f + yy * (-84.f + yy * (70.f - 20.f * yy)));
                const float dw = 140.f * (xx * xx * xx) * (y2 * yy);
                const float du = dx * ux + dy * uy + dz * uz;
                const float f3 = r2 > 0.f ? mj * ri * ri * ri : 0.f;
                const float kf = Kw * f3;
                const float kdot = -dw * du * ri * inv_dr_f;  // dK/dt
                const float c1 = kdot * f3 - 3.f * kf * du * ri * ri;
                Ff[0] += kf * dx, Ff[1] += kf * dy, Ff[2] += kf * dz;
                Jf[0] += kf * ux + c1 * dx;
                Jf[1] += kf * uy + c1 * dy;
                Jf[2] += kf * uz + c1 * dz;
            } else {
                const double d0 = dsub(a.x[j], xi), d1 = dsub(a.y[j], yi), d2 = dsub(a.z[j], zi);
                const double u0 = dsub(a.vx[j], uxi), u1 = dsub(a.vy[j], uyi),
                             u2 = dsub(a.vz[j], uzi);
                const double mj = a.m[j];
                // the oracle's operations, in its order
                const double r2 = dadd(dadd(dmul(d0, d0), dmul(d1, d1)), dmul(d2, d2));
                if (r2 == 0.0) continue;
                const double r = dsqrt(r2);
                const double y = ddiv(r, r_out), gamma = ddiv(r_in, r_out);
                const double x = ddiv(dsub(y, gamma), dsub(1.0, gamma));
                double W, dw;
                if (x < 0.0) {
                    W = 0.0, dw = 0.0;
                } else if (x >= 1.0) {
                    continue;  // K = 0, K' = 0
                } else {
                    const double x3 = dmul(dmul(x, x), x);
                    const double x4 = dmul(x3, x), x5 = dmul(x4, x), x6 = dmul(x5, x),
                                 x7 = dmul(x6, x);
                    W = dadd(dsub(dadd(dmul(-20.0, x7), dmul(70.0, x6)), dmul(84.0, x5)),
                             dmul(35.0, x4));
                    dw = dadd(dsub(dadd(dmul(-140.0, x6), dmul(420.0, x5)), dmul(420.0, x4)),
                              dmul(140.0, x3));
                }
                const double kk = dsub(1.0, W);
                if (kk == 0.0) continue;
                const double du = dadd(dadd(dmul(d0, u0), dmul(d1, u1)), dmul(d2, u2));
                const double kdot = ddiv(dmul(-dw, du), dmul(r, dr));
                const double f3 = ddiv(mj, dmul(r2, r));
                const double kf = dmul(kk, f3);
                const double c3 = dmul(dmul(dmul(3.0, kk), f3), ddiv(du, r2));
                const double kd = dmul(kdot, f3);
                const double d[3] = {d0, d1, d2}, u[3] = {u0, u1, u2};
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    F[q] = dadd(F[q], dmul(kf, d[q]));
                    J[q] = dadd(J[q], dadd(dsub(dmul(kf, u[q]), dmul(c3, d[q])), dmul(kd, d[q])));
                }
            }
        }
        if (MIXED) {
            // the lanes' FP32 partial sums summed in FP32; lane q < 6 widens and stores
            // component q (one FP64-pipe conversion per row)
#pragma unroll
            for (int q = 0; q < 3; q++) Ff[q] = warp_sum_f(Ff[q]), Jf[q] = warp_sum_f(Jf[q]);
            const float v = lane == 0 ? Ff[0] : lane == 1 ? Ff[1] : lane == 2 ? Ff[2]
                          : lane == 3 ? Jf[0] : lane == 4 ? Jf[1] : Jf[2];
            double *out = lane == 0 ? a.fx : lane == 1 ? a.fy : lane == 2 ? a.fz
                        : lane == 3 ? a.jx : lane == 4 ? a.jy : a.jz;
            if (lane < 6) out[i] = (double)v;
        } else {
#pragma unroll
            for (int q = 0; q < 3; q++) F[q] = warp_sum_d(F[q]), J[q] = warp_sum_d(J[q]);
            if (lane == 0) {
                a.fx[i] = F[0], a.fy[i] = F[1], a.fz[i] = F[2];
                a.jx[i] = J[0], a.jy[i] = J[1], a.jz[i] = J[2];
            }
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) latch_error(a.meta, P3T_ERR_INVALID_INPUT);
}

int irregular(p3t_ctx *c, int n, const int64_t *offs, const int32_t *idx, const double *x,
              const double *y, const double *z, const double *m, const double *vx,
              const double *vy, const double *vz, double *fx, double *fy, double *fz, double *jx,
              double *jy, double *jz)
{
    IrrArgs a;
    a.n = n;
    a.offs = offs, a.idx = idx;
    a.x = x, a.y = y, a.z = z, a.m = m, a.vx = vx, a.vy = vy, a.vz = vz;
    a.fx = fx, a.fy = fy, a.fz = fz, a.jx = jx, a.jy = jy, a.jz = jz;
    // the built tree holds these n particles (checked by the caller): key order,
    // cluster of every particle, frames and (per-cluster) radii
    a.order = c->tree.perm;
    a.inv = c->tree.inv;
    a.cid_s = c->tree.cid_s;
    a.cl = c->uniform_params ? nullptr : c->tree.cl;
    a.cl_frame = c->tree.cl;
    a.r_in = c->prm.r_in, a.r_out = c->prm.r_out;
    a.meta = c->meta;
    a.ds = nullptr;
    const int grid = 8 * c->sm_count;
    if (c->prm.precision == P3T_FP64) {
        irregular_kernel<false><<<grid, kIrrWarps * 32, 0, c->stream>>>(a);
    } else {
        const size_t need = sizeof(DsState) * (size_t)n;
        if (c->irr_bytes < need) {
            if (c->irr_buf) {
                cudaStreamSynchronize(c->stream);
                cudaFree(c->irr_buf);
                c->irr_buf = nullptr;
                c->irr_bytes = 0;
            }
            if (cudaMalloc(&c->irr_buf, need) != cudaSuccess) {
                cudaGetLastError();
                return P3T_ERR_OOM;
            }
            c->irr_bytes = need;
        }
        a.ds = (DsState *)c->irr_buf;
        irregular_split_kernel<<<4 * c->sm_count, 256, 0, c->stream>>>(a);
        irregular_kernel<true><<<grid, kIrrWarps * 32, 0, c->stream>>>(a);
    }
    return check_launch(c);
}

}  // namespace p3t
