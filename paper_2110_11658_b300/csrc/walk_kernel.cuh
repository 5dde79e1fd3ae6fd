// Group-wise tree walk and far-force evaluation (Sec. 2.1 Eqs. 1, 3, 6;
// Sec. 2.4 Barnes-Hut walk with opening angle theta).
//
// One warp walks the tree for one group of <= 32*TPL particles (a persistent
// grid takes groups from an atomic ticket).  The traversal keeps a stack of
// node ranges in shared memory; each step pops up to 32 nodes, one per lane,
// and tests them:
//   open  iff  dist(B_g, com_c)^2 < r_open_c^2   (opening angle, rule 8)
//         or   dist(B_g, box_c)^2  < r_out^2     (the cell may hold a pair with W < 1)
// The decision is defined in FP64.  In the mixed form it is first taken in
// FP32 on coordinates relative to the cube centre O, with an error band that
// bounds the FP32-vs-FP64 difference; only a test that falls inside the band
// is recomputed with the exact FP64 operations (counted in meta->fallback_tests).
// The interaction lists therefore equal the FP64 rule exactly.
//
// Accepted cells (monopole + quadrupole, W = 1) and opened leaves (particle
// terms weighted by W) are queued in shared memory and evaluated once `tile`
// of them are queued: every lane holds TPL target particles in registers and
// loops over the queue, read by broadcast.  In the mixed form the queue is
// pair-interleaved ({x_k, x_k+1, y_k, y_k+1}, ...) and two sources are
// evaluated at once with the packed FP32x2 instructions of sm_100+ (one
// instruction per two multiply-adds), which halves the issue slots of the
// arithmetic; an odd tail is padded with a massless copy of its partner,
// whose terms are exactly zero.  Relative coordinates x_source - c_g
// and x_i - c_g (c_g the group-box centre) are formed from double-single
// splits of the FP64 coordinates (hi + lo FP32 pairs made once per particle
// and node in FP64 by the build), which gives the FP32 difference to within
// 2^-23 of its magnitude without any FP64 instruction in the walk; interactions
// run in FP32 and each tile's partial sum is added to the running sum with
// Kahan compensation.  The FP64 form does everything in FP64.
// The mixed form's cell term takes the r^-5 form when every cluster of the tree
// keeps r^-5 and its products inside FP32, else the r^-3 form (eval_cells_x2; the
// far force launches the walk once per form, one of the two launches finding no
// work).
//
// In the mixed form the particle loop also counts, per target, the neighbours
// of Sec. 2.3 (pairs with |r| < r_list), with the same FP32 band + exact FP64
// decision as the neighbour kernels, so p3t_neighbours can skip its counting
// pass.  Every pair within r_out of a group particle lies in a leaf the walk
// opens.  For r_list > r_out (the buffer radius r_out + r_buff of Eq. 20) a
// cell the force accepts may still hold neighbours: its children are pushed as
// flagged, neighbour-only ranges, tested by the r_list box test alone, and the
// particles of such leaves are staged with mass 0, so they are counted and add
// exactly nothing to the force.  The force and its interaction counts do not
// depend on r_list.
#include <cstdint>
#include <type_traits>

#pragma once

#include "p3t_internal.cuh"

namespace p3t {

constexpr int kWalkWarps = 4;                // warps per block
constexpr int kStackCap = 32 * 22 + 64;      // ranges per warp; see the bound below
constexpr float kU = 5.9604644775390625e-8f;  // 2^-24, FP32 unit round-off
// pairs of cells per unrolled iteration: 4 in the force-only walk, 2 where the neighbour
// state holds registers
template <int NBR>
__host__ __device__ constexpr int cell_pair_unroll() { return NBR == 0 ? 4 : 2; }
constexpr int kPartPairUnroll = 2;           // pairs of particles per unrolled iteration
constexpr int kMinBlocksTpl1 = 6;            // resident blocks per SM at TPL = 1 (80 registers; 5 for
                                             // the row-mode walk, whose neighbour state needs more)

// Stack bound: children ranges are pushed so that the stack stays sorted by
// level (deepest on top).  Ranges of level l are created only while popping
// level l-1 nodes, which happens only after every level-l range above them is
// consumed; so at most 32 ranges per level are live: 32 * 22 in total.

struct WalkArgs {
    Tree T;  // every radius and frame comes from the tree's cluster table
    int tile;
    void *ax, *ay, *az;
    double *pot;
    unsigned long long *n_cell, *n_part;
    long long *grp_cells, *grp_parts;
    unsigned int *ticket;
    int32_t *nbr_count;          // fused neighbour count (original order) or null
    int32_t *rows;               // row mode: the targets' rows (key order), laid out by row_off
    const int64_t *row_off;
    long long row_entries;       // entries of the row scratch
};

template <typename Real>
struct Vec4;
template <>
struct Vec4<float> {
    using T = float4;
    using T2 = float2;
};
template <>
struct Vec4<double> {
    using T = double4_32a;
    using T2 = double2;
};

template <typename Real>
__device__ __forceinline__ Real rsqrt_(Real x);
template <>
__device__ __forceinline__ float rsqrt_<float>(float x)
{
    return rsqrtf(x);
}
template <>
__device__ __forceinline__ double rsqrt_<double>(double x)
{
    return 1.0 / sqrt(x);
}

template <typename Real>
__device__ __forceinline__ Real sat_(Real x);  // clamp to [0, 1], NaN -> 0
template <>
__device__ __forceinline__ float sat_<float>(float x)
{
    return __saturatef(x);
}
template <>
__device__ __forceinline__ double sat_<double>(double x)
{
    return x > 0.0 ? (x < 1.0 ? x : 1.0) : 0.0;
}

template <typename Real>
__device__ __forceinline__ Real to_real(double v);
template <>
__device__ __forceinline__ float to_real<float>(double v)
{
    return __double2float_rn(v);
}
template <>
__device__ __forceinline__ double to_real<double>(double v)
{
    return v;
}


// packed FP32x2 arithmetic (per component identical to the scalar fmaf/__fmul_rn/__fadd_rn)
__device__ __forceinline__ float2 f2(float a)
{
    return make_float2(a, a);
}
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c)
{
    return __ffma2_rn(a, b, c);
}
__device__ __forceinline__ float2 fmul2(float2 a, float2 b)
{
    return __fmul2_rn(a, b);
}
__device__ __forceinline__ float2 fadd2(float2 a, float2 b)
{
    return __fadd2_rn(a, b);
}

// r^2 below which 1/r is clamped in the particle loop: keeps (1/r)^3 finite for
// coincident pairs, whose weight W is then exactly 0 (r = 0 < r_in, or x = 0);
// for r_in >= 4.5e-13 the clamp never touches a pair with W > 0
constexpr float kR2Min = 4e-26f;

// shared-memory carve-up of one warp
template <typename Real>
struct WarpSmem {
    using R4 = typename Vec4<Real>::T;
    using R2 = typename Vec4<Real>::T2;
    // mixed form: cpos..cqb hold pairs of cells, 5 float4 per pair:
    // {-x0, -x1, -y0, -y1} {-z0, -z1, -M0, -M1} {Qxx} {Qxy} / {Qxz} {Qyy} / {Qyz} {Qzz}
    // (each {} one float2 of the two cells), and pp holds pairs of particles,
    // 2 float4 per pair: {x0, x1, y0, y1} {z0, z1, m0, m1}
    int *stk;
    R4 *cpos;  // {dx, dy, dz, M} of accepted cells, relative to c_g
    R4 *cqa;   // {Qxx, Qxy, Qxz, Qyy}
    R2 *cqb;   // {Qyz, Qzz}
    int2 *lq;  // opened leaves {first, count}
    int *lqo;  // exclusive prefix of leaf counts
    R4 *pp;    // staged source particles {dx, dy, dz, m}
    int *pj;   // their positions in key order
    int *po;   // row mode: their original indices
    // mixed form: the group box relative to c_g {lo xyz, hi x} {hi yz, t2, -}, t2 the
    // squared distance beyond which a source is r_out or more from the whole box
    float4 *gb;
    static __host__ __device__ size_t bytes(int tile)
    {
        size_t cb = tile + 32;
        size_t b = 4 * kStackCap;
        b += cb * (2 * sizeof(R4) + sizeof(R2));
        b += cb * 8 + (cb + 1) * 4;
        b = (b + 31) / 32 * 32;
        b += 32 * sizeof(R4) + 2 * 32 * 4 + 2 * sizeof(float4);
        return (b + 127) / 128 * 128;
    }
    __device__ void carve(char *base, int tile)
    {
        size_t cb = tile + 32;
        char *p = base;
        stk = (int *)p;
        p += 4 * kStackCap;
        cpos = (R4 *)p;
        p += cb * sizeof(R4);
        cqa = (R4 *)p;
        p += cb * sizeof(R4);
        cqb = (R2 *)p;
        p += cb * sizeof(R2);
        lq = (int2 *)p;
        p += cb * 8;
        lqo = (int *)p;
        p += (cb + 1) * 4;
        p = base + ((p - base + 31) / 32 * 32);
        pp = (R4 *)p;
        p += 32 * sizeof(R4);
        pj = (int *)p;
        p += 32 * 4;
        po = (int *)p;
        p += 32 * 4;
        gb = (float4 *)p;
    }
};

// per-lane accumulator of TPL targets
template <typename Real, int TPL>
struct Acc {
    Real s[TPL][4];  // running sums ax, ay, az, phi
    Real c[TPL][4];  // Kahan compensation (mixed form)
    Real p[TPL][4];  // partial sums of the current tile
    __device__ void zero_all()
    {
#pragma unroll
        for (int t = 0; t < TPL; t++)
#pragma unroll
            for (int k = 0; k < 4; k++) s[t][k] = c[t][k] = p[t][k] = Real(0);
    }
    __device__ void fold()
    {
#pragma unroll
        for (int t = 0; t < TPL; t++)
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (sizeof(Real) == 4) {
                    Real y = p[t][k] - c[t][k];
                    Real u = s[t][k] + y;
                    c[t][k] = (u - s[t][k]) - y;
                    s[t][k] = u;
                } else {
                    s[t][k] += p[t][k];
                }
                p[t][k] = Real(0);
            }
    }
};

// mixed form: partial sums of the current tile as float2 (even / odd sources)
template <int TPL>
struct AccX2 {
    float s[TPL][4];
    float c[TPL][4];
    float2 p[TPL][4];
    __device__ void zero_all()
    {
#pragma unroll
        for (int t = 0; t < TPL; t++)
#pragma unroll
            for (int k = 0; k < 4; k++) {
                s[t][k] = c[t][k] = 0.f;
                p[t][k] = make_float2(0.f, 0.f);
            }
    }
    __device__ void fold()
    {
#pragma unroll
        for (int t = 0; t < TPL; t++)
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float y = (p[t][k].x + p[t][k].y) - c[t][k];
                const float u = s[t][k] + y;
                c[t][k] = (u - s[t][k]) - y;
                s[t][k] = u;
                p[t][k] = make_float2(0.f, 0.f);
            }
    }
};

template <typename Real, int TPL, bool POT, bool QUAD>
__device__ __forceinline__ void eval_cells(const WarpSmem<Real> &W, int ncells, const Real (&px)[TPL],
                                           const Real (&py)[TPL], const Real (&pz)[TPL],
                                           Acc<Real, TPL> &A)
{
    using R4 = typename Vec4<Real>::T;
    using R2 = typename Vec4<Real>::T2;
    __syncwarp();
#pragma unroll 4
    for (int k = 0; k < ncells; k++) {
        const R4 s = W.cpos[k];
        R4 qa;
        R2 qb;
        if (QUAD) {
            qa = W.cqa[k];
            qb = W.cqb[k];
        }
#pragma unroll
        for (int t = 0; t < TPL; t++) {
            // r = x_i - com;  a = r^-3 [(-M - 5/2 (r.Q.r)/r^4) r + (Q r)/r^2]
            // (r^-3 applied last keeps every intermediate in FP32 range)
            const Real rx = px[t] - s.x, ry = py[t] - s.y, rz = pz[t] - s.z;
            const Real r2 = rx * rx + ry * ry + rz * rz;
            const Real ri = rsqrt_<Real>(r2);
            const Real q = ri * ri;
            const Real ri3 = ri * q;
            if (QUAD) {
                const Real qx = (qa.x * rx + qa.y * ry + qa.z * rz) * q;
                const Real qy = (qa.y * rx + qa.w * ry + qb.x * rz) * q;
                const Real qz = (qa.z * rx + qb.x * ry + qb.y * rz) * q;
                const Real rqr4 = (rx * qx + ry * qy + rz * qz) * q;  // r.Q.r / r^4
                const Real cf = -s.w - Real(2.5) * rqr4;
                A.p[t][0] += ri3 * (cf * rx + qx);
                A.p[t][1] += ri3 * (cf * ry + qy);
                A.p[t][2] += ri3 * (cf * rz + qz);
                if (POT) A.p[t][3] -= ri * (s.w + Real(0.5) * rqr4);
            } else {
                const Real mr3 = s.w * ri3;
                A.p[t][0] -= mr3 * rx;
                A.p[t][1] -= mr3 * ry;
                A.p[t][2] -= mr3 * rz;
                if (POT) A.p[t][3] -= s.w * ri;
            }
        }
    }
    A.fold();
    __syncwarp();
}

// Group frame: c_g in FP64 and its double-single split relative to O.
struct GroupFrame {
    double cx, cy, cz;       // c_g
    float hx, hy, hz;        // hi part of c_g - O
    float lx, ly, lz;        // lo part
};

// x_j - c_g from the double-single split of x_j - O (mixed form)
__device__ __forceinline__ float4 ds_rel(float4 h, float4 l, const GroupFrame &F)
{
    return make_float4((h.x - F.hx) + (l.x - F.lx), (h.y - F.hy) + (l.y - F.ly),
                       (h.z - F.hz) + (l.z - F.lz), h.w);
}

// Per-target neighbour counting state (fused counting in the mixed form).
template <int TPL>
struct NbrCount {
    int si[TPL];   // target positions in key order (-1: empty slot)
    int cnt[TPL];
    // row mode: wc entries written to the target's row in the row scratch, at
    // rows + row_off[si] (ids of the sources, the target itself left out; entries
    // past the row's capacity are dropped while cnt keeps counting)
    int wc[TPL];
    unsigned hit[TPL];  // neighbours among the 32 staged sources (bit = staging slot)
    bool beyond;   // the group's cluster lists neighbours beyond r_out (r_list > r_out)
    float lo, hi;  // r2 < lo: neighbour; r2 > hi: not; otherwise decide in FP64
    // |r2 - mid| <= rad covers [lo, hi] (the rare undecided band) with a 2x margin,
    // so rounding of mid and of r2 - mid cannot leave a band pair out
    float mid, rad;
    __device__ void set(float l, float h)  // l <= h; h infinite: every pair to FP64
    {
        lo = l, hi = h;
        mid = 0.5f * l + 0.5f * h;
        rad = h - l;
    }
    __device__ void off()  // no counting in this walk
    {
        lo = hi = -INFINITY;
        mid = 0.f, rad = -1.f;
    }
};

template <typename Real, int TPL, bool POT, int NBR>
__device__ __forceinline__ void eval_parts(const WarpSmem<Real> &W, const WalkArgs &P,
                                           const Cluster &K, int nleaves, int nparts,
                                           const GroupFrame &F, const Real (&px)[TPL],
                                           const Real (&py)[TPL], const Real (&pz)[TPL],
                                           Acc<Real, TPL> &A, NbrCount<TPL> &NC)
{
    using R4 = typename Vec4<Real>::T;
    constexpr bool kMixed = sizeof(Real) == 4;
    const int lane = threadIdx.x & 31;
    __syncwarp();
    // exclusive prefix of the queued leaf counts
    int carry = 0;
    for (int b = 0; b < nleaves; b += 32) {
        int i = b + lane;
        int v = i < nleaves ? W.lq[i].y : 0;
        int inc = warp_incl_scan(v);
        if (i < nleaves) W.lqo[i] = carry + inc - v;
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    __syncwarp();
    const Real inv_dr = kMixed ? Real(K.inv_dr_f) : Real(K.inv_dr_d);
    const Real rin_dr = kMixed ? Real(K.rin_dr_f) : Real(K.r_in * K.inv_dr_d);
    for (int c0 = 0; c0 < nparts; c0 += 32) {
        int pos = c0 + lane;
        if (pos < nparts) {
            int lo = 0, hi = nleaves;  // last leaf with lqo <= pos
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (W.lqo[mid] <= pos)
                    lo = mid;
                else
                    hi = mid;
            }
            int j = W.lq[lo].x + (pos - W.lqo[lo]);
            R4 v;
            if (kMixed) {
                float4 r = ds_rel(P.T.ph[j], P.T.pl[j], F);
                v.x = r.x, v.y = r.y, v.z = r.z, v.w = r.w;
            } else {
                double4_32a q = P.T.sp[j];
                v.x = to_real<Real>(dsub(q.x, F.cx));
                v.y = to_real<Real>(dsub(q.y, F.cy));
                v.z = to_real<Real>(dsub(q.z, F.cz));
                v.w = to_real<Real>(q.w);
            }
            W.pp[lane] = v;
            if (NBR) W.pj[lane] = j;
        }
        __syncwarp();
        const int ns = min(32, nparts - c0);
#pragma unroll 4
        for (int k = 0; k < ns; k++) {
            const R4 s = W.pp[k];
#pragma unroll
            for (int t = 0; t < TPL; t++) {
                // d = x_j - x_i
                const Real dx = s.x - px[t], dy = s.y - py[t], dz = s.z - pz[t];
                const Real r2 = dx * dx + dy * dy + dz * dz;
                const Real ri = rsqrt_<Real>(r2);
                const Real r = r2 * ri;
                // x = (r - r_in)/(r_out - r_in) clamped to [0, 1]; NaN (r2 = 0) maps to 0
                const Real x = sat_(r * inv_dr - rin_dr);
                Real w = (Real(-20) * x + Real(70)) * x + Real(-84);
                w = w * x + Real(35);
                const Real x2 = x * x;
                const Real Wt = w * (x2 * x2);
                Real f = s.w * Wt * (ri * ri * ri);
                f = Wt > Real(0) ? f : Real(0);
                A.p[t][0] += f * dx;
                A.p[t][1] += f * dy;
                A.p[t][2] += f * dz;
                if (POT) A.p[t][3] -= r2 > Real(0) ? s.w * ri : Real(0);
                if (NBR) {
                    // neighbour iff |x_j - x_i|^2 < r_list^2 in FP64; the pair with
                    // itself is counted here (r2 = 0) and removed at the end
                    const float r2f = (float)r2;
                    if (r2f < NC.lo) {
                        NC.cnt[t]++;
                    } else if (r2f <= NC.hi) {  // inside the band: decide in FP64
                        const int sj = W.pj[k];
                        const double4_32a a = P.T.sp[NC.si[t] < 0 ? sj : NC.si[t]], b = P.T.sp[sj];
                        const double ex = dsub(b.x, a.x), ey = dsub(b.y, a.y), ez = dsub(b.z, a.z);
                        NC.cnt[t] += dadd(dadd(dmul(ex, ex), dmul(ey, ey)), dmul(ez, ez)) < K.rl2_d;
                    }
                }
            }
        }
        __syncwarp();
    }
    A.fold();
}

// Mixed form, two queued cells at a time (layout above); same terms as eval_cells.
// PAD: pad an odd count here (one warp per group); with several warps per group the
// walking warp pads the queue once before they all read it.
// FAST: the quadrupole term as r^-5 [(-M r^2 - 5/2 (r.Q.r)/r^2) r + Q r], one packed
// operation fewer per pair of cells than the r^-3 form below.  r^-5 and the products
// stay inside the FP32 range (no overflow, no flush to zero) for r_out >= 1e-7, a
// frame half-size R <= 1e6 and a cluster mass <= 1e15, which the walk checks per
// group (every accepted cell lies at r >= r_out from each target of the group, and
// r <= 2 sqrt(3) R); otherwise the r^-3 form runs, which keeps every intermediate
// within r^-3.
template <int TPL, bool POT, bool QUAD, bool PAD, int UNROLL, bool FAST>
__device__ __forceinline__ void eval_cells_x2(const WarpSmem<float> &W, int ncells, const float (&px)[TPL],
                                              const float (&py)[TPL], const float (&pz)[TPL],
                                              AccX2<TPL> &A)
{
    const float4 *cq = reinterpret_cast<const float4 *>(W.cpos);
    __syncwarp();
    if (PAD && (ncells & 1) && (threadIdx.x & 31) == 0) {
        // pad: the partner's position with M = 0 and Q = 0 adds exactly zero
        float *b = reinterpret_cast<float *>(W.cpos) + 20 * (ncells >> 1);
        b[1] = b[0], b[3] = b[2], b[5] = b[4];
        b[7] = b[9] = b[11] = b[13] = b[15] = b[17] = b[19] = 0.f;
    }
    __syncwarp();
    float2 PX[TPL], PY[TPL], PZ[TPL];
#pragma unroll
    for (int t = 0; t < TPL; t++) PX[t] = f2(px[t]), PY[t] = f2(py[t]), PZ[t] = f2(pz[t]);
    const int npairs = (ncells + 1) >> 1;
#pragma unroll UNROLL
    for (int k = 0; k < npairs; k++) {
        const float4 a0 = cq[5 * k], a1 = cq[5 * k + 1];
        const float2 NX = make_float2(a0.x, a0.y), NY = make_float2(a0.z, a0.w);
        const float2 NZ = make_float2(a1.x, a1.y), NM = make_float2(a1.z, a1.w);
        float2 Qxx, Qxy, Qxz, Qyy, Qyz, Qzz;
        if (QUAD) {
            const float4 a2 = cq[5 * k + 2], a3 = cq[5 * k + 3], a4 = cq[5 * k + 4];
            Qxx = make_float2(a2.x, a2.y), Qxy = make_float2(a2.z, a2.w);
            Qxz = make_float2(a3.x, a3.y), Qyy = make_float2(a3.z, a3.w);
            Qyz = make_float2(a4.x, a4.y), Qzz = make_float2(a4.z, a4.w);
        }
#pragma unroll
        for (int t = 0; t < TPL; t++) {
            // r = x_i - com;  a = r^-3 [(-M - 5/2 (r.Q.r)/r^4) r + (Q r)/r^2]
            const float2 rx = fadd2(PX[t], NX), ry = fadd2(PY[t], NY), rz = fadd2(PZ[t], NZ);
            float2 r2 = fmul2(rx, rx);
            r2 = ffma2(ry, ry, r2);
            r2 = ffma2(rz, rz, r2);
            const float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
            const float2 q = fmul2(ri, ri);
            const float2 ri3 = fmul2(ri, q);
            if (QUAD && FAST) {
                float2 qx = fmul2(Qxx, rx), qy = fmul2(Qxy, rx), qz = fmul2(Qxz, rx);
                qx = ffma2(Qxy, ry, qx), qy = ffma2(Qyy, ry, qy), qz = ffma2(Qyz, ry, qz);
                qx = ffma2(Qxz, rz, qx), qy = ffma2(Qyz, rz, qy), qz = ffma2(Qzz, rz, qz);
                float2 rqr = fmul2(rx, qx);
                rqr = ffma2(ry, qy, rqr);
                rqr = ffma2(rz, qz, rqr);
                const float2 w = fmul2(rqr, q);                         // r.Q.r / r^2
                const float2 sc = ffma2(NM, r2, fmul2(f2(-2.5f), w));  // -M r^2 - 5/2 r.Q.r / r^2
                const float2 ri5 = fmul2(ri3, q);
                A.p[t][0] = ffma2(ri5, ffma2(sc, rx, qx), A.p[t][0]);
                A.p[t][1] = ffma2(ri5, ffma2(sc, ry, qy), A.p[t][1]);
                A.p[t][2] = ffma2(ri5, ffma2(sc, rz, qz), A.p[t][2]);
                if (POT) A.p[t][3] = ffma2(ri, ffma2(f2(-0.5f), fmul2(w, q), NM), A.p[t][3]);
            } else if (QUAD) {
                float2 qx = fmul2(Qxx, rx), qy = fmul2(Qxy, rx), qz = fmul2(Qxz, rx);
                qx = ffma2(Qxy, ry, qx), qy = ffma2(Qyy, ry, qy), qz = ffma2(Qyz, ry, qz);
                qx = ffma2(Qxz, rz, qx), qy = ffma2(Qyz, rz, qy), qz = ffma2(Qzz, rz, qz);
                qx = fmul2(qx, q), qy = fmul2(qy, q), qz = fmul2(qz, q);
                float2 rqr4 = fmul2(rx, qx);
                rqr4 = ffma2(ry, qy, rqr4);
                rqr4 = ffma2(rz, qz, rqr4);
                rqr4 = fmul2(rqr4, q);  // r.Q.r / r^4
                const float2 cf = ffma2(f2(-2.5f), rqr4, NM);
                A.p[t][0] = ffma2(ri3, ffma2(cf, rx, qx), A.p[t][0]);
                A.p[t][1] = ffma2(ri3, ffma2(cf, ry, qy), A.p[t][1]);
                A.p[t][2] = ffma2(ri3, ffma2(cf, rz, qz), A.p[t][2]);
                if (POT) A.p[t][3] = ffma2(ri, ffma2(f2(-0.5f), rqr4, NM), A.p[t][3]);
            } else {
                const float2 mr3 = fmul2(NM, ri3);  // -M / r^3
                A.p[t][0] = ffma2(mr3, rx, A.p[t][0]);
                A.p[t][1] = ffma2(mr3, ry, A.p[t][1]);
                A.p[t][2] = ffma2(mr3, rz, A.p[t][2]);
                if (POT) A.p[t][3] = ffma2(NM, ri, A.p[t][3]);
            }
        }
    }
    A.fold();
    __syncwarp();
}

// The neighbour test of one pair of staged particles against target t: neighbour
// iff |x_j - x_i|^2 < r_list^2 in FP64.  Below the band in FP32 counts at once;
// inside it (rare), the FP64 operations decide.  The pair with itself is counted
// (r2 = 0) and removed at the end.
template <int TPL, int NBR, bool TAIL>
__device__ __forceinline__ void pair_nbr(const WarpSmem<float> &W, const Tree &T, const Cluster &K, int k,
                                         int ns, int t, float2 r2, NbrCount<TPL> &NC)
{
    const bool yreal = !TAIL || 2 * k + 1 < ns;
    bool in0 = r2.x < NC.lo, in1 = yreal && r2.y < NC.lo;
    const float2 d = fadd2(r2, f2(-NC.mid));
    if (fminf(fabsf(d.x), fabsf(d.y)) <= NC.rad) {
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const float r2e = e ? r2.y : r2.x;
            if ((e == 0 || yreal) && r2e >= NC.lo && r2e <= NC.hi) {
                const int sj = W.pj[2 * k + e];
                const double4_32a a = T.sp[NC.si[t] < 0 ? sj : NC.si[t]], b = T.sp[sj];
                const double ex = dsub(b.x, a.x), ey = dsub(b.y, a.y), ez = dsub(b.z, a.z);
                const bool in = dadd(dadd(dmul(ex, ex), dmul(ey, ey)), dmul(ez, ez)) < K.rl2_d;
                if (e)
                    in1 = in;
                else
                    in0 = in;
            }
        }
    }
    if constexpr (NBR == 2)  // rows written once per staged chunk (write_rows)
        NC.hit[t] |= ((unsigned)in0 | ((unsigned)in1 << 1)) << (2 * k);
    else
        NC.cnt[t] += (int)in0 + (int)in1;
}

// One pair of staged particles (k: pair index) against this lane's targets.  A
// pair whose two sources come from leaves beyond r_out of the group box (or pads of
// mass 0; a clear bit pair in wm) has r >= r_out for every target: W = 1 exactly.
// Its sources may hold neighbours only if the cluster lists neighbours beyond r_out
// (bits in cm).  wm and cm are ballots over the staged slots, so the branches are
// warp-uniform.  ALL_FAR: wm = cm = 0 for the whole chunk; ALL_NEAR: every slot of
// the chunk needs W (no branch at all in either).
template <int TPL, bool POT, int NBR, bool SHELL, bool TAIL, bool ALL_FAR = false, bool ALL_NEAR = false>
__device__ __forceinline__ void part_pair(const WarpSmem<float> &W, const Tree &T, const Cluster &K,
                                          const float4 *pq, int k, int ns, unsigned wm, unsigned cm,
                                          float inv_dr,
                                          float nrin_dr,
                                          const float2 (&NPX)[TPL], const float2 (&NPY)[TPL],
                                          const float2 (&NPZ)[TPL], AccX2<TPL> &A, NbrCount<TPL> &NC)
{
    const float4 b0 = pq[2 * k], b1 = pq[2 * k + 1];
    const float2 X = make_float2(b0.x, b0.y), Y = make_float2(b0.z, b0.w);
    const float2 Z = make_float2(b1.x, b1.y), Mj = make_float2(b1.z, b1.w);
    const bool far = ALL_FAR || (!ALL_NEAR && ((wm >> (2 * k)) & 3u) == 0u);
#pragma unroll
    for (int t = 0; t < TPL; t++) {
        // d = x_j - x_i
        const float2 dx = fadd2(X, NPX[t]), dy = fadd2(Y, NPY[t]), dz = fadd2(Z, NPZ[t]);
        float2 r2 = fmul2(dx, dx);
        r2 = ffma2(dy, dy, r2);
        r2 = ffma2(dz, dz, r2);
        const float2 ri = make_float2(rsqrtf(fmaxf(r2.x, kR2Min)), rsqrtf(fmaxf(r2.y, kR2Min)));
        const float2 ri3 = fmul2(fmul2(ri, ri), ri);
        // W(r): x = (r - r_in)/(r_out - r_in) clamped to [0, 1], x^4 (35 - 84x + 70x^2 - 20x^3)
        auto weight = [&]() {
            const float2 r = fmul2(r2, ri);
            const float2 x = make_float2(__saturatef(fmaf(r.x, inv_dr, nrin_dr)),
                                         __saturatef(fmaf(r.y, inv_dr, nrin_dr)));
            float2 w = ffma2(f2(-20.f), x, f2(70.f));
            w = ffma2(w, x, f2(-84.f));
            w = ffma2(w, x, f2(35.f));
            const float2 x2 = fmul2(x, x);
            return fmul2(w, fmul2(x2, x2));
        };
        float2 f;
        if constexpr (ALL_FAR) {
            f = fmul2(Mj, ri3);
        } else if constexpr (NBR == 1 && !ALL_NEAR) {
            // the counting walk stays straight-line (a branch per pair measured slower
            // there): every pair's weight, then W = 1 for far pairs as in the other walks
            const float2 fw = fmul2(fmul2(Mj, weight()), ri3);
            const float2 f1 = fmul2(Mj, ri3);
            f = far ? f1 : fw;
        } else if (far) {
            f = fmul2(Mj, ri3);
            if constexpr (NBR == 2 && SHELL)  // neighbours beyond r_out (r_list > r_out) only
                if ((cm >> (2 * k)) & 3u) pair_nbr<TPL, NBR, TAIL>(W, T, K, k, ns, t, r2, NC);
        } else {
            f = fmul2(fmul2(Mj, weight()), ri3);
            if constexpr (NBR == 2)  // the row-mode walk tests the pairs that may hold neighbours
                pair_nbr<TPL, NBR, TAIL>(W, T, K, k, ns, t, r2, NC);
        }
        A.p[t][0] = ffma2(f, dx, A.p[t][0]);
        A.p[t][1] = ffma2(f, dy, A.p[t][1]);
        A.p[t][2] = ffma2(f, dz, A.p[t][2]);
        if (POT) {
            A.p[t][3].x -= r2.x > 0.f ? Mj.x * ri.x : 0.f;
            A.p[t][3].y -= r2.y > 0.f ? Mj.y * ri.y : 0.f;
        }
        if constexpr (NBR == 1 && !ALL_FAR)  // the counting walk tests every pair, straight-line
            pair_nbr<TPL, NBR, TAIL>(W, T, K, k, ns, t, r2, NC);
    }
}

// Mixed form, two staged particles at a time; same terms as eval_parts.
template <int TPL, bool POT, int NBR, bool SHELL>
__device__ __forceinline__ void eval_parts_x2(const WarpSmem<float> &W, const WalkArgs &P,
                                              const Cluster &K, int nleaves, int nparts,
                                              const GroupFrame &F, const float (&px)[TPL],
                                              const float (&py)[TPL], const float (&pz)[TPL],
                                              AccX2<TPL> &A, NbrCount<TPL> &NC)
{
    const int lane = threadIdx.x & 31;
    __syncwarp();
    int carry = 0;
    for (int b = 0; b < nleaves; b += 32) {
        int i = b + lane;
        int v = i < nleaves ? W.lq[i].y : 0;
        int inc = warp_incl_scan(v);
        if (i < nleaves) W.lqo[i] = carry + inc - v;
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    __syncwarp();
    const float inv_dr = K.inv_dr_f, nrin_dr = -K.rin_dr_f;
    float2 NPX[TPL], NPY[TPL], NPZ[TPL];
#pragma unroll
    for (int t = 0; t < TPL; t++) NPX[t] = f2(-px[t]), NPY[t] = f2(-py[t]), NPZ[t] = f2(-pz[t]);
    const float4 *pq = reinterpret_cast<const float4 *>(W.pp);
    float *pb = reinterpret_cast<float *>(W.pp) + 8 * (lane >> 1) + (lane & 1);
    for (int c0 = 0; c0 < nparts; c0 += 32) {
        int pos = c0 + lane;
        const int ns = min(32, nparts - c0);
        bool wneed = false;  // not from a leaf beyond r_out: the weight W(r) is needed
        bool cand = false;   // may be a neighbour of a target of the group
        if (pos < nparts) {
            int lo = 0, hi = nleaves;  // last leaf with lqo <= pos
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (W.lqo[mid] <= pos)
                    lo = mid;
                else
                    hi = mid;
            }
            // bit 31: neighbour-only leaf (staged with mass 0); bit 30: leaf beyond r_out
            const int lx = W.lq[lo].x;
            const int j = (lx & 0x3fffffff) + (pos - W.lqo[lo]);
            wneed = (lx & (int)kFarLeaf) == 0;
            const float4 r = ds_rel(P.T.ph[j], P.T.pl[j], F);
            if (wneed) {
                // a source r_out or more from the whole group box (FP32 with a margin
                // that covers its rounding) has W = 1 with every target, like the
                // sources of a leaf beyond r_out
                const float4 b0 = W.gb[0], b1 = W.gb[1];
                const float tx = fmaxf(fmaxf(b0.x - r.x, r.x - b0.w), 0.f);
                const float ty = fmaxf(fmaxf(b0.y - r.y, r.y - b1.x), 0.f);
                const float tz = fmaxf(fmaxf(b0.z - r.z, r.z - b1.y), 0.f);
                wneed = !(tx * tx + ty * ty + tz * tz > b1.z);
            }
            cand = wneed || (SHELL && NC.beyond);
            pb[0] = r.x, pb[2] = r.y, pb[4] = r.z, pb[6] = lx < 0 ? 0.f : r.w;
            if (NBR) W.pj[lane] = j;
            if (NBR == 2) W.po[lane] = P.T.rid[j];
        }
        __syncwarp();
        if ((ns & 1) && lane == 0) {
            // pad: the partner's position with m = 0 (never counted as a neighbour)
            float *b = reinterpret_cast<float *>(W.pp) + 8 * (ns >> 1);
            b[1] = b[0], b[3] = b[2], b[5] = b[4], b[7] = 0.f;
        }
        __syncwarp();
        // slots that need the weight polynomial (a slot from a leaf beyond r_out has
        // W = 1) and slots that may hold neighbours (the same unless the cluster
        // lists neighbours beyond r_out)
        const unsigned wm = __ballot_sync(0xffffffffu, wneed);
        const unsigned cm = NBR && SHELL ? __ballot_sync(0xffffffffu, cand) : wm;
        const int nfull = ns >> 1;
        if constexpr (NBR == 0) {
            // the force-only walk (no neighbour work, fewer live registers): deeper
            // unrolling and a branch-free loop for chunks of near sources too
            const unsigned all = ns == 32 ? 0xffffffffu : (1u << ns) - 1u;
            if (wm == 0u) {
#pragma unroll 4
                for (int k = 0; k < nfull; k++)
                    part_pair<TPL, POT, NBR, SHELL, false, true>(W, P.T, K, pq, k, ns, wm, cm, inv_dr, nrin_dr, NPX,
                                                                 NPY, NPZ, A, NC);
                if (ns & 1)
                    part_pair<TPL, POT, NBR, SHELL, true, true>(W, P.T, K, pq, nfull, ns, wm, cm, inv_dr, nrin_dr,
                                                                NPX, NPY, NPZ, A, NC);
            } else if (wm == all) {
#pragma unroll 4
                for (int k = 0; k < nfull; k++)
                    part_pair<TPL, POT, NBR, SHELL, false, false, true>(W, P.T, K, pq, k, ns, wm, cm, inv_dr,
                                                                        nrin_dr, NPX, NPY, NPZ, A, NC);
                if (ns & 1)
                    part_pair<TPL, POT, NBR, SHELL, true, false, true>(W, P.T, K, pq, nfull, ns, wm, cm, inv_dr,
                                                                       nrin_dr, NPX, NPY, NPZ, A, NC);
            } else {
#pragma unroll 4
                for (int k = 0; k < nfull; k++)
                    part_pair<TPL, POT, NBR, SHELL, false>(W, P.T, K, pq, k, ns, wm, cm, inv_dr, nrin_dr, NPX, NPY,
                                                           NPZ, A, NC);
                if (ns & 1)
                    part_pair<TPL, POT, NBR, SHELL, true>(W, P.T, K, pq, nfull, ns, wm, cm, inv_dr, nrin_dr, NPX,
                                                          NPY, NPZ, A, NC);
            }
        } else if ((wm | cm) == 0u) {
            // every source of the chunk from a leaf beyond r_out: W = 1, no neighbour
#pragma unroll kPartPairUnroll
            for (int k = 0; k < nfull; k++)
                part_pair<TPL, POT, NBR, SHELL, false, true>(W, P.T, K, pq, k, ns, wm, cm, inv_dr, nrin_dr, NPX, NPY, NPZ,
                                                      A, NC);
            if (ns & 1)
                part_pair<TPL, POT, NBR, SHELL, true, true>(W, P.T, K, pq, nfull, ns, wm, cm, inv_dr, nrin_dr, NPX, NPY,
                                                     NPZ, A, NC);
        } else {
#pragma unroll kPartPairUnroll
            for (int k = 0; k < nfull; k++)
                part_pair<TPL, POT, NBR, SHELL, false>(W, P.T, K, pq, k, ns, wm, cm, inv_dr, nrin_dr, NPX, NPY, NPZ, A,
                                                NC);
            if (ns & 1)  // the last pair holds the zero-mass pad
                part_pair<TPL, POT, NBR, SHELL, true>(W, P.T, K, pq, nfull, ns, wm, cm, inv_dr, nrin_dr, NPX, NPY, NPZ,
                                               A, NC);
        }
        if constexpr (NBR == 2) {
            // the chunk's neighbours of each target: counted (the target itself
            // included, removed at the end) and appended to its row but for itself;
            // entries past the row's capacity are dropped
#pragma unroll
            for (int t = 0; t < TPL; t++) {
                unsigned h = NC.hit[t];
                NC.hit[t] = 0u;
                NC.cnt[t] += __popc(h);
                if (h && NC.si[t] >= 0) {  // (an empty slot writes nothing)
                    long long lo;
                    int cap;
                    row_span(P.row_off, P.row_entries, NC.si[t], lo, cap);
                    // two hits an iteration, their loads issued together
                    while (h) {
                        const int b0 = __ffs(h) - 1;
                        h &= h - 1u;
                        const bool two = h != 0u;
                        const int b1 = two ? __ffs(h) - 1 : b0;
                        h &= h - 1u;
                        const int j0 = W.pj[b0], j1 = W.pj[b1], o0 = W.po[b0], o1 = W.po[b1];
                        if (j0 != NC.si[t]) {
                            if (NC.wc[t] < cap) P.rows[lo + NC.wc[t]] = o0;
                            NC.wc[t]++;
                        }
                        if (two && j1 != NC.si[t]) {
                            if (NC.wc[t] < cap) P.rows[lo + NC.wc[t]] = o1;
                            NC.wc[t]++;
                        }
                    }
                }
            }
        }
        __syncwarp();
    }
    A.fold();
}

// the mixed form evaluates pairs of sources, the FP64 form one at a time
template <typename Real, int TPL, bool POT, bool QUAD, bool PAD, int NBR, bool FAST, typename AccT>
__device__ __forceinline__ void eval_cells_any(const WarpSmem<Real> &W, int ncells, const Real (&px)[TPL],
                                               const Real (&py)[TPL], const Real (&pz)[TPL], AccT &A)
{
    if constexpr (sizeof(Real) == 4) {
        eval_cells_x2<TPL, POT, QUAD, PAD, cell_pair_unroll<NBR>(), FAST>(W, ncells, px, py, pz, A);
    } else {
        eval_cells<Real, TPL, POT, QUAD>(W, ncells, px, py, pz, A);
    }
}

template <typename Real, int TPL, bool POT, int NBR, bool SHELL, typename AccT>
__device__ __forceinline__ void eval_parts_any(const WarpSmem<Real> &W, const WalkArgs &P, const Cluster &K,
                                               int nleaves, int nparts, const GroupFrame &F,
                                               const Real (&px)[TPL], const Real (&py)[TPL],
                                               const Real (&pz)[TPL], AccT &A, NbrCount<TPL> &NC)
{
    if constexpr (sizeof(Real) == 4)
        eval_parts_x2<TPL, POT, NBR, SHELL>(W, P, K, nleaves, nparts, F, px, py, pz, A, NC);
    else
        eval_parts<Real, TPL, POT, NBR>(W, P, K, nleaves, nparts, F, px, py, pz, A, NC);
}

// Control block of a group walked by WPG > 1 warps (shared memory, after the
// warps' own areas): the group taken from the ticket, the lanes' largest target
// offset per warp (for the neighbour band), and what the walking warp queued for
// the current evaluation round.
struct GroupCtl {
    int g;
    int ncells, nleaves, nparts;
    int done;
    int parts_first;  // the round evaluates the particles before the cells
    float amax[4];
};

// Threads of a walk block: WPG = 1, kWalkWarps independent warps; WPG > 1, one
// group of WPG warps (so that the walking warp's queues and the control block sit
// at fixed offsets of the block's shared memory).
template <int WPG>
constexpr int walk_block_threads()
{
    return 32 * (WPG == 1 ? kWalkWarps : WPG);
}

// WPG warps per group (threads per group 32 WPG).  WPG = 1: one warp walks and
// evaluates its group, TPL targets per lane.  WPG > 1 (TPL = 1, one group per
// block): the first warp walks the tree and queues cells and leaves in its shared
// memory; whenever a queue reaches the tile (or the walk ends), every warp of the
// block evaluates the queues for its own 32 targets, between two block barriers.
// Every warp executes the same sequence of barriers: the round loop ends on the
// flag the walking warp writes before a round's first barrier and nobody changes
// before its second.
// FORM: 0 the FP64 form; a mixed walk is launched twice, 1 with the r^-5 cell term,
// which does the work when every cluster of the tree fits that form (fast_cells),
// and 2 with the r^-3 term, which does it otherwise; the other launch returns at once.
template <typename Real, int TPL, bool POT, bool QUAD, int NBR, bool SHELL, int WPG, int FORM = 0>
__global__ void __launch_bounds__(walk_block_threads<WPG>(),
                                  TPL == 1 ? (NBR == 2 ? 5 : kMinBlocksTpl1) * kWalkWarps / (WPG == 1 ? kWalkWarps : WPG) : 3)
    walk_kernel(WalkArgs P)
{
    pdl_wait();
    static_assert(WPG == 1 || TPL == 1, "several warps per group hold one target per lane");
    static_assert(FORM == 0 || sizeof(Real) == 4, "cell forms: mixed walks");
    extern __shared__ __align__(16) char smem[];
    using R4 = typename Vec4<Real>::T;
    using R2 = typename Vec4<Real>::T2;
    constexpr bool kMixed = sizeof(Real) == 4;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int warp = threadIdx.x >> 5;
    const int wig = WPG == 1 ? 0 : warp;  // warp within its group; 0 walks the tree
    const bool walker = wig == 0;
    const size_t wbytes = WarpSmem<Real>::bytes(P.tile);
    WarpSmem<Real> W;  // queues of the group's walking warp, staging of this warp
    W.carve(smem + warp * wbytes, P.tile);
    if constexpr (WPG > 1) {
        WarpSmem<Real> L;
        L.carve(smem, P.tile);
        W.stk = L.stk, W.cpos = L.cpos, W.cqa = L.cqa, W.cqb = L.cqb, W.lq = L.lq;
    }
    GroupCtl *ctl = reinterpret_cast<GroupCtl *>(smem + WPG * wbytes);
    const Tree &T = P.T;
    Meta *meta = T.meta;
    const int ng = meta->n_groups;
    const int nn = meta->n_nodes;
    const int tile = P.tile;
    // the r^-5 launch runs when every cluster fits that form, the r^-3 launch otherwise
    if (FORM != 0 && (meta->cell_forms[1] == 0) != (FORM == 1)) return;

    while (true) {
        int g = 0;
        if constexpr (WPG == 1) {
            if (lane == 0) g = (int)atomicAdd(P.ticket, 1u);
            g = __shfl_sync(0xffffffffu, g, 0);
        } else {
            if (walker && lane == 0) ctl->g = (int)atomicAdd(P.ticket, 1u);
            __syncthreads();
            g = ctl->g;
        }
        if (g >= ng) break;
        g = T.gorder[g];  // smallest group boxes first (made by the build)
        const int2 gr = T.grp[g];
        double4_32a glo, ghi;  // the FP64 form's group box (the mixed form reloads it when needed)
        if constexpr (!kMixed) glo = T.glo[g], ghi = T.ghi[g];
        // the group's cluster: its frame O, its root (node cid) and the filter bands
        // (|FP32 - FP64| of a squared distance <= k_rel (d2 + r2) + k_abs |t|_1 +
        // k_sq, about twice the derived bound, every coordinate relative to O being
        // within R and carrying <= 2^-24 R rounding; for a fixed threshold r this is
        // at most A d2 + B, see fp32_band).  Outside a safe range of scales the
        // filter is off and every test is exact FP64.
        const int cid = T.cid_s[gr.x];
        const Cluster &K = T.cl[cid];
        const double *fr = K.frame;
        const double Ox = fr[0], Oy = fr[1], Oz = fr[2];
        const float Rf = (float)fr[3] * 1.0001f;
        const float rout2_f = K.rout2_f;
        const double rout2_d = K.rout2_d;
        const bool filter_ok = Rf > 1e-6f && Rf < 1e12f && rout2_f > 1e-20f && rout2_f < 1e30f;
        // FORM 1 / 2: this launch takes only the groups of clusters whose cell term
        // stays / does not stay in the FP32 range in the r^-5 form (cell_forms_kernel)
        constexpr bool fast_cells = kMixed && FORM == 1;
        const bool count_here = NBR && K.counted;
        const bool shell = SHELL && count_here && K.rl2_d > rout2_d;  // neighbours beyond r_out
        const float rl2_f = K.rl2_f;
        const float k_rel = 8.f * kU, k_abs = 8.f * kU * Rf, k_sq = 16.f * kU * kU * Rf * Rf;
        const Band bb_band = fp32_band(Rf, rout2_f);  // the box-box test against r_out
        const Band bl_band = fp32_band(Rf, rl2_f);    // and against r_list (shell)
        GroupFrame F;
        float glx, gly, glz, ghx, ghy, ghz;  // group box relative to O for the FP32 filter
        if constexpr (kMixed) {
            // c_g's double-single split and the box, made once per build (group_frames_kernel)
            const float4 g0 = T.gfr[3 * (size_t)g], g1 = T.gfr[3 * (size_t)g + 1],
                         g2 = T.gfr[3 * (size_t)g + 2];
            F.cx = F.cy = F.cz = 0.0;  // (the mixed form works relative to O)
            F.hx = g0.x, F.hy = g0.y, F.hz = g0.z, F.lx = g0.w, F.ly = g1.x, F.lz = g1.y;
            glx = g1.z, gly = g1.w, glz = g2.x, ghx = g2.y, ghy = g2.z, ghz = g2.w;
        } else {
            F.cx = dmul(0.5, dadd(glo.x, ghi.x));
            F.cy = dmul(0.5, dadd(glo.y, ghi.y));
            F.cz = dmul(0.5, dadd(glo.z, ghi.z));
            ds_split(dsub(F.cx, Ox), F.hx, F.lx);
            ds_split(dsub(F.cy, Oy), F.hy, F.ly);
            ds_split(dsub(F.cz, Oz), F.hz, F.lz);
            glx = __double2float_rn(dsub(glo.x, Ox)), gly = __double2float_rn(dsub(glo.y, Oy));
            glz = __double2float_rn(dsub(glo.z, Oz));
            ghx = __double2float_rn(dsub(ghi.x, Ox)), ghy = __double2float_rn(dsub(ghi.y, Oy));
            ghz = __double2float_rn(dsub(ghi.z, Oz));
        }
        if constexpr (kMixed) {
            if (lane == 0) {
                // the source test of eval_parts_x2: box - c_g carries <= ~6 u R per
                // coordinate and a source offset about as much, so a distance above
                // r_out (1 + 1e-5) + 32 u R in FP32 is above r_out exactly
                const float t = sqrtf(rout2_f) * 1.00001f + 32.f * kU * Rf;
                W.gb[0] = make_float4((glx - F.hx) - F.lx, (gly - F.hy) - F.ly, (glz - F.hz) - F.lz,
                                      (ghx - F.hx) - F.lx);
                W.gb[1] = make_float4((ghy - F.hy) - F.ly, (ghz - F.hz) - F.lz, filter_ok ? t * t : INFINITY, 0.f);
            }
        }
        Real px[TPL], py[TPL], pz[TPL];
        NbrCount<TPL> NC;
        NC.beyond = false;
        float amax = 0.f;
#pragma unroll
        for (int t = 0; t < TPL; t++) {
            int s = gr.x + lane + 32 * (wig + WPG * t);
            NC.cnt[t] = 0;
            NC.si[t] = -1;
            if constexpr (NBR == 2) {
                // an empty slot (at c_g) must write nothing: its count starts past any cap
                NC.hit[t] = 0u;
                NC.wc[t] = s < gr.x + gr.y ? 0 : (1 << 30);
            }
            if (s < gr.x + gr.y) {
                if (kMixed) {
                    float4 r = ds_rel(T.ph[s], T.pl[s], F);
                    px[t] = r.x, py[t] = r.y, pz[t] = r.z;
                    amax = fmaxf(amax, fmaxf(fabsf(r.x), fmaxf(fabsf(r.y), fabsf(r.z))));
                } else {
                    double4_32a q = T.sp[s];
                    px[t] = to_real<Real>(dsub(q.x, F.cx));
                    py[t] = to_real<Real>(dsub(q.y, F.cy));
                    pz[t] = to_real<Real>(dsub(q.z, F.cz));
                }
                NC.si[t] = s;
            } else {
                px[t] = py[t] = pz[t] = Real(0);
            }
        }
        if (NBR) {
            // band of the neighbour pair test: coordinates relative to c_g carry
            // <= 2.01 u |x - c_g| + 8 u^2 R (double-single), targets within A of c_g
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
            if constexpr (WPG > 1) {
                // A is the group's: the largest offset over the targets of every warp
                if (lane == 0) ctl->amax[wig] = amax;
                __syncthreads();
#pragma unroll
                for (int w = 0; w < WPG; w++) amax = fmaxf(amax, ctl->amax[w]);
            }
            const float A = amax * 1.0001f;
            const float band = kU * (24.f * K.rl2_f + 32.f * A * K.rl_f + 128.f * kU * Rf * K.rl_f) +
                               64.f * kU * kU * (A + 2.f * K.rl_f) * (A + 2.f * K.rl_f);
            NC.beyond = shell;
            if (!count_here)
                NC.off();  // this cluster is counted elsewhere
            else if (filter_ok)
                NC.set(K.rl2_f - band, K.rl2_f + band);
            else
                NC.set(-1.f, INFINITY);  // filter off: every pair decided in FP64
        }
        typename std::conditional<kMixed, AccX2<TPL>, Acc<double, TPL>>::type A;
        A.zero_all();
        int sp = 1;
        if (walker && lane == 0) W.stk[0] = pack_range_f(cid, 1, false);
        __syncwarp();
        int cb = 0, lqn = 0, lqp = 0;
        long long ncell = 0, npart = 0;
        int nfallback = 0;
        int iters = 0;  // a valid walk pops every node at most once

        // One batch of the traversal (the walking warp): pop up to 32 nodes, test,
        // push the opened internal nodes, queue accepted cells and opened leaves.
        // Returns false when the walk must stop (a latched error).
        auto walk_batch = [&]() -> bool {
            if (++iters > nn + 1) {
                if (lane == 0) latch_error(meta, P3T_ERR_INTERNAL);
                return false;
            }
            // ---- pop up to 32 nodes, one per lane (flagged: neighbour-only range)
            bool nbr_only = false;
            int node;
            if constexpr (SHELL)
                node = pop_batch_f(W.stk, sp, nbr_only);
            else
                node = pop_batch(W.stk, sp);

            // ---- opening test (test and staging data come in one load batch)
            bool open = false, is_leaf = false, in_shell = false;
            bool beyond = false;  // box certainly r_out or more from the group box: W = 1
            int cinfo = 0, ccount = 0;
            float4 ra, rd, rq0, rq1;  // node record: COM hi / lo + M / quadrupole
            if (node >= 0) {
                if (kMixed) {
                    const auto rec = wrec_at(T.wn, node);
                    ra = rec[0];
                    const float4 b = rec[1], c = rec[2];
                    rd = rec[3];
                    rq0 = rec[4];
                    rq1 = rec[5];
                    cinfo = __float_as_int(b.w);
                    ccount = __float_as_int(c.w);
                    // FP32 tests with their error bands: the opening angle's band keeps the
                    // |t|_1 term (it follows sqrt(d2) for nodes of every size, down to
                    // single particles); the box test against r_out uses A d2 + B
                    bool dec_m = false, dec_b = false, in_m = false, in_b = false;
                    if (filter_ok) {
                        // point-box: COM against the group box
                        const float tx = fmaxf(fmaxf(glx - ra.x, ra.x - ghx), 0.f);
                        const float ty = fmaxf(fmaxf(gly - ra.y, ra.y - ghy), 0.f);
                        const float tz = fmaxf(fmaxf(glz - ra.z, ra.z - ghz), 0.f);
                        const float d2 = tx * tx + ty * ty + tz * tz;
                        const float dm = d2 - ra.w;  // -inf for theta = 0: always open
                        dec_m = isinf(ra.w) ||
                                fabsf(dm) > k_rel * (d2 + ra.w) + k_abs * (tx + ty + tz) + k_sq;
                        in_m = dm < 0.f;
                        // box-box against r_out
                        const float ux = fmaxf(fmaxf(b.x - ghx, glx - c.x), 0.f);
                        const float uy = fmaxf(fmaxf(b.y - ghy, gly - c.y), 0.f);
                        const float uz = fmaxf(fmaxf(b.z - ghz, glz - c.z), 0.f);
                        const float e2 = ux * ux + uy * uy + uz * uz;
                        const float db = e2 - rout2_f;
                        dec_b = fabsf(db) > fmaf(bb_band.a, e2, bb_band.b);
                        in_b = db < 0.f;
                    }
                    // (with r_list > r_out a force leaf beyond r_out may still hold neighbours)
                    beyond = dec_b && !in_b;
                    if (SHELL && nbr_only) {
                        // neighbour-only range: the box test against r_list alone
                        bool dec_l = false, in_l = false;
                        if (filter_ok) {
                            const float ux = fmaxf(fmaxf(b.x - ghx, glx - c.x), 0.f);
                            const float uy = fmaxf(fmaxf(b.y - ghy, gly - c.y), 0.f);
                            const float uz = fmaxf(fmaxf(b.z - ghz, glz - c.z), 0.f);
                            const float e2 = ux * ux + uy * uy + uz * uz;
                            const float dl = e2 - rl2_f;
                            dec_l = fabsf(dl) > fmaf(bl_band.a, e2, bl_band.b);
                            in_l = dl < 0.f;
                        }
                        if (!dec_l) {
                            nfallback += filter_ok;
                            const double4_32a cl = T.lo[node], ch = T.hi[node];
                            in_l = dist2_box_box(T.glo[g], T.ghi[g], cl, ch) < T.cl[cid].rl2_d;
                        }
                        open = in_l;
                    } else if ((dec_m && in_m) || (dec_b && in_b)) {
                        open = true;
                    } else if (dec_m && dec_b) {
                        open = false;
                    } else {
                        // undecided in FP32 (rare): the exact FP64 test; the group box and
                        // r_out^2 are reloaded so they need no registers during the walk
                        nfallback += filter_ok;
                        const double4_32a cm = T.comM[node], cl = T.lo[node], ch = T.hi[node];
                        const double4_32a bl = T.glo[g], bh = T.ghi[g];
                        open = dist2_point_box(cm.x, cm.y, cm.z, bl, bh) < cl.w ||
                               dist2_box_box(bl, bh, cl, ch) < T.cl[cid].rout2_d;
                    }
                    if (SHELL && shell && !nbr_only && !open) {
                        // a cell the force accepts may still hold neighbours (r_list > r_out)
                        bool dec_l = false, in_l = false;
                        if (filter_ok) {
                            const float ux = fmaxf(fmaxf(b.x - ghx, glx - c.x), 0.f);
                            const float uy = fmaxf(fmaxf(b.y - ghy, gly - c.y), 0.f);
                            const float uz = fmaxf(fmaxf(b.z - ghz, glz - c.z), 0.f);
                            const float e2 = ux * ux + uy * uy + uz * uz;
                            const float dl = e2 - rl2_f;
                            dec_l = fabsf(dl) > fmaf(bl_band.a, e2, bl_band.b);
                            in_l = dl < 0.f;
                        }
                        if (!dec_l) {
                            nfallback += filter_ok;
                            const double4_32a cl = T.lo[node], ch = T.hi[node];
                            in_l = dist2_box_box(T.glo[g], T.ghi[g], cl, ch) < T.cl[cid].rl2_d;
                        }
                        in_shell = in_l;
                    }
                } else {
                    const double4_32a cm = T.comM[node], cl = T.lo[node], ch = T.hi[node];
                    const auto rec = wrec_at(T.wn, node);
                    cinfo = __float_as_int(rec[1].w);
                    ccount = __float_as_int(rec[2].w);
                    open = dist2_point_box(cm.x, cm.y, cm.z, glo, ghi) < cl.w ||
                           dist2_box_box(glo, ghi, cl, ch) < rout2_d;
                }
                is_leaf = cinfo < 0;
            }
            // force: accepted cells and opened nodes of force ranges; neighbour count
            // only: flagged ranges that pass the r_list test and accepted shell cells
            const bool accept = node >= 0 && !open && !nbr_only;
            const bool go_nbr = node >= 0 && ((nbr_only && open) || in_shell);
            const bool open_int = node >= 0 && ((open && !nbr_only) || go_nbr) && !is_leaf;
            const bool open_leaf = node >= 0 && ((open && !nbr_only) || go_nbr) && is_leaf;
            // consistency of the child / particle ranges before following them
            const bool bad = (open_int && (ccount < 1 || ccount > 8 || cinfo + ccount > nn)) ||
                             (open_leaf && (ccount < 1 || -1 - cinfo + ccount > T.n_src));
            if (__any_sync(0xffffffffu, bad)) {
                if (lane == 0) latch_error(meta, P3T_ERR_INTERNAL);
                return false;
            }

            // ---- push child ranges (lane 0's, the deepest, ends on top)
            const unsigned pm = __ballot_sync(0xffffffffu, open_int);
            const int npush = __popc(pm);
            if (sp + npush > kStackCap) {
                if (lane == 0) latch_error(meta, P3T_ERR_CAPACITY);
                sp = 0;
                return false;
            }
            if (open_int) W.stk[sp + __popc(pm >> lane >> 1)] = pack_range_f(cinfo, ccount, go_nbr);
            sp += npush;

            // ---- queue accepted cells
            const unsigned am = __ballot_sync(0xffffffffu, accept);
            if (accept) {
                const int pos = cb + __popc(am & lt);
                R4 v;
                R4 qa;
                R2 qb;
                if (kMixed) {
                    // pair layout: negated position and mass, then the quadrupole
                    const float4 r = ds_rel(ra, rd, F);
                    float *b = reinterpret_cast<float *>(W.cpos) + 20 * (pos >> 1) + (pos & 1);
                    b[0] = -r.x, b[2] = -r.y, b[4] = -r.z, b[6] = -rd.w;
                    if (QUAD) {
                        b[8] = rq0.x, b[10] = rq0.y, b[12] = rq0.z, b[14] = rq0.w;
                        b[16] = rq1.x, b[18] = rq1.y;
                    }
                } else {
                    const double4_32a cm = T.comM[node];
                    v.x = to_real<Real>(dsub(cm.x, F.cx));
                    v.y = to_real<Real>(dsub(cm.y, F.cy));
                    v.z = to_real<Real>(dsub(cm.z, F.cz));
                    v.w = to_real<Real>(cm.w);
                    const double2 *q = reinterpret_cast<const double2 *>(T.q64 + 6 * (size_t)node);
                    const double2 q0 = q[0], q1 = q[1], q2 = q[2];
                    qa.x = q0.x, qa.y = q0.y, qa.z = q1.x, qa.w = q1.y, qb.x = q2.x, qb.y = q2.y;
                    W.cpos[pos] = v;
                    if (QUAD) {
                        W.cqa[pos] = qa;
                        W.cqb[pos] = qb;
                    }
                }
            }
            const int na = __popc(am);
            cb += na;
            ncell += na;

            // ---- queue opened leaves (neighbour-only ones flagged in bit 31 of .x)
            const unsigned lm = __ballot_sync(0xffffffffu, open_leaf);
            if (open_leaf)
                W.lq[lqn + __popc(lm & lt)] =
                    make_int2((int)((unsigned)(-1 - cinfo) | (go_nbr ? kRangeFlag : 0u) |
                                    (beyond ? kFarLeaf : 0u)),
                              ccount);
            lqn += __popc(lm);
            const int lc = (int)__reduce_add_sync(0xffffffffu, open_leaf ? (unsigned)ccount : 0u);
            lqp += lc;
            npart += shell ? (int)__reduce_add_sync(0xffffffffu, open_leaf && !go_nbr ? (unsigned)ccount : 0u)
                           : lc;
            return true;
        };

        if constexpr (WPG == 1) {
            while (sp > 0) {
                if (!walk_batch()) break;
                if (cb >= tile) {
                    eval_cells_any<Real, TPL, POT, QUAD, true, NBR, fast_cells>(W, cb, px, py, pz, A);
                    cb = 0;
                }
                if (lqp >= tile) {
                    eval_parts_any<Real, TPL, POT, NBR, SHELL>(W, P, K, lqn, lqp, F, px, py, pz, A, NC);
                    lqn = lqp = 0;
                }
            }
            if (cb > 0) eval_cells_any<Real, TPL, POT, QUAD, true, NBR, fast_cells>(W, cb, px, py, pz, A);
            if (lqp > 0) eval_parts_any<Real, TPL, POT, NBR, SHELL>(W, P, K, lqn, lqp, F, px, py, pz, A, NC);
        } else {
            // evaluation rounds: the walking warp fills the queues up to a tile, then
            // every warp of the group evaluates them for its own targets
            while (true) {
                if (walker) {
                    bool stop = false;
                    while (sp > 0 && cb < tile && lqp < tile)
                        if (!walk_batch()) {
                            stop = true;
                            break;
                        }
                    const bool fin = stop || sp == 0;
                    const int ec = (cb >= tile || fin) ? cb : 0;
                    const int ep = (lqp >= tile || fin) ? lqp : 0;
                    if (kMixed && (ec & 1) && lane == 0) {
                        // pad the pair layout once for every warp: the partner's position
                        // with M = 0 and Q = 0 adds exactly zero
                        float *b = reinterpret_cast<float *>(W.cpos) + 20 * (ec >> 1);
                        b[1] = b[0], b[3] = b[2], b[5] = b[4];
                        b[7] = b[9] = b[11] = b[13] = b[15] = b[17] = b[19] = 0.f;
                    }
                    if (lane == 0) {
                        ctl->ncells = ec;
                        ctl->nleaves = ep ? lqn : 0;
                        ctl->nparts = ep;
                        ctl->done = fin;
                        // the one-warp walk's order: due queues (a full tile) as the last
                        // batch left them, cells first, then at the end what remains; so
                        // when only the particles were due, they come before the cells
                        ctl->parts_first = lqp >= tile && cb < tile;
                    }
                }
                __syncthreads();  // the round's queues are complete
                const int ec = ctl->ncells, el = ctl->nleaves, ep = ctl->nparts;
                const bool fin = ctl->done != 0;
                const bool parts_first = ctl->parts_first != 0;
#pragma unroll 1
                for (int pass = 0; pass < 2; pass++) {  // one call site each (code size)
                    if ((pass == 0) != parts_first) {
                        if (ec > 0) eval_cells_any<Real, TPL, POT, QUAD, false, NBR, fast_cells>(W, ec, px, py, pz, A);
                    } else if (ep > 0) {
                        eval_parts_any<Real, TPL, POT, NBR, SHELL>(W, P, K, el, ep, F, px, py, pz, A, NC);
                    }
                }
                __syncthreads();  // every warp is done with them
                if (ec > 0) cb = 0;
                if (ep > 0) lqn = lqp = 0;
                if (fin) break;
            }
        }

        // ---- results, scattered to the original order
#pragma unroll
        for (int t = 0; t < TPL; t++) {
            int s = gr.x + lane + 32 * (wig + WPG * t);
            if (s < gr.x + gr.y) {
                int o = T.perm[s];
                if (kMixed) {
                    ((float *)P.ax)[o] = (float)(A.s[t][0] - A.c[t][0]);
                    ((float *)P.ay)[o] = (float)(A.s[t][1] - A.c[t][1]);
                    ((float *)P.az)[o] = (float)(A.s[t][2] - A.c[t][2]);
                    if (POT) P.pot[o] = (double)A.s[t][3] - (double)A.c[t][3];
                } else {
                    ((double *)P.ax)[o] = (double)A.s[t][0];
                    ((double *)P.ay)[o] = (double)A.s[t][1];
                    ((double *)P.az)[o] = (double)A.s[t][2];
                    if (POT) P.pot[o] = (double)A.s[t][3];
                }
                if (count_here) P.nbr_count[o] = NC.cnt[t] - 1;  // minus the pair with itself
                if constexpr (NBR == 2) {  // a row that outgrew its room: the fill pass rebuilds it
                    long long lo;
                    int cap;
                    row_span(P.row_off, P.row_entries, s, lo, cap);
                    if (NC.wc[t] > cap) meta->row_over = 1;
                }
            }
        }
        if (walker) {
            const unsigned nfb = __reduce_add_sync(0xffffffffu, (unsigned)nfallback);
            if (lane == 0) {
                if (P.n_cell) atomicAdd(P.n_cell, (unsigned long long)(ncell * gr.y));
                if (P.n_part) atomicAdd(P.n_part, (unsigned long long)(npart * gr.y));
                if (P.grp_cells) {
                    P.grp_cells[g] = ncell;
                    P.grp_parts[g] = npart;
                }
                if (nfb) atomicAdd((unsigned long long *)&meta->fallback_tests, (unsigned long long)nfb);
            }
        }
        __syncwarp();
    }
}

// Dynamic shared memory of one walk block: the warps' areas, then (WPG > 1) the
// group's control block.
inline size_t walk_smem_bytes(int tile, bool fp64, int wpg)
{
    const size_t w = fp64 ? WarpSmem<double>::bytes(tile) : WarpSmem<float>::bytes(tile);
    return wpg == 1 ? kWalkWarps * w : wpg * w + sizeof(GroupCtl);
}

template <typename Real, int TPL, bool POT, bool QUAD, int NBR, bool SHELL, int WPG, int FORM>
static int launch_walk(p3t_ctx *c, const WalkArgs &a)
{
    auto kern = walk_kernel<Real, TPL, POT, QUAD, NBR, SHELL, WPG, FORM>;
    const size_t smem = walk_smem_bytes(a.tile, sizeof(Real) == 8, WPG);
    constexpr int threads = walk_block_threads<WPG>();
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return P3T_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess ||
        per_sm < 1)
        return P3T_ERR_CUDA;
    if (launch_pdl_smem(kern, dim3(per_sm * c->sm_count), dim3(threads), smem, c->stream, a) != cudaSuccess)
        return P3T_ERR_CUDA;
    return check_launch(c);
}

template <typename Real, int TPL, int NBR, bool SHELL, int WPG, int FORM>
static int dispatch_pq(p3t_ctx *c, const WalkArgs &a, bool pot, bool quad)
{
    if (pot)
        return quad ? launch_walk<Real, TPL, true, true, NBR, SHELL, WPG, FORM>(c, a)
                    : launch_walk<Real, TPL, true, false, NBR, SHELL, WPG, FORM>(c, a);
    return quad ? launch_walk<Real, TPL, false, true, NBR, SHELL, WPG, FORM>(c, a)
                : launch_walk<Real, TPL, false, false, NBR, SHELL, WPG, FORM>(c, a);
}

// The variants of one warps-per-group count: precision, neighbour work (0 none,
// 1 count, 2 count and rows), neighbour-only ranges (shell), potential, quadrupole.
// FORM 0 is the FP64 form, 1 and 2 the mixed form's two launches.
template <int WPG, int FORM>
int dispatch_walk_wpg(p3t_ctx *c, const WalkArgs &a, int nbr, bool shell, bool pot, bool quad)
{
    if constexpr (FORM == 0) {
        return dispatch_pq<double, 1, 0, false, WPG, 0>(c, a, pot, quad);
    } else {
        if (shell)
            return nbr == 2 ? dispatch_pq<float, 1, 2, true, WPG, FORM>(c, a, pot, quad)
                            : dispatch_pq<float, 1, 1, true, WPG, FORM>(c, a, pot, quad);
        if (nbr == 2) return dispatch_pq<float, 1, 2, false, WPG, FORM>(c, a, pot, quad);
        if (nbr == 1) return dispatch_pq<float, 1, 1, false, WPG, FORM>(c, a, pot, quad);
        return dispatch_pq<float, 1, 0, false, WPG, FORM>(c, a, pot, quad);
    }
}

// One warp per group: TPL targets per lane for groups of up to 32 TPL particles.
template <typename Real, int NBR, bool SHELL, int FORM>
int dispatch_tpl(p3t_ctx *c, const WalkArgs &a, bool pot, bool quad)
{
    const int G = c->prm.group_size;
    if constexpr (NBR == 2) return dispatch_pq<Real, 1, 2, SHELL, 1, FORM>(c, a, pot, quad);  // G <= 32
    if (G <= 32) return dispatch_pq<Real, 1, NBR, SHELL, 1, FORM>(c, a, pot, quad);
    if (G <= 64) return dispatch_pq<Real, 2, NBR, SHELL, 1, FORM>(c, a, pot, quad);
    return dispatch_pq<Real, 4, NBR, SHELL, 1, FORM>(c, a, pot, quad);
}

// One launch of the mixed walk with cell form FORM (1 or 2) for the context's warps per
// group and neighbour work (0 none, 1 count, 2 count and rows; shell: neighbour-only
// ranges).  Instantiated in walk_f1.cu and walk_f2.cu, the several-warp variants in
// walk_wpg.cu, so that the translation units compile in parallel.
template <int FORM>
int mixed_walk(p3t_ctx *c, const WalkArgs &a, int wpg, int nbr, bool shell, bool pot, bool quad)
{
    if (wpg > 1)
        return wpg == 2 ? dispatch_walk_wpg<2, FORM>(c, a, nbr, shell, pot, quad)
                        : dispatch_walk_wpg<4, FORM>(c, a, nbr, shell, pot, quad);
    if (shell)
        return nbr == 2 ? dispatch_tpl<float, 2, true, FORM>(c, a, pot, quad)
                        : dispatch_tpl<float, 1, true, FORM>(c, a, pot, quad);
    if (nbr == 2) return dispatch_tpl<float, 2, false, FORM>(c, a, pot, quad);
    if (nbr == 1) return dispatch_tpl<float, 1, false, FORM>(c, a, pot, quad);
    return dispatch_tpl<float, 0, false, FORM>(c, a, pot, quad);
}

#define P3T_WPG_DECL(W, F) extern template int dispatch_walk_wpg<W, F>(p3t_ctx *, const WalkArgs &, int, bool, bool, bool);
P3T_WPG_DECL(2, 0)
P3T_WPG_DECL(2, 1)
P3T_WPG_DECL(2, 2)
P3T_WPG_DECL(4, 0)
P3T_WPG_DECL(4, 1)
P3T_WPG_DECL(4, 2)
#undef P3T_WPG_DECL
extern template int mixed_walk<1>(p3t_ctx *, const WalkArgs &, int, int, bool, bool, bool);
extern template int mixed_walk<2>(p3t_ctx *, const WalkArgs &, int, int, bool, bool, bool);

}  // namespace p3t
