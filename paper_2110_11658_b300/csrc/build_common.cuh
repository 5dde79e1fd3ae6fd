// Device helpers shared by the tree build (build_tree.cu) and the decomposed
// cluster's tree joins (decomp.cu): order-preserving encodings of doubles, exact
// boxes, Morton-key quantisation (rules 1-3), and the moments of an internal node
// from its children with its records (rules 6 and 8).
#pragma once

#include <cstdint>

#include "p3t_internal.cuh"

namespace p3t {

constexpr unsigned long long kQMax = (1ULL << 21) - 1;

// order-preserving map of non-NaN doubles onto unsigned integers
__device__ __forceinline__ unsigned long long enc_double(double v)
{
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ULL);
}
__device__ __forceinline__ double dec_double(unsigned long long e)
{
    unsigned long long u = (e >> 63) ? (e ^ 0x8000000000000000ULL) : ~e;
    return __longlong_as_double((long long)u);
}

__device__ __forceinline__ unsigned long long spread3(unsigned long long v)
{
    v &= 0x1fffffULL;
    v = (v | (v << 32)) & 0x1f00000000ffffULL;
    v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
    v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
    v = (v | (v << 2)) & 0x1249249249249249ULL;
    return v;
}

__device__ __forceinline__ unsigned long long quantise(double v, double lo, double s)
{
    double t = floor(dmul(dsub(v, lo), s));
    if (!(t >= 0.0)) return 0;  // also NaN
    if (t > (double)kQMax) return kQMax;
    return (unsigned long long)t;
}


// Exact box bounds on the integer pipes: min/max of the order-preserving
// encodings (no FP64 instruction).  Equal to the FP64 min/max except that -0
// orders below +0, which changes no distance, extent or centre computed later.
struct EncBox {
    unsigned long long lo[3], hi[3];
    __device__ void reset()
    {
        for (int d = 0; d < 3; d++) lo[d] = ~0ULL, hi[d] = 0ULL;
    }
    __device__ void add(double x, double y, double z)
    {
        unsigned long long e[3] = {enc_double(x), enc_double(y), enc_double(z)};
#pragma unroll
        for (int d = 0; d < 3; d++) {
            lo[d] = e[d] < lo[d] ? e[d] : lo[d];
            hi[d] = e[d] > hi[d] ? e[d] : hi[d];
        }
    }
    __device__ void add_box(const double4_32a &l, const double4_32a &h)
    {
        unsigned long long a[3] = {enc_double(l.x), enc_double(l.y), enc_double(l.z)};
        unsigned long long b[3] = {enc_double(h.x), enc_double(h.y), enc_double(h.z)};
#pragma unroll
        for (int d = 0; d < 3; d++) {
            lo[d] = a[d] < lo[d] ? a[d] : lo[d];
            hi[d] = b[d] > hi[d] ? b[d] : hi[d];
        }
    }
    __device__ void get(double *l, double *h) const
    {
        for (int d = 0; d < 3; d++) l[d] = dec_double(lo[d]), h[d] = dec_double(hi[d]);
    }
};


template <bool Q64>
__device__ void write_node(Tree &T, int k, double M, const double com[3], const double lo[3],
                           const double hi[3], const double *q, double, int4 tp)
{
    const Cluster &K = T.cl[T.cid_s[tp.x < T.n ? tp.x : 0]];
    const double theta = K.theta;
    // opening radius l/theta + delta
    double l = dsub(hi[0], lo[0]);
    if (dsub(hi[1], lo[1]) > l) l = dsub(hi[1], lo[1]);
    if (dsub(hi[2], lo[2]) > l) l = dsub(hi[2], lo[2]);
    double cx = dsub(dmul(0.5, dadd(lo[0], hi[0])), com[0]);
    double cy = dsub(dmul(0.5, dadd(lo[1], hi[1])), com[1]);
    double cz = dsub(dmul(0.5, dadd(lo[2], hi[2])), com[2]);
    double delta = dsqrt(dadd(dadd(dmul(cx, cx), dmul(cy, cy)), dmul(cz, cz)));
    double ro2;
    if (theta > 0.0) {
        double ro = dadd(ddiv(l, theta), delta);
        ro2 = dmul(ro, ro);
    } else {
        ro2 = INFINITY;
    }
    T.comM[k] = make_double4_32a(com[0], com[1], com[2], M);
    T.lo[k] = make_double4_32a(lo[0], lo[1], lo[2], ro2);
    T.hi[k] = make_double4_32a(hi[0], hi[1], hi[2], 0.0);
    if (Q64) {
        double2 *q2 = reinterpret_cast<double2 *>(T.q64 + 6 * (size_t)k);
        q2[0] = make_double2(q[0], q[1]);
        q2[1] = make_double2(q[2], q[3]);
        q2[2] = make_double2(q[4], q[5]);
    } else {
        float2 *q2 = reinterpret_cast<float2 *>(T.q32 + 6 * (size_t)k);
        q2[0] = make_float2((float)q[0], (float)q[1]);
        q2[1] = make_float2((float)q[2], (float)q[3]);
        q2[2] = make_float2((float)q[4], (float)q[5]);
    }
    const double *O = K.frame;
    const bool leaf = tp.z < 0;
    float chx, chy, chz, clx, cly, clz;
    ds_split(dsub(com[0], O[0]), chx, clx);
    ds_split(dsub(com[1], O[1]), chy, cly);
    ds_split(dsub(com[2], O[2]), chz, clz);
    const auto w = wrec_at(T.wn, k);
    w[0] = make_float4(chx, chy, chz, __double2float_rn(ro2));
    w[1] = make_float4(__double2float_rn(dsub(lo[0], O[0])), __double2float_rn(dsub(lo[1], O[1])),
                       __double2float_rn(dsub(lo[2], O[2])), __int_as_float(leaf ? -1 - tp.x : tp.z));
    w[2] = make_float4(__double2float_rn(dsub(hi[0], O[0])), __double2float_rn(dsub(hi[1], O[1])),
                       __double2float_rn(dsub(hi[2], O[2])), __int_as_float(leaf ? tp.y : tp.w));
    w[3] = make_float4(clx, cly, clz, __double2float_rn(M));
    w[4] = make_float4((float)q[0], (float)q[1], (float)q[2], (float)q[3]);
    w[5] = make_float4((float)q[4], (float)q[5], 0.f, 0.f);
}


// L2-coherent load of a value written by another block in this kernel
__device__ __forceinline__ double4_32a ldcg_d4(const double4_32a *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 a = __ldcg(q), b = __ldcg(q + 1);
    return make_double4_32a(a.x, a.y, b.x, b.y);
}

template <bool Q64>
__device__ void internal_moments(Tree &T, int k, int4 tp, double theta)
{
    const int c0 = tp.z, c1 = tp.z + tp.w;
    double M = 0.0, S[3] = {0, 0, 0}, lo[3], hi[3], com[3];
    EncBox box;
    box.reset();
    // at most 8 children: every child's record is loaded before the
    // (sequential, octant-order) sums
    const int nc = c1 - c0;
    double4_32a cm[8];
#pragma unroll
    for (int i = 0; i < 8; i++)
        if (i < nc) cm[i] = ldcg_d4(&T.comM[c0 + i]);
#pragma unroll
    for (int i = 0; i < 8; i++) {
        if (i < nc) {
            const double4_32a cl = ldcg_d4(&T.lo[c0 + i]);
            const double4_32a ch = ldcg_d4(&T.hi[c0 + i]);
            M = dadd(M, cm[i].w);
            S[0] = dadd(S[0], dmul(cm[i].w, cm[i].x));
            S[1] = dadd(S[1], dmul(cm[i].w, cm[i].y));
            S[2] = dadd(S[2], dmul(cm[i].w, cm[i].z));
            box.add_box(cl, ch);
        }
    }
    box.get(lo, hi);
    for (int d = 0; d < 3; d++) com[d] = M > 0.0 ? ddiv(S[d], M) : dmul(0.5, dadd(lo[d], hi[d]));
    double q[6];
    if (Q64) {
        double Q[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int i = 0; i < 8; i++) {
            if (i >= nc) break;
            const int c = c0 + i;
            const double *Qc = T.q64 + 6 * (size_t)c;
            double Mc = cm[i].w;
            double dx = dsub(cm[i].x, com[0]), dy = dsub(cm[i].y, com[1]), dz = dsub(cm[i].z, com[2]);
            double d2 = dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz));
            Q[0] = dadd(Q[0], dadd(__ldcg(Qc + 0), dmul(Mc, dsub(dmul(dmul(3.0, dx), dx), d2))));
            Q[1] = dadd(Q[1], dadd(__ldcg(Qc + 1), dmul(Mc, dmul(dmul(3.0, dx), dy))));
            Q[2] = dadd(Q[2], dadd(__ldcg(Qc + 2), dmul(Mc, dmul(dmul(3.0, dx), dz))));
            Q[3] = dadd(Q[3], dadd(__ldcg(Qc + 3), dmul(Mc, dsub(dmul(dmul(3.0, dy), dy), d2))));
            Q[4] = dadd(Q[4], dadd(__ldcg(Qc + 4), dmul(Mc, dmul(dmul(3.0, dy), dz))));
            Q[5] = dadd(Q[5], dadd(__ldcg(Qc + 5), dmul(Mc, dsub(dmul(dmul(3.0, dz), dz), d2))));
        }
        for (int a = 0; a < 6; a++) q[a] = Q[a];
    } else {
        // offsets from the double-single COMs relative to the cluster's frame O (the
        // children's records and the node's own split)
        const double *O = T.cl[T.cid_s[tp.x < T.n ? tp.x : 0]].frame;
        float ch[3], cl[3];
        for (int d = 0; d < 3; d++) ds_split(dsub(com[d], O[d]), ch[d], cl[d]);
        float Q[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int i = 0; i < 8; i++) {
            if (i >= nc) break;
            const int c = c0 + i;
            const float *Qc = T.q32 + 6 * (size_t)c;
            const float4 w0 = __ldcg(&T.wn[wrec(c, 0)]), w3 = __ldcg(&T.wn[wrec(c, 3)]);
            const float Mc = w3.w;
            const float dx = (w0.x - ch[0]) + (w3.x - cl[0]);
            const float dy = (w0.y - ch[1]) + (w3.y - cl[1]);
            const float dz = (w0.z - ch[2]) + (w3.z - cl[2]);
            float d2 = dx * dx + dy * dy + dz * dz;
            Q[0] += __ldcg(Qc + 0) + Mc * (3.f * dx * dx - d2);
            Q[1] += __ldcg(Qc + 1) + Mc * (3.f * dx * dy);
            Q[2] += __ldcg(Qc + 2) + Mc * (3.f * dx * dz);
            Q[3] += __ldcg(Qc + 3) + Mc * (3.f * dy * dy - d2);
            Q[4] += __ldcg(Qc + 4) + Mc * (3.f * dy * dz);
            Q[5] += __ldcg(Qc + 5) + Mc * (3.f * dz * dz - d2);
        }
        for (int a = 0; a < 6; a++) q[a] = Q[a];
    }
    write_node<Q64>(T, k, M, com, lo, hi, q, theta, tp);
}


}  // namespace p3t
