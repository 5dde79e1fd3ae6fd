// Neighbour lists of the constant neighbour radius (Sec. 2.3), handed to the
// irregular (Hermite) side: row i lists every j != i with |x_i - x_j| < r_list,
// by ascending original index; empty rows are legal.
//
// Passes, one warp per walk group:
//   count  walk opening every cell whose box lies within r_list of the group
//          box, test each target against the particles of the opened leaves
//          (skipped for the clusters the mixed far-force walk already counted)
//   scan   counts -> int64 row offsets (look-back scan)
//   fill   the same walk, writing original indices; then each row is sorted
//          (bitonic networks by row-length class, see below).
// The pair test is defined in FP64 as r2 = (dx*dx + dy*dy) + dz*dz < r_list^2.
// It is first taken in FP32 on coordinates relative to the group centre
// (double-single differences); a pair inside the FP32 error band is re-tested
// with the exact FP64 operations, so the lists equal the FP64 definition bit
// for bit.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <type_traits>

#include "p3t_internal.cuh"

namespace p3t {

constexpr int kNbrWarps = 4;
constexpr int kNbrStack = 32 * 22 + 64;
constexpr int kNbrLeafQ = 96;  // flush threshold 64 + up to 32 leaves from one step
constexpr float kUn = 5.9604644775390625e-8f;

struct NbrArgs {
    Tree T;  // list radii and frames come from the tree's cluster table
    int32_t *count;        // per particle, original order
    const int64_t *offs;   // row offsets (fill pass)
    int32_t *idx;          // entries (fill pass)
    long long capacity;
    int skip_counted;      // count pass: skip clusters whose neighbours the walk counted
    unsigned int *ticket;
    int row_cap;           // fill pass in row mode (> 0): only groups with a row longer than its span
    int32_t *rows;         // count pass in row mode: the targets' rows (key order, laid out by
                           // row_off; ids as the far-force walk writes them)
    const int64_t *row_off;
    long long row_entries;
};

struct NbrSmem {
    int stk[kNbrStack];
    int2 lq[kNbrLeafQ];
    int lqo[kNbrLeafQ + 1];
    // staged sources in the pair layout: slots [0, 32) are tested as one chunk of
    // 16 pairs, [32, 64) take what a candidate chunk adds beyond 32
    float4 pp[64];
    int pj[64];  // their positions in key order
};

template <int TPL, bool FILL, bool ROWS = false>
__global__ void __launch_bounds__(kNbrWarps * 32) nbr_kernel(NbrArgs P)
{
    __shared__ NbrSmem sm[kNbrWarps];
    NbrSmem &W = sm[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const Tree &T = P.T;
    Meta *meta = T.meta;
    const int ng = meta->n_groups;
    const int nn = meta->n_nodes;
    // the fill pass runs right before the rows' length classes are counted: it clears
    // their counters (block 0, before any return)
    if (FILL && blockIdx.x == 0 && threadIdx.x < (int)(sizeof(meta->row_class) / sizeof(int)))
        meta->row_class[threadIdx.x] = 0;
    bool allowed = true;
    if (FILL) allowed = P.offs[T.n] <= P.capacity;
    if (FILL && !allowed) {
        if (blockIdx.x == 0 && threadIdx.x == 0) latch_error(meta, P3T_ERR_CAPACITY);
        return;
    }
    // nothing to do: row mode with every row within its room, or a count pass after a
    // walk that counted every cluster
    if (FILL && P.row_cap > 0 && meta->row_over == 0) return;
    if (!FILL && P.skip_counted && meta->uncounted == 0) return;

    while (true) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(P.ticket, 1u);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ng) break;
        const int2 gr = T.grp[g];
        const double4_32a glo = T.glo[g], ghi = T.ghi[g];
        const int cid = T.cid_s[gr.x];  // the group's cluster: frame, root, radius, band
        const Cluster &K = T.cl[cid];
        // counting: clusters the far-force walk already counted are skipped
        if (!FILL && P.skip_counted && K.counted) continue;
        if (FILL && P.row_cap > 0) {  // row mode: every row within its span is written
            bool longer = false;
#pragma unroll
            for (int t = 0; t < TPL; t++) {
                const int s = gr.x + lane + 32 * t;
                if (s < gr.x + gr.y) {
                    long long lo;
                    int cap;
                    row_span(P.row_off, P.row_entries, s, lo, cap);
                    longer |= P.count[T.perm[s]] > cap;
                }
            }
            if (!__any_sync(0xffffffffu, longer)) continue;
        }
        const float Rf = (float)K.frame[3] * 1.0001f;
        const float rl_f = K.rl_f, rl2_f = K.rl2_f;
        const double rl2_d = K.rl2_d;
        const bool filter_ok = Rf > 1e-6f && Rf < 1e12f && rl2_f > 1e-20f && rl2_f < 1e30f;
        const Band bl_band = fp32_band(Rf, rl2_f);  // box-box test against r_list
        // double-single split of c_g - O and the box - O, made once per build
        const float4 g0 = T.gfr[3 * (size_t)g], g1 = T.gfr[3 * (size_t)g + 1],
                     g2 = T.gfr[3 * (size_t)g + 2];
        const float fhx = g0.x, fhy = g0.y, fhz = g0.z, flx = g0.w, fly = g1.x, flz = g1.y;
        const float glx = g1.z, gly = g1.w, glz = g2.x, ghx = g2.y, ghy = g2.z, ghz = g2.w;
        // targets: coordinates relative to c_g, original index `me`; an empty slot sits
        // at 1e30 so that no FP32 test counts it (its rare FP64 path checks si < 0)
        float px[TPL], py[TPL], pz[TPL];
        int si[TPL], cnt[TPL], me[TPL];  // me: the target's row id (as its sources carry)
        int32_t *wp[TPL];  // fill: next entry of the target's row
        // count pass in row mode: neighbours among the staged chunk (bit = slot), the
        // target's scratch row and its entries (an empty slot writes nothing)
        unsigned hit[TPL];
        int32_t *rrow[TPL];
        int rwc[TPL], rcap[TPL];
        float A = 0.f;
#pragma unroll
        for (int t = 0; t < TPL; t++) {
            int s = gr.x + lane + 32 * t;
            cnt[t] = 0;
            wp[t] = P.idx;
            if (ROWS) {
                hit[t] = 0u;
                long long lo = 0;
                rcap[t] = 0;
                if (s < gr.x + gr.y) row_span(P.row_off, P.row_entries, s, lo, rcap[t]);
                rrow[t] = P.rows + lo;
                rwc[t] = s < gr.x + gr.y ? 0 : (1 << 30);
            }
            if (s < gr.x + gr.y) {
                const float4 h = T.ph[s], l = T.pl[s];
                px[t] = (h.x - fhx) + (l.x - flx);
                py[t] = (h.y - fhy) + (l.y - fly);
                pz[t] = (h.z - fhz) + (l.z - flz);
                si[t] = s;
                A = fmaxf(A, fmaxf(fabsf(px[t]), fmaxf(fabsf(py[t]), fabsf(pz[t]))));
                me[t] = T.rid[s];
                if (FILL) wp[t] = P.idx + P.offs[T.perm[s]];
            } else {
                px[t] = py[t] = pz[t] = 1e30f;
                si[t] = -1;
                me[t] = -1;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) A = fmaxf(A, __shfl_xor_sync(0xffffffffu, A, o));
        A *= 1.0001f;
        // band of the pair test (FP32 vs FP64 squared distance), factor ~2 spare:
        // coordinates relative to c_g carry <= 2.01 u |x - c_g| + 8 u^2 R
        const float tpair = kUn * (24.f * rl2_f + 32.f * A * rl_f + 128.f * kUn * Rf * rl_f) +
                            64.f * kUn * kUn * (A + 2.f * rl_f) * (A + 2.f * rl_f);
        const bool pair_filter = filter_ok && A < 1e12f;
        // r2 < in_lo: neighbour; r2 > in_hi: not; otherwise decide in FP64
        const float in_lo = pair_filter ? rl2_f - tpair : -1.f;
        const float in_hi = pair_filter ? rl2_f + tpair : INFINITY;
        // |r2 - in_mid| <= in_rad covers [in_lo, in_hi] with a 2x margin (infinite: filter off)
        const float in_mid = 0.5f * in_lo + 0.5f * in_hi, in_rad = in_hi - in_lo;
        // Source filter: a source whose distance to the group box is r_list or more
        // (with a margin) is nobody's neighbour and is not staged.  The box relative
        // to c_g and the source offsets carry at most ~8 u R error per coordinate
        // (u = 2^-24), so d > r_list (1 + 1e-5) + 32 u R in FP32 implies an exact
        // distance above r_list, far outside the FP64 test's rounding.
        const float bxl = (glx - fhx) - flx, byl = (gly - fhy) - fly, bzl = (glz - fhz) - flz;
        const float bxh = (ghx - fhx) - flx, byh = (ghy - fhy) - fly, bzh = (ghz - fhz) - flz;
        const float thr = rl_f * 1.00001f + 32.f * kUn * Rf;
        const float src_thr2 = pair_filter ? thr * thr : INFINITY;
        float2 NPX[TPL], NPY[TPL], NPZ[TPL];
#pragma unroll
        for (int t = 0; t < TPL; t++)
            NPX[t] = make_float2(-px[t], -px[t]), NPY[t] = make_float2(-py[t], -py[t]),
            NPZ[t] = make_float2(-pz[t], -pz[t]);
        const float4 *pq = W.pp;
        float *pb = reinterpret_cast<float *>(W.pp) + 8 * (lane >> 1) + (lane & 1);
        // one pair of staged sources (pair layout {x0 x1 y0 y1} {z0 z1 o0 o1}, o the
        // original index) against this lane's targets; FP32x2 distances
        auto test_pair = [&](int k, int ns, auto tail) {
            constexpr bool kTail = decltype(tail)::value;
            const float4 b0 = pq[2 * k], b1 = pq[2 * k + 1];
            const float2 X = make_float2(b0.x, b0.y), Y = make_float2(b0.z, b0.w);
            const float2 Z = make_float2(b1.x, b1.y);
            const int o0 = __float_as_int(b1.z), o1 = __float_as_int(b1.w);
#pragma unroll
            for (int t = 0; t < TPL; t++) {
                const float2 dx = __fadd2_rn(X, NPX[t]), dy = __fadd2_rn(Y, NPY[t]), dz = __fadd2_rn(Z, NPZ[t]);
                float2 r2 = __fmul2_rn(dx, dx);
                r2 = __ffma2_rn(dy, dy, r2);
                r2 = __ffma2_rn(dz, dz, r2);
                // (the pair of a target with itself is counted here, r2 = 0, and taken off
                // at the end; the fill pass leaves it out at once)
                bool in0 = r2.x < in_lo && (!FILL || o0 != me[t]);
                bool in1 = r2.y < in_lo && (!FILL || o1 != me[t]);
                const float2 d = __fadd2_rn(r2, make_float2(-in_mid, -in_mid));
                if (fminf(fabsf(d.x), fabsf(d.y)) <= in_rad) {  // an undecided pair (rare)
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        const float r2e = e ? r2.y : r2.x;
                        const int oe = e ? o1 : o0;
                        if (si[t] >= 0 && (!kTail || e == 0 || 2 * k + 1 < ns) && (!FILL || oe != me[t]) &&
                            r2e >= in_lo && r2e <= in_hi) {
                            const double4_32a a = T.sp[si[t]], b = T.sp[W.pj[2 * k + e]];
                            double ex = dsub(b.x, a.x), ey = dsub(b.y, a.y), ez = dsub(b.z, a.z);
                            const bool in = dadd(dadd(dmul(ex, ex), dmul(ey, ey)), dmul(ez, ez)) < rl2_d;
                            if (e)
                                in1 = in;
                            else
                                in0 = in;
                        }
                    }
                }
                if (FILL) {
                    if (in0) *wp[t] = o0;
                    wp[t] += in0;
                    if (in1) *wp[t] = o1;
                    wp[t] += in1;
                } else if (ROWS) {
                    hit[t] |= ((unsigned)in0 | ((unsigned)in1 << 1)) << (2 * k);
                } else {
                    cnt[t] += (int)in0 + (int)in1;
                }
            }
        };

        int sp = 1;
        if (lane == 0) W.stk[0] = pack_range(cid, 1);
        __syncwarp();
        // the staged sources [0, ns) against the targets (ns <= 32; an odd ns is padded
        // by the caller), then, in row mode, their neighbours appended to the rows
        auto test_chunk = [&](int ns) {
            const int nfull = ns >> 1;
#pragma unroll 2
            for (int k = 0; k < nfull; k++) test_pair(k, ns, std::false_type());
            if (ns & 1) test_pair(nfull, ns, std::true_type());
            if (ROWS) {  // count the chunk's neighbours and append them to the rows
                const int *po = reinterpret_cast<const int *>(W.pp);
#pragma unroll
                for (int t = 0; t < TPL; t++) {
                    unsigned h = hit[t];
                    hit[t] = 0u;
                    cnt[t] += __popc(h);
                    // two hits an iteration, their loads issued together; the target
                    // itself is left out
                    while (h) {
                        const int b0 = __ffs(h) - 1;
                        h &= h - 1u;
                        const bool two = h != 0u;
                        const int b1 = two ? __ffs(h) - 1 : b0;
                        h &= h - 1u;
                        const int o0 = po[8 * (b0 >> 1) + 6 + (b0 & 1)], o1 = po[8 * (b1 >> 1) + 6 + (b1 & 1)];
                        if (o0 != me[t]) {
                            if (rwc[t] < rcap[t]) rrow[t][rwc[t]] = o0;
                            rwc[t]++;
                        }
                        if (two && o1 != me[t]) {
                            if (rwc[t] < rcap[t]) rrow[t][rwc[t]] = o1;
                            rwc[t]++;
                        }
                    }
                }
            }
            __syncwarp();
        };
        int lqn = 0, lqp = 0;
        int nst = 0;  // staged sources waiting for a full chunk (< 32 between chunks)
        int iters = 0;  // a valid walk pops every node at most once
        while (true) {
            if (++iters > nn + 2) {
                if (lane == 0) latch_error(meta, P3T_ERR_INTERNAL);
                break;
            }
            if (sp > 0) {
                const int node = pop_batch(W.stk, sp);
                bool open = false, is_leaf = false;
                int cinfo = 0, ccount = 0;
                if (node >= 0) {
                    const auto rec = wrec_at(T.wn, node);
                    const float4 b = rec[1], cc = rec[2];
                    cinfo = __float_as_int(b.w);
                    ccount = __float_as_int(cc.w);
                    is_leaf = cinfo < 0;
                    int bb = 2;
                    if (filter_ok) {
                        float ux = fmaxf(fmaxf(b.x - ghx, glx - cc.x), 0.f);
                        float uy = fmaxf(fmaxf(b.y - ghy, gly - cc.y), 0.f);
                        float uz = fmaxf(fmaxf(b.z - ghz, glz - cc.z), 0.f);
                        float e2 = ux * ux + uy * uy + uz * uz;
                        const float db = e2 - rl2_f;
                        bb = fabsf(db) > fmaf(bl_band.a, e2, bl_band.b) ? (db < 0.f ? 1 : 0) : 2;
                    }
                    if (bb == 2) {
                        bb = dist2_box_box(glo, ghi, T.lo[node], T.hi[node]) < rl2_d;
                        if (filter_ok) atomicAdd((unsigned long long *)&meta->fallback_tests, 1ULL);
                    }
                    open = bb == 1;
                }
                const bool open_int = open && !is_leaf;
                const bool open_leaf = open && is_leaf;
                const bool bad = (open_int && (ccount < 1 || ccount > 8 || cinfo + ccount > nn)) ||
                                 (open_leaf && (ccount < 1 || -1 - cinfo + ccount > T.n_src));
                if (__any_sync(0xffffffffu, bad)) {
                    if (lane == 0) latch_error(meta, P3T_ERR_INTERNAL);
                    break;
                }
                const unsigned pm = __ballot_sync(0xffffffffu, open_int);
                const int npush = __popc(pm);
                if (sp + npush > kNbrStack) {
                    if (lane == 0) latch_error(meta, P3T_ERR_CAPACITY);
                    sp = 0;
                    break;
                }
                if (open_int) W.stk[sp + __popc(pm >> lane >> 1)] = pack_range(cinfo, ccount);
                sp += npush;
                const unsigned lm = __ballot_sync(0xffffffffu, open_leaf);
                if (open_leaf) W.lq[lqn + __popc(lm & lt)] = make_int2(-1 - cinfo, ccount);
                lqn += __popc(lm);
                lqp += (int)__reduce_add_sync(0xffffffffu, open_leaf ? (unsigned)ccount : 0u);
                if (lqp < 64 && sp > 0) continue;
            }
            if (lqp > 0) {
                // ---- stage the queued leaves' particles that pass the source filter
                __syncwarp();
                {
                    int carry = 0;
                    for (int b0 = 0; b0 < lqn; b0 += 32) {
                        int i = b0 + lane;
                        int v = i < lqn ? W.lq[i].y : 0;
                        int inc = warp_incl_scan(v);
                        if (i < lqn) W.lqo[i] = carry + inc - v;
                        carry += __shfl_sync(0xffffffffu, inc, 31);
                    }
                }
                __syncwarp();
                for (int c0 = 0; c0 < lqp; c0 += 32) {
                    const int pos = c0 + lane;
                    bool keep = false;
                    float rx = 0.f, ry = 0.f, rz = 0.f;
                    int j = 0;
                    if (pos < lqp) {
                        int lo = 0, hi = lqn;
                        while (hi - lo > 1) {
                            int mid = (lo + hi) >> 1;
                            if (W.lqo[mid] <= pos)
                                lo = mid;
                            else
                                hi = mid;
                        }
                        j = W.lq[lo].x + (pos - W.lqo[lo]);
                        const float4 h = T.ph[j], l = T.pl[j];
                        rx = (h.x - fhx) + (l.x - flx);
                        ry = (h.y - fhy) + (l.y - fly);
                        rz = (h.z - fhz) + (l.z - flz);
                        const float tx = fmaxf(fmaxf(bxl - rx, rx - bxh), 0.f);
                        const float ty = fmaxf(fmaxf(byl - ry, ry - byh), 0.f);
                        const float tz = fmaxf(fmaxf(bzl - rz, rz - bzh), 0.f);
                        keep = !(tx * tx + ty * ty + tz * tz > src_thr2);
                    }
                    const unsigned km = __ballot_sync(0xffffffffu, keep);
                    if (keep) {
                        const int sl = nst + __popc(km & lt);  // < 64
                        float *b = reinterpret_cast<float *>(W.pp) + 8 * (sl >> 1) + (sl & 1);
                        b[0] = rx, b[2] = ry, b[4] = rz, b[6] = __int_as_float(T.rid[j]);
                        W.pj[sl] = j;
                    }
                    nst += __popc(km);
                    if (nst >= 32) {
                        __syncwarp();
                        test_chunk(32);
                        // the staged sources beyond the chunk move down to slots [0, nst - 32)
                        const int rem = nst - 32;
                        if (lane < rem) {
                            const float *src = reinterpret_cast<const float *>(W.pp) + 8 * ((32 + lane) >> 1) + (lane & 1);
                            float *dst = reinterpret_cast<float *>(W.pp) + 8 * (lane >> 1) + (lane & 1);
                            const float v0 = src[0], v1 = src[2], v2 = src[4], v3 = src[6];
                            const int pjv = W.pj[32 + lane];
                            dst[0] = v0, dst[2] = v1, dst[4] = v2, dst[6] = v3;
                            W.pj[lane] = pjv;
                        }
                        __syncwarp();
                        nst = rem;
                    }
                }
                lqn = lqp = 0;
            }
            if (sp == 0) break;
        }
        if (nst > 0) {  // the last staged sources
            __syncwarp();
            if ((nst & 1) && lane == 0) {  // pad: far away, never a neighbour
                float *b = reinterpret_cast<float *>(W.pp) + 8 * (nst >> 1);
                b[1] = b[3] = b[5] = 1e30f;
                b[7] = __int_as_float(-1);
            }
            __syncwarp();
            test_chunk(nst);
        }
        if (!FILL) {
            // each target met itself once (its leaf is opened and it passes the source
            // filter) and counted itself iff 0 < r_list^2
            const int self = rl2_d > 0.0 ? 1 : 0;
#pragma unroll
            for (int t = 0; t < TPL; t++)
                if (si[t] >= 0) P.count[T.perm[si[t]]] = cnt[t] - self;
        }
        if (ROWS) {
#pragma unroll
            for (int t = 0; t < TPL; t++)
                if (si[t] >= 0 && rwc[t] > rcap[t]) meta->row_over = 1;
        }
        __syncwarp();
    }
}

// ---- per-row ascending sort --------------------------------------------------
// Rows are distinct indices in [0, n), so the sorted row is unique and any
// correct sort writes the same bytes.  The rows are first binned by length into
// per-class lists (two cheap passes over the row offsets), then each class is
// sorted by its own launch, one warp per listed row (one thread for the
// shortest), so that no launch scans the rows of other classes and only one
// class's code is resident in the instruction cache:
//   [1, 4]        a 5-comparator network in one thread's registers (a row of
//                 one entry is only copied, from the walk's scratch in row mode)
//   (4, 1024]     bitonic network in registers, K = 1, 2, 4, 8, 16, 32 entries
//                 per lane: up to 128 in the strided layout (element e = 32 r +
//                 lane in register r; partners 32 apart or more are in the same
//                 lane, closer ones are exchanged by shuffles), above in the
//                 transposed layout (warp_bitonic_row_t)
//   (1024, 2048]  loop-based bitonic network (below) in shared memory
//   > 2048        the same network in global memory.
// The loop network puts the smaller value at the lower index in every
// compare-exchange (each merge stage starts by comparing mirrored positions of a
// block), so a row of any length sorts in place as if padded with +infinity: a
// pair whose upper index is past the end never moves.  (An LSD radix sort in
// shared memory, ranks from ballots, was slower than these networks for every
// class of the 10^6-particle Plummer workload.)
constexpr int kRowClasses = 9;
// class c holds the rows with kClassLen[c] < len <= kClassLen[c + 1]
__constant__ int kClassLenDev[kRowClasses + 1] = {0, 4, 32, 64, 128, 256, 512, 1024, 2048, INT_MAX};
constexpr int kClassLen[kRowClasses + 1] = {0, 4, 32, 64, 128, 256, 512, 1024, 2048, INT_MAX};
static_assert(2 * kRowClasses <= (int)(sizeof(Meta::row_class) / sizeof(int)), "class counters and cursors");
constexpr int kSortWarps = 4;
constexpr int kRowLoadBatch = 8;  // global loads a lane issues before storing any
// bit c set: class c uses the transposed register network (faster for
// (128, 1024], slower for (64, 128] on the 10^6-particle Plummer rows)
constexpr unsigned kTransposed = (1u << 4) | (1u << 5) | (1u << 6);

__device__ __forceinline__ int row_class(int len)
{
    int c = 0;
#pragma unroll
    for (int k = 1; k < kRowClasses; k++) c += len > kClassLenDev[k];
    return len > 0 ? c : -1;
}

// counts of the classes -> Meta.row_class[0 .. 7]
__global__ void row_class_count_kernel(int n, const int64_t *__restrict__ offs, long long capacity,
                                       Meta *meta)
{
    pdl_wait();
    __shared__ int cnt[kRowClasses];
    if (threadIdx.x < kRowClasses) cnt[threadIdx.x] = 0;
    __syncthreads();
    if (offs[n] <= capacity) {
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
            const int c = row_class((int)(offs[i + 1] - offs[i]));
            if (c >= 0) atomicAdd(&cnt[c], 1);
        }
    }
    __syncthreads();
    if (threadIdx.x < kRowClasses && cnt[threadIdx.x])
        atomicAdd(&meta->row_class[threadIdx.x], cnt[threadIdx.x]);
}

// row ids -> list, class c at [sum of the counts below c, + count c) (in any
// order inside a class); cursors in Meta.row_class[8 .. 15]
__global__ void row_class_fill_kernel(int n, const int64_t *__restrict__ offs, long long capacity,
                                      Meta *meta, int32_t *list)
{
    pdl_wait();
    __shared__ int cnt[kRowClasses], base[kRowClasses];
    if (offs[n] > capacity) return;
    const int stride = gridDim.x * blockDim.x;
    for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
        if (threadIdx.x < kRowClasses) cnt[threadIdx.x] = 0;
        __syncthreads();
        const int i = i0 + threadIdx.x;
        const int c = i < n ? row_class((int)(offs[i + 1] - offs[i])) : -1;
        const int rank = c >= 0 ? atomicAdd(&cnt[c], 1) : 0;
        __syncthreads();
        if (threadIdx.x < kRowClasses) {
            int start = 0;
            for (int q = 0; q < (int)threadIdx.x; q++) start += meta->row_class[q];
            base[threadIdx.x] =
                start + (cnt[threadIdx.x] ? atomicAdd(&meta->row_class[kRowClasses + threadIdx.x],
                                                      cnt[threadIdx.x])
                                          : 0);
        }
        __syncthreads();
        if (c >= 0) list[base[c] + rank] = i;
        __syncthreads();
    }
}

// Where the entries of row i come from: the row itself in idx (filled by the
// fill pass), or, in row mode, the far-force walk's scratch row of the target
// (cap entries per particle in key order, holding original indices) when the
// row has at most cap entries.
struct RowSrc {
    const int32_t *rows;  // null: every row is in idx
    const int32_t *inv;   // original -> key order
    const int64_t *row_off;
    long long entries;
};

// Where one row's entries are read from: its scratch row, else its place in idx.
struct RowLoad {
    const int32_t *sr;  // scratch row, or null
    const int32_t *row;
    __device__ __forceinline__ const int32_t *base() const { return sr ? sr : row; }
};

// The rows of class C, one warp each: f(row pointer in idx, length, loader).
template <int C, typename F>
__device__ __forceinline__ void for_class_rows(const Meta *meta, const int32_t *list,
                                               const int64_t *offs, int32_t *idx, RowSrc src,
                                               F &&f)
{
    int start = 0;
#pragma unroll
    for (int q = 0; q < C; q++) start += meta->row_class[q];
    const int count = meta->row_class[C];
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < count;
         k += (gridDim.x * blockDim.x) >> 5) {
        const int i = list[start + k];
        const long long o = offs[i];
        const int len = (int)(offs[i + 1] - o);
        RowLoad ld;
        ld.sr = nullptr;
        if (src.rows) {
            long long lo;
            int cap;
            row_span(src.row_off, src.entries, src.inv[i], lo, cap);
            if (len <= cap) ld.sr = src.rows + lo;
        }
        ld.row = idx + o;
        f(idx + o, len, ld);
        __syncwarp();
    }
}

template <int K>
__device__ __forceinline__ void warp_bitonic_row(int32_t *row, int len, const RowLoad &ld)
{
    const int lane = threadIdx.x & 31;
    const int32_t *src = ld.base();
    int v[K];
#pragma unroll
    for (int r = 0; r < K; r++) {
        int e = 32 * r + lane;
        v[r] = e < len ? src[e] : INT_MAX;
    }
#pragma unroll
    for (int k = 2; k <= 32 * K; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int rj = j >> 5;
#pragma unroll
                for (int r = 0; r < K; r++) {
                    const int r2 = r ^ rj;
                    if (r2 > r) {
                        const bool up = ((32 * r + lane) & k) == 0;
                        const int a = v[r], bb = v[r2];
                        const int lo = min(a, bb), hi = max(a, bb);
                        v[r] = up ? lo : hi;
                        v[r2] = up ? hi : lo;
                    }
                }
            } else {
                const bool lower = (lane & j) == 0;
#pragma unroll
                for (int r = 0; r < K; r++) {
                    const bool up = ((32 * r + lane) & k) == 0;
                    const int p = __shfl_xor_sync(0xffffffffu, v[r], j);
                    v[r] = (lower == up) ? min(v[r], p) : max(v[r], p);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < K; r++) {
        int e = 32 * r + lane;
        if (e < len) row[e] = v[r];
    }
}

// The same network in the transposed layout: lane holds the K consecutive
// elements e = K lane + r, so the stages with partners less than K apart are
// compare-exchanges between registers and only the wider ones need shuffles.
// Descending blocks are handled by complementing their values (~v reverses the
// order of int32), so that every compare-exchange is ascending; the complement
// pattern changes once per merge level.  The row passes through shared memory
// (sb: 32 K + K words, index e + e / 32 keeps both access patterns free of bank
// conflicts) so that the global loads and stores stay coalesced; all K loads of
// a lane are issued before the first store.
template <int K>
__device__ __forceinline__ void warp_bitonic_row_t(int32_t *row, int len, int32_t *sb,
                                                   const RowLoad &ld)
{
    constexpr int N = 32 * K;
    const int lane = threadIdx.x & 31;
    const int32_t *src = ld.base();
    int v[K];
#pragma unroll
    for (int r = 0; r < K; r++) {
        const int e = 32 * r + lane;
        v[r] = e < len ? src[e] : INT_MAX;
    }
#pragma unroll
    for (int r = 0; r < K; r++) {
        const int e = 32 * r + lane;
        sb[e + (e >> 5)] = v[r];
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < K; r++) {
        const int e = K * lane + r;
        v[r] = sb[e + (e >> 5)] ^ ((e & 2) ? -1 : 0);
    }
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
        if (k > 2) {
#pragma unroll
            for (int r = 0; r < K; r++) {
                const int e = K * lane + r;
                v[r] ^= ((e & k) ? -1 : 0) ^ ((e & (k >> 1)) ? -1 : 0);
            }
        }
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < K) {
#pragma unroll
                for (int r = 0; r < K; r++) {
                    const int r2 = r ^ j;
                    if (r2 > r) {
                        const int a = v[r], b = v[r2];
                        v[r] = min(a, b);
                        v[r2] = max(a, b);
                    }
                }
            } else {
                const int lj = j / K;
                const bool lower = (lane & lj) == 0;
#pragma unroll
                for (int r = 0; r < K; r++) {
                    const int p = __shfl_xor_sync(0xffffffffu, v[r], lj);
                    v[r] = lower ? min(v[r], p) : max(v[r], p);
                }
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < K; r++) {
        const int e = K * lane + r;
        sb[e + (e >> 5)] = v[r];  // level N has no descending block: v is the value
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < K; r++) {
        const int e = 32 * r + lane;
        if (e < len) row[e] = sb[e + (e >> 5)];
    }
}

// ascending compare-exchange of a[i] and a[h] (i < h), skipped past the end
__device__ __forceinline__ void cmpx(int32_t *a, int i, int h, int len)
{
    if (h < len) {
        const int32_t x = a[i], y = a[h];
        if (y < x) {
            a[i] = y;
            a[h] = x;
        }
    }
}

// Warp-cooperative sort of a[0 .. len) (shared or global memory).
__device__ void warp_sort_mem(int32_t *a, int len)
{
    const int lane = threadIdx.x & 31;
    int P = 1;
    while (P < len) P <<= 1;
    const int half = P >> 1;
    for (int k = 2; k <= P; k <<= 1) {
        const int hk = k >> 1;
        for (int i = lane; i < half; i += 32) {  // mirrored pairs within blocks of k
            const int lo = ((i & ~(hk - 1)) << 1) | (i & (hk - 1));
            cmpx(a, lo, lo ^ (k - 1), len);
        }
        __syncwarp();
        for (int j = k >> 2; j > 0; j >>= 1) {
            for (int i = lane; i < half; i += 32) {
                const int lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
                cmpx(a, lo, lo | j, len);
            }
            __syncwarp();
        }
    }
}

// ascending compare-exchange of two registers
__device__ __forceinline__ void cx2(int &a, int &b)
{
    const int lo = min(a, b), hi = max(a, b);
    a = lo, b = hi;
}

// rows of class C (at most 4 entries), one thread each: a 5-comparator network
template <int C>
__global__ void __launch_bounds__(kSortWarps * 32)
    row_sort_tiny_kernel(const Meta *meta, const int32_t *list, const int64_t *__restrict__ offs,
                         int32_t *idx, RowSrc src)
{
    pdl_wait();
    static_assert(kClassLen[C + 1] == 4, "four entries per row");
    int start = 0;
#pragma unroll
    for (int q = 0; q < C; q++) start += meta->row_class[q];
    const int count = meta->row_class[C];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const int i = list[start + k];
        const long long o = offs[i];
        const int len = (int)(offs[i + 1] - o);
        const int32_t *s = idx + o;
        if (src.rows) {
            long long lo;
            int cap;
            row_span(src.row_off, src.entries, src.inv[i], lo, cap);
            if (len <= cap) s = src.rows + lo;
        }
        int v0 = s[0], v1 = len > 1 ? s[1] : INT_MAX, v2 = len > 2 ? s[2] : INT_MAX, v3 = len > 3 ? s[3] : INT_MAX;
        cx2(v0, v1);
        cx2(v2, v3);
        cx2(v0, v2);
        cx2(v1, v3);
        cx2(v1, v2);
        int32_t *row = idx + o;
        row[0] = v0;
        if (len > 1) row[1] = v1;
        if (len > 2) row[2] = v2;
        if (len > 3) row[3] = v3;
    }
}

template <int C, int K>
__global__ void __launch_bounds__(kSortWarps * 32)
    row_sort_reg_kernel(const Meta *meta, const int32_t *list, const int64_t *__restrict__ offs,
                        int32_t *idx, RowSrc src)
{
    pdl_wait();
    for_class_rows<C>(meta, list, offs, idx, src, [](int32_t *row, int len, const RowLoad &ld) {
        warp_bitonic_row<K>(row, len, ld);
    });
}

template <int C, int K>
__global__ void __launch_bounds__(kSortWarps * 32)
    row_sort_tr_kernel(const Meta *meta, const int32_t *list, const int64_t *__restrict__ offs,
                       int32_t *idx, RowSrc src)
{
    pdl_wait();
    __shared__ int32_t sbuf[kSortWarps][33 * K];
    int32_t *sb = sbuf[threadIdx.x >> 5];
    for_class_rows<C>(meta, list, offs, idx, src, [&](int32_t *row, int len, const RowLoad &ld) {
        warp_bitonic_row_t<K>(row, len, sb, ld);
    });
}

// rows of class C sorted by the loop network in shared memory
template <int C>
__global__ void __launch_bounds__(kSortWarps * 32)
    row_sort_smem_kernel(const Meta *meta, const int32_t *list, const int64_t *__restrict__ offs,
                         int32_t *idx, RowSrc src)
{
    pdl_wait();
    __shared__ int32_t sbuf[kSortWarps][kClassLen[C + 1]];
    const int lane = threadIdx.x & 31;
    int32_t *sb = sbuf[threadIdx.x >> 5];
    for_class_rows<C>(meta, list, offs, idx, src, [&](int32_t *row, int len, const RowLoad &ld) {
        const int32_t *s = ld.base();
        for (int e0 = 0; e0 < len; e0 += 32 * kRowLoadBatch) {  // loads in flight together
            int t[kRowLoadBatch];
#pragma unroll
            for (int r = 0; r < kRowLoadBatch; r++) {
                const int e = e0 + 32 * r + lane;
                t[r] = e < len ? s[e] : 0;
            }
#pragma unroll
            for (int r = 0; r < kRowLoadBatch; r++) {
                const int e = e0 + 32 * r + lane;
                if (e < len) sb[e] = t[r];
            }
        }
        __syncwarp();
        warp_sort_mem(sb, len);
        for (int e = lane; e < len; e += 32) row[e] = sb[e];
    });
}

// rows of class C sorted by the loop network in global memory (a scratch row is
// first copied into place)
template <int C>
__global__ void __launch_bounds__(kSortWarps * 32)
    row_sort_global_kernel(const Meta *meta, const int32_t *list, const int64_t *__restrict__ offs,
                           int32_t *idx, RowSrc src)
{
    pdl_wait();
    const int lane = threadIdx.x & 31;
    for_class_rows<C>(meta, list, offs, idx, src, [&](int32_t *row, int len, const RowLoad &ld) {
        if (ld.sr) {
            for (int e = lane; e < len; e += 32) row[e] = ld.sr[e];
            __syncwarp();
        }
        warp_sort_mem(row, len);
    });
}

template <typename Kern>
static int launch_sort(p3t_ctx *c, Kern kern, const int64_t *offsets, int32_t *idx, RowSrc src,
                       cudaStream_t st)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSortWarps * 32, 0) !=
            cudaSuccess ||
        per_sm < 1)
        return P3T_ERR_CUDA;
    if (launch_pdl(kern, dim3(per_sm * c->sm_count), dim3(kSortWarps * 32), st, (const Meta *)c->meta,
                   (const int32_t *)c->row_list, offsets, idx, src) != cudaSuccess)
        return P3T_ERR_CUDA;
    return check_launch(c);
}

// Sorts every row of the filled lists (offsets[n] <= capacity; otherwise nothing),
// reading rows of at most src.cap entries from the walk's scratch in row mode.
static int sort_rows(p3t_ctx *c, const int64_t *offsets, int32_t *idx, long long capacity,
                     RowSrc src)
{
    cudaStream_t s = c->stream;
    const int n = c->n;
    // (Meta.row_class was cleared by the fill pass launched just before)
    const int grid = (int)std::min<long long>(((long long)n + 255) / 256, 4LL * c->sm_count);
    if (launch_pdl(row_class_count_kernel, dim3(grid), dim3(256), s, n, offsets, capacity, c->meta) != cudaSuccess ||
        launch_pdl(row_class_fill_kernel, dim3(grid), dim3(256), s, n, offsets, capacity, c->meta, c->row_list) !=
            cudaSuccess)
        return P3T_ERR_CUDA;
    int e = check_launch(c);
    if (e) return e;
    // the length classes sort disjoint rows: the longest class on the context's stream,
    // the other classes on two side streams beside it (joined before returning, also
    // after a failed launch, so that a captured stream is always joined)
    const bool fork = c->side_stream != nullptr;
    const cudaStream_t s1 = fork ? c->side_stream : s;
    const cudaStream_t s2 = c->side_stream2 ? c->side_stream2 : s1;
    if (fork && (cudaEventRecord(c->fork_ev, s) != cudaSuccess || cudaStreamWaitEvent(s1, c->fork_ev, 0) != cudaSuccess ||
                 cudaStreamWaitEvent(s2, c->fork_ev, 0) != cudaSuccess))
        return P3T_ERR_CUDA;
    auto run = [&]() -> int {
        int e2;
        if ((e2 = launch_sort(c, row_sort_tiny_kernel<0>, offsets, idx, src, s2))) return e2;
        if ((e2 = launch_sort(c, row_sort_reg_kernel<1, 1>, offsets, idx, src, s2))) return e2;
        if ((e2 = launch_sort(c, row_sort_reg_kernel<2, 2>, offsets, idx, src, s2))) return e2;
        if (kTransposed & (1u << 3))
            e2 = launch_sort(c, row_sort_tr_kernel<3, 4>, offsets, idx, src, s2);
        else
            e2 = launch_sort(c, row_sort_reg_kernel<3, 4>, offsets, idx, src, s2);
        if (e2) return e2;
        if (n > kClassLen[4] + 1) {  // longer rows need more than 128 distinct indices
            if (kTransposed & (1u << 4))
                e2 = launch_sort(c, row_sort_tr_kernel<4, 8>, offsets, idx, src, s1);
            else
                e2 = launch_sort(c, row_sort_reg_kernel<4, 8>, offsets, idx, src, s1);
            if (e2) return e2;
            if (kTransposed & (1u << 5))
                e2 = launch_sort(c, row_sort_tr_kernel<5, 16>, offsets, idx, src, s);
            else
                e2 = launch_sort(c, row_sort_reg_kernel<5, 16>, offsets, idx, src, s);
            if (e2) return e2;
            if ((e2 = launch_sort(c, row_sort_tr_kernel<6, 32>, offsets, idx, src, s1))) return e2;
            if ((e2 = launch_sort(c, row_sort_smem_kernel<7>, offsets, idx, src, s1))) return e2;
            if ((e2 = launch_sort(c, row_sort_global_kernel<8>, offsets, idx, src, s1))) return e2;
        }
        return P3T_OK;
    };
    e = run();
    if (fork) {
        const bool ok = cudaEventRecord(c->join_ev, s1) == cudaSuccess && cudaStreamWaitEvent(s, c->join_ev, 0) == cudaSuccess &&
                        (s2 == s1 || (cudaEventRecord(c->join_ev2, s2) == cudaSuccess &&
                                      cudaStreamWaitEvent(s, c->join_ev2, 0) == cudaSuccess));
        if (!ok && !e) e = P3T_ERR_CUDA;
    }
    if (e) return e;
    return P3T_OK;
}

template <int TPL, bool FILL, bool ROWS = false>
static int launch_nbr(p3t_ctx *c, const NbrArgs &a)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nbr_kernel<TPL, FILL, ROWS>,
                                                      kNbrWarps * 32, 0) != cudaSuccess ||
        per_sm < 1)
        return P3T_ERR_CUDA;
    if (cudaMemsetAsync(a.ticket, 0, sizeof(unsigned int), c->stream) != cudaSuccess)
        return P3T_ERR_CUDA;
    nbr_kernel<TPL, FILL, ROWS><<<per_sm * c->sm_count, kNbrWarps * 32, 0, c->stream>>>(a);
    return check_launch(c);
}

template <bool FILL>
static int dispatch_nbr(p3t_ctx *c, const NbrArgs &a)
{
    const int G = c->prm.group_size;
    if (G <= 32) return launch_nbr<1, FILL>(c, a);
    if (G <= 64) return launch_nbr<2, FILL>(c, a);
    return launch_nbr<4, FILL>(c, a);
}

// Row mode: the pass that counts the neighbours (the far-force walk, or the
// count pass when the lists come first) also writes each neighbour into the
// target's row of a scratch, so that the lists need no fill walk.  Each tree's
// rows are laid out from the last counts of the same particles (row_caps_kernel:
// c + c/8 + 8 entries for a particle that had c neighbours), and the synchronous
// lists size the scratch once: the entries of such a layout of their counts plus
// a sixteenth (about 1.3 times the lists' entries at 100 neighbours a particle),
// so a row overflows only when its particle gained more than an eighth of its
// neighbours and 8 since the counts were taken (and the rows at the end when the
// layout as a whole grew by more than a sixteenth).  Such a row is filled by
// the fill pass for its group.  A failed allocation leaves row mode off.
// Reallocating drops the rows of the current tree (rows_valid), which the fill
// pass then rebuilds.
static void size_row_scratch(p3t_ctx *c, long long total)
{
    // (rows need one target per lane in the walk: G <= threads per group)
    if (c->built_precision != P3T_FP32_MIXED || c->prm.group_size > c->prm.threads_per_group || c->n <= 0)
        return;
    const long long layout = total + total / 8 + 8LL * c->n;
    const size_t need = (size_t)((layout + layout / 16 + 4095) / 4096 * 4096);
    const long long cap = std::max(1LL, (long long)(need / (size_t)c->n));
    if (need > c->row_scratch_entries) {
        cudaStreamSynchronize(c->stream);
        if (c->row_scratch) cudaFree(c->row_scratch);
        c->row_scratch = nullptr;
        c->row_scratch_entries = 0;
        c->rows_valid = 0;
        c->row_cap = 0;
        c->gen++;  // graphs captured with the old scratch refuse to launch
        void *p = nullptr;
        if (cudaMalloc(&p, need * sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        c->row_scratch = (int32_t *)p;
        c->row_scratch_entries = need;
    }
    c->row_cap = (int)std::min(cap, (long long)INT32_MAX);
}

// capacity of each target's row (key order) from the last count of its particle
__global__ void __launch_bounds__(256)
    row_caps_kernel(int n, const int32_t *__restrict__ perm, const int32_t *__restrict__ count,
                    int32_t *__restrict__ cap, int *row_over, unsigned long long *scan_status, int scan_words,
                    unsigned int *scan_ticket)
{
    pdl_wait();
    if (blockIdx.x == 0) {  // the layout's overflow flag and its scan's state
        clear_scan_state(scan_status, scan_words, scan_ticket);
        if (threadIdx.x == 0) *row_over = 0;
    }
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int cnt = count[perm[s]];
    cap[s] = cnt < (1 << 24) ? cnt + (cnt >> 3) + 8 : (1 << 24);
}

// equal rows of `cap` entries (no counts of these particles yet)
__global__ void __launch_bounds__(256) row_uniform_kernel(int n, long long cap, int64_t *__restrict__ row_off,
                                                          int *row_over)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0) *row_over = 0;
    if (s <= n) row_off[s] = (long long)s * cap;
}

// Lay out the current tree's rows in the scratch (row_off) when row mode is on:
// from the last counts of these particles when known, else in equal rows (a
// context that steps different particle sets, such as a serving slot's batches);
// returns whether the rows can be written.
int prepare_rows(p3t_ctx *c)
{
    c->rows_cap_used = 0;
    if (c->row_cap <= 0 || !c->row_scratch || c->n <= 0) return 0;
    const int n = c->n;
    if (c->counts_n == n) {
        if (launch_pdl(row_caps_kernel, dim3((n + 255) / 256), dim3(256), c->stream, n, (const int32_t *)c->tree.perm,
                       (const int32_t *)c->nbr_count, c->row_list, &c->meta->row_over, c->scan_status,
                       scan_status_words(n), &c->meta->tickets[26]) != cudaSuccess)
            return 0;
        if (scan_excl_i32_to_i64_cleared(c->row_list, c->row_off, n, c->row_off + n, c->scan_status,
                                         &c->meta->tickets[26], c->meta, c->stream) != P3T_OK)
            return 0;
    } else {
        const long long cap = (long long)(c->row_scratch_entries / (size_t)n);
        if (cap < 1) return 0;
        row_uniform_kernel<<<(n + 256) / 256, 256, 0, c->stream>>>(n, cap, c->row_off, &c->meta->row_over);
    }
    c->rows_cap_used = 1;
    return 1;
}

int neighbours(p3t_ctx *c, int64_t *offsets, int32_t *idx, long long capacity, int64_t *total_dev,
               bool sync, int64_t *total_host)
{
    cudaStream_t s = c->stream;
    const int n = c->n;
    NbrArgs a;
    a.T = c->tree;
    a.count = c->nbr_count;
    a.offs = offsets;
    a.idx = idx;
    a.capacity = capacity;
    a.ticket = &c->meta->tickets[23];
    a.row_cap = 0;
    a.rows = nullptr;
    a.row_off = c->row_off;
    a.row_entries = (long long)c->row_scratch_entries;
    int e;
    a.skip_counted = c->walk_counted;
    if (!c->counts_valid) {  // the far-force walk did not count every cluster
        // row mode in the count pass: when the walk counted nothing (the lists come
        // before the far force), or wrote the rows of what it counted
        const bool can = c->prm.group_size <= 32 && c->built_precision == P3T_FP32_MIXED;
        const bool rows = can && (c->walk_counted ? c->rows_valid != 0 : prepare_rows(c) != 0);
        if (rows) {
            a.rows = c->row_scratch;
            e = launch_nbr<1, false, true>(c, a);
        } else {
            e = dispatch_nbr<false>(c, a);
        }
        if (e) return e;
        c->counts_valid = 1;
        c->counts_n = n;
        c->rows_valid = rows;
    }
    e = scan_excl_i32_to_i64(c->nbr_count, offsets, n, offsets + n, c->scan_status,
                             &c->meta->tickets[29], c->meta, s);
    if (e) return e;
    if (sync) {
        int64_t tot = 0;
        if (cudaMemcpyAsync(&tot, offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return P3T_ERR_CUDA;
        *total_host = tot;
        size_row_scratch(c, tot);
        int err = 0;
        if (cudaMemcpy(&err, &c->meta->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return P3T_ERR_CUDA;
        if (err) {
            int zero = 0;
            cudaMemcpy(&c->meta->err, &zero, sizeof(int), cudaMemcpyHostToDevice);
            return err;
        }
        if (tot > capacity) return P3T_ERR_CAPACITY;
    } else {
        if (cudaMemcpyAsync(total_dev, offsets + n, sizeof(int64_t), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
            return P3T_ERR_CUDA;
    }
    if (capacity == 0) return P3T_OK;
    RowSrc src{nullptr, nullptr, nullptr, 0};
    if (c->rows_valid) {  // the rows were written: fill only groups with a longer row
        a.row_cap = 1;
        src = RowSrc{c->row_scratch, c->tree.inv, c->row_off, (long long)c->row_scratch_entries};
    }
    e = dispatch_nbr<true>(c, a);
    if (e) return e;
    return sort_rows(c, offsets, idx, capacity, src);
}

}  // namespace p3t
