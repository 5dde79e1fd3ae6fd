/*
 * p3t_oracle.c -- plain, slow FP64 CPU oracle of the distant-force path of the
 * P3T scheme (arXiv:2110.11658, Sec. 2).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The CUDA library never
 * links, includes or calls it, and it shares no code with the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (see build.py).
 * -ffp-contract=off keeps every a*b+c as two rounded operations, so the
 * decisions below (keys, opening tests, neighbour tests) are reproducible
 * operation by operation.
 *
 * Part 1, the plain definition (Sec. 2.1, Eqs. 1, 3, 4, 6, 8-10):
 *   far  a_i = sum_{j!=i} W(r_ij) m_j (x_j - x_i) / r_ij^3
 *   near a_i = sum_{j!=i} K(r_ij) m_j (x_j - x_i) / r_ij^3,   K = 1 - W
 *   full = near + far,  phi_i = -sum_{j!=i} m_j / r_ij      (G = 1)
 * The sign is read as attraction (Eq. 1 prints r_ij = x_i - x_j, which would
 * be repulsive); coincident pairs (r = 0) are skipped.
 *
 * Part 2, the reference Barnes-Hut tree (Sec. 2.4: "Barnes-Hut tree" with an
 * opening angle theta; theta = 0 reproduces direct summation).  The paper
 * fixes no key layout, node rule, moment order or opening test, so the rules
 * written here ARE the definition the GPU path must reproduce:
 *   1. bounding cube: exact FP64 min/max per axis; side = max extent (1 if 0);
 *      s = 2^21 / side.
 *   2. q_d = floor((x_d - min_d) * s), clamped to [0, 2^21 - 1].
 *   3. 63-bit Morton key: bit 3k+2 <- bit k of q_x, 3k+1 <- q_y, 3k <- q_z.
 *   4. stable order by (key, original index).
 *   5. canonical octree: a level-l node holds the particles sharing the top
 *      3l key bits; it is split iff count > leaf_cap and l < 21; its children
 *      are its non-empty octants in ascending order; nodes are numbered
 *      breadth first (by level, then by key prefix); single-child chains stay.
 *   6. moments in a fixed order: leaves sum their particles in sorted order,
 *      internal nodes combine their children in octant order; COM, traceless
 *      quadrupole Q = sum m (3 d d^T - |d|^2 I), tight AABB; massless nodes
 *      put the COM at the AABB centre.
 *   7. groups: let B = 16 G.  A node with count <= B whose parent has count > B
 *      (or the root if n <= B), and a leaf with count > B, are cut into
 *      consecutive chunks of G particles in key order (the last chunk of a
 *      node may be smaller); the chunks, ordered by first particle, are the
 *      walk groups.  Groups therefore stay inside nodes of at most 16 G
 *      particles and are full except at node ends.
 *   8. opening test of cell c for group g (box B_g): open iff
 *         dist(B_g, com_c)^2 < r_open_c^2,  r_open = l_c/theta + delta_c
 *      (l_c longest side of the cell box, delta_c = |com_c - box centre|,
 *      theta = 0 opens every cell)  OR  dist(B_g, box_c)^2 < r_out^2.
 *      An accepted cell lies at least r_out from every group particle, so
 *      W = 1 for all its mass; an opened leaf gives particle-particle terms.
 *   9. cell term at r = x_i - com (multipole expansion to quadrupole order):
 *         a = -M r/r^3 + Q r/r^5 - (5/2)(r.Q.r) r/r^7
 *         phi = -M/r - (1/2) r.Q.r / r^5
 *  10. particle term: a += W(r) m_j (x_j - x_i)/r^3, phi -= m_j/r (r > 0).
 *  11. neighbours of i: all j != i with |x_i - x_j|^2 < r_list^2, the square
 *      formed as (dx*dx + dy*dy) + dz*dz, listed by ascending original index.
 *  12. leapfrog kick (Eq. 12): v += (dt/2) a_far.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_LEVELS 21
#define ORC_QMAX 2097151LL /* 2^21 - 1 */
#define ORC_GROUP_NODE_FACTOR 16 /* rule 7: groups are cut from nodes of <= 16 G particles */

/* ------------------------------------------------------------------------ */
/* Part 1: changeover function and the direct split sum                      */
/* ------------------------------------------------------------------------ */

/* W = 1 - K of Eq. 6, with x = (y - gamma)/(1 - gamma), y = r/r_cut,
 * gamma = r_in/r_cut (Eqs. 8-10); r_cut is the outer radius r_out. */
double orc_changeover_W(double r, double r_in, double r_out)
{
    double y = r / r_out;
    double gamma = r_in / r_out;
    double x = (y - gamma) / (1.0 - gamma);
    if (x < 0.0) return 0.0;
    if (x >= 1.0) return 1.0;
    double x4 = x * x * x * x;
    double x5 = x4 * x, x6 = x5 * x, x7 = x6 * x;
    return -20.0 * x7 + 70.0 * x6 - 84.0 * x5 + 35.0 * x4;
}

/* K of Eq. 6, the near (irregular) weight. */
double orc_changeover_K(double r, double r_in, double r_out)
{
    return 1.0 - orc_changeover_W(r, r_in, r_out);
}

/* Direct split sum over all pairs for the listed targets (Eqs. 1, 3).
 * Outputs are (nt x 3) row-major; any of them may be NULL. */
void orc_direct_split(int64_t n, const double *x, const double *y, const double *z,
                      const double *m, double r_in, double r_out, int64_t nt,
                      const int64_t *targets, double *far, double *near, double *full,
                      double *pot)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets[t];
        double fa[3] = {0, 0, 0}, na[3] = {0, 0, 0}, ua[3] = {0, 0, 0}, ph = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double d[3] = {x[j] - x[i], y[j] - y[i], z[j] - z[i]};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            double f = m[j] / (r2 * r);
            double w = orc_changeover_W(r, r_in, r_out);
            double k = 1.0 - w;
            for (int c = 0; c < 3; c++) {
                fa[c] += w * f * d[c];
                na[c] += k * f * d[c];
                ua[c] += f * d[c];
            }
            ph -= m[j] / r;
        }
        for (int c = 0; c < 3; c++) {
            if (far) far[3 * t + c] = fa[c];
            if (near) near[3 * t + c] = na[c];
            if (full) full[3 * t + c] = ua[c];
        }
        if (pot) pot[t] = ph;
    }
}

/* Neighbour test of rule 11, shared by the brute-force and tree searches. */
static int orc_is_neighbour(double xi, double yi, double zi, double xj, double yj, double zj,
                            double rl2)
{
    double dx = xj - xi, dy = yj - yi, dz = zj - zi;
    double r2 = (dx * dx + dy * dy) + dz * dz;
    return r2 < rl2;
}

/* Brute-force neighbour lists (rule 11) of the listed targets.  Pass idx=NULL
 * to count only: counts[t] is always written; with idx, the rows are packed
 * back to back in target order (caller sizes idx from the counts). */
void orc_neighbours_brute(int64_t n, const double *x, const double *y, const double *z,
                          double r_list, int64_t nt, const int64_t *targets, int64_t *counts,
                          const int64_t *row_offsets, int32_t *idx)
{
    double rl2 = r_list * r_list;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets[t], c = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            if (orc_is_neighbour(x[i], y[i], z[i], x[j], y[j], z[j], rl2)) {
                if (idx) idx[row_offsets[t] + c] = (int32_t)j;
                c++;
            }
        }
        counts[t] = c;
    }
}

/* Leapfrog velocity kick of Eq. 12: v += (dt/2) a. */
void orc_kick(int64_t n, double dt, const double *ax, const double *ay, const double *az,
              double *vx, double *vy, double *vz)
{
    double h = 0.5 * dt;
    for (int64_t i = 0; i < n; i++) {
        vx[i] += h * ax[i];
        vy[i] += h * ay[i];
        vz[i] += h * az[i];
    }
}

/* dW/dx of Eq. 6 in the variable x of Eqs. 8-10: the bracket of Eq. 7,
 * -140 x^6 + 420 x^5 - 420 x^4 + 140 x^3 (= 140 x^3 (1 - x)^3) for 0 <= x < 1,
 * and 0 outside. */
double orc_changeover_dWdx(double r, double r_in, double r_out)
{
    double y = r / r_out;
    double gamma = r_in / r_out;
    double x = (y - gamma) / (1.0 - gamma);
    if (x < 0.0 || x >= 1.0) return 0.0;
    double x3 = x * x * x;
    double x4 = x3 * x, x5 = x4 * x, x6 = x5 * x;
    return -140.0 * x6 + 420.0 * x5 - 420.0 * x4 + 140.0 * x3;
}

/* Irregular (neighbour) force of Eq. 1 and its time derivative of Eq. 2 for
 * every particle, summed over the particle's neighbour row (offsets / idx as
 * produced by rule 11, original indices):
 *   F_I,i = sum_j K m_j d / r^3
 *   dF_I,i/dt = sum_j m_j [K (u / r^3 - 3 (d.u) d / r^5) + Kdot d / r^3]
 * with d = x_j - x_i, u = v_j - v_i (attraction, as in Part 1) and
 *   Kdot = dK/dt = -dW/dx (d.u) / (r (r_cut - r_in)),
 * the chain rule through x = (r/r_cut - gamma)/(1 - gamma).  Readings: Eq. 2
 * as printed drops m_j and K from its middle term and Eq. 7 prints K' with the
 * opposite sign; both are taken as the exact derivative of Eq. 1.  Pairs at
 * r = 0 (singular) and at r >= r_cut (K = K' = 0) contribute nothing.  The
 * sums run over the row in its order.  scale_f / scale_j (nullable) receive the
 * sums of the magnitudes of the terms, sum K m / r^2 and
 * sum m (K |u| / r^3 + 3 K |d.u| / r^4 + |Kdot| / r^2), per particle. */
void orc_irregular(int64_t n, const double *x, const double *y, const double *z,
                   const double *m, const double *vx, const double *vy, const double *vz,
                   double r_in, double r_out, const int64_t *offsets, const int32_t *idx,
                   double *f, double *jerk, double *scale_f, double *scale_j)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        double F[3] = {0, 0, 0}, J[3] = {0, 0, 0}, sf = 0.0, sj = 0.0;
        for (int64_t e = offsets[i]; e < offsets[i + 1]; e++) {
            int64_t j = idx[e];
            double d[3] = {x[j] - x[i], y[j] - y[i], z[j] - z[i]};
            double u[3] = {vx[j] - vx[i], vy[j] - vy[i], vz[j] - vz[i]};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            double k = orc_changeover_K(r, r_in, r_out);
            if (k == 0.0) continue;
            double du = d[0] * u[0] + d[1] * u[1] + d[2] * u[2];
            double kdot = -orc_changeover_dWdx(r, r_in, r_out) * du / (r * (r_out - r_in));
            double f3 = m[j] / (r2 * r);
            for (int c = 0; c < 3; c++) {
                F[c] += k * f3 * d[c];
                J[c] += k * f3 * u[c] - 3.0 * k * f3 * (du / r2) * d[c] + kdot * f3 * d[c];
            }
            sf += k * m[j] / r2;
            sj += m[j] * (k * sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) / (r2 * r) +
                          3.0 * k * fabs(du) / (r2 * r2) + fabs(kdot) / r2);
        }
        for (int c = 0; c < 3; c++) {
            f[3 * i + c] = F[c];
            jerk[3 * i + c] = J[c];
        }
        if (scale_f) scale_f[i] = sf;
        if (scale_j) scale_j[i] = sj;
    }
}

/* k nearest neighbours of sampled particles by brute force (the core-quantity
 * search of Sec. 4: a random sample of min(N, sqrt(5000 N)) particles, each
 * with its 6 nearest neighbours).  For sample t (particle i = sample[t]) the
 * k particles j != i with the smallest squared distance (dx*dx + dy*dy) + dz*dz
 * (FP64, as rule 11), ties broken by the smaller original index, in ascending
 * order: idx[t*k + q], d2[t*k + q].  Fewer than k candidates leave -1 / inf. */
void orc_knn(int64_t n, const double *x, const double *y, const double *z, int k, int64_t s,
             const int32_t *sample, int32_t *idx, double *d2)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < s; t++) {
        int64_t i = sample[t];
        int32_t *bi = idx + t * k;
        double *bd = d2 + t * k;
        for (int q = 0; q < k; q++) {
            bi[q] = -1;
            bd[q] = INFINITY;
        }
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];
            double r2 = (dx * dx + dy * dy) + dz * dz;
            /* (r2, j) against the current k-th: j ascends, so ties keep the earlier */
            if (!(r2 < bd[k - 1])) continue;
            int q = k - 1;
            while (q > 0 && r2 < bd[q - 1]) {
                bd[q] = bd[q - 1];
                bi[q] = bi[q - 1];
                q--;
            }
            bd[q] = r2;
            bi[q] = (int32_t)j;
        }
    }
}

/* Core quantities from the 6 nearest neighbours of a sample (the density
 * estimator and density-weighted averages of Casertano & Hut, which Sec. 4
 * cites and does not print; this is the reading):
 *   rho_t   = 3 (m of the 5 nearest) / (4 pi r_6^3)        per sample particle
 *   x_d     = sum rho_t x_t / sum rho_t                     density centre
 *   r_core  = sqrt(sum rho_t^2 |x_t - x_d|^2 / sum rho_t^2)
 *   rho_core = sum rho_t^2 / sum rho_t
 *   n_core  = #{ all particles j : |x_j - x_d|^2 < r_core^2 }
 * Sums run over the sample in its order.  A sampled particle without 6
 * neighbours (a system of fewer than 7 particles) gets rho = 0.  out = {x_d,
 * y_d, z_d, r_core, rho_core, n_core}; rho (s values) may be NULL. */
void orc_core_quantities(int64_t n, const double *x, const double *y, const double *z,
                         const double *m, int64_t s, const int32_t *sample, const int32_t *idx6,
                         const double *d26, double *rho, double *out)
{
    const double pi = 3.14159265358979323846;
    double w = 0.0, w2 = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
    double *r = (double *)malloc(sizeof(double) * (size_t)(s > 0 ? s : 1));
    for (int64_t t = 0; t < s; t++) {
        double mass = 0.0;
        for (int q = 0; q < 5; q++)
            if (idx6[6 * t + q] >= 0) mass += m[idx6[6 * t + q]];
        double r6 = sqrt(d26[6 * t + 5]); /* inf without a 6th neighbour: rho = 0 */
        r[t] = 3.0 * mass / (4.0 * pi * (r6 * r6 * r6));
        int64_t i = sample[t];
        w += r[t];
        w2 += r[t] * r[t];
        cx += r[t] * x[i];
        cy += r[t] * y[i];
        cz += r[t] * z[i];
    }
    cx /= w;
    cy /= w;
    cz /= w;
    double a = 0.0;
    for (int64_t t = 0; t < s; t++) {
        int64_t i = sample[t];
        double dx = x[i] - cx, dy = y[i] - cy, dz = z[i] - cz;
        a += r[t] * r[t] * ((dx * dx + dy * dy) + dz * dz);
    }
    double rc = sqrt(a / w2);
    double rc2 = rc * rc;
    int64_t cnt = 0;
    for (int64_t j = 0; j < n; j++) {
        double dx = x[j] - cx, dy = y[j] - cy, dz = z[j] - cz;
        if ((dx * dx + dy * dy) + dz * dz < rc2) cnt++;
    }
    out[0] = cx;
    out[1] = cy;
    out[2] = cz;
    out[3] = rc;
    out[4] = w2 / w;
    out[5] = (double)cnt;
    if (rho)
        for (int64_t t = 0; t < s; t++) rho[t] = r[t];
    free(r);
}

/* ------------------------------------------------------------------------ */
/* Part 2: the reference tree                                                */
/* ------------------------------------------------------------------------ */

/* Rule 1: out = {min_x, min_y, min_z, side}. */
void orc_bounding_cube(int64_t n, const double *x, const double *y, const double *z,
                       double *out)
{
    const double *p[3] = {x, y, z};
    double side = 0.0;
    for (int d = 0; d < 3; d++) {
        double lo = p[d][0], hi = p[d][0];
        for (int64_t i = 1; i < n; i++) {
            if (p[d][i] < lo) lo = p[d][i];
            if (p[d][i] > hi) hi = p[d][i];
        }
        out[d] = lo;
        double ext = hi - lo;
        if (ext > side) side = ext;
    }
    if (side == 0.0) side = 1.0;
    out[3] = side;
}

/* Rules 2-3: quantised coordinate and the interleaved 63-bit key. */
static int64_t orc_quantise(double v, double lo, double s)
{
    double t = floor((v - lo) * s);
    if (t < 0.0) return 0;
    if (t > (double)ORC_QMAX) return ORC_QMAX;
    return (int64_t)t;
}

uint64_t orc_interleave(int64_t qx, int64_t qy, int64_t qz)
{
    uint64_t key = 0;
    for (int k = 0; k < ORC_LEVELS; k++) {
        key |= (uint64_t)((qx >> k) & 1) << (3 * k + 2);
        key |= (uint64_t)((qy >> k) & 1) << (3 * k + 1);
        key |= (uint64_t)((qz >> k) & 1) << (3 * k);
    }
    return key;
}

void orc_morton_keys(int64_t n, const double *x, const double *y, const double *z,
                     uint64_t *keys)
{
    double cube[4];
    orc_bounding_cube(n, x, y, z, cube);
    double s = 2097152.0 / cube[3];
    for (int64_t i = 0; i < n; i++)
        keys[i] = orc_interleave(orc_quantise(x[i], cube[0], s), orc_quantise(y[i], cube[1], s),
                                 orc_quantise(z[i], cube[2], s));
}

typedef struct {
    int64_t n;
    double theta, r_out;
    int leaf_cap, group_size;
    uint64_t *keys; /* sorted */
    int32_t *perm;  /* sorted position -> original index */
    double *xs, *ys, *zs, *ms;
    int64_t n_nodes, cap_nodes;
    int32_t *level, *first, *count, *child, *nchild, *parent;
    double *M, *com, *Q, *lo, *hi, *ropen2; /* com/lo/hi: 3 per node, Q: 6 */
    int64_t n_groups;
    int32_t *g_first, *g_count;
    double *g_lo, *g_hi; /* 3 per group */
} orc_tree;

static const uint64_t *g_sort_keys; /* qsort has no user pointer */

static int orc_cmp_key_idx(const void *a, const void *b)
{
    int32_t i = *(const int32_t *)a, j = *(const int32_t *)b;
    uint64_t ki = g_sort_keys[i], kj = g_sort_keys[j];
    if (ki < kj) return -1;
    if (ki > kj) return 1;
    return (i > j) - (i < j);
}

static void orc_node_push(orc_tree *t, int32_t lvl, int32_t f, int32_t c, int32_t par)
{
    if (t->n_nodes == t->cap_nodes) {
        t->cap_nodes = t->cap_nodes ? 2 * t->cap_nodes : 1024;
        t->level = realloc(t->level, t->cap_nodes * sizeof(int32_t));
        t->first = realloc(t->first, t->cap_nodes * sizeof(int32_t));
        t->count = realloc(t->count, t->cap_nodes * sizeof(int32_t));
        t->child = realloc(t->child, t->cap_nodes * sizeof(int32_t));
        t->nchild = realloc(t->nchild, t->cap_nodes * sizeof(int32_t));
        t->parent = realloc(t->parent, t->cap_nodes * sizeof(int32_t));
    }
    int64_t k = t->n_nodes++;
    t->level[k] = lvl;
    t->first[k] = f;
    t->count[k] = c;
    t->child[k] = -1;
    t->nchild[k] = 0;
    t->parent[k] = par;
}

/* Rule 6 for one node, children (if any) already done. */
static void orc_node_moments(orc_tree *t, int64_t k)
{
    double M = 0.0, S[3] = {0, 0, 0}, lo[3] = {INFINITY, INFINITY, INFINITY},
           hi[3] = {-INFINITY, -INFINITY, -INFINITY}, com[3], Q[6] = {0, 0, 0, 0, 0, 0};
    if (t->nchild[k] == 0) {
        int32_t b = t->first[k], e = b + t->count[k];
        for (int32_t i = b; i < e; i++) {
            double p[3] = {t->xs[i], t->ys[i], t->zs[i]};
            M += t->ms[i];
            for (int d = 0; d < 3; d++) {
                S[d] += t->ms[i] * p[d];
                if (p[d] < lo[d]) lo[d] = p[d];
                if (p[d] > hi[d]) hi[d] = p[d];
            }
        }
        for (int d = 0; d < 3; d++) com[d] = M > 0.0 ? S[d] / M : 0.5 * (lo[d] + hi[d]);
        for (int32_t i = b; i < e; i++) {
            double m = t->ms[i];
            double dx = t->xs[i] - com[0], dy = t->ys[i] - com[1], dz = t->zs[i] - com[2];
            double r2 = (dx * dx + dy * dy) + dz * dz;
            Q[0] += m * (3.0 * dx * dx - r2);
            Q[1] += m * (3.0 * dx * dy);
            Q[2] += m * (3.0 * dx * dz);
            Q[3] += m * (3.0 * dy * dy - r2);
            Q[4] += m * (3.0 * dy * dz);
            Q[5] += m * (3.0 * dz * dz - r2);
        }
    } else {
        int32_t c0 = t->child[k], c1 = c0 + t->nchild[k];
        for (int32_t c = c0; c < c1; c++) {
            M += t->M[c];
            for (int d = 0; d < 3; d++) {
                S[d] += t->M[c] * t->com[3 * c + d];
                if (t->lo[3 * c + d] < lo[d]) lo[d] = t->lo[3 * c + d];
                if (t->hi[3 * c + d] > hi[d]) hi[d] = t->hi[3 * c + d];
            }
        }
        for (int d = 0; d < 3; d++) com[d] = M > 0.0 ? S[d] / M : 0.5 * (lo[d] + hi[d]);
        for (int32_t c = c0; c < c1; c++) {
            double Mc = t->M[c];
            double dx = t->com[3 * c] - com[0], dy = t->com[3 * c + 1] - com[1],
                   dz = t->com[3 * c + 2] - com[2];
            double d2 = (dx * dx + dy * dy) + dz * dz;
            const double *Qc = t->Q + 6 * c;
            Q[0] += Qc[0] + Mc * (3.0 * dx * dx - d2);
            Q[1] += Qc[1] + Mc * (3.0 * dx * dy);
            Q[2] += Qc[2] + Mc * (3.0 * dx * dz);
            Q[3] += Qc[3] + Mc * (3.0 * dy * dy - d2);
            Q[4] += Qc[4] + Mc * (3.0 * dy * dz);
            Q[5] += Qc[5] + Mc * (3.0 * dz * dz - d2);
        }
    }
    t->M[k] = M;
    for (int d = 0; d < 3; d++) {
        t->com[3 * k + d] = com[d];
        t->lo[3 * k + d] = lo[d];
        t->hi[3 * k + d] = hi[d];
    }
    for (int a = 0; a < 6; a++) t->Q[6 * k + a] = Q[a];
    /* rule 8: opening radius l/theta + delta */
    double l = hi[0] - lo[0];
    if (hi[1] - lo[1] > l) l = hi[1] - lo[1];
    if (hi[2] - lo[2] > l) l = hi[2] - lo[2];
    double cx = 0.5 * (lo[0] + hi[0]) - com[0], cy = 0.5 * (lo[1] + hi[1]) - com[1],
           cz = 0.5 * (lo[2] + hi[2]) - com[2];
    double delta = sqrt((cx * cx + cy * cy) + cz * cz);
    if (t->theta > 0.0) {
        double ro = l / t->theta + delta;
        t->ropen2[k] = ro * ro;
    } else {
        t->ropen2[k] = INFINITY;
    }
}

static void orc_group_push(orc_tree *t, int32_t f, int32_t c, int64_t *cap)
{
    if (t->n_groups == *cap) {
        *cap = *cap ? 2 * *cap : 1024;
        t->g_first = realloc(t->g_first, *cap * sizeof(int32_t));
        t->g_count = realloc(t->g_count, *cap * sizeof(int32_t));
    }
    t->g_first[t->n_groups] = f;
    t->g_count[t->n_groups] = c;
    t->n_groups++;
}

static int orc_cmp_group(const void *a, const void *b)
{
    const int32_t *p = a, *q = b;
    return (p[0] > q[0]) - (p[0] < q[0]);
}

orc_tree *orc_tree_build(int64_t n, const double *x, const double *y, const double *z,
                         const double *m, double theta, double r_out, int leaf_cap,
                         int group_size)
{
    orc_tree *t = calloc(1, sizeof(orc_tree));
    t->n = n;
    t->theta = theta;
    t->r_out = r_out;
    t->leaf_cap = leaf_cap;
    t->group_size = group_size;
    /* rules 1-4 */
    uint64_t *keys = malloc(n * sizeof(uint64_t));
    orc_morton_keys(n, x, y, z, keys);
    t->perm = malloc(n * sizeof(int32_t));
    for (int64_t i = 0; i < n; i++) t->perm[i] = (int32_t)i;
    g_sort_keys = keys;
    qsort(t->perm, n, sizeof(int32_t), orc_cmp_key_idx);
    t->keys = malloc(n * sizeof(uint64_t));
    t->xs = malloc(n * sizeof(double));
    t->ys = malloc(n * sizeof(double));
    t->zs = malloc(n * sizeof(double));
    t->ms = malloc(n * sizeof(double));
    for (int64_t s = 0; s < n; s++) {
        int32_t i = t->perm[s];
        t->keys[s] = keys[i];
        t->xs[s] = x[i];
        t->ys[s] = y[i];
        t->zs[s] = z[i];
        t->ms[s] = m[i];
    }
    free(keys);
    /* rule 5: breadth-first canonical octree */
    orc_node_push(t, 0, 0, (int32_t)n, -1);
    for (int64_t k = 0; k < t->n_nodes; k++) {
        int32_t lvl = t->level[k];
        if (t->count[k] <= leaf_cap || lvl >= ORC_LEVELS) continue;
        int shift = 63 - 3 * (lvl + 1);
        int32_t b = t->first[k], e = b + t->count[k];
        int32_t first_child = (int32_t)t->n_nodes, nc = 0;
        int32_t run = b;
        for (int32_t i = b + 1; i <= e; i++) {
            if (i == e || (t->keys[i] >> shift) != (t->keys[run] >> shift)) {
                orc_node_push(t, lvl + 1, run, i - run, (int32_t)k);
                nc++;
                run = i;
            }
        }
        t->child[k] = first_child;
        t->nchild[k] = nc;
    }
    int64_t nn = t->n_nodes;
    t->M = malloc(nn * sizeof(double));
    t->com = malloc(3 * nn * sizeof(double));
    t->Q = malloc(6 * nn * sizeof(double));
    t->lo = malloc(3 * nn * sizeof(double));
    t->hi = malloc(3 * nn * sizeof(double));
    t->ropen2 = malloc(nn * sizeof(double));
    /* rule 6: children before parents */
    for (int64_t k = nn - 1; k >= 0; k--) orc_node_moments(t, k);
    /* rule 7: groups, then ordered by first particle */
    int64_t gcap = 0;
    int64_t big = (int64_t)ORC_GROUP_NODE_FACTOR * group_size;
    for (int64_t k = 0; k < nn; k++) {
        int32_t c = t->count[k];
        int parent_big = (k == 0) || t->count[t->parent[k]] > big;
        if (!parent_big) continue;
        if (c <= big || t->nchild[k] == 0) {
            for (int32_t f = 0; f < c; f += group_size)
                orc_group_push(t, t->first[k] + f, c - f < group_size ? c - f : group_size, &gcap);
        }
    }
    int32_t *pairs = malloc(2 * t->n_groups * sizeof(int32_t));
    for (int64_t g = 0; g < t->n_groups; g++) {
        pairs[2 * g] = t->g_first[g];
        pairs[2 * g + 1] = t->g_count[g];
    }
    qsort(pairs, t->n_groups, 2 * sizeof(int32_t), orc_cmp_group);
    t->g_lo = malloc(3 * t->n_groups * sizeof(double));
    t->g_hi = malloc(3 * t->n_groups * sizeof(double));
    for (int64_t g = 0; g < t->n_groups; g++) {
        t->g_first[g] = pairs[2 * g];
        t->g_count[g] = pairs[2 * g + 1];
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int32_t i = t->g_first[g]; i < t->g_first[g] + t->g_count[g]; i++) {
            double p[3] = {t->xs[i], t->ys[i], t->zs[i]};
            for (int d = 0; d < 3; d++) {
                if (p[d] < lo[d]) lo[d] = p[d];
                if (p[d] > hi[d]) hi[d] = p[d];
            }
        }
        for (int d = 0; d < 3; d++) {
            t->g_lo[3 * g + d] = lo[d];
            t->g_hi[3 * g + d] = hi[d];
        }
    }
    free(pairs);
    return t;
}

void orc_tree_free(orc_tree *t)
{
    if (!t) return;
    void *bufs[] = {t->keys, t->perm, t->xs, t->ys, t->zs, t->ms, t->level, t->first, t->count,
                    t->child, t->nchild, t->parent, t->M, t->com, t->Q, t->lo, t->hi, t->ropen2,
                    t->g_first, t->g_count, t->g_lo, t->g_hi};
    for (size_t i = 0; i < sizeof(bufs) / sizeof(bufs[0]); i++) free(bufs[i]);
    free(t);
}

int64_t orc_tree_n_nodes(const orc_tree *t) { return t->n_nodes; }
int64_t orc_tree_n_groups(const orc_tree *t) { return t->n_groups; }

/* Copy the tree out; any pointer may be NULL.  Node arrays have n_nodes rows
 * (com/lo/hi 3 columns, Q 6 columns), group arrays n_groups rows. */
void orc_tree_export(const orc_tree *t, uint64_t *keys, int32_t *perm, int32_t *level,
                     int32_t *first, int32_t *count, int32_t *child, int32_t *nchild,
                     double *M, double *com, double *Q, double *lo, double *hi, double *ropen2,
                     int32_t *g_first, int32_t *g_count, double *g_lo, double *g_hi)
{
    int64_t n = t->n, nn = t->n_nodes, ng = t->n_groups;
    if (keys) memcpy(keys, t->keys, n * sizeof(uint64_t));
    if (perm) memcpy(perm, t->perm, n * sizeof(int32_t));
    if (level) memcpy(level, t->level, nn * sizeof(int32_t));
    if (first) memcpy(first, t->first, nn * sizeof(int32_t));
    if (count) memcpy(count, t->count, nn * sizeof(int32_t));
    if (child) memcpy(child, t->child, nn * sizeof(int32_t));
    if (nchild) memcpy(nchild, t->nchild, nn * sizeof(int32_t));
    if (M) memcpy(M, t->M, nn * sizeof(double));
    if (com) memcpy(com, t->com, 3 * nn * sizeof(double));
    if (Q) memcpy(Q, t->Q, 6 * nn * sizeof(double));
    if (lo) memcpy(lo, t->lo, 3 * nn * sizeof(double));
    if (hi) memcpy(hi, t->hi, 3 * nn * sizeof(double));
    if (ropen2) memcpy(ropen2, t->ropen2, nn * sizeof(double));
    if (g_first) memcpy(g_first, t->g_first, ng * sizeof(int32_t));
    if (g_count) memcpy(g_count, t->g_count, ng * sizeof(int32_t));
    if (g_lo) memcpy(g_lo, t->g_lo, 3 * ng * sizeof(double));
    if (g_hi) memcpy(g_hi, t->g_hi, 3 * ng * sizeof(double));
}

/* Squared distance from a point to a box, per axis max(0, lo - p, p - hi). */
static double orc_dist2_point_box(const double *p, const double *lo, const double *hi)
{
    double t[3];
    for (int d = 0; d < 3; d++) {
        double a = lo[d] - p[d], b = p[d] - hi[d];
        double v = a > b ? a : b;
        t[d] = v > 0.0 ? v : 0.0;
    }
    return (t[0] * t[0] + t[1] * t[1]) + t[2] * t[2];
}

/* Squared distance between two boxes, per axis max(0, lo_c - hi_g, lo_g - hi_c). */
static double orc_dist2_box_box(const double *glo, const double *ghi, const double *clo,
                                const double *chi)
{
    double t[3];
    for (int d = 0; d < 3; d++) {
        double a = clo[d] - ghi[d], b = glo[d] - chi[d];
        double v = a > b ? a : b;
        t[d] = v > 0.0 ? v : 0.0;
    }
    return (t[0] * t[0] + t[1] * t[1]) + t[2] * t[2];
}

/* Rule 8. */
static int orc_opens(const orc_tree *t, int64_t g, int64_t c, double r_out2)
{
    const double *glo = t->g_lo + 3 * g, *ghi = t->g_hi + 3 * g;
    if (orc_dist2_point_box(t->com + 3 * c, glo, ghi) < t->ropen2[c]) return 1;
    return orc_dist2_box_box(glo, ghi, t->lo + 3 * c, t->hi + 3 * c) < r_out2;
}

/* Far force (rules 8-10) on the particles of the listed groups (all groups if
 * groups == NULL).  ax/ay/az/pot are indexed by ORIGINAL particle index and
 * only the selected groups' particles are written; pot may be NULL.
 * n_cell/n_part (nullable, one entry per listed group) receive the number of
 * accepted cells and of source particles in opened leaves of that group. */
void orc_tree_far(const orc_tree *t, int quadrupole, double r_in, double r_out, int64_t ng_sel,
                  const int64_t *groups, double *ax, double *ay, double *az, double *pot,
                  int64_t *n_cell, int64_t *n_part)
{
    int64_t ng = groups ? ng_sel : t->n_groups;
    double r_out2 = r_out * r_out;
#pragma omp parallel
    {
        int32_t *stack = malloc((8 * ORC_LEVELS + 16) * 8 * sizeof(int32_t));
#pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < ng; q++) {
            int64_t g = groups ? groups[q] : q;
            int32_t gb = t->g_first[g], gc = t->g_count[g];
            int64_t ncell = 0, npart = 0;
            double *acc = calloc(4 * (size_t)gc, sizeof(double));
            int sp = 0;
            stack[sp++] = 0;
            while (sp > 0) {
                int32_t c = stack[--sp];
                if (orc_opens(t, g, c, r_out2)) {
                    if (t->nchild[c] == 0) {
                        int32_t jb = t->first[c], je = jb + t->count[c];
                        npart += je - jb;
                        for (int32_t s = 0; s < gc; s++) {
                            int32_t i = gb + s;
                            for (int32_t j = jb; j < je; j++) {
                                double d[3] = {t->xs[j] - t->xs[i], t->ys[j] - t->ys[i],
                                               t->zs[j] - t->zs[i]};
                                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                                if (r2 == 0.0) continue;
                                double r = sqrt(r2);
                                double f = orc_changeover_W(r, r_in, r_out) * t->ms[j] / (r2 * r);
                                for (int k = 0; k < 3; k++) acc[4 * s + k] += f * d[k];
                                acc[4 * s + 3] -= t->ms[j] / r;
                            }
                        }
                    } else {
                        for (int32_t k = 0; k < t->nchild[c]; k++) stack[sp++] = t->child[c] + k;
                    }
                } else {
                    ncell++;
                    const double *Q = t->Q + 6 * c;
                    double M = t->M[c];
                    for (int32_t s = 0; s < gc; s++) {
                        int32_t i = gb + s;
                        double r[3] = {t->xs[i] - t->com[3 * c], t->ys[i] - t->com[3 * c + 1],
                                       t->zs[i] - t->com[3 * c + 2]};
                        double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                        double ri = 1.0 / sqrt(r2);
                        double ri2 = ri * ri, ri3 = ri * ri2, ri5 = ri3 * ri2, ri7 = ri5 * ri2;
                        double a[3], ph = -M * ri;
                        for (int k = 0; k < 3; k++) a[k] = -M * r[k] * ri3;
                        if (quadrupole) {
                            double Qr[3] = {Q[0] * r[0] + Q[1] * r[1] + Q[2] * r[2],
                                            Q[1] * r[0] + Q[3] * r[1] + Q[4] * r[2],
                                            Q[2] * r[0] + Q[4] * r[1] + Q[5] * r[2]};
                            double rQr = r[0] * Qr[0] + r[1] * Qr[1] + r[2] * Qr[2];
                            for (int k = 0; k < 3; k++)
                                a[k] += Qr[k] * ri5 - 2.5 * rQr * r[k] * ri7;
                            ph -= 0.5 * rQr * ri5;
                        }
                        for (int k = 0; k < 3; k++) acc[4 * s + k] += a[k];
                        acc[4 * s + 3] += ph;
                    }
                }
            }
            for (int32_t s = 0; s < gc; s++) {
                int32_t o = t->perm[gb + s];
                ax[o] = acc[4 * s];
                ay[o] = acc[4 * s + 1];
                az[o] = acc[4 * s + 2];
                if (pot) pot[o] = acc[4 * s + 3];
            }
            if (n_cell) n_cell[q] = ncell;
            if (n_part) n_part[q] = npart;
            free(acc);
        }
        free(stack);
    }
}

static int orc_cmp_i32(const void *a, const void *b)
{
    int32_t p = *(const int32_t *)a, q = *(const int32_t *)b;
    return (p > q) - (p < q);
}

/* Neighbour lists (rule 11) of the particles of the listed groups, found by
 * opening every cell whose box lies within r_list of the group box.
 * counts[] is indexed by ORIGINAL particle index (only the selected groups'
 * particles are written).  If idx != NULL, row_offsets (indexed by original
 * index) give where each row starts in idx; rows are sorted ascending. */
void orc_tree_neighbours(const orc_tree *t, double r_list, int64_t ng_sel, const int64_t *groups,
                         int64_t *counts, const int64_t *row_offsets, int32_t *idx)
{
    int64_t ng = groups ? ng_sel : t->n_groups;
    double rl2 = r_list * r_list;
#pragma omp parallel
    {
        int32_t *stack = malloc((8 * ORC_LEVELS + 16) * 8 * sizeof(int32_t));
#pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < ng; q++) {
            int64_t g = groups ? groups[q] : q;
            int32_t gb = t->g_first[g], gc = t->g_count[g];
            const double *glo = t->g_lo + 3 * g, *ghi = t->g_hi + 3 * g;
            for (int32_t s = 0; s < gc; s++) counts[t->perm[gb + s]] = 0;
            int sp = 0;
            stack[sp++] = 0;
            while (sp > 0) {
                int32_t c = stack[--sp];
                if (!(orc_dist2_box_box(glo, ghi, t->lo + 3 * c, t->hi + 3 * c) < rl2)) continue;
                if (t->nchild[c] > 0) {
                    for (int32_t k = 0; k < t->nchild[c]; k++) stack[sp++] = t->child[c] + k;
                    continue;
                }
                int32_t jb = t->first[c], je = jb + t->count[c];
                for (int32_t s = 0; s < gc; s++) {
                    int32_t i = gb + s, oi = t->perm[i];
                    for (int32_t j = jb; j < je; j++) {
                        if (j == i) continue;
                        if (orc_is_neighbour(t->xs[i], t->ys[i], t->zs[i], t->xs[j], t->ys[j],
                                             t->zs[j], rl2)) {
                            if (idx) idx[row_offsets[oi] + counts[oi]] = t->perm[j];
                            counts[oi]++;
                        }
                    }
                }
            }
            if (idx)
                for (int32_t s = 0; s < gc; s++) {
                    int32_t oi = t->perm[gb + s];
                    qsort(idx + row_offsets[oi], counts[oi], sizeof(int32_t), orc_cmp_i32);
                }
        }
        free(stack);
    }
}
