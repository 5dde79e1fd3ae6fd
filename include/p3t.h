/*
 * p3t.h -- C ABI of the distant-force ("regular force") path of the P3T scheme
 * (Particle-Particle Particle-Tree; arXiv:2110.11658, Sec. 2) on one NVIDIA
 * B300 GPU (sm_103a).
 *
 * The paper's regular-force step (Sec. 2.2, integration steps 1-2 and 4-5;
 * Sec. 2.4) takes FP64 positions and masses, builds a Barnes-Hut tree,
 * returns the regular (far) acceleration F_R of Eq. 3 -- the Newtonian force
 * weighted by W = 1 - K of Eq. 6 -- and the neighbour lists of the constant
 * neighbour radius (Sec. 2.3), and applies the leapfrog kick of Eq. 12.
 *
 * Conventions shared by every call:
 *  - G = 1 (Henon units, Sec. 3.1).  Accelerations are attractive:
 *    a_i = sum_j W(r_ij) m_j (x_j - x_i) / r_ij^3.
 *  - Array arguments are DEVICE pointers owned by the caller (except the
 *    *_host variants), indexed by the caller's ORIGINAL particle order, in
 *    structure-of-arrays form (one array per component).
 *  - Work is enqueued on the context's CUDA stream and is asynchronous unless
 *    a call says it synchronises.  Errors found on the device (non-finite or
 *    negative inputs, capacity, a bounded wait that ran out) are latched in the
 *    context and returned by the next synchronising call (p3t_status,
 *    p3t_neighbours, p3t_tree_info, p3t_step_host).
 *  - Every call returns P3T_OK (0) or one of the P3T_ERR_* codes; no call
 *    throws across the ABI.  Contexts are independent (no global state).
 *  - A context is not thread-safe: use one per host thread.
 */
#ifndef P3T_H
#define P3T_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define P3T_OK 0
#define P3T_ERR_INVALID_ARG 1   /* n <= 0, theta < 0, r_in >= r_out, null pointer, bad tuning value */
#define P3T_ERR_INVALID_INPUT 2 /* a non-finite position or mass, or a negative mass */
#define P3T_ERR_OOM 3           /* device allocation failed */
#define P3T_ERR_CAPACITY 4      /* caller buffer too small; the required size is reported */
#define P3T_ERR_ORDER 5         /* a call that needs a tree came before p3t_build_tree */
#define P3T_ERR_TIMEOUT 6       /* a bounded device-side wait ran out */
#define P3T_ERR_CUDA 7          /* a CUDA runtime call failed */
#define P3T_ERR_INTERNAL 8      /* a device-side consistency check failed (tree walk aborted) */

#define P3T_FP32_MIXED 0 /* FP32 interactions on FP64-subtracted relative coordinates, compensated sums */
#define P3T_FP64 1       /* every interaction in FP64 */

/* Tuning and physics parameters.
 *  theta        opening angle of the Barnes-Hut test (Sec. 2.4); 0 opens every cell.
 *  r_in, r_out  inner and outer radii of the changeover W (Eqs. 6, 8-10; r_out is
 *               the paper's r_cut).  0 <= r_in < r_out.
 *  r_list       neighbour-list radius (Sec. 2.3); a pair is listed iff |r| < r_list.
 *  leaf_cap     a node holding more than leaf_cap particles is split (below level 21).
 *  group_size   G, the largest particle group that walks the tree together (32, 64 or 128).
 *  tile         interaction-list tile: a group evaluates its buffered cells and
 *               particles once `tile` of them are queued (32..256, multiple of 32).
 *  threads_per_group  threads that evaluate one group: 32 (one warp; a lane holds
 *               G/32 targets when G > 32), 64 or 128 (2 or 4 warps, one target per
 *               thread, G <= threads_per_group: the first warp walks the tree for the
 *               group and every warp evaluates the queued cells and particles).
 *  precision    P3T_FP32_MIXED or P3T_FP64.
 *  quadrupole   1: monopole + quadrupole cell terms; 0: monopole only. */
typedef struct {
    double theta, r_in, r_out, r_list;
    int32_t leaf_cap, group_size, tile, threads_per_group, precision, quadrupole;
} p3t_params;

typedef struct p3t_ctx p3t_ctx; /* opaque; owns the tree and all scratch memory */

/* Fill *p with defaults: theta 0.5, r_in 0.005, r_out 0.05, r_list 0.05, leaf_cap 16,
 * group_size 32, tile 64, threads_per_group 32, P3T_FP32_MIXED, quadrupole 1. */
int p3t_default_params(p3t_params *p);

/* Create a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the handle. */
int p3t_create(p3t_ctx **out, const p3t_params *p, void *cuda_stream);

/* Free every device buffer of the context (synchronises its stream). */
int p3t_destroy(p3t_ctx *c);

/* Replace the parameters; they take effect at the next p3t_build_tree. */
int p3t_set_params(p3t_ctx *c, const p3t_params *p);

/* Build the tree of n particles (Sec. 2.4): bounding cube, 63-bit Morton keys,
 * stable radix sort by (key, index), canonical octree, centre-of-mass,
 * quadrupole and bounding-box moments, walk groups.  x, y, z, m: device FP64
 * arrays of length n, read only; they are copied in sorted order, so the
 * caller may change them afterwards.  Grows the context's scratch if n
 * exceeds every earlier n (that growth allocates and synchronises).
 * Errors: P3T_ERR_INVALID_ARG (n <= 0 or n >= 2^31, null pointer);
 * non-finite coordinates or masses and negative masses are reported later
 * as P3T_ERR_INVALID_INPUT. */
int p3t_build_tree(p3t_ctx *c, int64_t n, const double *x, const double *y, const double *z,
                   const double *m);

/* Build the trees of n_clusters independent clusters at once (the ensemble
 * form): cluster k holds the particles [seg_offsets[k], seg_offsets[k+1]) of
 * the concatenated arrays x, y, z, m (device double[n]).  seg_offsets is a
 * DEVICE int64 array of n_clusters + 1 entries, 0 = seg_offsets[0] <
 * seg_offsets[1] < ... < seg_offsets[n_clusters] = n (every cluster non-empty).
 * cluster_params: nullable DEVICE double array of 4 per cluster {theta, r_in,
 * r_out, r_list} (meaning as in p3t_params); NULL gives every cluster the
 * context's values.  Invalid offsets or radii are reported as
 * P3T_ERR_INVALID_INPUT.  Each cluster gets its own bounding cube and tree
 * exactly as p3t_build_tree would build it alone with its parameters, so every
 * later call (far force, neighbours, kick) gives each cluster the same result,
 * bit for bit, as a build of that cluster alone; neighbour lists never cross
 * clusters.  (One exception: the mixed far force evaluates cells in the r^-5 form
 * when every cluster of the tree has r_out >= 1e-7, a frame half-size <= 1e6 and
 * a mass <= 1e15, else in the r^-3 form; a batch holding a cluster outside those
 * bounds gives the others forces equal to their builds alone to FP32 rounding,
 * lists still bit for bit.)  Original indices in outputs refer to the concatenated order.  No
 * host synchronisation: a whole step can be captured in a CUDA graph once the
 * context's scratch has been sized by an earlier build of the same n. */
int p3t_build_tree_batch(p3t_ctx *c, int32_t n_clusters, int64_t n, const int64_t *seg_offsets,
                         const double *cluster_params, const double *x, const double *y,
                         const double *z, const double *m);

/* Far (regular) acceleration F_R of Eq. 3 for every particle of the last built
 * tree: the group-wise walk opens a cell iff it fails the opening-angle test
 * or lies within r_out of the group's box; accepted cells give monopole (+
 * quadrupole) terms, opened leaves give particle terms weighted by W (Eq. 6).
 * ax, ay, az: device arrays of n float (P3T_FP32_MIXED) or double (P3T_FP64),
 * written in original order.  pot: nullable device double[n], the unsplit
 * Newtonian potential -sum m_j / r_ij (for energy diagnostics).
 * n_cell_inter, n_part_inter: nullable device int64 counters; the call ADDS
 * the number of particle-cell and particle-particle interactions evaluated.
 * Errors: P3T_ERR_ORDER if no tree was built; P3T_ERR_INVALID_ARG for a null
 * acceleration pointer. */
int p3t_far_force(p3t_ctx *c, void *ax, void *ay, void *az, double *pot, int64_t *n_cell_inter,
                  int64_t *n_part_inter);

/* Neighbour lists of the last built tree (Sec. 2.3): for each particle i all
 * j != i with |x_i - x_j| < r_list, the distance formed and compared in FP64,
 * as original indices in ascending order.  Rows may be empty.  CSR layout:
 * offsets: device int64[n + 1], row i is idx[offsets[i] .. offsets[i+1]);
 * idx: device int32[capacity].  *total (host) receives the number of entries.
 * Synchronises the stream once to read the total.  If total > capacity the
 * call returns P3T_ERR_CAPACITY with *total and offsets set and idx untouched.
 * Row mode (mixed precision, one target per lane: group_size <= 32, or <=
 * threads_per_group): this call also sizes a context-owned scratch of int32
 * entries, about 1.3 times the lists' entries at 100 neighbours a particle;
 * for the following trees the pass that counts the neighbours (the far-force
 * walk, or the lists' own count pass when they come first) writes each neighbour
 * into its target's row there, each row having room for c + c/8 + 8 entries when
 * its particle had c neighbours at the last count of the same n particles (equal
 * rows otherwise), and the lists only sort those rows (a row that outgrew its
 * room is rebuilt by a second walk of its group).  The lists are the same either way; a
 * failed allocation of the scratch leaves row mode off. */
int p3t_neighbours(p3t_ctx *c, int64_t *offsets, int32_t *idx, int64_t capacity, int64_t *total);

/* As p3t_neighbours without the synchronisation: *total_dev is a device
 * int64 written on the stream.  If the total exceeds capacity no entry is
 * written and P3T_ERR_CAPACITY is latched for the next synchronising call. */
int p3t_neighbours_async(p3t_ctx *c, int64_t *offsets, int32_t *idx, int64_t capacity,
                         int64_t *total_dev);

/* Leapfrog kick of Eq. 12, v += (dt/2) a, for the n particles of the last
 * built tree.  dt is the regular step Delta t_reg.  ax, ay, az: device arrays
 * of float (P3T_FP32_MIXED) or double (P3T_FP64) as written by p3t_far_force;
 * vx, vy, vz: device double[n], updated in place.  Arithmetic in FP64. */
int p3t_kick(p3t_ctx *c, double dt, const void *ax, const void *ay, const void *az, double *vx,
             double *vy, double *vz);

/* Drift x += dt v over n particles (device FP64 arrays).  Not part of the
 * paper's regular step: a stand-in for the Hermite integration that moves
 * the particles between regular steps in benchmarks. */
int p3t_drift(p3t_ctx *c, int64_t n, double dt, double *x, double *y, double *z, const double *vx,
              const double *vy, const double *vz);

/* One whole regular step from HOST memory, the paper's REGF + RKICK boundary
 * (Sec. 2.4, Eq. 12): copy x, y, z, m, vx, vy, vz (host double[n]) to the
 * device, build, neighbours, far force, kick, and copy back a_far (host
 * float or double[n] per precision, SoA ax/ay/az), the kicked velocities
 * (in place in vx, vy, vz) and the neighbour lists (host int64 offsets[n+1],
 * int32 idx[capacity]).  The lists are copied on a second stream of the
 * context while the far force runs; the call synchronises both streams
 * before it returns.  Page-locked host memory gives full copy bandwidth
 * (and is needed for the copy to overlap the far force).  *total receives the neighbour count; P3T_ERR_CAPACITY as
 * in p3t_neighbours (velocities are then kicked but idx is not written). */
int p3t_step_host(p3t_ctx *c, int64_t n, double dt, const double *x, const double *y,
                  const double *z, const double *m, double *vx, double *vy, double *vz, void *ax,
                  void *ay, void *az, int64_t *offsets, int32_t *idx, int64_t capacity,
                  int64_t *total);

/* Synchronise the stream and return the first latched device error (then
 * clear it), or the first CUDA error. */
int p3t_status(p3t_ctx *c);

/* Sizes of the last built tree (synchronises): particles, nodes, groups and
 * the deepest level; any pointer may be NULL. */
int p3t_tree_info(p3t_ctx *c, int64_t *n, int64_t *n_nodes, int64_t *n_groups, int32_t *depth);

/* Copy the last built tree into caller device buffers for inspection (any
 * pointer may be NULL).  Particle arrays have n entries in sorted order:
 * keys (uint64), perm (int32 sorted -> original).  Node arrays have n_nodes
 * entries in breadth-first order: level, first, count, child (first child or
 * -1), nchild (int32); M (double); com, lo, hi (double, n_nodes x 3
 * row-major); Q (double, n_nodes x 6 as xx, xy, xz, yy, yz, zz; FP32 values
 * widened in P3T_FP32_MIXED); ropen2 (double).  Group arrays have n_groups
 * entries in particle order: g_first, g_count (int32). */
int p3t_export_tree(p3t_ctx *c, uint64_t *keys, int32_t *perm, int32_t *level, int32_t *first,
                    int32_t *count, int32_t *child, int32_t *nchild, double *M, double *com,
                    double *Q, double *lo, double *hi, double *ropen2, int32_t *g_first,
                    int32_t *g_count);

/* Per-group interaction counts of the last p3t_far_force (device int64
 * n_groups each, in group order): accepted cells and source particles in
 * opened leaves.  Filled only when the walk ran after p3t_set_debug(c, 1). */
int p3t_group_counts(p3t_ctx *c, int64_t *n_cell, int64_t *n_part);

/* Irregular (neighbour) force F_I of Eq. 1 and its time derivative (Eq. 2) of
 * every particle, summed over the particle's neighbour row: the near side of
 * the changeover (K = 1 - W of Eq. 6) that the Hermite integrator needs.
 *   F_I,i     = sum_j K m_j d / r^3
 *   dF_I,i/dt = sum_j m_j [K (u / r^3 - 3 (d.u) d / r^5) + Kdot d / r^3]
 * with d = x_j - x_i, u = v_j - v_i (attraction), Kdot = dK/dt =
 * -dW/dx (d.u) / (r (r_out - r_in)) (the exact derivative of Eq. 1; Eq. 2 as
 * printed drops m_j and K from its middle term and Eq. 7 prints K' with the
 * opposite sign).  Pairs at r = 0 and at r >= r_out contribute nothing, so rows
 * must hold every j with r < r_out (r_list >= r_out).
 * Arguments (device, original order, n particles): offsets int64[n+1] and idx
 * int32 (row i = idx[offsets[i] .. offsets[i+1]), indices in [0, n)), x, y, z,
 * m, vx, vy, vz double[n]; outputs f* (F_I) and j* (dF_I/dt) double[n].  r_in
 * and r_out are the context's, or each particle's cluster radii after a
 * p3t_build_tree_batch with cluster parameters of these n particles.  The
 * context's precision selects the arithmetic: P3T_FP64 repeats the FP64
 * operations of the definition pair by pair; P3T_FP32_MIXED forms d and u in
 * FP64 and evaluates each pair in FP32 (through double-single splits of every
 * position and velocity, made once per call in a scratch buffer of the context
 * of 64 bytes per particle, allocated on first use).  Positions and velocities
 * may differ from those the tree was built on (predicted states).  Requires a
 * built tree of the same n particles (P3T_ERR_ORDER); an index outside [0, n)
 * latches P3T_ERR_INVALID_INPUT and is skipped.  Asynchronous on the context's
 * stream (except the first mixed call, which allocates). */
int p3t_irregular(p3t_ctx *c, int64_t n, const int64_t *offsets, const int32_t *idx,
                  const double *x, const double *y, const double *z, const double *m,
                  const double *vx, const double *vy, const double *vz, double *fx, double *fy,
                  double *fz, double *jx, double *jy, double *jz);

/* ---- core quantities (Sec. 4) -------------------------------------------
 * The core radius, density and membership are estimated from the 6 nearest
 * neighbours of a random sample of min(N, sqrt(5000 N)) particles found by a
 * brute-force search (Sec. 4), with the density estimator and density-weighted
 * averages of Casertano & Hut, which the paper cites without printing.
 *
 * p3t_sample_knn6: for each sampled particle (sample: device int32[s], original
 * indices drawn by the caller) its 6 nearest other particles among the n
 * particles of the last p3t_build_tree (one cluster; positions of that build),
 * by exact FP64 squared distance (dx*dx + dy*dy) + dz*dz, ties broken by the
 * smaller original index, ascending: nn_idx device int32[s*6] (original
 * indices; -1 where fewer than 6 exist), nn_d2 device double[s*6] (inf there).
 * The search walks the built tree, pruning nodes whose box lies beyond an
 * upper bound of the 6th distance; the lists equal those of a brute-force
 * search.  Errors: P3T_ERR_ORDER without a one-cluster tree of these n
 * particles; a sample index outside [0, n) latches P3T_ERR_INVALID_INPUT (its
 * row is left unset).
 *
 * p3t_sample_knn6_brute: the same lists by the paper's brute-force search,
 * every sampled particle against every particle.  Uses a scratch buffer of the
 * context (allocated on first use, ~72 bytes per sampled particle and chunk of
 * candidates).  Same arguments and errors.
 *
 * p3t_core_quantities: from those neighbours (device arrays in original order
 * x, y, z, m of n particles): rho[t] = 3 (mass of the 5 nearest) / (4 pi r_6^3)
 * per sampled particle, then out (device double[6]) = {density centre x, y, z,
 * core radius sqrt(sum rho^2 |x - x_d|^2 / sum rho^2), core density
 * sum rho^2 / sum rho, number of particles within the core radius}; a sampled
 * particle with fewer than 6 neighbours (n < 7) gets rho = 0.  Requires
 * a context that has built a tree (its metadata block holds a counter).
 * Both calls are asynchronous on the context's stream. */
int p3t_sample_knn6(p3t_ctx *c, int64_t n, int64_t s, const int32_t *sample, int32_t *nn_idx,
                    double *nn_d2);
int p3t_sample_knn6_brute(p3t_ctx *c, int64_t n, int64_t s, const int32_t *sample, int32_t *nn_idx,
                          double *nn_d2);
int p3t_core_quantities(p3t_ctx *c, int64_t n, const double *x, const double *y, const double *z,
                        const double *m, int64_t s, const int32_t *sample, const int32_t *nn_idx,
                        const double *nn_d2, double *rho, double *out);

/* Number of exact FP64 decisions the FP32 filters have handed over (opening
 * and box tests that fell inside their error bands) since the last build;
 * host int64.  A diagnostic of the filters' efficiency: the results do not
 * depend on it.  Synchronises the context's stream. */
int p3t_filter_fallbacks(p3t_ctx *c, int64_t *count);

/* Row mode of the neighbour lists (see p3t_neighbours), host values, no
 * synchronisation: *row_cap = the row scratch's entries per particle, on average
 * (0: row mode off); *rows_valid = 1 if the last walk on the current tree
 * wrote its rows, so that the next lists only sort them.  Either pointer may
 * be NULL. */
int p3t_row_mode(p3t_ctx *c, int32_t *row_cap, int32_t *rows_valid);

/* 1: record per-group counts in the walk (slightly slower); 0: off (default). */
int p3t_set_debug(p3t_ctx *c, int on);

/* Bounded device-side waits (the look-back of the device-wide prefix sums in
 * the sort, the topology, the groups and the neighbour offsets; no part of the
 * paper's method, a guard that keeps every kernel finite): a wait that has
 * polled `polls` times without its predecessor publishing gives up, latches
 * P3T_ERR_TIMEOUT (returned by the next synchronising call, e.g. p3t_status)
 * and lets the kernel finish with a partial result.  polls = 0 restores the
 * default, 2^22 polls (about 1.1 s of backoff sleeps).  Synchronises the
 * context's stream when the device block already exists.  Errors:
 * P3T_ERR_INVALID_ARG (polls < 0), P3T_ERR_CUDA. */
int p3t_set_spin_limit(p3t_ctx *c, int64_t polls);

/* Test hook for the bounded waits: runs one exclusive prefix sum over n
 * entries of the context's neighbour-count buffer in which tile 0's work item is
 * never handed out, so the tiles after it wait on a status word that nothing
 * writes until their spin limit (p3t_set_spin_limit) runs out.  Synchronises
 * and returns the context's status: P3T_ERR_TIMEOUT is the expected outcome,
 * read and cleared like any latched error, after which the context is usable.
 * Needs scratch for n particles (p3t_reserve or a build; else P3T_ERR_ORDER);
 * invalidates the cached neighbour counts (the next p3t_neighbours recounts). */
int p3t_debug_stalled_scan(p3t_ctx *c, int64_t n);

/* Static description of an error code. */
const char *p3t_error_string(int code);

/* Size the context's device scratch for n particles in n_clusters clusters
 * now, so that later builds up to that size allocate nothing (a serving loop
 * pre-sizes its contexts this way).  May synchronise the context's stream when
 * it reallocates.  Errors: P3T_ERR_INVALID_ARG, P3T_ERR_OOM. */
int p3t_reserve(p3t_ctx *c, int64_t n, int32_t n_clusters);

/* Device bytes a context with parameters p allocates for n particles in
 * n_clusters clusters (scratch plus cluster table); *bytes is host memory.
 * For admission by device-memory footprint.  Errors: P3T_ERR_INVALID_ARG. */
int p3t_scratch_bytes(const p3t_params *p, int64_t n, int32_t n_clusters, int64_t *bytes);

/* ---- one whole step as a CUDA graph -------------------------------------
 * The distant-force step of the P3T scheme (Sec. 2.4, Eq. 12): tree build,
 * far force, neighbour lists, kick and (optionally) the drift that stands in
 * for the Hermite side, recorded once into a CUDA graph and replayed with a
 * single launch per step.  Batching many clusters this way leaves one graph
 * launch per step for the whole ensemble (one persistent walk kernel inside).
 *
 * p3t_step_args (all pointers device pointers owned by the caller; they and
 * every size are baked into the graph at capture, so replays must use the same
 * buffers, whose contents may change between launches):
 *   n_clusters, n, seg_offsets, cluster_params: as p3t_build_tree_batch;
 *     seg_offsets may be null with n_clusters == 1 (then p3t_build_tree).
 *   x, y, z, m: positions and masses (drift updates x, y, z in place).
 *   vx, vy, vz: velocities kicked by kick_dt (Eq. 12), or all null: no kick.
 *   ax, ay, az, pot, n_cell, n_part: as p3t_far_force.
 *   offsets, idx, capacity, total: as p3t_neighbours_async; offsets null: no lists.
 *   drift_dt: x += drift_dt * v after the kick; 0: no drift.
 *   events: five optional cudaEvent_t handles (null entries skipped), recorded
 *     into the graph as event nodes at the start of the step, after the build,
 *     after the far force, after the lists and at the end (lists_first: after the
 *     lists, then after the far force), so that one launch can be timed phase by
 *     phase (cudaEventElapsedTime after it completes).
 *   lists_first: 0, the far force before the lists (its walk counts the
 *     neighbours and, in row mode, writes their rows); 1, the lists first (their
 *     own count pass, then a far force that computes forces only), which is
 *     faster when the rows are short.  Both orders give the same lists, and
 *     the same forces bit for bit unless a cluster lists neighbours beyond its
 *     r_out (then to rounding: the counting walk stages that cluster's
 *     neighbour-only sources with mass 0, which changes how the pair sums are
 *     split).
 * p3t_graph_capture sizes the context's scratch for the step first, then
 * records the step on a private stream, so nothing runs or allocates during
 * capture; the graph is launched on the context's stream.  The context's
 * host-side state after capture is that of before it: launch the graph
 * before further entry points rely on its tree.  A launch restores the
 * state the captured step leaves (so p3t_export_tree, p3t_tree_info ...
 * describe the graph's tree after it).  If the context's scratch is
 * reallocated later (a larger eager build), the graph's pointers are stale and
 * p3t_graph_launch returns P3T_ERR_ORDER.  Destroy a context's graphs before
 * the context.  Errors: those of the captured
 * calls, P3T_ERR_INVALID_ARG for inconsistent arguments, P3T_ERR_CUDA when
 * capture or instantiation fails.  Device-side errors (capacity, invalid
 * input) latch as for the eager calls; read them with p3t_status. */
typedef struct p3t_graph p3t_graph;
typedef struct {
    int32_t n_clusters;
    int64_t n;
    const int64_t *seg_offsets;
    const double *cluster_params;
    double *x, *y, *z;
    const double *m;
    double *vx, *vy, *vz;
    void *ax, *ay, *az;
    double *pot;
    int64_t *n_cell, *n_part;
    int64_t *offsets;
    int32_t *idx;
    int64_t capacity;
    int64_t *total;
    double kick_dt;
    double drift_dt;
    void *events[5];
    int32_t lists_first;
} p3t_step_args;
int p3t_graph_capture(p3t_ctx *c, const p3t_step_args *a, p3t_graph **out);
int p3t_graph_launch(p3t_graph *g);
int p3t_graph_destroy(p3t_graph *g);

/* ---- serving: batches of resident clusters --------------------------------
 * A server keeps many clusters resident in one device arena and steps an
 * arbitrary subset of them together: their particles are gathered into a
 * contiguous staging area, stepped with one batched call sequence
 * (p3t_build_tree_batch ... p3t_kick, one persistent walk for all of them),
 * and the results scattered back.  A batch of n_seg clusters is described by
 * batch_off (device int64[n_seg + 1], ascending, batch_off[0] = 0: the
 * segment offsets in the staging area, i.e. the batch's seg_offsets) and
 * arena_off (device int64[n_seg]: each cluster's first particle in the arena).
 * n_batch = batch_off[n_seg] (host copy; it sizes the grid).
 *
 * p3t_batch_move copies n_arrays (<= 10) parallel arrays between arena and
 * staging: element i of the staging area <-> element arena_off[k] + (i -
 * batch_off[k]) of the arena, k the segment holding i; to_batch = 1 gathers
 * (arena -> staging), 0 scatters back.  Elements are 4 or 8 bytes
 * (elem_bytes).  Segments must not overlap in the arena.
 *
 * p3t_batch_scatter_neighbours turns the batch's neighbour lists (offsets
 * int64[n_batch + 1], idx int32 with batch indices, capacity max_entries) into
 * cluster-local lists in the arena: cluster k's n_k + 1 row offsets start at
 * arena_offsets[row_arena_off[k]] (from 0), its entries at
 * arena_idx[ent_arena_off[k]] with indices relative to the cluster (0 .. n_k -
 * 1).  A cluster whose entries exceed ent_arena_cap[k], or a batch whose
 * total exceeds max_entries, sets *status (device int32) to P3T_ERR_CAPACITY
 * and is not copied.
 * Both run on `cuda_stream` without synchronising; they return
 * P3T_ERR_INVALID_ARG for bad arguments and P3T_ERR_CUDA for launch errors. */
typedef struct {
    void *arena;
    void *batch;
    int32_t elem_bytes;
} p3t_seg_array;
int p3t_batch_move(void *cuda_stream, int32_t n_seg, int64_t n_batch, const int64_t *batch_off,
                   const int64_t *arena_off, int32_t n_arrays, const p3t_seg_array *arrays,
                   int32_t to_batch);
int p3t_batch_scatter_neighbours(void *cuda_stream, int32_t n_seg, int64_t n_batch,
                                 int64_t max_entries, const int64_t *batch_off,
                                 const int64_t *row_arena_off, const int64_t *ent_arena_off,
                                 const int64_t *ent_arena_cap, const int64_t *offsets,
                                 const int32_t *idx, int64_t *arena_offsets, int32_t *arena_idx,
                                 int32_t *status);

/* Morton order of n particles WITHOUT ANY DEVICE ALLOCATION.  The paper has
 * no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc where they need it -- a host whose own memory pool already owns
 * the GPU's memory and hands out only buffers it allocated, or a loop that
 * must not allocate once running because an allocation can synchronise the
 * device and stall other streams.
 * It computes what p3t_build_tree computes first: the bounding cube, the
 * 63-bit Morton keys and the stable sort by (key, original index).  Outputs:
 * keys (device uint64[n], ascending) and perm (device int32[n], sorted
 * position -> original index); inputs x, y, z, m are device double[n] as in
 * p3t_build_tree.  All scratch memory lives in one static device array of the
 * library sized for P3T_NOALLOC_MAX_N particles (about 0.8 MB, held by every
 * GPU that loads the library until the process exits); n above that returns
 * P3T_ERR_CAPACITY, n <= 0 or a null pointer P3T_ERR_INVALID_ARG.
 * The first call on a device looks up the array's device address on the
 * current device; make that first call before any stream capture.  Every
 * call, the first and each later one, runs on `cuda_stream` and ends by
 * synchronising it to read its status; it returns P3T_ERR_INVALID_INPUT for
 * non-finite or negative inputs as p3t_build_tree would, and a latched error
 * never carries over into the next call.  Every call
 * shares the one array: calls that overlap on a GPU (other streams or host
 * threads at the same time) race on it. */
#define P3T_NOALLOC_MAX_N 65536
int p3t_morton_order_noalloc(int64_t n, const double *x, const double *y, const double *z,
                             const double *m, uint64_t *keys, int32_t *perm, void *cuda_stream);

/* ---- one cluster over several ranks (multi-GPU domain decomposition) -------
 * The multi-GPU force calculator the paper leaves as future work (Sec. 4):
 * rank r holds the particles whose Morton keys (rules 1-3, on the bounding box
 * of the whole cluster) lie in [b_r, b_r+1).  The splitters b are cell
 * boundaries of the global octree chosen so that every cell straddling one (a
 * "top cell") holds more than max(16 G, leaf_cap) particles; the global tree is
 * then the top cells plus complete subtrees that each belong to one rank, and
 * every walk group of the whole cluster lies in one rank.  Each rank builds its
 * part (p3t_build_tree_range), ships every other rank the part of its subtrees
 * that the receiver's domain box opens (p3t_let_export: the locally essential
 * tree, by rule 8 with r_out, or r_list when that is larger), and joins what it
 * receives (p3t_tree_join).  Its groups then walk the global tree: interaction
 * lists, forces and neighbour rows equal those of one build of the whole cluster,
 * neighbour rows holding global indices.  The caller moves the data between
 * ranks (NCCL or any transport): every array below is device memory of this
 * rank unless marked host.  These calls synchronise the context's stream.
 *
 * p3t_local_bbox: exact min xyz, max xyz (host double[6]) of n device points.
 * p3t_key_range_counts: counts[r] (host) = number of the n points whose key, in
 *   the cube of global_box (host double[6], the ranks' boxes reduced), lies in
 *   [lo[r], hi[r]) (host uint64, at most 1024 intervals).
 * p3t_partition: the n particles packed by destination rank, rank r taking the
 *   keys in [bounds[r], bounds[r+1]) (host, n_ranks + 1 bounds, bounds[0] = 0,
 *   bounds[n_ranks] = 2^63): every src[a] (n 8-byte elements) is copied to dst[a]
 *   (n elements), rank 0's particles first, each rank's in their input order;
 *   counts (host, n_ranks) receives the particles per rank.
 * p3t_build_tree_range: the rank's tree of its n particles (all inside its key
 *   range), on the cube and frame of global_box (host), with the n_top top cells
 *   (host: first key and level of each, at most 256, levels < 21) split whatever
 *   their local count and never cut into groups; gid (device int64[n], < 2^31) the
 *   particles' global indices, which order equal keys and fill neighbour rows.
 *   Errors as p3t_build_tree; P3T_ERR_INVALID_INPUT when a particle lies outside
 *   global_box.
 * p3t_subtree_boxes: after p3t_build_tree_range, the exact boxes (host,
 *   min xyz, max xyz, 6 doubles each, at most cap) of this rank's subtree roots,
 *   the nodes below the top cells; every walk group of the rank lies in one of
 *   them.  *n_boxes = their number (P3T_ERR_CAPACITY when above cap).
 * p3t_let_export: after p3t_build_tree_range, the locally essential tree of this
 *   rank's subtrees for a receiver whose subtree boxes are boxes (host, n_boxes x
 *   6 doubles, at most 4096) and radius r_halo (max(r_out, r_list)): a node is
 *   shipped opened iff rule 8 opens it for one of the boxes (so for any group of
 *   the receiver that opens it); *n_roots subtree roots first, then the opened
 *   nodes' children level by level, as *n_nodes records of P3T_LET_NODE_BYTES, and
 *   the *n_parts particles of opened leaves (P3T_LET_PART_BYTES each).  With
 *   cap_nodes = 0 only the sizes are returned (P3T_ERR_CAPACITY when they exceed
 *   the capacities, sizes still set).
 * p3t_tree_join: after p3t_build_tree_range, the rank's tree joined with the
 *   locally essential trees of the n_let other ranks (device buffers as exported,
 *   with their sizes and root counts; host arrays of n_let): the top cells'
 *   moments are formed from the joined children (rule 6), and p3t_far_force,
 *   p3t_neighbours and p3t_kick then work on the rank's own particles, in its input
 *   order.  The joined tree holds copies of the remote nodes and particles; the
 *   next build returns to the rank's own tree.  P3T_ERR_INVALID_INPUT when the
 *   subtree roots do not complete the top cells (a missing or duplicated rank). */
#define P3T_LET_NODE_BYTES 288
#define P3T_LET_PART_BYTES 96
int p3t_local_bbox(p3t_ctx *c, int64_t n, const double *x, const double *y, const double *z, double *box);
int p3t_key_range_counts(p3t_ctx *c, int64_t n, const double *x, const double *y, const double *z,
                         const double *global_box, int32_t n_ranges, const uint64_t *lo, const uint64_t *hi,
                         int64_t *counts);
int p3t_partition(p3t_ctx *c, int64_t n, const double *x, const double *y, const double *z,
                  const double *global_box, int32_t n_ranks, const uint64_t *bounds, int32_t n_arrays,
                  const void *const *src, void *const *dst, int64_t *counts);
int p3t_build_tree_range(p3t_ctx *c, int64_t n, const double *x, const double *y, const double *z,
                         const double *m, const int64_t *gid, const double *global_box, int32_t n_top,
                         const uint64_t *top_key, const int32_t *top_level);
int p3t_subtree_boxes(p3t_ctx *c, int32_t cap, double *boxes, int32_t *n_boxes);
int p3t_let_export(p3t_ctx *c, int32_t n_boxes, const double *boxes, double r_halo, int64_t cap_nodes, void *nodes,
                   int64_t cap_parts, void *parts, int64_t *n_nodes, int64_t *n_parts, int32_t *n_roots);
int p3t_tree_join(p3t_ctx *c, int32_t n_let, const void *const *let_nodes, const int64_t *let_n_nodes,
                  const int32_t *let_n_roots, const void *const *let_parts, const int64_t *let_n_parts);

#ifdef __cplusplus
}
#endif

#endif /* P3T_H */
