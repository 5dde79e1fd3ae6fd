// Far-force entry (p3t_far_force): picks the walk variant of walk_kernel.cuh for
// the context's precision, parameters and neighbour state.  Walks with one warp per
// group are instantiated here, those with 2 and 4 warps per group in walk_wpg.cu.
#include "walk_kernel.cuh"

namespace p3t {

extern template int dispatch_walk_wpg<2>(p3t_ctx *, const WalkArgs &, bool, int, bool, bool, bool);
extern template int dispatch_walk_wpg<4>(p3t_ctx *, const WalkArgs &, bool, int, bool, bool, bool);

template <typename Real, int NBR, bool SHELL = false>
static int dispatch_tpl(p3t_ctx *c, const WalkArgs &a, bool pot, bool quad)
{
    const int G = c->prm.group_size;
    if constexpr (NBR == 2) return dispatch_pq<Real, 1, 2, SHELL, 1>(c, a, pot, quad);  // G <= 32
    if (G <= 32) return dispatch_pq<Real, 1, NBR, SHELL, 1>(c, a, pot, quad);
    if (G <= 64) return dispatch_pq<Real, 2, NBR, SHELL, 1>(c, a, pot, quad);
    return dispatch_pq<Real, 4, NBR, SHELL, 1>(c, a, pot, quad);
}

int far_force(p3t_ctx *c, void *ax, void *ay, void *az, double *pot, int64_t *nc, int64_t *np)
{
    const p3t_params &P = c->prm;
    WalkArgs a;
    a.T = c->tree;
    a.tile = P.tile;
    a.ax = ax, a.ay = ay, a.az = az;
    a.pot = pot;
    a.n_cell = (unsigned long long *)nc;
    a.n_part = (unsigned long long *)np;
    a.grp_cells = c->debug ? (long long *)c->grp_cells : nullptr;
    a.grp_parts = c->debug ? (long long *)c->grp_parts : nullptr;
    a.ticket = &c->meta->tickets[22];
    // the mixed walk counts the neighbours of every cluster with a list radius
    // (beyond r_out through neighbour-only ranges); with a per-cluster table the
    // walk decides per group.  Counts already taken for this tree (p3t_neighbours
    // ran first) are not taken again.
    const bool fuse_nbr = !c->counts_valid && c->built_precision == P3T_FP32_MIXED &&
                          (!c->uniform_params || P.r_list > 0.0);
    a.nbr_count = fuse_nbr ? c->nbr_count : nullptr;
    // row mode: the walk also writes each neighbour it counts into the row scratch,
    // so that p3t_neighbours only sorts (one target per lane)
    const int wpg = P.threads_per_group / 32;  // warps per group
    // (rows laid out from the last counts of these particles, before the walk
    // overwrites them)
    const bool rows = fuse_nbr && P.group_size <= 32 * wpg && prepare_rows(c);
    a.rows = rows ? c->row_scratch : nullptr;
    a.row_off = c->row_off;
    a.row_entries = (long long)c->row_scratch_entries;
    if (cudaMemsetAsync(a.ticket, 0, sizeof(unsigned int), c->stream) != cudaSuccess)
        return P3T_ERR_CUDA;
    const bool quad = P.quadrupole != 0;
    const bool want_pot = pot != nullptr;
    int e;
    // neighbour-only ranges are needed when a list radius exceeds r_out (with a
    // per-cluster table the host cannot tell, so they are compiled in)
    const bool shell = fuse_nbr && (!c->uniform_params || P.r_list > P.r_out);
    if (wpg > 1) {
        const bool fp64 = c->built_precision == P3T_FP64;
        const int nbr = fp64 || !fuse_nbr ? 0 : (rows ? 2 : 1);
        e = wpg == 2 ? dispatch_walk_wpg<2>(c, a, fp64, nbr, shell, want_pot, quad)
                     : dispatch_walk_wpg<4>(c, a, fp64, nbr, shell, want_pot, quad);
    } else if (c->built_precision == P3T_FP64)
        e = dispatch_tpl<double, 0>(c, a, want_pot, quad);
    else if (shell)
        e = rows ? dispatch_tpl<float, 2, true>(c, a, want_pot, quad)
                 : dispatch_tpl<float, 1, true>(c, a, want_pot, quad);
    else if (fuse_nbr)
        e = rows ? dispatch_tpl<float, 2>(c, a, want_pot, quad)
                 : dispatch_tpl<float, 1>(c, a, want_pot, quad);
    else
        e = dispatch_tpl<float, 0>(c, a, want_pot, quad);
    if (e == P3T_OK && fuse_nbr) {
        c->walk_counted = 1;
        c->rows_valid = rows;
        c->counts_valid = c->uniform_params;  // every cluster counted
        if (c->counts_valid) c->counts_n = c->n;
    }
    return e;
}

}  // namespace p3t
