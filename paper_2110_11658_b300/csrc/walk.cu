// Far-force entry (p3t_far_force): picks the walk variant of walk_kernel.cuh for
// the context's precision, parameters and neighbour state.  The FP64 walk with one
// warp per group is instantiated here, the mixed walks in walk_f1.cu / walk_f2.cu
// (the two cell forms) and those with 2 and 4 warps per group in walk_wpg*.cu.
#include "walk_kernel.cuh"

namespace p3t {

// Which clusters may take the r^-5 cell term (eval_cells_x2): r_out >= 1e-7, frame
// half-size R <= 1e6 and cluster mass (the root record's) <= 1e15, all finite.  One
// block; the counts of both kinds go to Meta.cell_forms: the r^-5 walk runs when no
// cluster is outside that range, the r^-3 walk otherwise (for every cluster, so that
// the form is one per launch).
__global__ void __launch_bounds__(256) cell_forms_kernel(Tree T, unsigned int *ticket1, unsigned int *ticket2)
{
    pdl_wait();
    __shared__ int cnt[2];
    if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
    if (threadIdx.x == 0) *ticket1 = 0u, *ticket2 = 0u;  // the two walks' group tickets
    __syncthreads();
    int nf = 0, ns = 0;
    for (int c = threadIdx.x; c < T.n_clusters; c += blockDim.x) {
        Cluster &K = T.cl[c];
        const float R = (float)K.frame[3];
        const float M = T.wn[wrec(c, 3)].w;
        const bool fast = K.rout2_f >= 1e-14f && K.rout2_f < 1e30f && R >= 0.f && R <= 1e6f &&
                          M >= 0.f && M <= 1e15f;
        K.fast_cells = fast;
        nf += fast;
        ns += !fast;
    }
    if (nf) atomicAdd(&cnt[0], nf);
    if (ns) atomicAdd(&cnt[1], ns);
    __syncthreads();
    if (threadIdx.x < 2) T.meta->cell_forms[threadIdx.x] = cnt[threadIdx.x];
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
    const bool quad = P.quadrupole != 0;
    const bool want_pot = pot != nullptr;
    int e;
    // neighbour-only ranges are needed when a list radius exceeds r_out (with a
    // per-cluster table the host cannot tell, so they are compiled in)
    const bool shell = fuse_nbr && (!c->uniform_params || P.r_list > P.r_out);
    if (c->built_precision == P3T_FP64) {
        if (cudaMemsetAsync(a.ticket, 0, sizeof(unsigned int), c->stream) != cudaSuccess) return P3T_ERR_CUDA;
        e = wpg == 1 ? dispatch_tpl<double, 0, false, 0>(c, a, want_pot, quad)
                     : (wpg == 2 ? dispatch_walk_wpg<2, 0>(c, a, 0, false, want_pot, quad)
                                 : dispatch_walk_wpg<4, 0>(c, a, 0, false, want_pot, quad));
    } else {
        // the r^-5 walk, then the r^-3 walk: one of the two finds its form chosen
        // (cell_forms_kernel) and walks every group, the other returns at once
        const int nbr = !fuse_nbr ? 0 : (rows ? 2 : 1);
        WalkArgs b = a;
        b.ticket = &c->meta->tickets[24];
        e = launch_pdl(cell_forms_kernel, dim3(1), dim3(256), c->stream, c->tree, a.ticket, b.ticket) == cudaSuccess
                ? check_launch(c)
                : P3T_ERR_CUDA;
        if (!e) e = mixed_walk<1>(c, a, wpg, nbr, shell, want_pot, quad);
        if (!e) e = mixed_walk<2>(c, b, wpg, nbr, shell, want_pot, quad);
    }
    if (e == P3T_OK && fuse_nbr) {
        c->walk_counted = 1;
        c->rows_valid = rows;
        c->counts_valid = c->uniform_params;  // every cluster counted
        if (c->counts_valid) c->counts_n = c->n;
    }
    return e;
}

}  // namespace p3t
