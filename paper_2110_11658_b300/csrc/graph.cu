// One distant-force step (build, far force, neighbour lists, kick, drift) as a
// CUDA graph: the entry points of ctx.cu are recorded on a private stream and
// replayed with one launch.  Used by the ensemble and serving loops, where the
// launch overhead of ~85 kernels per step would otherwise be paid per step.
#include <cmath>
#include <new>

#include "p3t_internal.cuh"

using namespace p3t;

struct p3t_graph {
    p3t_ctx *c;
    cudaGraphExec_t exec;
    unsigned long long gen;  // context generation the pointers belong to
    HostState after;         // host-side state the captured step leaves
};

// an event node of the graph (the step's phase boundaries), if the caller gave one
static int mark(p3t_ctx *c, const p3t_step_args *a, int k)
{
    if (!a->events[k]) return P3T_OK;
    return cudaEventRecordWithFlags((cudaEvent_t)a->events[k], c->stream, cudaEventRecordExternal) ==
                   cudaSuccess
               ? P3T_OK
               : P3T_ERR_CUDA;
}

static int record_step(p3t_ctx *c, const p3t_step_args *a)
{
    int e = mark(c, a, 0);
    if (e) return e;
    e = a->seg_offsets ? p3t_build_tree_batch(c, a->n_clusters, a->n, a->seg_offsets,
                                              a->cluster_params, a->x, a->y, a->z, a->m)
                       : p3t_build_tree(c, a->n, a->x, a->y, a->z, a->m);
    if (e || (e = mark(c, a, 1))) return e;
    // the far force and the lists, in the order asked for
    for (int ph = 0; ph < 2; ph++) {
        if ((ph == 0) == (a->lists_first == 0)) {
            e = p3t_far_force(c, a->ax, a->ay, a->az, a->pot, a->n_cell, a->n_part);
        } else if (a->offsets) {
            e = p3t_neighbours_async(c, a->offsets, a->idx, a->capacity, a->total);
        }
        if (e || (e = mark(c, a, 2 + ph))) return e;
    }
    if (a->vx) {
        e = p3t_kick(c, a->kick_dt, a->ax, a->ay, a->az, a->vx, a->vy, a->vz);
        if (e) return e;
        if (a->drift_dt != 0.0) {
            e = p3t_drift(c, a->n, a->drift_dt, a->x, a->y, a->z, a->vx, a->vy, a->vz);
            if (e) return e;
        }
    }
    return mark(c, a, 4);
}

extern "C" {

int p3t_graph_capture(p3t_ctx *c, const p3t_step_args *a, p3t_graph **out)
{
    if (!c || !a || !out) return P3T_ERR_INVALID_ARG;
    *out = nullptr;
    if (a->n <= 0 || a->n >= (1LL << 31) - 1 || a->n_clusters < 1 || a->n_clusters > a->n)
        return P3T_ERR_INVALID_ARG;
    if (!a->seg_offsets && a->n_clusters != 1) return P3T_ERR_INVALID_ARG;
    if (!a->x || !a->y || !a->z || !a->m || !a->ax || !a->ay || !a->az) return P3T_ERR_INVALID_ARG;
    const bool kick = a->vx || a->vy || a->vz;
    if (kick && (!a->vx || !a->vy || !a->vz || !std::isfinite(a->kick_dt)))
        return P3T_ERR_INVALID_ARG;
    if (a->drift_dt != 0.0 && (!kick || !std::isfinite(a->drift_dt))) return P3T_ERR_INVALID_ARG;
    if (a->offsets && (!a->total || a->capacity < 0 || (a->capacity > 0 && !a->idx)))
        return P3T_ERR_INVALID_ARG;
    if (a->lists_first != 0 && a->lists_first != 1) return P3T_ERR_INVALID_ARG;
    // scratch first: nothing may allocate while the stream is being captured
    int e = reserve(c, a->n, a->n_clusters);
    if (e) return e;
    p3t_graph *g = new (std::nothrow) p3t_graph();
    if (!g) return P3T_ERR_OOM;
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return P3T_ERR_CUDA;
    }
    const HostState before = save_state(c);
    cudaStream_t saved = c->stream;
    c->stream = cap;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        e = P3T_ERR_CUDA;
    } else {
        e = record_step(c, a);
        const cudaError_t ce = cudaStreamEndCapture(cap, &graph);
        if (!e && ce != cudaSuccess) e = P3T_ERR_CUDA;
    }
    c->stream = saved;
    g->after = save_state(c);
    restore_state(c, before);  // nothing of the captured step has run yet
    if (!e && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) e = P3T_ERR_CUDA;
    // upload now, so that the first launch does not pay for it
    if (!e && cudaGraphUpload(g->exec, c->stream) != cudaSuccess) e = P3T_ERR_CUDA;
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (e) {
        cudaGetLastError();
        delete g;
        return e;
    }
    g->c = c;
    g->gen = c->gen;
    *out = g;
    return P3T_OK;
}

int p3t_graph_launch(p3t_graph *g)
{
    if (!g || !g->c) return P3T_ERR_INVALID_ARG;
    p3t_ctx *c = g->c;
    if (g->gen != c->gen) return P3T_ERR_ORDER;  // scratch moved since capture
    if (cudaGraphLaunch(g->exec, c->stream) != cudaSuccess) {
        cudaGetLastError();
        return P3T_ERR_CUDA;
    }
    restore_state(c, g->after);
    return P3T_OK;
}

int p3t_graph_destroy(p3t_graph *g)
{
    if (!g) return P3T_ERR_INVALID_ARG;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    delete g;
    return P3T_OK;
}

}  // extern "C"
