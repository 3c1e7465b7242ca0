// Batched shadow XL-BOMD steps of several systems (the serving loop's MD work).
//
// A serving GPU holds many small periodic systems at once, each with its own
// context (neighbour list, PME mesh, shadow charge history resident on the
// device).  Stepping them one call at a time costs every system a host
// synchronisation (the skin check) and a graph launch per step.  A batch step
// instead queues every member's integrator update and displacement kernel on
// one stream, synchronises once for all of them, rebuilds the lists of the
// members past skin / 2, and launches ONE CUDA graph whose parallel branches are
// the members' captured evaluations (charges, forces, Krylov kernel, second
// half kick).  The parent graph is cached and rebuilt only when the set of
// members or one of their step graphs changes.  Each member runs exactly the
// kernels of its own qeq_shadow_step, so results equal separate steps.

#include <algorithm>
#include <vector>

#include "internal.cuh"

struct qeq_batch {
    std::vector<qeq_ctx *> members;  // members of the cached parent graph, in order
    std::vector<uint64_t> gens;      // their step-graph generations at that time
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double *h_d2 = nullptr;          // pinned: one displacement check per member
    int h_cap = 0;
    int64_t parent_builds = 0;
    int64_t launches = 0;
};

namespace qeq {
namespace {

void drop_parent(qeq_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->members.clear();
    b->gens.clear();
}

int reserve_host(qeq_batch *b, int n) {
    if (n <= b->h_cap) return QEQ_OK;
    const int cap = std::max(n, 2 * b->h_cap + 16);
    if (b->h_d2) cudaFreeHost(b->h_d2);
    b->h_d2 = nullptr;
    b->h_cap = 0;
    if (cudaMallocHost(&b->h_d2, sizeof(double) * cap) != cudaSuccess) {
        cudaGetLastError();
        return set_error(nullptr, QEQ_ERR_NOMEM, "batch step: pinned host buffer");
    }
    b->h_cap = cap;
    return QEQ_OK;
}

// The parent graph: one child-graph node per member, no edges between them.
int build_parent(qeq_batch *b, const std::vector<qeq_ctx *> &m) {
    drop_parent(b);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    for (size_t k = 0; k < m.size() && e == cudaSuccess; ++k) {
        cudaGraphNode_t node;
        e = cudaGraphAddChildGraphNode(&node, g, nullptr, 0, m[k]->step_graph);
    }
    cudaGraphExec_t x = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, cudaGraphInstantiateFlagUseNodePriority);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return set_error(nullptr, QEQ_ERR_CUDA, "batch step: parent graph: %s", cudaGetErrorString(e));
    }
    b->graph = g;
    b->exec = x;
    b->members = m;
    for (qeq_ctx *c : m) b->gens.push_back(c->graph_gen);
    b->parent_builds++;
    return QEQ_OK;
}

}  // namespace
}  // namespace qeq

using namespace qeq;

QEQ_API int qeq_batch_create(qeq_batch **out) {
    if (!out) return set_error(nullptr, QEQ_ERR_INVALID, "batch create: NULL output");
    *out = new (std::nothrow) qeq_batch();
    return *out ? QEQ_OK : set_error(nullptr, QEQ_ERR_NOMEM, "batch create: host allocation");
}

QEQ_API void qeq_batch_destroy(qeq_batch *b) {
    if (!b) return;
    drop_parent(b);
    if (b->h_d2) cudaFreeHost(b->h_d2);
    delete b;
}

QEQ_API int qeq_batch_stats(const qeq_batch *b, int64_t *out2) {
    if (!b || !out2) return QEQ_ERR_INVALID;
    out2[0] = b->parent_builds;
    out2[1] = b->launches;
    return QEQ_OK;
}

QEQ_API int qeq_batch_step(qeq_batch *b, int32_t n, qeq_ctx *const *ctxs, const qeq_md_params *prms,
                           qeq_md_state *sts, void *stream) {
    NvtxRange nvtx_range("qeq_batch_step");
    if (!b || n < 0 || (n > 0 && (!ctxs || !prms || !sts)))
        return set_error(nullptr, QEQ_ERR_INVALID, "batch step: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (!s) return set_error(nullptr, QEQ_ERR_INVALID, "batch step: needs a non-default stream");
    for (int32_t k = 0; k < n; ++k) {
        qeq_ctx *c = ctxs[k];
        if (!c) return set_error(nullptr, QEQ_ERR_INVALID, "batch step: member %d is NULL", k);
        for (int32_t j = 0; j < k; ++j)
            if (ctxs[j] == c)
                return set_error(nullptr, QEQ_ERR_INVALID, "batch step: member %d repeated", k);
        int rc = check_md(c, &prms[k], &sts[k]);
        if (rc) return rc;
        if (!c->list_valid) return set_error(c, QEQ_ERR_NOLIST, "call qeq_shadow_init first");
    }
    int rc = reserve_host(b, n);
    if (rc) return rc;
    // 1. every member's kick, drift and n update, and its displacement check.
    //    A member's kernels run beside the other members' (parallel branches of
    //    the parent graph), so none waits on the device for its predecessor
    //    (pdl off: its step graph is captured again without the attribute)
    for (int32_t k = 0; k < n; ++k) {
        ctxs[k]->pdl = false;
        rc = shadow_advance_queue(ctxs[k], &prms[k], &sts[k], s);
        if (rc) return rc;
        cudaMemcpyAsync(&b->h_d2[k], ctxs[k]->scal + kScMaxDisp2, sizeof(double),
                        cudaMemcpyDeviceToHost, s);
    }
    // 2. one synchronisation for all skin checks; rebuild where an atom moved
    //    more than skin / 2
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(nullptr, QEQ_ERR_CUDA, "batch step: skin checks: %s", cudaGetErrorString(e));
    }
    std::vector<qeq_ctx *> graphed;
    graphed.reserve(n);
    for (int32_t k = 0; k < n; ++k) {
        qeq_ctx *c = ctxs[k];
        const double half = 0.5 * c->p.skin;
        if (!(b->h_d2[k] <= half * half)) {
            rc = nl_build(c, sts[k].R, s);
            if (rc) return rc;
        }
    }
    // 3. the evaluations: members that replay a graph go into the parent graph,
    //    the others (tolerance-driven rank, callback, profiler) run kernel by kernel
    for (int32_t k = 0; k < n; ++k) {
        qeq_ctx *c = ctxs[k];
        if (step_graphable(c, s)) {
            rc = ensure_step_graph(c, &prms[k], &sts[k], s);
            if (rc) return rc;
            graphed.push_back(c);
        } else {
            rc = shadow_evaluate(c, &prms[k], &sts[k], s);
            if (!rc) rc = shadow_finish(c, &prms[k], &sts[k], true, s, true);
            if (rc) return rc;
        }
    }
    if (graphed.empty()) return QEQ_OK;
    bool same = b->exec && b->members == graphed;
    for (size_t k = 0; k < graphed.size() && same; ++k) same = b->gens[k] == graphed[k]->graph_gen;
    if (!same) {
        rc = build_parent(b, graphed);
        if (rc) return rc;
    }
    for (qeq_ctx *c : graphed) count_step_replay(c);
    b->launches++;
    e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(nullptr, QEQ_ERR_CUDA, "batch step: graph launch: %s", cudaGetErrorString(e));
    }
    return QEQ_OK;
}
