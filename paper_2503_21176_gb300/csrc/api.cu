// Exported C entry points of include/qeq.h: parameter checks, context lifetime,
// error reporting, and the thin wrappers around the neighbour, Coulomb and
// shadow-step code.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>

#include "internal.cuh"

namespace {
thread_local std::string g_create_error;
}

namespace qeq {

int set_error(qeq_ctx *ctx, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx)
        ctx->err = buf;
    else
        g_create_error = buf;
    return code;
}

int cuda_check(qeq_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return QEQ_OK;
    cudaGetLastError();
    return set_error(ctx, QEQ_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int dev_alloc(qeq_ctx *ctx, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = ctx->async_alloc ? cudaMallocAsync(p, bytes, ctx->alloc_stream)
                                     : cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(ctx, QEQ_ERR_NOMEM, "device allocation of %zu bytes failed (%s)", bytes,
                         cudaGetErrorString(e));
    }
    return QEQ_OK;
}

void dev_free(qeq_ctx *ctx, void *p) {
    if (!p) return;
    if (ctx->async_alloc)
        cudaFreeAsync(p, ctx->alloc_stream);
    else
        cudaFree(p);
}

static int validate(const qeq_params *p) {
    if (!p) return set_error(nullptr, QEQ_ERR_INVALID, "params is NULL");
    if (p->n_atoms < 1 || p->n_atoms > kIndexMask)
        return set_error(nullptr, QEQ_ERR_INVALID, "n_atoms must be in [1, %d]", kIndexMask);
    for (int d = 0; d < 3; ++d) {
        if (!(p->box[d] > 0.0) || !std::isfinite(p->box[d]))
            return set_error(nullptr, QEQ_ERR_INVALID, "box[%d] must be positive and finite", d);
        if (p->mesh[d] < 4 || p->mesh[d] > 4096)
            return set_error(nullptr, QEQ_ERR_INVALID, "mesh[%d] must be in [4, 4096]", d);
        if (p->mesh[d] < p->order)
            return set_error(nullptr, QEQ_ERR_INVALID, "mesh[%d] is smaller than the spline order", d);
    }
    if ((int64_t)p->mesh[0] * p->mesh[1] * p->mesh[2] > INT32_MAX)
        return set_error(nullptr, QEQ_ERR_UNSUPPORTED, "mesh of more than 2^31 - 1 points");
    if (!(p->alpha > 0.0)) return set_error(nullptr, QEQ_ERR_INVALID, "alpha must be positive");
    if (!(p->r_cut > 0.0)) return set_error(nullptr, QEQ_ERR_INVALID, "r_cut must be positive");
    if (!(p->skin >= 0.0)) return set_error(nullptr, QEQ_ERR_INVALID, "skin must be >= 0");
    if (p->order < 4 || p->order > 8)
        return set_error(nullptr, QEQ_ERR_UNSUPPORTED, "B-spline order must be in [4, 8]");
    if (p->precision != QEQ_FP64 && p->precision != QEQ_FP32_MIXED)
        return set_error(nullptr, QEQ_ERR_INVALID, "unknown precision %d", p->precision);
    if (!(p->k_e > 0.0)) return set_error(nullptr, QEQ_ERR_INVALID, "k_e must be positive");
    if (p->recip != QEQ_RECIP_PME && p->recip != QEQ_RECIP_EWALD)
        return set_error(nullptr, QEQ_ERR_INVALID, "unknown reciprocal method %d", p->recip);
    if (p->recip == QEQ_RECIP_EWALD && p->precision != QEQ_FP64)
        return set_error(nullptr, QEQ_ERR_UNSUPPORTED, "the explicit k-sum runs in FP64 only");
    if (!(p->k_cut >= 0.0)) return set_error(nullptr, QEQ_ERR_INVALID, "k_cut must be >= 0");
    if (!(p->krylov_tol >= 0.0))
        return set_error(nullptr, QEQ_ERR_INVALID, "krylov_tol must be >= 0");
    if (p->krylov_rank < 1 || p->krylov_rank > kMaxRank)
        return set_error(nullptr, QEQ_ERR_INVALID, "krylov_rank must be in [1, %d]", kMaxRank);
    if (p->dissipation_k < 3 || p->dissipation_k > 7)
        return set_error(nullptr, QEQ_ERR_INVALID, "dissipation_k must be in [3, 7]");
    if (p->short_range != QEQ_SHORT_NONE && p->short_range != QEQ_SHORT_WATER)
        return set_error(nullptr, QEQ_ERR_INVALID, "unknown short_range model %d", p->short_range);
    if (p->short_range == QEQ_SHORT_WATER && p->n_atoms % 3 != 0)
        return set_error(nullptr, QEQ_ERR_INVALID, "the water model needs atoms ordered O, H, H");
    if (!(p->dt > 0.0)) return set_error(nullptr, QEQ_ERR_INVALID, "dt must be positive");
    if (!(p->mass_unit > 0.0)) return set_error(nullptr, QEQ_ERR_INVALID, "mass_unit must be positive");
    if (p->max_neighbors < 0) return set_error(nullptr, QEQ_ERR_INVALID, "max_neighbors must be >= 0");
    return QEQ_OK;
}

static void drop_graph(qeq_ctx *ctx) {
    if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
    if (ctx->step_graph) cudaGraphDestroy(ctx->step_graph);
    ctx->step_exec = nullptr;
    ctx->step_graph = nullptr;
}

static void destroy(qeq_ctx *ctx) {
    if (!ctx) return;
    if (!ctx->async_alloc) cudaDeviceSynchronize();
    drop_graph(ctx);
    for (cudaEvent_t e : ctx->prof.ev) cudaEventDestroy(e);
    solver_free(ctx);
    shadow_free(ctx);
    coulomb_free(ctx);
    nl_free(ctx);
    cudaGetLastError();
    delete ctx;
}

}  // namespace qeq

using namespace qeq;

QEQ_API void qeq_params_default(qeq_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->n_atoms = 0;
    p->alpha = 0.34;
    p->r_cut = 8.0;
    p->skin = 1.0;
    p->mesh[0] = p->mesh[1] = p->mesh[2] = 32;
    p->order = 4;
    p->precision = QEQ_FP64;
    p->gaussian_self = 1;
    p->k_e = 14.3996454784;
    p->max_neighbors = 0;
    p->krylov_rank = 2;
    p->krylov_tol = 0.0;
    p->recip = QEQ_RECIP_PME;
    p->k_cut = 0.0;
    p->q_tot = 0.0;
    p->dissipation_k = 5;
    p->short_range = QEQ_SHORT_NONE;
    p->dt = 0.5;
    p->mass_unit = 103.6427;
}

namespace {

int create(const qeq_params *p, cudaStream_t stream, bool async_alloc, qeq_ctx **out) {
    if (!out) return set_error(nullptr, QEQ_ERR_INVALID, "out is NULL");
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    qeq_ctx *ctx = new (std::nothrow) qeq_ctx();
    if (!ctx) return set_error(nullptr, QEQ_ERR_NOMEM, "host allocation failed");
    ctx->async_alloc = async_alloc;
    ctx->alloc_stream = stream;
    ctx->p = *p;
    ctx->n = p->n_atoms;
    ctx->fp32 = p->precision == QEQ_FP32_MIXED;
    cudaGetDevice(&ctx->device);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) == cudaSuccess &&
        sms > 0) {
        ctx->sm_count = sms;
        ctx->red_grid = std::min(kRedBlocks, kRedPerSm * sms);
    }
    cudaGetLastError();
    rc = nl_configure(ctx);
    if (!rc) rc = nl_alloc(ctx);
    if (!rc) rc = coulomb_alloc(ctx);
    if (!rc) rc = shadow_alloc(ctx);
    // stream-ordered creation returns without waiting: the set-up kernels and copies
    // (from process-lifetime host tables only) are ordered before the caller's work
    // on the same stream
    if (!rc)
        rc = cuda_check(ctx, async_alloc ? cudaGetLastError() : cudaDeviceSynchronize(), "create");
    if (rc) {
        g_create_error = ctx->err;
        destroy(ctx);
        return rc;
    }
    *out = ctx;
    return QEQ_OK;
}

}  // namespace

QEQ_API int qeq_create(const qeq_params *p, qeq_ctx **out) { return create(p, nullptr, false, out); }

QEQ_API int qeq_create_async(const qeq_params *p, void *stream, qeq_ctx **out) {
    // Keep freed blocks in the pool so that the next context reuses them without
    // returning memory to the driver.
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    return create(p, (cudaStream_t)stream, true, out);
}

QEQ_API void qeq_destroy(qeq_ctx *ctx) { destroy(ctx); }

QEQ_API const char *qeq_last_error(const qeq_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

QEQ_API int qeq_get_sizes(const qeq_ctx *ctx, int64_t *n_atoms, int32_t *width) {
    if (!ctx) return QEQ_ERR_INVALID;
    if (n_atoms) *n_atoms = ctx->n;
    if (width) *width = ctx->width;
    return QEQ_OK;
}

QEQ_API int qeq_neighbor_build(qeq_ctx *ctx, const double *R, void *stream) {
    NvtxRange nvtx_range("qeq_neighbor_build");
    if (!ctx) return QEQ_ERR_INVALID;
    if (!R) return set_error(ctx, QEQ_ERR_INVALID, "R is NULL");
    ctx->err.clear();
    return nl_build(ctx, R, (cudaStream_t)stream);
}

QEQ_API int qeq_neighbor_export(qeq_ctx *ctx, int32_t *counts, int32_t *nbr, int8_t *shift) {
    if (!ctx) return QEQ_ERR_INVALID;
    if (!ctx->list_valid) return set_error(ctx, QEQ_ERR_NOLIST, "no neighbour list built yet");
    return nl_export(ctx, counts, nbr, shift);
}

QEQ_API int qeq_neighbor_export_coo(qeq_ctx *ctx, int64_t capacity, int32_t *pair_i,
                                    int32_t *pair_j, int8_t *image_code, int64_t *n_pairs,
                                    void *stream) {
    if (!ctx) return QEQ_ERR_INVALID;
    if (!pair_i || !pair_j || !image_code || !n_pairs)
        return set_error(ctx, QEQ_ERR_INVALID, "NULL argument");
    if (!ctx->list_valid) return set_error(ctx, QEQ_ERR_NOLIST, "no neighbour list built yet");
    return nl_export_coo(ctx, capacity, pair_i, pair_j, image_code, n_pairs, (cudaStream_t)stream);
}

QEQ_API int qeq_neighbor_displacement(qeq_ctx *ctx, const double *R, double *max_disp2,
                                      void *stream) {
    if (!ctx) return QEQ_ERR_INVALID;
    if (!R || !max_disp2) return set_error(ctx, QEQ_ERR_INVALID, "NULL argument");
    if (!ctx->list_valid) return set_error(ctx, QEQ_ERR_NOLIST, "no neighbour list built yet");
    return nl_displacement(ctx, R, (cudaStream_t)stream, max_disp2);
}

QEQ_API int qeq_build_info(int32_t *bounds_checked) {
    if (!bounds_checked) return set_error(nullptr, QEQ_ERR_INVALID, "NULL argument");
#ifdef QEQ_BOUNDS
    *bounds_checked = 1;
#else
    *bounds_checked = 0;
#endif
    return QEQ_OK;
}

QEQ_API int qeq_bounds_status(qeq_ctx *ctx, int32_t *site) {
    if (!ctx) return QEQ_ERR_INVALID;
    if (!site) return set_error(ctx, QEQ_ERR_INVALID, "NULL argument");
    int32_t v = 0;
    cudaError_t e = cudaDeviceSynchronize();  // the context's kernels may run on any stream
    if (e == cudaSuccess)
        e = cudaMemcpy(&v, ctx->d_flags + kFlagBounds, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_flags + kFlagBounds, 0, sizeof(int32_t));
    const int rc = cuda_check(ctx, e, "bounds status");
    if (rc) return rc;
    *site = v;
    if (v) return set_error(ctx, QEQ_ERR_BOUNDS, "bounds check failed at site %d", (int)v);
    return QEQ_OK;
}

QEQ_API int qeq_neighbor_plan(const qeq_params *p, qeq_nl_plan *out) {
    if (!out) return set_error(nullptr, QEQ_ERR_INVALID, "out is NULL");
    int rc = validate(p);
    if (rc) return rc;
    qeq_ctx *ctx = new (std::nothrow) qeq_ctx();
    if (!ctx) return set_error(nullptr, QEQ_ERR_NOMEM, "host allocation failed");
    ctx->p = *p;
    ctx->n = p->n_atoms;
    rc = nl_configure(ctx);  // host arithmetic only
    if (rc) {
        set_error(nullptr, rc, "%s", ctx->err.c_str());
    } else {
        const BrickGeom &g = ctx->geom;
        for (int d = 0; d < 3; ++d) {
            out->nc[d] = ctx->nc[d];
            out->reach[d] = ctx->reach[d];
            out->brick[d] = g.B[d];
            out->bricks[d] = g.nb[d];
            out->tile_reach[d] = g.br[d];
            out->cell_width[d] = ctx->cw[d];
        }
        out->tile_bricks = g.T;
        out->n_bricks = g.nbricks;
        out->r_list = ctx->rl;
        out->band_lo = ctx->rl2f_lo;
        out->band_hi = ctx->rl2f_hi;
    }
    delete ctx;
    return rc;
}

QEQ_API int qeq_coulomb_apply(qeq_ctx *ctx, const double *R, const double *q, const double *sigma,
                              double *v, double *E, double *F, double *energy, void *stream) {
    NvtxRange nvtx_range("qeq_coulomb_apply");
    if (!ctx) return QEQ_ERR_INVALID;
    if (!R || !q || !sigma || !v) return set_error(ctx, QEQ_ERR_INVALID, "NULL input or output");
    const bool field = E || F;
    return coulomb_apply_impl(ctx, R, q, sigma, v, E, F, energy, field, (cudaStream_t)stream);
}

namespace qeq {
int check_md(qeq_ctx *ctx, const qeq_md_params *prm, const qeq_md_state *st) {
    if (!ctx) return QEQ_ERR_INVALID;
    if (!prm || !st) return set_error(ctx, QEQ_ERR_INVALID, "NULL md params or state");
    if (!prm->chi || !prm->eta || !prm->sigma || !prm->mass)
        return set_error(ctx, QEQ_ERR_INVALID, "NULL parameter array");
    if (!st->R || !st->V || !st->F || !st->Kf || !st->n_hist || !st->q || !st->energies)
        return set_error(ctx, QEQ_ERR_INVALID, "NULL state array");
    ctx->err.clear();
    return QEQ_OK;
}
}  // namespace qeq

QEQ_API int qeq_shadow_init(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st,
                            void *stream) {
    NvtxRange nvtx_range("qeq_shadow_init");
    int rc = check_md(ctx, prm, st);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (!ctx->list_valid) {
        rc = nl_build(ctx, st->R, s);
        if (rc) return rc;
    }
    rc = shadow_evaluate(ctx, prm, st, s);
    if (rc) return rc;
    return shadow_finish(ctx, prm, st, false, s, true);
}

// The evaluation and the second half kick of a fixed-rank shadow step contain
// no host synchronisation, so they are captured once into a CUDA graph and
// replayed.  The graph is re-captured when the state, parameter or neighbour-list
// buffers it was recorded with change, or the launch capacities of the
// real-space kernels (tile and brick size) grow.  It is not used with a tolerance-driven
// Krylov rank (host reads), with the profiler on, with a user short-range
// callback, or on the legacy default stream (which cannot be captured).
namespace qeq {

std::atomic<uint64_t> g_graph_generation{0};

bool step_graphable(const qeq_ctx *ctx, cudaStream_t s) {
    return ctx->use_graphs && s != nullptr && !(ctx->p.krylov_tol > 0.0) && !ctx->prof.on &&
           !ctx->short_fn;
}


int ensure_step_graph(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, cudaStream_t s) {
    const void *key[14] = {st->R, st->V, st->F, st->Kf, st->n_hist, st->q, st->energies,
                           prm->chi, prm->eta, prm->sigma, prm->mass, ctx->nbr, ctx->tile_scratch,
                           nullptr};
    bool same = ctx->step_exec && ctx->graph_width == ctx->width &&
                ctx->graph_tile == ctx->tile_cap && ctx->graph_rows == ctx->rows_cap &&
                ctx->graph_pdl == ctx->pdl;
    for (int k = 0; k < 14 && same; ++k) same = key[k] == ctx->graph_key[k];
    if (same) return QEQ_OK;
    drop_graph(ctx);
    const int64_t l0 = ctx->launches, a0 = ctx->applies;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_check(ctx, e, "graph capture begin");
    int rc = shadow_evaluate(ctx, prm, st, s);
    if (!rc) rc = shadow_finish(ctx, prm, st, true, s, true);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_check(ctx, e, "graph capture end");
    // node priorities on: the mesh chain's kernels keep the priority of the
    // side stream they were captured on
    e = cudaGraphInstantiate(&ctx->step_exec, g, cudaGraphInstantiateFlagUseNodePriority);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_check(ctx, e, "graph instantiate");
    }
    ctx->step_graph = g;
    ctx->graph_width = ctx->width;
    ctx->graph_tile = ctx->tile_cap;
    ctx->graph_rows = ctx->rows_cap;
    ctx->graph_pdl = ctx->pdl;
    ctx->graph_launches = ctx->launches - l0;
    ctx->launches = l0;
    ctx->applies = a0;
    for (int k = 0; k < 14; ++k) ctx->graph_key[k] = key[k];
    ctx->graph_captures++;
    ctx->graph_gen = ++g_graph_generation;
    return QEQ_OK;
}

// Counters of one replay of the step graph (the graph's kernels, m + 1 applies).
void count_step_replay(qeq_ctx *ctx) {
    ctx->graph_replays++;
    ctx->launches += ctx->graph_launches;
    ctx->applies += ctx->p.krylov_rank + 1;
}

}  // namespace qeq

static int evaluate_and_finish(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st,
                               cudaStream_t s) {
    if (!step_graphable(ctx, s)) {
        int rc = shadow_evaluate(ctx, prm, st, s);
        if (rc) return rc;
        return shadow_finish(ctx, prm, st, true, s, true);
    }
    int rc = ensure_step_graph(ctx, prm, st, s);
    if (rc) return rc;
    count_step_replay(ctx);
    return cuda_check(ctx, cudaGraphLaunch(ctx->step_exec, s), "graph launch");
}

QEQ_API int qeq_shadow_step(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st,
                            void *stream) {
    NvtxRange nvtx_range("qeq_shadow_step");
    int rc = check_md(ctx, prm, st);
    if (rc) return rc;
    if (!ctx->list_valid) return set_error(ctx, QEQ_ERR_NOLIST, "call qeq_shadow_init first");
    cudaStream_t s = (cudaStream_t)stream;
    rc = shadow_advance(ctx, prm, st, s);
    if (rc) return rc;
    return evaluate_and_finish(ctx, prm, st, s);
}

QEQ_API int qeq_set_short_range(qeq_ctx *ctx, qeq_short_fn fn, void *user) {
    if (!ctx) return QEQ_ERR_INVALID;
    if (fn && !ctx->F_short)
        return set_error(ctx, QEQ_ERR_UNSUPPORTED, "this context has no short-range buffer");
    ctx->short_fn = fn;
    ctx->short_user = fn ? user : nullptr;
    drop_graph(ctx);  // a captured step holds the previous short-range term
    return QEQ_OK;
}

// Smallest n' >= n whose prime factors are all 2, 3, 5 or 7.
static int64_t smooth_size(int64_t n) {
    for (;; ++n) {
        int64_t m = n;
        for (int f : {2, 3, 5, 7})
            while (m % f == 0) m /= f;
        if (m == 1) return n;
    }
}

QEQ_API int qeq_params_from_tolerance(qeq_params *p, double delta) {
    if (!p) return set_error(nullptr, QEQ_ERR_INVALID, "params_from_tolerance: NULL params");
    if (!(delta > 0.0 && delta < 0.5))
        return set_error(nullptr, QEQ_ERR_INVALID, "params_from_tolerance: delta %g outside (0, 0.5)",
                         delta);
    if (!(p->r_cut > 0.0) || !std::isfinite(p->r_cut))
        return set_error(nullptr, QEQ_ERR_INVALID, "params_from_tolerance: r_cut must be positive");
    const double lg = std::sqrt(-std::log(2.0 * delta));
    const double alpha = lg / p->r_cut;
    int32_t mesh[3];
    for (int d = 0; d < 3; ++d) {
        if (!(p->box[d] > 0.0) || !std::isfinite(p->box[d]))
            return set_error(nullptr, QEQ_ERR_INVALID, "params_from_tolerance: box[%d] invalid", d);
        const double bound = 2.0 * alpha * p->box[d] / (3.0 * std::pow(delta, 0.2));
        const int64_t k = smooth_size(std::max<int64_t>(std::max(4, p->order), (int64_t)std::ceil(bound)));
        if (k > 4096)
            return set_error(nullptr, QEQ_ERR_INVALID,
                             "params_from_tolerance: mesh %lld on axis %d exceeds 4096", (long long)k, d);
        mesh[d] = (int32_t)k;
    }
    p->alpha = alpha;
    for (int d = 0; d < 3; ++d) p->mesh[d] = mesh[d];
    p->k_cut = 2.0 * alpha * lg;
    return QEQ_OK;
}

QEQ_API int qeq_set_neighbor_method(qeq_ctx *ctx, int method) {
    if (!ctx) return QEQ_ERR_INVALID;
    if (method != QEQ_NL_BRICK && method != QEQ_NL_ATOM)
        return set_error(ctx, QEQ_ERR_INVALID, "unknown neighbour method %d", method);
    ctx->nl_method = method;
    return QEQ_OK;
}

QEQ_API int qeq_set_graphs(qeq_ctx *ctx, int on) {
    if (!ctx) return QEQ_ERR_INVALID;
    ctx->use_graphs = on != 0;
    if (!ctx->use_graphs) drop_graph(ctx);
    return QEQ_OK;
}

QEQ_API int qeq_shadow_run(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st,
                           int32_t n_steps, void *stream) {
    NvtxRange nvtx_range("qeq_shadow_run");
    for (int32_t k = 0; k < n_steps; ++k) {
        int rc = qeq_shadow_step(ctx, prm, st, stream);
        if (rc) return rc;
    }
    return QEQ_OK;
}

static const char *kPhaseNames[kNumPhases] = {
    "neighbor_build", "gather_in", "real_space", "pme_spread", "fft_forward",
    "pme_influence",  "fft_inverse", "pme_gather", "shadow_reductions", "integrate"};

QEQ_API int qeq_profile_enable(qeq_ctx *ctx, int on) {
    if (!ctx) return QEQ_ERR_INVALID;
    Profiler &P = ctx->prof;
    if (on && P.ev.empty()) {
        const int pool = 8192;
        P.ev.resize(pool);
        P.phase.resize(pool / 2);
        for (int k = 0; k < pool; ++k) {
            cudaError_t e = cudaEventCreate(&P.ev[k]);
            if (e != cudaSuccess) {
                P.ev.resize(k);
                return cuda_check(ctx, e, "profiler event pool");
            }
        }
    }
    P.on = on != 0;
    P.used = 0;
    P.open = false;
    return QEQ_OK;
}

QEQ_API int qeq_profile_read(qeq_ctx *ctx, double *ms, int64_t *counts, int n_phases) {
    if (!ctx) return QEQ_ERR_INVALID;
    Profiler &P = ctx->prof;
    int rc = cuda_check(ctx, cudaDeviceSynchronize(), "profile read");
    if (rc) return rc;
    for (int k = 0; k < P.used / 2; ++k) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, P.ev[2 * k], P.ev[2 * k + 1]) == cudaSuccess) {
            P.ms[P.phase[k]] += t;
            P.count[P.phase[k]] += 1;
        }
    }
    cudaGetLastError();
    P.used = 0;
    P.open = false;
    for (int k = 0; k < n_phases && k < kNumPhases; ++k) {
        if (ms) ms[k] = P.ms[k];
        if (counts) counts[k] = P.count[k];
        P.ms[k] = 0.0;
        P.count[k] = 0;
    }
    return QEQ_OK;
}

QEQ_API const char *qeq_profile_phase_name(int phase) {
    return (phase >= 0 && phase < kNumPhases) ? kPhaseNames[phase] : "";
}

QEQ_API int qeq_graph_stats(const qeq_ctx *ctx, int64_t *out2) {
    if (!ctx || !out2) return QEQ_ERR_INVALID;
    out2[0] = ctx->graph_captures;
    out2[1] = ctx->graph_replays;
    return QEQ_OK;
}

QEQ_API int qeq_get_counters(const qeq_ctx *ctx, int64_t *out4) {
    if (!ctx || !out4) return QEQ_ERR_INVALID;
    out4[0] = ctx->launches;
    out4[1] = ctx->n_builds;
    out4[2] = ctx->applies;
    out4[3] = ctx->fft_execs;
    return QEQ_OK;
}

namespace qeq {
int erfc32_selftest(const float *x, float *out, int64_t n, cudaStream_t s);
}

QEQ_API int qeq_selftest_erfc32(const float *x, float *out, int64_t n, void *stream) {
    if (!x || !out || n < 0) return set_error(nullptr, QEQ_ERR_INVALID, "selftest: bad argument");
    if (n == 0) return QEQ_OK;
    return erfc32_selftest(x, out, n, (cudaStream_t)stream);
}

namespace qeq {
int pair_table_eval_host(int which, double alpha, double smax, int64_t n, const double *arg,
                         double *F, double *G, int32_t *in, int32_t *kept);
int pair64_selftest(qeq_ctx *ctx, int which, const double *arg, double *F, double *G, int32_t *in,
                    int64_t n, cudaStream_t s);
}

QEQ_API int qeq_pair_table_eval(double alpha, double smax, int32_t which, int64_t n, const double *arg,
                                double *F, double *G, int32_t *in_table, int32_t *kept) {
    if ((which != 0 && which != 1) || n < 0 || !kept || (n > 0 && (!arg || !F || !G || !in_table)))
        return set_error(nullptr, QEQ_ERR_INVALID, "pair_table_eval: bad argument");
    if (which == 0 && !(alpha > 0.0 && smax > 0.0))
        return set_error(nullptr, QEQ_ERR_INVALID, "pair_table_eval: alpha and smax must be positive");
    return pair_table_eval_host(which, alpha, smax, n, arg, F, G, in_table, kept);
}

QEQ_API int qeq_selftest_pair64(qeq_ctx *ctx, int32_t which, const double *arg, double *F, double *G,
                                int32_t *in_table, int64_t n, void *stream) {
    if (!ctx) return QEQ_ERR_INVALID;
    if ((which != 0 && which != 1) || n < 0 || (n > 0 && (!arg || !F || !G || !in_table)))
        return set_error(ctx, QEQ_ERR_INVALID, "selftest: bad argument");
    if (n == 0) return QEQ_OK;
    return pair64_selftest(ctx, which, arg, F, G, in_table, n, (cudaStream_t)stream);
}

namespace qeq {
int erfc64_selftest(qeq_ctx *ctx, const double *x, double *out, double *dout, int64_t n,
                    cudaStream_t s);
}

QEQ_API int qeq_selftest_erfc64(qeq_ctx *ctx, const double *x, double *out, double *dout, int64_t n,
                                void *stream) {
    if (!ctx) return QEQ_ERR_INVALID;
    if (!x || !out || !dout || n < 0) return set_error(ctx, QEQ_ERR_INVALID, "selftest: bad argument");
    if (n == 0) return QEQ_OK;
    return erfc64_selftest(ctx, x, out, dout, n, (cudaStream_t)stream);
}

// ---- regular QEq by GMRES, regular BO-MD ----

QEQ_API int qeq_solve(qeq_ctx *ctx, const double *R, const double *chi, const double *eta,
                      const double *sigma, double *q, double tol, int32_t max_iter, int32_t restart,
                      qeq_solve_info *info, void *stream) {
    NvtxRange nvtx_range("qeq_solve");
    if (!ctx) return QEQ_ERR_INVALID;
    if (!R || !chi || !eta || !sigma || !q) return set_error(ctx, QEQ_ERR_INVALID, "NULL argument");
    if (!(tol > 0.0) || max_iter < 1 || restart < 1)
        return set_error(ctx, QEQ_ERR_INVALID, "tol, max_iter and restart must be positive");
    if (!ctx->list_valid) return set_error(ctx, QEQ_ERR_NOLIST, "qeq_solve before neighbor_build");
    ctx->err.clear();
    cudaStream_t s = (cudaStream_t)stream;
    int rc = solver_alloc(ctx, restart > 64 ? 64 : restart);
    if (rc) return rc;
    if (!ctx->gmSol) {
        rc = dev_alloc(ctx, (void **)&ctx->gmSol, sizeof(double) * (ctx->n + 1));
        if (rc) return rc;
    }
    cudaMemsetAsync(ctx->gmSol, 0, sizeof(double) * (ctx->n + 1), s);
    cudaMemcpyAsync(ctx->gmSol, q, sizeof(double) * ctx->n, cudaMemcpyDeviceToDevice, s);
    qeq_solve_info local{};
    rc = gmres_solve(ctx, R, chi, eta, sigma, ctx->gmSol, tol, max_iter, restart, true, &local, s);
    if (rc) return rc;
    cudaMemcpyAsync(q, ctx->gmSol, sizeof(double) * ctx->n, cudaMemcpyDeviceToDevice, s);
    if (info) *info = local;
    return cuda_check(ctx, cudaStreamSynchronize(s), "qeq_solve");
}

static int check_bo(qeq_ctx *ctx, const qeq_md_params *prm, const qeq_md_state *st) {
    if (!ctx) return QEQ_ERR_INVALID;
    if (!prm || !st || !prm->chi || !prm->eta || !prm->sigma || !prm->mass)
        return set_error(ctx, QEQ_ERR_INVALID, "NULL md params");
    if (!st->R || !st->V || !st->F || !st->q || !st->energies)
        return set_error(ctx, QEQ_ERR_INVALID, "NULL state array");
    ctx->err.clear();
    return QEQ_OK;
}

QEQ_API int qeq_bomd_init(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, double tol,
                          int32_t max_iter, qeq_solve_info *info, void *stream) {
    NvtxRange nvtx_range("qeq_bomd_init");
    int rc = check_bo(ctx, prm, st);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (!ctx->list_valid) {
        rc = nl_build(ctx, st->R, s);
        if (rc) return rc;
    }
    rc = bomd_evaluate(ctx, prm, st, tol, max_iter, info, s);
    if (rc) return rc;
    return shadow_finish(ctx, prm, st, false, s, false);
}

QEQ_API int qeq_bomd_step(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, double tol,
                          int32_t max_iter, qeq_solve_info *info, void *stream) {
    NvtxRange nvtx_range("qeq_bomd_step");
    int rc = check_bo(ctx, prm, st);
    if (rc) return rc;
    if (!ctx->list_valid) return set_error(ctx, QEQ_ERR_NOLIST, "call qeq_bomd_init first");
    cudaStream_t s = (cudaStream_t)stream;
    rc = bomd_advance(ctx, prm, st, s);
    if (!rc) rc = bomd_evaluate(ctx, prm, st, tol, max_iter, info, s);
    if (!rc) rc = shadow_finish(ctx, prm, st, true, s, false);
    return rc;
}
