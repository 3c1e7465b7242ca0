/*
 * qeq.h -- C ABI of the GB300 shadow charge-equilibration Coulomb library.
 *
 * The library evaluates the periodic Coulomb potential operator v = Phi q and
 * its field on one GPU.  Kaymak et al., "GPU-Accelerated Charge-Equilibration
 * for Shadow Molecular Dynamics in Python" (arXiv 2503.21176), needs it several
 * times per shadow MD step (Sec. 3.4 matrix-free C v = u o v + dE_Coul/dv;
 * Sec. 3.5).  The library also advances that shadow XL-BOMD step.
 *
 * Conventions for every call:
 *  - Array arguments are DEVICE pointers owned by the caller, unless a comment
 *    says "host".  Positions are row-major [N][3] doubles.  Per-atom scalars are
 *    [N] doubles.  The library never frees or keeps caller memory past the call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is queued on it and the call returns without waiting,
 *    except where a comment says the call synchronises.
 *  - The ABI is FP64.  With QEQ_FP32_MIXED the pair sum, spreading, FFT and
 *    gather run in FP32 internally, and the inputs and outputs stay FP64.
 *  - Return value: QEQ_OK (0) or a negative QEQ_ERR_* code.  qeq_last_error()
 *    returns a message for the last failing call on that context.  No C++
 *    exception crosses the ABI.
 *  - Units follow the caller.  The water workloads use Angstrom, e, eV, amu
 *    and fs, with k_e = 14.3996454784 eV*A/e^2.
 *  - A context is not thread safe.  Use one context per host thread.
 */
#ifndef QEQ_GB300_H
#define QEQ_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QEQ_ABI_VERSION 1

enum qeq_status {
    QEQ_OK = 0,
    QEQ_ERR_INVALID = -1,     /* bad argument or parameter (message says which) */
    QEQ_ERR_UNSUPPORTED = -2, /* valid request outside what this build supports */
    QEQ_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    QEQ_ERR_CUFFT = -4,       /* a cuFFT call failed */
    QEQ_ERR_NOMEM = -5,       /* device allocation failed */
    QEQ_ERR_NOLIST = -6,      /* coulomb_apply before any neighbor_build */
    QEQ_ERR_NONFINITE = -7,   /* NaN or Inf found in the inputs */
    QEQ_ERR_CAPACITY = -8,    /* a neighbour row exceeds the hard width limit */
    QEQ_ERR_BOUNDS = -9       /* bounds-checked build: a kernel index check failed */
};

enum qeq_precision {
    QEQ_FP64 = 0,       /* every step in FP64 */
    QEQ_FP32_MIXED = 1  /* FP32 pair sum, spreading, FFT and gather with FP64 sums */
};

enum qeq_recip_method {
    QEQ_RECIP_PME = 0,   /* smooth PME on the K^3 mesh (Alg. 2) */
    QEQ_RECIP_EWALD = 1  /* explicit k-vector sum (Eq. ewald_rec), FP64 only */
};

enum qeq_short_model {
    QEQ_SHORT_NONE = 0, /* no short-range potential */
    QEQ_SHORT_WATER = 1 /* built-in flexible-water stand-in (not from the paper) */
};

/*
 * Parameters of one periodic system.  qeq_params_default() fills the water
 * workload defaults.
 *
 *  n_atoms         N >= 1, at most 2^24 - 1.
 *  box             orthorhombic edge lengths (Sec. 3.2: "length of the unit
 *                  cell").  Each edge must be at least (r_cut + skin) / 2.
 *  alpha           Ewald splitting parameter of Eqs. ewald_real, ewald_rec and
 *                  ewald_self, in 1/length.
 *  r_cut           real-space cutoff.  Pairs at distance exactly r_cut are
 *                  excluded.
 *  skin            neighbour-list skin.  The list radius is r_cut + skin, and
 *                  a rebuild is due when an atom has moved more than skin / 2
 *                  since the last build (Sec. 4.2.3).
 *  mesh            PME mesh K[3], each between 4 and 4096, K0 K1 K2 <= 2^31 - 1 (Alg. 2).
 *  order           B-spline points per dimension p, 4..8 (Alg. 2, step 1).
 *  precision       enum qeq_precision.
 *  k_e             Coulomb constant multiplying every term.
 *  gaussian_self   1 adds the Gaussian self-energy k_e sqrt(2/pi)/sigma_i to
 *                  Phi_ii.  0 leaves it absorbed in the hardness.
 *  max_neighbors   initial ELLPACK width (0 = estimate from density).  The
 *                  list grows by itself on overflow (Sec. 3.1).
 *  q_tot           total charge Q_tot of the constraint (Eq. linear_qeq).
 *  krylov_rank     m in 1..8, rank of the low-rank kernel update (Sec. 3.5);
 *                  with krylov_tol > 0 it is the largest rank allowed.
 *  krylov_tol      0: fixed rank m.  > 0: Krylov vectors are added until the
 *                  least-squares residual |R c - f| / |f| of the kernel update
 *                  is <= krylov_tol (the tolerance of the paper's Krylov solve
 *                  of Eq. Jnddot).  Costs one host sync per added vector.
 *  dissipation_k   K_d in 3..7, the XL-BOMD dissipation window.
 *  dt              MD time step, in the time unit.
 *  short_range     enum qeq_short_model.
 *  mass_unit       length^2 * mass / time^2 expressed in the energy unit
 *                  (103.6427 for A, amu, fs, eV).
 *  recip           enum qeq_recip_method: how Eq. ewald_rec is evaluated.
 *  k_cut           |k| cutoff of the explicit k-sum (0: where
 *                  exp(-k^2 / 4 alpha^2) falls below 1e-16).
 */
typedef struct qeq_params {
    int64_t n_atoms;
    double box[3];
    double alpha;
    double r_cut;
    double skin;
    int32_t mesh[3];
    int32_t order;
    int32_t precision;
    int32_t gaussian_self;
    double k_e;
    int32_t max_neighbors;
    int32_t krylov_rank;
    double krylov_tol;
    double q_tot;
    int32_t dissipation_k;
    int32_t short_range;
    double dt;
    double mass_unit;
    int32_t recip;
    double k_cut;
} qeq_params;

typedef struct qeq_ctx qeq_ctx;

/*
 * Accuracy-driven Ewald parameters.  The paper picks alpha and the mesh from a
 * requested accuracy with the heuristics of OpenMM (Sec. 3.2, Sec. 3.3); this
 * is that rule, as the OpenMM User Guide states it for PME:
 *   alpha   = sqrt(-ln(2 delta)) / r_cut,
 *   mesh[d] = the smallest K >= max(order, 2 alpha box[d] / (3 delta^(1/5)))
 *             whose prime factors are all 2, 3, 5 or 7 (fast FFT sizes),
 * and, for the explicit k-vector sum, k_cut = 2 alpha sqrt(-ln(2 delta)), where
 * the reciprocal factor exp(-k^2 / 4 alpha^2) falls to the same 2 delta (this
 * library's choice; OpenMM states no k-sum rule in this form).  delta is about
 * the relative RMS error of the forces; the mesh rule assumes fifth-order
 * B-splines (order 5), and lower orders give larger errors at small delta.
 * Reads p->r_cut, p->box, p->order and writes p->alpha, p->mesh, p->k_cut.
 * Host only.  QEQ_ERR_INVALID for delta outside (0, 0.5), a non-positive cutoff
 * or box edge, or a mesh above 4096.
 */
int qeq_params_from_tolerance(qeq_params *p, double delta);

/* Fill *p with the defaults: alpha 0.34, r_cut 8, skin 1, mesh 32^3, order 4,
 * FP64, Gaussian self-energy on, k_e 14.3996454784, rank 2, K_d 5, dt 0.5,
 * no short-range model.  The caller still sets n_atoms and box. */
void qeq_params_default(qeq_params *p);

/* Check *p and allocate every device buffer.  The buffers are the cell arrays,
 * the ELLPACK neighbour list at its initial width, the PME meshes, the
 * influence table, the cuFFT plans and the Krylov / reduction scratch (FP64
 * precision adds the pair-function tables of the real-space kernel, built on
 * the host once per alpha and cutoff).  The context also takes one
 * high-priority non-blocking stream and two events, used inside each apply,
 * from a process-wide pool per device (returned by qeq_destroy).
 * Uses the current CUDA device.
 * On failure *out is NULL and the return code says why.  Synchronises. */
int qeq_create(const qeq_params *p, qeq_ctx **out);

/* Same as qeq_create, but every device buffer, including the cuFFT work
 * area, comes from the device's default stream-ordered memory pool
 * (cudaMallocAsync on `stream`).  The set-up kernels, uploads and memsets are
 * ordered on `stream`, and the call returns without waiting for them (it never
 * synchronises the device; only the explicit k-vector Ewald set-up waits for
 * `stream`).  cuFFT plans come from a process-wide pool keyed by device, mesh
 * and transform: qeq_destroy of any context returns its plans there.
 * qeq_destroy then frees with cudaFreeAsync on that stream.  Creating and
 * destroying contexts this way does not stall work on other streams.  The
 * serving loop relies on that to admit and retire requests while others run.
 * The pool is set to keep freed memory cached (release threshold = max) for
 * reuse by later contexts.  Use the context on `stream`, or synchronise its
 * work before qeq_destroy. */
int qeq_create_async(const qeq_params *p, void *stream, qeq_ctx **out);

/* Free everything qeq_create allocated (its cuFFT plans go back to the plan
 * pool).  NULL is ignored.  Synchronises the device (contexts from
 * qeq_create_async: stream-ordered frees, no sync). */
void qeq_destroy(qeq_ctx *ctx);

/* Message for the last failing call on ctx ("" when none).  ctx may be NULL,
 * and then the message is that of the last failing qeq_create. */
const char *qeq_last_error(const qeq_ctx *ctx);

/* Number of atoms, and the current ELLPACK width (list capacity per row). */
int qeq_get_sizes(const qeq_ctx *ctx, int64_t *n_atoms, int32_t *width);

/*
 * Cell-list neighbour build (Sec. 3.1, Alg. 1).
 * Steps: wrap positions into the box (x + w, w = -(L floor(x / L))); bin into
 * cells of edge >= (r_cut + skin) / 2, paired into 2 x 2 x 2 bricks on axes
 * with four or more cells (qeq_neighbor_plan); counting sort brick-major
 * (ascending atom id inside a cell); emit, for every atom, each (j, image) with
 * |x_j - x_i + s L| < r_cut + skin into an ELLPACK row.  The pair decision
 * runs in FP64 with a fixed operation order and no fused multiply-add, so
 * the pair set is exactly the geometric one.
 * R: device [N][3] positions (any periodic image).
 * The call synchronises once to read the overflow flag.  When a row does not
 * fit, the list grows and is rebuilt before returning.
 * Returns QEQ_OK, or QEQ_ERR_NONFINITE for a non-finite coordinate.
 */
int qeq_neighbor_build(qeq_ctx *ctx, const double *R, void *stream);

/*
 * Neighbour search used by qeq_neighbor_build (Sec. 3.1, Alg. 1).  Both write
 * the same list: the same pair set, bit for bit, in the same three distance
 * classes per row (only the order inside a class differs), so every other call
 * is unaffected.  QEQ_NL_BRICK (the default): one block per brick of
 * 2 x 2 x 2 cells, four lanes per row walking the candidate cells that the
 * rows of a cell share.  QEQ_NL_ATOM: one thread per atom looping over the
 * cells around its own, with a counting pass and a placing pass, the form of
 * the paper's Triton kernel (one program per atom).  Host only; takes effect
 * at the next build.  QEQ_ERR_INVALID for another value.
 */
enum qeq_nl_method { QEQ_NL_BRICK = 0, QEQ_NL_ATOM = 1 };
int qeq_set_neighbor_method(qeq_ctx *ctx, int method);

/*
 * Host only (touches no device): the cell and brick decomposition that
 * qeq_create / qeq_neighbor_build use for *p, and the FP32 prefilter band of
 * the pair decision.  Per axis: nc cells of width cell_width >= r_list / 2
 * (r_list = r_cut + skin; nc made even when >= 4), reach = cells a pair can
 * span, brick = cells per brick (2, or 1 on axes with fewer than 4 cells),
 * bricks = nc / brick, tile_reach = bricks a tile extends on each side;
 * tile_bricks = prod (2 tile_reach + 1), n_bricks = prod bricks.  The emit
 * keeps a candidate whose FP32 squared distance is below band_lo and drops
 * one above band_hi without the FP64 test; inside the band the FP64 test
 * decides.  Returns QEQ_ERR_INVALID / QEQ_ERR_UNSUPPORTED as qeq_create does.
 */
typedef struct qeq_nl_plan {
    int32_t nc[3];
    int32_t reach[3];
    int32_t brick[3];
    int32_t bricks[3];
    int32_t tile_reach[3];
    int32_t tile_bricks;
    int64_t n_bricks;
    double cell_width[3];
    double r_list;
    float band_lo, band_hi;
} qeq_nl_plan;
int qeq_neighbor_plan(const qeq_params *p, qeq_nl_plan *out);

/*
 * Copy the current list to HOST memory in original atom numbering (for tests).
 * counts: host [N] int32, entries per row.  nbr: host [N][width] int32
 * neighbour atom ids.  shift: host [N][width][3] int8 image vectors s, so that
 * the displacement is x_j - x_i + s * box.  Unused slots are left untouched.
 * Any output may be NULL.  Synchronises.
 */
int qeq_neighbor_export(qeq_ctx *ctx, int32_t *counts, int32_t *nbr, int8_t *shift);

/*
 * COO copy of the current list (Sec. 3.1: the sparse "coordinate list" format
 * beside ELLPACK), written on the device: pair k is (pair_i[k], pair_j[k],
 * image_code[k]).  Atom ids are in original numbering.  The image code is
 * (sx + 2) * 25 + (sy + 2) * 5 + (sz + 2), so that the displacement is
 * x_j - x_i + s * box.  Pairs are grouped by row in the list's row order.
 * capacity: the length of the three device arrays.  *n_pairs (host)
 * receives the number of pairs.  When that exceeds the capacity, nothing is
 * written and QEQ_ERR_CAPACITY is returned.  Synchronises `stream`.
 */
int qeq_neighbor_export_coo(qeq_ctx *ctx, int64_t capacity, int32_t *pair_i, int32_t *pair_j,
                            int8_t *image_code, int64_t *n_pairs, void *stream);

/*
 * Largest squared displacement of any atom since the last build, written to
 * *max_disp2 (host double).  A rebuild is due when it exceeds (skin / 2)^2
 * (Sec. 4.2.3).  Synchronises.
 */
int qeq_neighbor_displacement(qeq_ctx *ctx, const double *R, double *max_disp2, void *stream);

/*
 * Allocation-free neighbour build.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc / cudaFree.  Examples
 * are an engine plugin whose host owns all device memory through its own
 * arena, a latency-critical loop that cannot take the device-wide
 * synchronisation of cudaFree, and a process under a hard memory budget.
 * It builds the same pair set as qeq_neighbor_build (same wrap, cells, FP64
 * decision and strict r_list comparison) without a qeq_ctx.  The scratch is
 * one file-scope device array of about 3.5 MB per device, which every GPU
 * that loads the library holds until the process exits.
 *
 * Limits: n_atoms <= 32768, each box edge >= r_list / 2, and at most 32768
 * cells (larger cells are used when the grid would not fit).  Larger inputs
 * are rejected with QEQ_ERR_CAPACITY before any GPU work.
 * R:       device [N][3] positions.     box: HOST double[3] orthorhombic edges.
 * r_list:  list radius (pairs at exactly r_list excluded).
 * width:   row capacity of nbr.
 * counts:  device [N] int32 output, entries per row.
 * nbr:     device [N][width] int32 output, row-major in original numbering.
 *          Entry = j | (code << 24), where j is the neighbour atom id and
 *          code = (sx + 2) * 25 + (sy + 2) * 5 + (sz + 2) encodes the image,
 *          so that the displacement is x_j - x_i + s * box.
 * max_row: HOST int32 output (nullable).  When a row needs more than width
 *          entries, the call returns QEQ_ERR_CAPACITY, writes the needed
 *          width here, and leaves the rows truncated.
 * Errors are reported through qeq_last_error(NULL).
 * The first call on each device looks up the device address of the scratch
 * array (cudaGetSymbolAddress) with that device current.  Make that first
 * call before any stream capture.  The call calls no cudaMalloc, cudaFree or
 * allocating library routine.  It synchronises `stream` once to read the
 * overflow and non-finite flags.  Every call reuses the same array and
 * clears what must start at zero.  Calls whose GPU work overlaps (other
 * streams, other host threads) race on the array and must be serialised.
 */
int qeq_neighbor_build_noalloc(const double *R, int64_t n_atoms, const double *box, double r_list,
                               int32_t width, int32_t *counts, int32_t *nbr, int32_t *max_row,
                               void *stream);

/*
 * Coulomb apply: v = Phi q with its field (Sec. 3.4, matrix-free form of
 * C v = u o v + dE_Coul/dv).  Phi is Eq. ewald_real (over the current list,
 * plain truncation at r_cut, Gaussian-charge correction
 * -erfc(r / sqrt(sigma_i^2 + sigma_j^2)) / r), plus smooth PME for Eq. ewald_rec
 * (Alg. 2: spread, FFT, influence function with |b(m)|^2, inverse FFT, gather),
 * plus the self term of Eq. ewald_self (-2 alpha / sqrt(pi) q_i).  With
 * gaussian_self it also carries the Gaussian self-energy.
 * R:      device [N][3] current positions.  They must lie within skin / 2 of the
 *         positions of the last neighbour build (not checked here; see
 *         qeq_neighbor_displacement).
 * q:      device [N] charges.   sigma: device [N] Gaussian widths (0 = point).
 * v:      device [N] output potential dE_Coul / dq_i.
 * E:      device [N][3] output field -d v_i / d r_i (nullable).
 * F:      device [N][3] output Coulomb force q_i E_i (nullable).
 * energy: device [4] output doubles (nullable): total 1/2 q.v, real-space part,
 *         reciprocal mesh energy 1/2 sum G |Q^|^2, self part.
 * Ordering: all work is ordered on `stream`.  Inside, the mesh chain (spread,
 * FFTs, influence) runs on the context's own stream, forked from `stream`
 * after the gathers and joined back into it before the outputs are written,
 * so to the caller the apply is one step of `stream` (capturable in a graph).
 * FP32-mixed results agree between runs to the rounding of the mesh's float
 * reductions, not bit for bit.
 * Returns QEQ_ERR_NOLIST before the first neighbour build.
 */
int qeq_coulomb_apply(qeq_ctx *ctx, const double *R, const double *q, const double *sigma,
                      double *v, double *E, double *F, double *energy, void *stream);

/*
 * Shadow XL-BOMD state (Sec. 3.5).  Everything is a caller-owned device array:
 *   R [N][3] positions, V [N][3] velocities, F [N][3] forces of the current
 *   state, Kf [N] kernel-times-residual of the current state,
 *   n_hist [K_d + 1][N] auxiliary charges n(t), n(t - dt), ..., q [N] the
 *   shadow charges q[n] of the current state.
 * chi, eta, sigma, mass: device [N] parameters (eta is the hardness u).
 * energies: device [8] doubles written by every evaluation:
 *   0 kinetic, 1 shadow potential (Eq. qeq_energy + short range),
 *   2 total, 3 short-range part, 4 Lagrange multiplier lambda,
 *   5 sum of q, 6 |q[n] - n|, 7 number of Coulomb applies in the evaluation.
 */
typedef struct qeq_md_state {
    double *R;
    double *V;
    double *F;
    double *Kf;
    double *n_hist;
    double *q;
    double *energies;
} qeq_md_state;

typedef struct qeq_md_params {
    const double *chi;
    const double *eta;
    const double *sigma;
    const double *mass;
} qeq_md_params;

/*
 * Evaluate the shadow potential at (R, n_hist[0]) without moving anything.
 * It computes the shadow charges q[n] (Eq. diag_linear_qeq, closed form,
 * one Coulomb apply), the forces F = q o E[n] + n o E[q - n] (+ short range),
 * and the rank-m Krylov approximation Kf of J^{-1} (q[n] - n) for
 * Eq. Jnddot (m - 1 further potential-only applies).
 * Rebuilds the neighbour list first if none exists.  Synchronises once.
 */
int qeq_shadow_init(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, void *stream);

/*
 * One shadow XL-BOMD step.  First a velocity-Verlet half kick and drift of R.
 * Then the dissipative Verlet update of n,
 *   n(t+dt) = 2 n(t) - n(t-dt) - kappa Kf(t) + a sum_k c_k n(t - k dt),
 * with the history shifted.  Then a neighbour rebuild if an atom moved more
 * than skin / 2, a full evaluation (as qeq_shadow_init), and the second half
 * kick.  The integrator constants are those of Niklasson et al., J. Chem.
 * Phys. 130, 214109 (2009); the paper does not print them.
 * Synchronises once (the skin check).
 */
int qeq_shadow_step(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, void *stream);

/* Replay of qeq_shadow_step through a CUDA graph (default on).  The
 * evaluation and second half kick of a fixed-rank step are captured on the
 * first step and replayed afterwards (re-captured when buffers change).  It
 * is skipped with krylov_tol > 0, with the profiler on, and on the legacy
 * default stream.  on = 0 always launches kernel by kernel. */
int qeq_set_graphs(qeq_ctx *ctx, int on);

/*
 * User short-range model.  A callback of this type replaces the
 * parameter-selected short-range term (qeq_params.short_range) in
 * qeq_shadow_init / qeq_shadow_step / qeq_shadow_run and the BO-MD calls:
 * each evaluation calls it on the host with the current positions
 * R (device [n_atoms][3]) and it writes the short-range forces F (device
 * [n_atoms][3], overwritten) and energy (device double, overwritten), with
 * all its work ordered on `stream` (it may be asynchronous; it must not wait
 * for other streams' work).  It returns 0, or non-zero to fail the call
 * (QEQ_ERR_INVALID).  qeq_set_short_range(ctx, NULL, NULL) restores the
 * parameter-selected term.  While a callback is set the step is not captured
 * into a CUDA graph (the callback may allocate or launch anything).  The call
 * itself allocates nothing and queues no GPU work: the force buffer the
 * callback writes belongs to the context from its creation.  Clearing or
 * replacing a callback drops a captured step graph, which the next fixed-rank
 * step re-captures.
 */
typedef int (*qeq_short_fn)(void *user, int64_t n_atoms, const double *R, double *F, double *energy,
                            void *stream);
int qeq_set_short_range(qeq_ctx *ctx, qeq_short_fn fn, void *user);

/*
 * Batched shadow steps, for a server holding many systems at once.  One
 * qeq_batch_step advances each of the n member contexts (ctxs[k] with its own
 * parameters prms[k] and state sts[k], all on the current device, each set up
 * by qeq_shadow_init) by one step of qeq_shadow_step.  Every member's integrator
 * update and displacement check is queued on `stream`; ONE host
 * synchronisation then reads all skin checks; members with an atom past
 * skin / 2 rebuild their lists; and ONE CUDA graph, whose parallel branches are
 * the members' captured evaluations and second half kicks, runs them all.
 * Members that cannot replay a graph (tolerance-driven rank, user short-range
 * callback, profiler on) are evaluated kernel by kernel on the same stream.
 * The batch caches that parent graph and rebuilds it only when the member list
 * (order included) or a member's captured step changes.  Each member runs the
 * kernels of its own qeq_shadow_step, so results equal n separate steps.  A
 * context stepping on its own launches its shadow-step kernels with
 * programmatic dependent launch (each scheduled while its predecessor
 * finishes); from its first batched step on, a member launches them without
 * it, since its evaluation runs beside the other members' (its step graph is
 * captured again once).
 * `stream` must not be the legacy default stream; the members' earlier work
 * must be ordered before it (same stream, or an event).  A member appears at
 * most once.  Synchronises once (plus once per rebuilding member).
 * qeq_batch_stats: host int64 out2[2] = parent graphs built, graph launches.
 */
typedef struct qeq_batch qeq_batch;
int qeq_batch_create(qeq_batch **out);
void qeq_batch_destroy(qeq_batch *b);
int qeq_batch_step(qeq_batch *b, int32_t n, qeq_ctx *const *ctxs, const qeq_md_params *prms,
                   qeq_md_state *sts, void *stream);
int qeq_batch_stats(const qeq_batch *b, int64_t *out2);

/* Same as qeq_shadow_step repeated n_steps times. */
int qeq_shadow_run(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, int32_t n_steps,
                   void *stream);

/*
 * Regular charge equilibration (Sec. 3.4, Eq. linear_qeq):
 *   [diag(u) + Phi, 1; 1^T, 0] [q; lambda] = [-chi; Q_tot],
 * solved matrix-free (one potential-only Coulomb apply per iteration) by
 * restarted GMRES with a right Jacobi preconditioner, as the paper does for
 * its regular BO-MD (Sec. 4.1).  The preconditioner diagonal is u_i plus the
 * Gaussian self-energy when that term is on.  Iteration stops when
 * ||b - A x|| / ||b|| <= tol (the paper's solver tolerance) or after max_iter
 * iterations.
 * q: device [N], the initial guess on entry and the solution on exit (lambda
 * starts at 0).  info (host, nullable) receives iterations, Coulomb applies,
 * the final true relative residual and lambda.  Synchronises once per
 * iteration.  Needs a current neighbour list.
 */
typedef struct qeq_solve_info {
    int32_t iterations;
    int32_t applies;
    double rel_residual;
    double lambda;
} qeq_solve_info;

int qeq_solve(qeq_ctx *ctx, const double *R, const double *chi, const double *eta,
              const double *sigma, double *q, double tol, int32_t max_iter, int32_t restart,
              qeq_solve_info *info, void *stream);

/*
 * Regular Born-Oppenheimer MD (Sec. 3.4), with the same state layout as the
 * shadow step.  Kf and n_hist are unused and may be NULL.  q is the solution
 * and also the warm start of the next solve.
 * qeq_bomd_init: solve at the current R, then compute forces F = q o E[q]
 * (+ short range) and energies.
 * qeq_bomd_step: velocity-Verlet half kick and drift, a neighbour rebuild
 * when due, the same evaluation, and the second half kick.
 * energies (device [8]): 0 kinetic, 1 potential sum q chi + 1/2 sum u q^2 +
 * 1/2 q.Phi q (+ short range), 2 total, 3 short range, 4 lambda, 5 sum q,
 * 6 final relative residual, 7 Coulomb applies in the evaluation.
 */
int qeq_bomd_init(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, double tol,
                  int32_t max_iter, qeq_solve_info *info, void *stream);
int qeq_bomd_step(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, double tol,
                  int32_t max_iter, qeq_solve_info *info, void *stream);

/*
 * Diagnostic: evaluate the FP32 complementary error function used by the
 * FP32-mixed real-space kernel (Abramowitz & Stegun eq. 7.1.26, absolute
 * error <= 1.5e-7 for x >= 0) on n device inputs x, writing device out.
 * Lets tests check the approximation against a reference erfc.
 */
int qeq_selftest_erfc32(const float *x, float *out, int64_t n, void *stream);

/*
 * Diagnostic: evaluate the FP64 complementary error function and its
 * derivative used by the FP64 real-space kernel.  It is a piecewise
 * polynomial through Chebyshev nodes of a long-double erfc: 256 pieces of
 * degree 9 on [0, 6.5), and 0 beyond.  Inputs are n device doubles x >= 0.
 * The outputs out (erfc) and dout (d erfc / dx) are device doubles.
 */
int qeq_selftest_erfc64(qeq_ctx *ctx, const double *x, double *out, double *dout, int64_t n,
                        void *stream);

/*
 * Diagnostic, host only (touches no device): the FP64 real-space kernel's
 * piecewise pair functions, built and evaluated exactly as a context builds
 * and the kernel evaluates them (same tables, same bit indexing, same fused
 * Horner steps).  which = 0: F(s) = erfc(alpha sqrt s) / sqrt s and
 * G(s) = -(F(s) + (2 alpha / sqrt pi) exp(-alpha^2 s)) / s, the table of a
 * context with this alpha and r_cut^2 = smax (both > 0); which = 1: the same
 * functions at alpha = 1 of t = r^2 / gamma^2, the Gaussian-correction table
 * (alpha and smax ignored).  For the n host arguments arg[k] > 0 it writes
 * F[k], G[k] (host doubles) and in_table[k] = 1 where arg[k] falls in the
 * kept pieces, else in_table[k] = 0 and leaves F[k], G[k] (the kernel then
 * takes its direct erfc path).  *kept: the number of kept pieces.
 * Returns QEQ_ERR_INVALID for a bad argument.
 */
int qeq_pair_table_eval(double alpha, double smax, int32_t which, int64_t n, const double *arg,
                        double *F, double *G, int32_t *in_table, int32_t *kept);

/*
 * Diagnostic: the same evaluation on the device, with the tables of an FP64
 * context (which as in qeq_pair_table_eval); arg, F, G, in_table are device
 * arrays of n entries.  QEQ_ERR_INVALID for an FP32-mixed context.
 */
int qeq_selftest_pair64(qeq_ctx *ctx, int32_t which, const double *arg, double *F, double *G,
                        int32_t *in_table, int64_t n, void *stream);

/*
 * Diagnostic: measured throughput of the pipes the real-space pair sum is
 * bound by, on the current device at its present clocks.  Writes host
 * out4[0] FP32 FLOP/s (a fused multiply-add counts two), out4[1] FP64 FLOP/s,
 * out4[2] special-function (MUFU reciprocal square root) operations/s and
 * out4[3] the SM count (cudaDevAttrMultiProcessorCount).  Each rate is the
 * best of three launches of a few milliseconds of independent dependency
 * chains on every SM, timed with CUDA events on `stream`.  Allocates a small
 * sink buffer and synchronises.  Errors go to qeq_last_error(NULL).
 */
int qeq_measure_peaks(double *out4, void *stream);

/*
 * Bounds-checked build.  Compiled with -DQEQ_BOUNDS (libqeq_bounds.so), the
 * kernels check their data-dependent indices (list entries against the tile,
 * the sorted-order permutation, tile slots in the emit) and, where one fails,
 * record the first failing site and skip the access instead of reading or
 * writing out of range.  qeq_build_info: *bounds_checked = 1 in that build,
 * 0 otherwise (host only).  qeq_bounds_status: synchronises, writes the first
 * failing site (0: none) to *site, clears it, and returns QEQ_ERR_BOUNDS when
 * a check failed since the last call.
 */
int qeq_build_info(int32_t *bounds_checked);
int qeq_bounds_status(qeq_ctx *ctx, int32_t *site);

/*
 * Tracing.  The paper reports a per-component time breakdown of its MD runs
 * (Sec. 4.2.3, Fig. MD_simulation).  These calls give the same breakdown per
 * library phase, measured with CUDA events on the caller's stream.
 * Phase ids 0..9: neighbor_build, gather_in, real_space, pme_spread,
 * fft_forward, pme_influence, fft_inverse, pme_gather, shadow_reductions,
 * integrate (qeq_profile_phase_name gives the strings).
 */
#define QEQ_NUM_PHASES 10

/* on = 1 starts recording event pairs around every phase (pool of 4096
 * pairs; pairs beyond the pool are dropped).  on = 0 stops.  Resets the pool. */
int qeq_profile_enable(qeq_ctx *ctx, int on);

/* Synchronise the device, then return the accumulated milliseconds and launch
 * counts per phase since the last read.  The host arrays ms[n_phases] and
 * counts[n_phases] are both nullable.  The totals are reset afterwards. */
int qeq_profile_read(qeq_ctx *ctx, double *ms, int64_t *counts, int n_phases);

/* Name of a phase id, or "" when out of range. */
const char *qeq_profile_phase_name(int phase);

/* Host int64 out4[4]: this library's kernel launches (cuFFT excluded),
 * neighbour builds, Coulomb applies and cuFFT executions since creation. */
int qeq_get_counters(const qeq_ctx *ctx, int64_t *out4);

/* Host int64 out2[2]: shadow-step CUDA graphs captured, and shadow steps
 * replayed from a captured graph, since creation (qeq_set_graphs).  Host only;
 * QEQ_ERR_INVALID for a NULL argument. */
int qeq_graph_stats(const qeq_ctx *ctx, int64_t *out2);

#ifdef __cplusplus
}
#endif

#endif /* QEQ_GB300_H */
