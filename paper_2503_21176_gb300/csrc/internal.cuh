// Internal declarations of the GB300 Coulomb / shadow-QEq library.
// Only qeq_* entry points (include/qeq.h) are exported from the shared object.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "qeq.h"

#define QEQ_API extern "C" __attribute__((visibility("default")))

// #pragma unroll with a macro argument (loop-shape tunables)
#define QEQ_PRAGMA_(x) _Pragma(#x)
#define QEQ_UNROLL_(n) QEQ_PRAGMA_(unroll n)
#define QEQ_UNROLL(n) QEQ_UNROLL_(n)

namespace qeq {

constexpr int kThreads = 256;
// Fixed reduction grid: grid-stride kernels that reduce run on the context's
// red_grid blocks (kRedPerSm x the device's SM count from
// cudaDevAttrMultiProcessorCount, read at creation: 304 on a 152-SM GB300) and
// write one partial per block into a [slot][kRedBlocks] table; a finalize sums
// each slot's red_grid partials in a fixed order, so results are deterministic
// on a given device.  kRedBlocks is the table's stride and the largest grid.
#ifndef QEQ_RED_BLOCKS
#define QEQ_RED_BLOCKS 1024
#endif
#ifndef QEQ_RED_PER_SM
#define QEQ_RED_PER_SM 2
#endif
constexpr int kRedBlocks = QEQ_RED_BLOCKS;
constexpr int kRedPerSm = QEQ_RED_PER_SM;
constexpr int kMaxRank = 8;
// Reduction slots: the largest user is the GMRES multi-dot (restart <= 64
// vectors plus the norm); the Krylov normal equations need
// kMaxRank (kMaxRank + 1) / 2 + kMaxRank.
constexpr int kMaxGmresRestart = 64;
constexpr int kMaxRedSlots = 72;
static_assert(kMaxRank * (kMaxRank + 1) / 2 + kMaxRank <= kMaxRedSlots, "reduction slots");
static_assert(kMaxGmresRestart + 1 <= kMaxRedSlots, "reduction slots");
constexpr int kMaxHist = 8;
// An entry of the allocation-free list packs the atom index (low 24 bits) and
// the image code (high 8 bits): code = (sx + 2) * 25 + (sy + 2) * 5 + (sz + 2),
// |s| <= 2.  The atom count is limited to the 24-bit index range.
constexpr int kIndexBits = 24;
constexpr int32_t kIndexMask = (1 << kIndexBits) - 1;
constexpr int kMaxWidthLimit = 1 << 16;

constexpr double kTwoOverSqrtPi = 1.12837916709551257390;
constexpr double kSqrtTwoOverPi = 0.79788456080286535588;
constexpr double kPi = 3.14159265358979323846;

// Device-side status words (int32).
// kFlagSigmaMax: float bits of max |sigma| of the last FP32 apply's inputs.
// kFlagMaxTile / kFlagMaxRows: largest tile (atoms) and brick (rows) of the last build.
// kFlagTileOverflow: a real-space block met a tile larger than its capacity
// (cannot happen for a list built by this context; the block then skips its brick).
enum Flag {
    kFlagMaxRow = 0,
    kFlagNonFinite = 1,
    kFlagSigmaMax = 2,
    kFlagMaxTile = 3,
    kFlagMaxRows = 4,
    kFlagTileOverflow = 5,
    kFlagBounds = 6,  // bounds-checked build: first failing check site (kept across builds)
    kNumFlags = 8
};

// Sites of the bounds checks (the value kFlagBounds records).
enum BoundsSite {
    kSiteReal32Entry = 1,
    kSiteReal64Entry = 2,
    kSiteGatherPerm = 3,
    kSiteEmitTile = 4,
};

// Bounds-checked build (-DQEQ_BOUNDS): QEQ_IN_BOUNDS(cond, flags, site) is
// cond, and records site in flags[kFlagBounds] (first one wins) where cond is
// false, so the caller skips the access.  Without QEQ_BOUNDS it is true and no
// check is compiled.
#ifdef QEQ_BOUNDS
__device__ __forceinline__ bool qeq_bounds_check(bool ok, int32_t *flags, int site) {
    if (!ok) atomicCAS(&flags[kFlagBounds], 0, site);
    return ok;
}
#define QEQ_IN_BOUNDS(cond, flags, site) qeq_bounds_check((cond), (flags), (site))
#else
#define QEQ_IN_BOUNDS(cond, flags, site) true
#endif

// ---------------------------------------------------------------------------
// Brick tiling of the cell grid.
//
// Cells are at least r_list / 2 wide, so a pair inside r_list lies at most
// reach <= 2 cells apart per axis.  Cells are grouped into bricks of B x B x B
// cells (B = 2 per axis, or 1 on an axis with a single cell).  The tile of a
// brick is the (2 br + 1)^3 block of bricks around it, br = ceil(reach / B),
// each with its periodic image shift; it holds every atom that a row of the
// brick can pair with (27 bricks, about 2,000 atoms, for water at r_list 9 A).
// Atoms are sorted brick-major (brick, then cell inside the brick, then atom
// id), so a brick's atoms are one contiguous range.  Neighbour entries are
// 16-bit indices into the tile of the row's brick: the tile is the
// concatenation of its bricks in tile order (oz fastest), so the entry of
// sorted atom j of tile brick rb is off[rb] + (j - start[rb]).
// ---------------------------------------------------------------------------
constexpr int kMaxTileBricks = 125;   // (2 br + 1)^3 with br <= 2
// 16-bit entries; index t_total (one past a brick's tile) is the padding entry
// the emit writes after a row's last entry up to its 16-entry stripe.
constexpr int kMaxTileAtoms = 65534;

struct BrickGeom {
    int nc[3];    // cells per axis
    int B[3];     // cells per brick per axis (1 or 2)
    int nb[3];    // bricks per axis
    int br[3];    // tile radius in bricks per axis
    int td[3];    // tile extent in bricks, 2 br + 1
    int T;        // bricks in a tile
    int bvol;     // cells per brick
    int center;   // tile index of the brick itself
    int64_t nbricks;
};

__host__ __device__ __forceinline__ int floor_div(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

__host__ __device__ __forceinline__ int64_t brick_index(const BrickGeom &g, int bx, int by, int bz) {
    return ((int64_t)bx * g.nb[1] + by) * g.nb[2] + bz;
}

// Brick-major index of cell (cx, cy, cz), 0 <= c < nc.
__host__ __device__ __forceinline__ int cell_index(const BrickGeom &g, int cx, int cy, int cz) {
    const int bx = cx / g.B[0], by = cy / g.B[1], bz = cz / g.B[2];
    const int lx = cx - bx * g.B[0], ly = cy - by * g.B[1], lz = cz - bz * g.B[2];
    return (int)(brick_index(g, bx, by, bz) * g.bvol + (lx * g.B[1] + ly) * g.B[2] + lz);
}

__host__ __device__ __forceinline__ void cell_coords(const BrickGeom &g, int c, int &cx, int &cy,
                                                     int &cz) {
    const int b = c / g.bvol, l = c - b * g.bvol;
    const int bz = b % g.nb[2], by = (b / g.nb[2]) % g.nb[1], bx = b / (g.nb[2] * g.nb[1]);
    const int lz = l % g.B[2], ly = (l / g.B[2]) % g.B[1], lx = l / (g.B[2] * g.B[1]);
    cx = bx * g.B[0] + lx;
    cy = by * g.B[1] + ly;
    cz = bz * g.B[2] + lz;
}

// Tile brick rb of brick b: the wrapped brick index and the image shift s per axis.
__host__ __device__ __forceinline__ int64_t tile_brick(const BrickGeom &g, int64_t b, int rb, int s[3]) {
    const int bz = (int)(b % g.nb[2]), by = (int)((b / g.nb[2]) % g.nb[1]);
    const int bx = (int)(b / ((int64_t)g.nb[2] * g.nb[1]));
    const int o[3] = {rb / (g.td[2] * g.td[1]) - g.br[0], (rb / g.td[2]) % g.td[1] - g.br[1],
                      rb % g.td[2] - g.br[2]};
    const int u[3] = {bx + o[0], by + o[1], bz + o[2]};
    int w[3];
    for (int d = 0; d < 3; ++d) {
        s[d] = floor_div(u[d], g.nb[d]);
        w[d] = u[d] - s[d] * g.nb[d];
    }
    return brick_index(g, w[0], w[1], w[2]);
}

// List layout: row i (sorted) keeps its entry k at list_index(k, i, n).  The
// real-space kernels give a row kListLanes lanes, lane s taking the entries
// k = s, s + 4, s + 8, ...  Rows are stored in stripes of kListStripe = 16
// entries ([width / 16][N][16]); inside a stripe, lane s's 4 entries are
// adjacent (one 8-byte load), and a warp's 8 rows read one contiguous 256-byte
// span per stripe.  The width is a multiple of 16.
constexpr int kListLanes = 4;
constexpr int kListStripe = 16;
__host__ __device__ __forceinline__ size_t list_index(int k, int64_t i, int64_t n) {
    return ((size_t)(k / kListStripe) * n + i) * kListStripe + (k % kListLanes) * 4 +
           (k / kListLanes) % 4;
}

// Tile table of brick b, built by one warp (all 32 lanes): for every tile brick
// rb the first sorted atom of its (wrapped) brick in start[rb], base[rb] =
// off[rb] - start[rb] (a sorted atom j of rb has tile index j + base[rb]), the
// image shift code (sx + 2) * 25 + (sy + 2) * 5 + (sz + 2) in code[rb] (when
// code is not null), and the tile size in *total.  off[rb] is the exclusive
// prefix sum of the brick counts in tile order: T <= 125 = 4 bricks a lane and
// one warp scan.
__device__ __forceinline__ void tile_table(const BrickGeom &g, int64_t b,
                                           const int32_t *__restrict__ cell_start, int *start,
                                           int *base, int *code, int *total) {
    const int lane = threadIdx.x & 31;
    int cn[4], st[4], sum = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int rb = lane * 4 + k;
        cn[k] = 0;
        st[k] = 0;
        if (rb < g.T) {
            int s[3];
            const int64_t wb = tile_brick(g, b, rb, s);
            st[k] = cell_start[wb * g.bvol];
            cn[k] = cell_start[(wb + 1) * g.bvol] - st[k];
            if (code) code[rb] = (s[0] + 2) * 25 + (s[1] + 2) * 5 + (s[2] + 2);
        }
        sum += cn[k];
    }
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    int run = x - sum;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int rb = lane * 4 + k;
        if (rb < g.T) {
            start[rb] = st[k];
            base[rb] = run - st[k];
        }
        run += cn[k];
    }
    if (lane == 31) *total = x;
}

// Tile index -> (tile brick, sorted atom): the last rb with off[rb] <= e, where
// off[rb] = start[rb] + base[rb] is non-decreasing in rb.
__device__ __forceinline__ int tile_locate(int e, int T, const int *start, const int *base) {
    int lo = 0, hi = T - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] + base[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Device scalar table (double).  Slot 4 holds the last max displacement^2;
// shadow.cu uses slots 32..127 for its reductions.
enum Scal { kScMaxDisp2 = 4, kNumScal = 160 };

// Phases timed by the optional CUDA-event profiler (qeq_profile_*).
enum Phase {
    kPhNeighbor = 0,
    kPhGatherIn,
    kPhReal,
    kPhSpread,
    kPhFftFwd,
    kPhInfluence,
    kPhFftInv,
    kPhGatherOut,
    kPhShadow,
    kPhIntegrate,
    kNumPhases
};

struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> ev;  // pool of event pairs, recorded in order
    std::vector<int> phase;       // phase of pair k
    int used = 0;                 // events used since the last read
    bool open = false;
    double ms[kNumPhases] = {};
    int64_t count[kNumPhases] = {};
    int64_t dropped = 0;
};

}  // namespace qeq

struct qeq_ctx {
    qeq_params p{};
    std::string err;
    int device = 0;
    // Stream-ordered allocation (qeq_create_async): every device buffer comes
    // from the device's default memory pool on alloc_stream.
    bool async_alloc = false;
    cudaStream_t alloc_stream = nullptr;
    int64_t n = 0;
    bool fp32 = false;

    // ---- cell grid (Sec. 3.1) ----
    int nc[3] = {1, 1, 1};
    int reach[3] = {1, 1, 1};  // cells per axis a list pair can span
    int64_t ncell = 1;
    double cw[3] = {0, 0, 0};
    double rl = 0, rl2 = 0;
    float rl2f_lo = 0, rl2f_hi = 0;

    // ---- neighbour list buffers (sorted numbering) ----
    int32_t *cell_of = nullptr;     // [N] cell of atom (original numbering)
    int32_t *cell_count = nullptr;  // [ncell]
    int32_t *cell_start = nullptr;  // [ncell + 1]
    int32_t *cell_fill = nullptr;   // [ncell]
    int32_t *tmp_list = nullptr;    // [N]
    int32_t *perm = nullptr;        // [N] sorted slot -> original atom
    int32_t *cell_s = nullptr;      // [N] cell of sorted slot
    double *wrap_off = nullptr;     // [N][3] wrap offsets w (original numbering)
    double *R_build = nullptr;      // [N][3] positions at the last build
    double4_32a *xs64 = nullptr;        // [N] wrapped positions at build (sorted)
    float4 *xs32 = nullptr;         // [N] FP32 copy
    uint16_t *nbr = nullptr;        // [width][N] tile-local entries (list_index layout)
    uint32_t *nbr_scratch = nullptr;  // same shape, 32-bit: the emit's kept entries with their class
    int32_t *cnt = nullptr;         // [N] entries per sorted row
    int width = 0;
    qeq::BrickGeom geom{};
    int max_tile = 0;               // largest brick tile of the current list (atoms)
    int max_rows = 0;               // largest brick (rows) of the current list
    // Launch capacities of the real-space kernels: grown (never shrunk) past the
    // largest tile / brick seen, in steps, so that rebuilds rarely change the
    // launch shape of a captured graph.
    int tile_cap = 0, rows_cap = 0;
    int4 *tile_tab = nullptr;       // [nbricks][T] (first sorted atom, tile base, image code, 0)
    int32_t *tile_tot = nullptr;    // [nbricks] tile size
    unsigned char *tile_scratch = nullptr;  // [nbricks][tile_cap] tiles when shared memory is too small
    size_t tile_scratch_bytes = 0;
    int32_t *d_flags = nullptr;     // [kNumFlags]
    int32_t *h_flags = nullptr;     // pinned host mirror
    bool list_valid = false;
    int64_t n_builds = 0;

    // ---- apply buffers (sorted numbering) ----
    double4_32a *xq64 = nullptr;   // [N] (x, y, z, q) FP64
    double *sg64 = nullptr;    // [N] sigma
    float4 *xq32 = nullptr;    // [N] FP32 copies
    float *sg32 = nullptr;
    bool gathered = false;     // sorted positions / sigma / spline bases current (cleared by a build)
    double *v_s = nullptr;     // [N] real-space potential (sorted)
    double *E_s = nullptr;     // [N][3] real-space field (sorted)
    int4 *sbase = nullptr;     // [N] B-spline base mesh index floor(K x / L) (sorted)
    void *sfrac = nullptr;     // [N] (fraction x, y, z, q) in the compute precision (sorted)

    // ---- PME (Alg. 2) ----
    int K[3] = {0, 0, 0};
    int64_t mesh_n = 0, meshc_n = 0;
    void *mesh = nullptr;      // [K1][K2][K3] real (double or float)
    void *meshc = nullptr;     // [K1][K2][K3/2+1] complex
    void *G = nullptr;         // influence function on the half spectrum (double or float)
    cufftHandle plan_r2c = 0, plan_c2r = 0;
    size_t plan_ws[2] = {0, 0};  // work-area sizes of the two plans
    bool have_plans = false;
    void *fft_work = nullptr;  // cuFFT work area (shared by both plans, one stream at a time)
    // High-priority side stream of the mesh chain (spread, FFTs, influence) and
    // its fork / join events: the chain runs beside the real-space kernel.
    cudaStream_t pme_stream = nullptr;
    cudaEvent_t pme_fork = nullptr, pme_join = nullptr;
    double *erfc_tab64 = nullptr;  // piecewise erfc coefficients of the FP64 real-space kernel
    double *fg_tab64 = nullptr;    // piecewise pair functions F(r^2), G(r^2) of the FP64 kernel
    int fg_pieces = 0;
    double *gc_tab64 = nullptr;    // piecewise F_1(t), G_1(t) of the Gaussian correction (FP64)
    int gc_pieces = 0;
    float4 *xf_pre = nullptr;      // [N] FP32 positions (sorted) of the FP64 kernel's prefilter

    // ---- explicit k-vector Ewald (ewald.cu) ----
    void *ewald_k = nullptr;        // [nk] double4 (kx, ky, kz, g)
    void *ewald_S = nullptr;        // [nk] double2 structure factor
    void *ewald_partial = nullptr;  // [nchunk][nk] double2
    int ewald_nk = 0, ewald_nchunk = 0;

    // ---- reductions ----
    double *part = nullptr;    // [kMaxRedSlots][kRedBlocks]
    unsigned int *ticket = nullptr;  // last-block counter of finalize_last_block (0 between kernels)
    double *scal = nullptr;    // [kNumScal]
    double *h_scal = nullptr;  // pinned host mirror

    // ---- shadow-step scratch (original numbering) ----
    double *v_n = nullptr, *E_n = nullptr, *phi = nullptr, *E_f = nullptr, *fvec = nullptr;
    double *Wb = nullptr;      // [m][N] Krylov basis
    double *Rb = nullptr;      // [m][N] J applied to the basis
    double *F_short = nullptr; // [N][3]
    qeq_short_fn short_fn = nullptr;  // user short-range model (qeq_set_short_range)
    void *short_user = nullptr;
    double *inv_u = nullptr;   // [N] 1 / u of the current evaluation
    double *half_kick = nullptr;  // [N] dt / (2 m mass_unit) of the current step

    // ---- GMRES solver of the regular QEq (solver.cu) ----
    double *gmV = nullptr;     // [restart + 1][N + 1] Arnoldi basis
    double *gmW = nullptr;     // [2][N + 1] work vectors
    double *gmZ = nullptr;     // [N + 1] preconditioned vector
    double *gmDinv = nullptr;  // [N + 1] Jacobi inverse diagonal
    double *gmH = nullptr;     // small device scratch
    double *gmSol = nullptr;   // [N + 1] BO-MD solution [q; lambda]
    int gm_restart = 0;
    double *energy4 = nullptr; // [4] energy parts of the last apply

    // ---- CUDA graph of the shadow evaluation + second half kick (api.cu) ----
    cudaGraph_t step_graph = nullptr;
    cudaGraphExec_t step_exec = nullptr;
    const void *graph_key[14] = {};  // state / parameter / list pointers it was captured with
    int graph_width = 0;
    int graph_tile = 0, graph_rows = 0;  // launch geometry of the real-space kernel at capture
    int64_t graph_launches = 0;      // this library's kernels inside the graph
    int red_grid = 2 * 152;          // blocks of the reduction grid (set at creation)
    int sm_count = 152;              // SMs of the device (set at creation)
    int kf_rank = 0;                 // Krylov vectors of the last shadow evaluation
    uint64_t graph_gen = 0;          // process-wide generation of the current step graph
    int64_t graph_captures = 0;      // step graphs captured since creation
    int64_t graph_replays = 0;       // step graph launches since creation
    bool use_graphs = true;
    int nl_method = QEQ_NL_BRICK;  // neighbour search (qeq_set_neighbor_method)
    bool pdl = true;       // shadow-step kernels by programmatic dependent launch
    bool graph_pdl = true; // ... as the captured step graph launches them

    // ---- tracing ----
    qeq::Profiler prof;
    int64_t launches = 0;     // kernels of this library launched (cuFFT excluded)
    int64_t applies = 0;      // Coulomb applies
    int64_t fft_execs = 0;    // cuFFT executions
};

namespace qeq {

// ---- error helpers (api.cu) ----
int set_error(qeq_ctx *ctx, int code, const char *fmt, ...);
int cuda_check(qeq_ctx *ctx, cudaError_t e, const char *what);

// ---- device memory (api.cu): cudaMalloc, or cudaMallocAsync on ctx->alloc_stream ----
int dev_alloc(qeq_ctx *ctx, void **p, size_t bytes);
void dev_free(qeq_ctx *ctx, void *p);

// ---- neighbour list (nlist.cu) ----
int nl_configure(qeq_ctx *ctx);  // cell grid from params
// Short-range term of an evaluation: the user callback, else the
// parameter-selected model, else zero; forces into ctx->F_short, energies into
// e_slot[0..1], on stream s.  has_short: whether ctx->F_short holds forces.
int short_range_eval(qeq_ctx *ctx, const double *R, const double *mass, double *e_slot,
                     cudaStream_t s);
inline bool has_short(const qeq_ctx *ctx) {
    return ctx->short_fn != nullptr || ctx->p.short_range == QEQ_SHORT_WATER;
}
int nl_alloc(qeq_ctx *ctx);
int nl_alloc_list(qeq_ctx *ctx, int width);
int nl_build(qeq_ctx *ctx, const double *R, cudaStream_t s);
int nl_export(qeq_ctx *ctx, int32_t *counts, int32_t *nbr, int8_t *shift);
int nl_export_coo(qeq_ctx *ctx, int64_t capacity, int32_t *coo_i, int32_t *coo_j, int8_t *coo_code,
                  int64_t *n_pairs, cudaStream_t s);
int nl_displacement(qeq_ctx *ctx, const double *R, cudaStream_t s, double *max_disp2);
void nl_free(qeq_ctx *ctx);

// ---- Coulomb operator (coulomb.cu) ----
int coulomb_alloc(qeq_ctx *ctx);
// Global tile scratch of the real-space kernels when the tile capacity exceeds
// shared memory (after each neighbour build; allocates only when it must grow).
int real_tile_reserve(qeq_ctx *ctx);
// cuFFT plan pool (coulomb.cu): take an idle plan of this device, mesh and type
// (or make one), and give it back when the context goes.
cufftResult plan_acquire(int dev, const int K[3], cufftType type, cufftHandle *out, size_t *ws);
void plan_release(int dev, const int K[3], cufftType type, cufftHandle h, size_t ws);
void coulomb_free(qeq_ctx *ctx);
// v, E, F in original numbering; E / F / energy4 may be null; need_field=false
// skips every field computation (potential-only apply).
// same_R: R and sigma are those of the previous apply of this context (no
// neighbour build since), so only the charges are gathered again.
int coulomb_apply_impl(qeq_ctx *ctx, const double *R, const double *q, const double *sigma,
                       double *v, double *E, double *F, double *energy4, bool need_field,
                       cudaStream_t s, bool same_R = false);

// ---- explicit k-vector Ewald (ewald.cu) ----
int ewald_alloc(qeq_ctx *ctx);
void ewald_free(qeq_ctx *ctx);
int ewald_recip_and_combine(qeq_ctx *ctx, const double *q, const double *sigma, double *v,
                            double *E, double *F, bool need_field, cudaStream_t s);

// ---- reductions (coulomb.cu) ----
// Sum nslots partial tables of kRedBlocks entries each, starting at part, into out[0..nslots).
void launch_finalize(const qeq_ctx *ctx, const double *part, int nslots, double *out, cudaStream_t s);

// ---- shadow step (shadow.cu) ----
int shadow_alloc(qeq_ctx *ctx);
void shadow_free(qeq_ctx *ctx);
int shadow_evaluate(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, cudaStream_t s);
int shadow_advance(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, cudaStream_t s);
// The integrator half of shadow_advance: kick, drift and n update, then the
// displacement kernel, all queued on s with no host synchronisation.
int shadow_advance_queue(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, cudaStream_t s);
// Step graphs (api.cu): whether the step of ctx on s can replay a graph, the
// capture (or reuse) of that graph, and the counters of one replay.
int check_md(qeq_ctx *ctx, const qeq_md_params *prm, const qeq_md_state *st);
bool step_graphable(const qeq_ctx *ctx, cudaStream_t s);
int ensure_step_graph(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, cudaStream_t s);
void count_step_replay(qeq_ctx *ctx);
// Second half kick (kick), kinetic and total energies, and with kf the kernel
// update Kf = W c of the preceding shadow evaluation.
int shadow_finish(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, bool kick,
                  cudaStream_t s, bool kf);

// ---- regular QEq / BO-MD (solver.cu) ----
int solver_alloc(qeq_ctx *ctx, int restart);
void solver_free(qeq_ctx *ctx);
int gmres_solve(qeq_ctx *ctx, const double *R, const double *chi, const double *u,
                const double *sigma, double *z, double tol, int max_iter, int restart,
                bool final_check, qeq_solve_info *info, cudaStream_t s);
int bomd_advance(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, cudaStream_t s);
int bomd_evaluate(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, double tol,
                  int max_iter, qeq_solve_info *info, cudaStream_t s);

// ---- device helpers ----
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Programmatic dependent launch (sm_90 and later).  A kernel launched by
// launch_pdl may be scheduled while the kernel before it on the stream is still
// running; pdl_begin() then holds every thread until that kernel has completed
// and its writes are visible, and lets the next kernel launch in turn.  Each such
// kernel calls it first, before any access to memory; without the launch
// attribute both instructions do nothing.  Inside a captured graph the
// dependency becomes a programmatic edge.  The shadow-step kernels use it (a
// chain of short grid-stride kernels: about 0.9 us per boundary) when their
// context steps on its own (pdl true).  Where other work runs beside them the
// early-launched successor's waiting blocks take SM resources from it: the
// Coulomb apply kernels, whose mesh chain runs on a side stream beside the
// real-space kernel, do not use it (the step graph ran 85 us slower), nor do
// the members of a batched step, whose evaluations are parallel branches of
// one graph (FP64 serving steps ran 5% slower).
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

#ifndef QEQ_PDL
#define QEQ_PDL 1  // 0: the same kernels launched without the attribute
#endif
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block,
                              size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = &attr;
    cfg.numAttrs = QEQ_PDL && pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Block-wide sum of NV values (blockDim.x == kThreads); result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sh[NV][kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double t = warp_sum(v[k]);
        if (lane == 0) sh[k][wid] = t;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = lane < kThreads / 32 ? sh[k][lane] : 0.0;
            v[k] = warp_sum(t);
        }
    }
    __syncthreads();
}

// Conversions between float and double on the integer pipe: GB300 runs the
// conversion instructions on its 1/64-rate FP64 pipe.
// Double to float by truncation toward zero: relative error below 2^-23,
// magnitudes below 2^-126 become zero.  Valid for |x| < 2^128.
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int sign = hi & (int)0x80000000;
    const int ex = ((hi >> 20) & 0x7FF) - 1023 + 127;
    if (ex <= 0) return __int_as_float(sign);
    return __int_as_float(sign | (ex << 23) | ((hi & 0xFFFFF) << 3) | (int)(lo >> 29));
}
// Float to double by rebuilding the IEEE-754 fields: exact for normal numbers
// (exponent rebiased from 127 to 1023, mantissa shifted by 29 bits), zero for
// zero and subnormals, infinities and NaNs kept.
__device__ __forceinline__ double f32_to_f64_exact(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned long long ed = e == 0xffu ? 0x7ffull : (unsigned long long)(e + 896u);
    const unsigned long long bits = sign | (ed << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double(e == 0 ? sign : bits);
}

// Grid reduction without a second launch.  Every block has written its NV
// partial sums to part[k * kRedBlocks + blockIdx.x]; the last block to arrive
// (ticket counter, then reset to 0 for the next kernel) sums them in the fixed
// order of k_finalize into out[0..NV).  Returns true in all threads of that
// block; out is written by its thread 0 before the block's final barrier.
template <int NV>
__device__ __forceinline__ bool finalize_last_block(const double *part, double *out,
                                                    unsigned int *ticket) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        v[k] = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
            v[k] += __ldcg(part + (size_t)k * kRedBlocks + b);
    }
    block_sum<NV>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = v[k];
        *ticket = 0u;
    }
    __syncthreads();
    return true;
}

// Grid maximum of non-negative values without a second launch: block maxima
// into part[blockIdx.x], and the last block to arrive (ticket counter, reset to
// 0) writes the maximum of them to *out.
__device__ __forceinline__ void max_last_block(double m, double *part, double *out,
                                               unsigned int *ticket) {
    __shared__ double sh[kThreads / 32];
    __shared__ bool is_last;
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
        t = warp_max(t);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double v = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) v = fmax(v, __ldcg(part + k));
    v = warp_max(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
        t = warp_max(t);
        if (threadIdx.x == 0) {
            *out = t;
            *ticket = 0u;
        }
    }
}

// NVTX range over a library entry point (host side: a timeline tool shows where
// each call enqueues its work; without a tool attached the calls do nothing).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Record the start / end event of a profiled phase on stream s (no-op when off).
inline void prof_begin(qeq_ctx *c, int ph, cudaStream_t s) {
    Profiler &P = c->prof;
    if (!P.on || P.open) return;
    if (P.used + 2 > (int)P.ev.size()) {
        ++P.dropped;
        return;
    }
    cudaEventRecord(P.ev[P.used], s);
    P.phase[P.used / 2] = ph;
    P.open = true;
}

inline void prof_end(qeq_ctx *c, cudaStream_t s) {
    Profiler &P = c->prof;
    if (!P.on || !P.open) return;
    cudaEventRecord(P.ev[P.used + 1], s);
    P.used += 2;
    P.open = false;
}

inline int grid_for(int64_t n, int threads = kThreads) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace qeq
