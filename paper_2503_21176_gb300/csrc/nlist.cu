// Cell-list neighbour build (Sec. 3.1, Alg. 1) for one GB300.
//
// The paper gathers a [N, 27, C_max] candidate tensor and filters it (Alg. 1).
// Its Triton variant instead loops over neighbouring cells per atom, writing a
// buffer sized by a neighbour-count estimate.  Here:
//   1. wrap + bin            one thread per atom: wrap offsets, brick-major cell index,
//                            cell histogram
//   2. scan                  one block, exclusive scan of the cell histogram
//   3. scatter               one thread per atom: slot in its cell (atomic)
//   4. cell sort             one warp per cell: rank by atom id, so the order in a cell
//                            is ascending atom id whatever order step 3 gave
//   5. pair emit             one block per brick: the tile table of the brick (the
//                            bricks around it and their offsets), then one thread per
//                            row sweeps the (2 reach + 1)^3 cell images; FP32 distance
//                            prefilter, FP64 decision inside a band around the list
//                            radius; 16-bit tile-local entries, column-major rows
// The FP64 decision is d = (xw_j - xw_i) + s * L per axis, then
// d2 = (dx*dx + dy*dy) + dz*dz < r_list^2, every operation explicitly rounded
// (no fused multiply-add), so the emitted set is exactly the geometric one.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <vector>

#include "internal.cuh"

namespace qeq {

namespace {

__global__ void k_wrap_bin(int n, const double *__restrict__ R, double Lx, double Ly, double Lz,
                           double cwx, double cwy, double cwz, BrickGeom g,
                           int32_t *__restrict__ cell_of, int32_t *__restrict__ cell_count,
                           double *__restrict__ wrap_off, double *__restrict__ R_build,
                           int32_t *__restrict__ flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double L[3] = {Lx, Ly, Lz};
    const double cw[3] = {cwx, cwy, cwz};
    const int nc[3] = {g.nc[0], g.nc[1], g.nc[2]};
    int c[3];
    bool finite = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double x = R[3 * (size_t)i + d];
        finite = finite && isfinite(x);
        // w = -(L * floor(x / L)), xw = x + w: one IEEE rounding per operation
        const double fl = floor(__ddiv_rn(x, L[d]));
        const double w = -__dmul_rn(L[d], fl);
        const double xw = __dadd_rn(x, w);
        wrap_off[3 * (size_t)i + d] = w;
        R_build[3 * (size_t)i + d] = x;
        int cc = isfinite(xw) ? (int)floor(xw / cw[d]) : 0;
        c[d] = min(max(cc, 0), nc[d] - 1);
    }
    if (!finite) atomicExch(&flags[kFlagNonFinite], 1);
    const int cell = cell_index(g, c[0], c[1], c[2]);
    cell_of[i] = cell;
    atomicAdd(&cell_count[cell], 1);
}

// Single-block exclusive scan of ncell ints (any size), launched with kScanThreads
// threads.  Tiles of kScanTile counts are loaded coalesced into shared memory;
// each thread scans kScanPer consecutive counts, a warp-shuffle scan of the
// thread sums and one of the warp sums give the offsets, and the tile is
// written back coalesced with the running carry.  Also zeroes fill.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

__global__ void __launch_bounds__(kScanThreads)
k_scan(int64_t ncell, const int32_t *__restrict__ count, int32_t *__restrict__ start,
       int32_t *__restrict__ fill) {
    // stride kScanPer + 1 per thread keeps the per-thread reads conflict-free
    __shared__ int32_t tile[kScanThreads * (kScanPer + 1)];
    __shared__ int32_t warp_sum[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    int32_t carry = 0;
    for (int64_t base = 0; base < ncell; base += kScanTile) {
        for (int k = t; k < kScanTile; k += kScanThreads) {
            const int64_t g = base + k;
            tile[(k / kScanPer) * (kScanPer + 1) + k % kScanPer] = g < ncell ? count[g] : 0;
        }
        __syncthreads();
        int32_t v[kScanPer];
        int32_t s = 0;
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            v[j] = tile[t * (kScanPer + 1) + j];
            s += v[j];
        }
        int32_t x = s;  // inclusive scan of the thread sums within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int32_t w = warp_sum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_sum[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        int32_t run = carry + (wid > 0 ? warp_sum[wid - 1] : 0) + (x - s);
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            tile[t * (kScanPer + 1) + j] = run;
            run += v[j];
        }
        carry += warp_sum[31];
        __syncthreads();
        for (int k = t; k < kScanTile; k += kScanThreads) {
            const int64_t g = base + k;
            if (g < ncell) {
                start[g] = tile[(k / kScanPer) * (kScanPer + 1) + k % kScanPer];
                fill[g] = 0;
            }
        }
        __syncthreads();
    }
    if (t == 0) start[ncell] = carry;
}

__global__ void k_scatter(int n, const int32_t *__restrict__ cell_of,
                          const int32_t *__restrict__ start, int32_t *__restrict__ fill,
                          int32_t *__restrict__ tmp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cell_of[i];
    const int slot = atomicAdd(&fill[c], 1);
    tmp[start[c] + slot] = i;
}

// One warp per cell: the rank of an atom inside its cell is the number of atoms
// of that cell with a smaller id.  Writes the permutation, the sorted cell id and
// the wrapped positions (recomputed from R and w with the same roundings).
__global__ void k_cell_sort(int64_t ncell, const int32_t *__restrict__ start,
                            const int32_t *__restrict__ tmp, const double *__restrict__ R,
                            const double *__restrict__ wrap_off, int32_t *__restrict__ perm,
                            int32_t *__restrict__ cell_s, double4_32a *__restrict__ xs64,
                            float4 *__restrict__ xs32) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= ncell) return;
    const int b = start[warp], e = start[warp + 1];
    for (int k = b + lane; k < e; k += 32) {
        const int id = tmp[k];
        int rank = 0;
        for (int t = b; t < e; ++t) rank += tmp[t] < id;
        const int slot = b + rank;
        perm[slot] = id;
        cell_s[slot] = (int)warp;
        const double x = __dadd_rn(R[3 * (size_t)id], wrap_off[3 * (size_t)id]);
        const double y = __dadd_rn(R[3 * (size_t)id + 1], wrap_off[3 * (size_t)id + 1]);
        const double z = __dadd_rn(R[3 * (size_t)id + 2], wrap_off[3 * (size_t)id + 2]);
        xs64[slot] = make_double4_32a(x, y, z, 0.0);
        xs32[slot] = make_float4((float)x, (float)y, (float)z, 0.f);
    }
}

// Cells per list radius.  With cells r_list / 2 wide the emit visits 125 cells
// holding about 1.16 (4 pi / 3)^-1 x 125 / 8 = 4.6x the atoms of the list ball,
// against 27 cells and 6.4x with cells r_list wide.  The brick tiling needs it.
constexpr int kCellDiv = 2;
// Unroll of the candidate loop of the emit (independent candidate loads in flight).
#ifndef QEQ_NL_UNROLL
#define QEQ_NL_UNROLL 1
#endif
constexpr int kEmitThreads = 128;
constexpr int kEmitBlocksPerSm = 4;

// s L for an image index s in [-2, 2]: exact in FP64 (a multiple of L by 0, 1 or
// 2), selected without an FP64 multiply.
__device__ __forceinline__ double image_shift(int s, double L, double L2) {
    // selected and negated on the integer pipe (sign bit flipped): the compiler
    // hoists this out of the candidate loops, and FP64 selects or negations
    // there would occupy GB300's 1/64-rate FP64 pipe once per cell
    const long long a = __double_as_longlong((s == 1 || s == -1) ? L : L2);
    const long long m = s < 0 ? (a ^ (long long)0x8000000000000000ull) : a;
    return __longlong_as_double(s == 0 ? 0ll : m);
}

struct EmitArgs {
    int n;
    int ncx, ncy, ncz;
    int rx, ry, rz;
    double Lx, Ly, Lz;
    double L2x, L2y, L2z;  // 2 L, exact
    float Lfx, Lfy, Lfz;
    double rl2;
    float lo, hi;
    float t_near, t_cut;  // class thresholds on the FP32 d^2
    int width;
};

// Rows are written in three distance classes: near (d^2 < r_list^2 / 3, where
// the Gaussian-charge correction of the real-space sum lives for water-like
// widths), inside the cutoff (d^2 < r_cut^2) and the skin beyond it.  Lanes that
// run the same iteration of the real-space kernel then hold neighbours of the
// same class, so its distance branches (cutoff test, Gaussian correction) agree
// across the warp.
// Lanes per row in the emit: lane s of a row tests atoms s, s + 4, ... of each
// of the row's candidate cells (its cell's (2 reach + 1)^3 neighbour cells).
// Rows of one cell visit the same cells, so the 8 rows of a warp (mostly one
// cell of about 9 atoms) walk them in lockstep and share each candidate load.
constexpr int kEmitLanes = 4;
constexpr int kMaxBrickCells = 8;
constexpr int kCenterCode = 62;  // image code of the zero shift

// The exact decision inside the FP32 band: d = (xw_j - xw_i) + s L per axis and
// d^2 = (dx dx + dy dy) + dz dz, each operation explicitly rounded.  Not inlined,
// and reading the arguments from the block's shared copy: inlined, the selection
// of its image shifts was hoisted into the per-cell prologue of the candidate
// loop and ran for every cell (the band holds a few candidates per row), about a
// quarter of the emit's instructions.
__device__ __noinline__ bool band_keep(const EmitArgs *ap, int code, const double4_32a *pj,
                                       const double4_32a *pi) {
    const EmitArgs &a = *ap;
    const double4_32a xj64 = *pj, xi = *pi;
    const double dx = __dadd_rn(__dsub_rn(xj64.x, xi.x), image_shift(code / 25 - 2, a.Lx, a.L2x));
    const double dy = __dadd_rn(__dsub_rn(xj64.y, xi.y), image_shift((code / 5) % 5 - 2, a.Ly, a.L2y));
    const double dz = __dadd_rn(__dsub_rn(xj64.z, xi.z), image_shift(code % 5 - 2, a.Lz, a.L2z));
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return d2 < a.rl2;
}

// The test pass of one lane, as a double loop: over the row's candidate ranges
// (its cell's neighbour cells, merged where they continue one sorted range; one
// table entry and one image shift per range, the shift folded into the row's
// own position), and over each range's atoms with stride kEmitLanes (lane s
// takes atoms s, s + 4, ...).  The decision is FP32 outside the band [lo, hi]
// and FP64 with a fixed operation order inside it; the distance class comes
// from the FP32 d^2.  A kept entry goes, with its class in bits 16-17, to the
// lane's slots 4 m + s of the 32-bit scratch list (m < cap = width / 4), and the
// classes are counted; counts keep running past cap (an overflow, reported for
// the regrowth).
__device__ __forceinline__ void emit_cells(const EmitArgs &a, const EmitArgs *sa, int i, int s,
                                           const int4 *__restrict__ tab,
                                           const float4 *__restrict__ shtab, int ncand,
                                           const float4 &xf,
                                           const double4_32a *__restrict__ xs64,
                                           const float4 *__restrict__ xs32, int cap, int (&c)[3],
                                           uint32_t *__restrict__ scr, int t_total,
                                           int32_t *__restrict__ flags) {
    // this lane's scratch slots 4 m + s of row i: stripe m / 4, word m % 4
    const size_t stripe = (size_t)a.n * kListStripe;
    size_t base = (size_t)i * kListStripe + (size_t)s * 4u;
    int m = 0, near = 0, inside = 0;
    for (int k = 0; k < ncand; ++k) {
        const int4 ct = tab[k];
        const float4 sh = shtab[ct.w];
        const float px = xf.x - sh.x, py = xf.y - sh.y, pz = xf.z - sh.z;
        const bool home = ct.w == kCenterCode;
        for (int j = ct.x + s; j < ct.y; j += kEmitLanes) {
            const float4 xj = xs32[j];
            const float dxf = xj.x - px, dyf = xj.y - py, dzf = xj.z - pz;
            const float d2f = fmaf(dzf, dzf, fmaf(dyf, dyf, dxf * dxf));
            if (d2f > a.hi) continue;
            if (home && j == i) continue;
            if (!(d2f < a.lo) && !band_keep(sa, ct.w, xs64 + j, xs64 + i)) continue;
            const int e = j + ct.z;
            if (!QEQ_IN_BOUNDS((unsigned)e < (unsigned)t_total, flags, kSiteEmitTile)) continue;
            const int cls = (d2f >= a.t_near) + (d2f >= a.t_cut);
            near += cls == 0;
            inside += cls == 1;
            if (m < cap) scr[base + (m & 3)] = (uint32_t)e | ((uint32_t)cls << 16);
            ++m;
            if ((m & 3) == 0) base += stripe;
        }
    }
    c[0] = near;
    c[1] = inside;
    c[2] = m - near - inside;
}

// One block per brick.  Warp 0 builds the tile table, then the block builds the
// candidate-cell table of each cell of the brick (first / end sorted atom, tile
// base and image code of each of its (2 reach + 1)^3 neighbour cells).  Warps
// take the brick's rows 8 at a time, kEmitLanes lanes a row.  The block also
// records the largest tile and brick for the real-space launch, and writes no
// entry when the tile exceeds 16-bit indices.
__global__ void __launch_bounds__(kEmitThreads)
k_emit(EmitArgs a, BrickGeom g, int nchunk, const double4_32a *__restrict__ xs64,
       const float4 *__restrict__ xs32, const int32_t *__restrict__ cell_s,
       const int32_t *__restrict__ cell_start, uint16_t *__restrict__ nbr, uint32_t *__restrict__ scr,
       int32_t *__restrict__ cnt, int4 *__restrict__ tile_tab, int32_t *__restrict__ tile_tot,
       int32_t *__restrict__ flags) {
    __shared__ int t_start[kMaxTileBricks], t_base[kMaxTileBricks], t_code[kMaxTileBricks], t_total;
    __shared__ int4 ctab[kMaxBrickCells][kMaxTileBricks];
    __shared__ float4 shtab[kMaxTileBricks];  // image shift s L of each code (sx + 2) * 25 + ...
    __shared__ int nrange[kMaxBrickCells];  // table entries (ranges) of each cell
    __shared__ EmitArgs sargs;  // the band decision's copy of the arguments
    if (threadIdx.x == 0) sargs = a;
    // nchunk blocks share a brick: chunk c takes the brick's groups of 32 rows
    // c, c + nchunk, ... (more blocks in flight for boxes of few bricks)
    const int64_t b = blockIdx.x / nchunk;
    const int chunk = (int)(blockIdx.x - b * nchunk);
    if (threadIdx.x < 32) tile_table(g, b, cell_start, t_start, t_base, t_code, &t_total);
    for (int code = threadIdx.x; code < 125; code += blockDim.x)
        shtab[code] = make_float4((float)(code / 25 - 2) * a.Lfx, (float)((code / 5) % 5 - 2) * a.Lfy,
                                  (float)(code % 5 - 2) * a.Lfz, 0.f);
    __syncthreads();
    const int i0 = t_start[g.center], i1 = cell_start[(b + 1) * g.bvol];
    if (chunk == 0) {
        // the tile table of the brick, for the real-space kernels of this list
        for (int rb = threadIdx.x; rb < g.T; rb += blockDim.x)
            tile_tab[b * g.T + rb] = make_int4(t_start[rb], t_base[rb], t_code[rb], 0);
        if (threadIdx.x == 0) {
            tile_tot[b] = t_total;
            atomicMax(&flags[kFlagMaxTile], t_total);
            atomicMax(&flags[kFlagMaxRows], i1 - i0);
        }
    }
    const int dx = 2 * a.rx + 1, dy = 2 * a.ry + 1, dz = 2 * a.rz + 1;
    const int ncand = dx * dy * dz;
    const int bz = (int)(b % g.nb[2]), by = (int)((b / g.nb[2]) % g.nb[1]);
    const int bx = (int)(b / ((int64_t)g.nb[2] * g.nb[1]));
    // Bricks are 1 or 2 cells per axis, so every division by B is a shift (lb =
    // log2 B); the flat index splits by FP32 reciprocals (exact below 2^22); and
    // with at least reach cells per axis a neighbour cell's image shift is -1, 0
    // or 1 by comparison (fewer cells take the general floor division).  Runtime
    // integer divisions made a sizeable part of the emit's instructions.
    const int lb0 = g.B[0] - 1, lb1 = g.B[1] - 1, lb2 = g.B[2] - 1;
    const bool near = a.ncx >= a.rx && a.ncy >= a.ry && a.ncz >= a.rz;
    const float inv_ncand = 1.0f / (float)ncand, inv_yz = 1.0f / (float)(dy * dz),
                inv_z = 1.0f / (float)dz;
    for (int t = threadIdx.x; t < g.bvol * ncand; t += blockDim.x) {
        const int lc = __float2int_rz(((float)t + 0.5f) * inv_ncand), kk = t - lc * ncand;
        const int lz = lc & lb2, ly = (lc >> lb2) & lb1, lx = lc >> (lb2 + lb1);
        const int cx = (bx << lb0) + lx, cy = (by << lb1) + ly, cz = (bz << lb2) + lz;
        const int qx = __float2int_rz(((float)kk + 0.5f) * inv_yz), rem = kk - qx * (dy * dz);
        const int qy = __float2int_rz(((float)rem + 0.5f) * inv_z);
        const int ux = cx + qx - a.rx, uy = cy + qy - a.ry, uz = cz + (rem - qy * dz) - a.rz;
        int sx, sy, sz;
        if (near) {
            sx = ux < 0 ? -1 : (ux >= a.ncx ? 1 : 0);
            sy = uy < 0 ? -1 : (uy >= a.ncy ? 1 : 0);
            sz = uz < 0 ? -1 : (uz >= a.ncz ? 1 : 0);
        } else {
            sx = floor_div(ux, a.ncx);
            sy = floor_div(uy, a.ncy);
            sz = floor_div(uz, a.ncz);
        }
        const int wx = ux - sx * a.ncx, wy = uy - sy * a.ncy, wz = uz - sz * a.ncz;
        const int tx = (ux >> lb0) - bx + g.br[0];
        const int ty = (uy >> lb1) - by + g.br[1];
        const int tz = (uz >> lb2) - bz + g.br[2];
        const int cn = (int)(brick_index(g, wx >> lb0, wy >> lb1, wz >> lb2) * g.bvol +
                             (((wx & lb0) << lb1 | (wy & lb1)) << lb2 | (wz & lb2)));
        ctab[lc][kk] = make_int4(cell_start[cn], cell_start[cn + 1],
                                 t_base[(tx * g.td[1] + ty) * g.td[2] + tz],
                                 (sx + 2) * 25 + (sy + 2) * 5 + (sz + 2));
    }
    __syncthreads();
    // each cell's table as ranges: consecutive entries that continue one sorted
    // range in the same tile brick under the same image shift merge, and empty
    // cells drop out
    if (threadIdx.x < g.bvol) {
        int4 *row = ctab[threadIdx.x];
        int m = 0;
        for (int k = 0; k < ncand; ++k) {
            const int4 e = row[k];
            if (e.x == e.y) continue;
            if (m > 0 && row[m - 1].y == e.x && row[m - 1].z == e.z && row[m - 1].w == e.w)
                row[m - 1].y = e.y;
            else
                row[m++] = e;
        }
        nrange[threadIdx.x] = m;
    }
    __syncthreads();
    if (t_total > kMaxTileAtoms) {
        if (chunk == 0)
            for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) cnt[i] = 0;
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int s = lane % kEmitLanes;
    const int nrows = i1 - i0;
    const int rows_per_warp = 32 / kEmitLanes;
    const int cap = a.width / kEmitLanes;
    for (int r0 = (chunk * nw + warp) * rows_per_warp; r0 < nrows;
         r0 += nchunk * nw * rows_per_warp) {
        const int r = r0 + lane / kEmitLanes;
        const bool act = r < nrows;
        const int i = i0 + (act ? r : 0);
        int c[3] = {0, 0, 0};
        if (act) {
            const int lc = cell_s[i] - (int)(b * g.bvol);
            emit_cells(a, &sargs, i, s, ctab[lc], shtab, nrange[lc], xs32[i], xs64, xs32, cap, c, scr,
                       t_total, flags);
        }
        const int mine = c[0] + c[1] + c[2];
        // this lane's first row slot in each class: the classes in order, and in
        // each class the lanes in order (exclusive scan over the row's 4 lanes)
        int start[3], row_tot = 0, lane_max = mine;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            int incl = c[k];
#pragma unroll
            for (int o = 1; o < kEmitLanes; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (s >= o) incl += y;
            }
            const int tot_k = __shfl_sync(0xffffffffu, incl, (lane / kEmitLanes) * kEmitLanes + kEmitLanes - 1);
            start[k] = row_tot + incl - c[k];
            row_tot += tot_k;
        }
#pragma unroll
        for (int o = 1; o < kEmitLanes; o <<= 1)
            lane_max = max(lane_max, __shfl_xor_sync(0xffffffffu, lane_max, o));
        const bool fits = lane_max <= cap && row_tot <= a.width;
        if (act && fits) {
            // move this lane's entries to their row slots (class order, lanes
            // interleaved inside a class), then pad to the stripe end with the
            // tile's far sentinel slot
            for (int m = 0; m < mine; ++m) {
                const uint32_t v = scr[list_index(kEmitLanes * m + s, i, a.n)];
                const int cls = (int)(v >> 16);
                const int slot = cls == 0 ? start[0]++ : (cls == 1 ? start[1]++ : start[2]++);
                nbr[list_index(slot, i, a.n)] = (uint16_t)(v & 0xffffu);
            }
            const int pad_end = (row_tot + kListStripe - 1) / kListStripe * kListStripe;
            for (int k = row_tot + ((s - row_tot) % kEmitLanes + kEmitLanes) % kEmitLanes; k < pad_end;
                 k += kEmitLanes)
                nbr[list_index(k, i, a.n)] = (uint16_t)t_total;
        }
        if (act && s == 0) {
            cnt[i] = fits ? row_tot : 0;
            if (!fits) atomicMax(&flags[kFlagMaxRow], max(row_tot, kEmitLanes * lane_max));
        }
    }
}

// Per-atom search (qeq_set_neighbor_method QEQ_NL_ATOM): the form of the paper's
// Triton neighbour kernel (Sec. 3.1), one thread per atom looping over the
// cells around its own, written in this library's list format so that the
// real-space kernels take either list.  First the tile table of every brick
// (one warp a brick), then one thread per sorted atom: a counting pass over its
// (2 reach + 1)^3 neighbour cells gives the sizes of the three distance
// classes, and a placing pass writes each kept candidate at the next slot of
// its class.  Both passes take the same pair decision as k_emit (FP32 outside
// the band, FP64 with a fixed operation order inside), so the pair set is the
// same bit for bit; only the order inside a class differs.
__global__ void __launch_bounds__(32)
k_tile_tables(BrickGeom g, const int32_t *__restrict__ cell_start, int4 *__restrict__ tile_tab,
              int32_t *__restrict__ tile_tot, int32_t *__restrict__ flags) {
    __shared__ int t_start[kMaxTileBricks], t_base[kMaxTileBricks], t_code[kMaxTileBricks], t_total;
    const int64_t b = blockIdx.x;
    tile_table(g, b, cell_start, t_start, t_base, t_code, &t_total);
    __syncwarp();
    for (int rb = threadIdx.x; rb < g.T; rb += 32)
        tile_tab[b * g.T + rb] = make_int4(t_start[rb], t_base[rb], t_code[rb], 0);
    if (threadIdx.x == 0) {
        tile_tot[b] = t_total;
        atomicMax(&flags[kFlagMaxTile], t_total);
        atomicMax(&flags[kFlagMaxRows], cell_start[(b + 1) * g.bvol] - cell_start[b * g.bvol]);
    }
}

// One candidate test of the per-atom search: keep (FP32 outside the band, FP64
// inside) and the distance class from the FP32 squared distance.
__device__ __forceinline__ bool atom_pair_keep(const EmitArgs &a, const double4_32a &xi,
                                               const float4 &xf, const float4 &xj,
                                               const double4_32a *__restrict__ xs64, int j,
                                               int sx, int sy, int sz, float shx, float shy,
                                               float shz, int &cls) {
    const float dxf = (xj.x - xf.x) + shx;
    const float dyf = (xj.y - xf.y) + shy;
    const float dzf = (xj.z - xf.z) + shz;
    const float d2f = dxf * dxf + dyf * dyf + dzf * dzf;
    cls = (d2f >= a.t_near) + (d2f >= a.t_cut);
    if (d2f < a.lo) return true;
    if (d2f > a.hi) return false;
    const double4_32a xj64 = xs64[j];
    const double dx = __dadd_rn(__dsub_rn(xj64.x, xi.x), image_shift(sx, a.Lx, a.L2x));
    const double dy = __dadd_rn(__dsub_rn(xj64.y, xi.y), image_shift(sy, a.Ly, a.L2y));
    const double dz = __dadd_rn(__dsub_rn(xj64.z, xi.z), image_shift(sz, a.Lz, a.L2z));
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return d2 < a.rl2;
}

template <bool PLACE>
__device__ __forceinline__ void atom_search(const EmitArgs &a, const BrickGeom &g, int i, int cx,
                                            int cy, int cz, int64_t b, const double4_32a &xi,
                                            const float4 &xf, const double4_32a *__restrict__ xs64,
                                            const float4 *__restrict__ xs32,
                                            const int32_t *__restrict__ cell_start,
                                            const int4 *__restrict__ ttab, int (&k)[3],
                                            uint16_t *__restrict__ nbr) {
    const int bx = cx / g.B[0], by = cy / g.B[1], bz = cz / g.B[2];
    for (int ox = -a.rx; ox <= a.rx; ++ox) {
        const int ux = cx + ox, sx = floor_div(ux, a.ncx), wx = ux - sx * a.ncx;
        const int tx = floor_div(ux, g.B[0]) - bx + g.br[0];
        const float shx = (float)sx * a.Lfx;
        for (int oy = -a.ry; oy <= a.ry; ++oy) {
            const int uy = cy + oy, sy = floor_div(uy, a.ncy), wy = uy - sy * a.ncy;
            const int ty = floor_div(uy, g.B[1]) - by + g.br[1];
            const float shy = (float)sy * a.Lfy;
            for (int oz = -a.rz; oz <= a.rz; ++oz) {
                const int uz = cz + oz, sz = floor_div(uz, a.ncz), wz = uz - sz * a.ncz;
                const int tz = floor_div(uz, g.B[2]) - bz + g.br[2];
                const float shz = (float)sz * a.Lfz;
                const bool self_img = (sx == 0) && (sy == 0) && (sz == 0);
                const int cn = cell_index(g, wx, wy, wz);
                const int jb = cell_start[cn], je = cell_start[cn + 1];
                const int tbase = PLACE ? ttab[(tx * g.td[1] + ty) * g.td[2] + tz].y : 0;
                for (int j = jb; j < je; ++j) {
                    if (self_img && j == i) continue;
                    int cls;
                    if (!atom_pair_keep(a, xi, xf, xs32[j], xs64, j, sx, sy, sz, shx, shy, shz, cls))
                        continue;
                    if (PLACE) {
                        const int slot = k[cls]++;
                        if (slot < a.width) nbr[list_index(slot, i, a.n)] = (uint16_t)(j + tbase);
                    } else {
                        ++k[cls];
                    }
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kEmitThreads)
k_emit_atom(EmitArgs a, BrickGeom g, const double4_32a *__restrict__ xs64,
            const float4 *__restrict__ xs32, const int32_t *__restrict__ cell_s,
            const int32_t *__restrict__ cell_start, const int4 *__restrict__ tile_tab,
            const int32_t *__restrict__ tile_tot, uint16_t *__restrict__ nbr,
            int32_t *__restrict__ cnt, int32_t *__restrict__ flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int c = cell_s[i];
    int cx, cy, cz;
    cell_coords(g, c, cx, cy, cz);
    const int64_t b = c / g.bvol;
    const int total = tile_tot[b];
    if (total > kMaxTileAtoms) {  // the host reports the oversized tile
        cnt[i] = 0;
        return;
    }
    const double4_32a xi = xs64[i];
    const float4 xf = xs32[i];
    const int4 *ttab = tile_tab + b * g.T;
    int k[3] = {0, 0, 0};
    atom_search<false>(a, g, i, cx, cy, cz, b, xi, xf, xs64, xs32, cell_start, ttab, k, nbr);
    const int row_tot = k[0] + k[1] + k[2];
    if (row_tot > a.width) {
        cnt[i] = 0;
        atomicMax(&flags[kFlagMaxRow], row_tot);
        return;
    }
    int start[3] = {0, k[0], k[0] + k[1]};
    atom_search<true>(a, g, i, cx, cy, cz, b, xi, xf, xs64, xs32, cell_start, ttab, start, nbr);
    const int pad_end = (row_tot + kListStripe - 1) / kListStripe * kListStripe;
    for (int q = row_tot; q < pad_end; ++q) nbr[list_index(q, i, a.n)] = (uint16_t)total;
    cnt[i] = row_tot;
}

// COO scatter, one block per brick: sorted row i with entries k < cnt[i] goes to
// slots offset[i] + k as (original i, original j, image code), so the pair order
// is the list's.
__global__ void __launch_bounds__(kEmitThreads)
k_coo_scatter(int n, BrickGeom g, const int32_t *__restrict__ cell_start,
              const int32_t *__restrict__ perm, const uint16_t *__restrict__ nbr,
              const int32_t *__restrict__ cnt, const int32_t *__restrict__ offset,
              int32_t *__restrict__ coo_i, int32_t *__restrict__ coo_j, int8_t *__restrict__ coo_code) {
    __shared__ int t_start[kMaxTileBricks], t_base[kMaxTileBricks], t_code[kMaxTileBricks], t_total;
    const int64_t b = blockIdx.x;
    if (threadIdx.x < 32) tile_table(g, b, cell_start, t_start, t_base, t_code, &t_total);
    __syncthreads();
    const int i0 = t_start[g.center], i1 = cell_start[(b + 1) * g.bvol];
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int c = cnt[i];
        const int off = offset[i];
        const int ai = perm[i];
        for (int k = 0; k < c; ++k) {
            const int e = nbr[list_index(k, i, n)];
            const int rb = tile_locate(e, g.T, t_start, t_base);
            coo_i[off + k] = ai;
            coo_j[off + k] = perm[e - t_base[rb]];
            coo_code[off + k] = (int8_t)t_code[rb];
        }
    }
}

// Max squared displacement since the last build: block maxima, and the last
// block to finish (ticket counter, reset to 0) reduces them into *out.
__global__ void k_max_disp2(int n, const double *__restrict__ R, const double *__restrict__ R0,
                            double *__restrict__ part, double *__restrict__ out,
                            unsigned int *__restrict__ ticket) {
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double dx = R[3 * (size_t)i] - R0[3 * (size_t)i];
        const double dy = R[3 * (size_t)i + 1] - R0[3 * (size_t)i + 1];
        const double dz = R[3 * (size_t)i + 2] - R0[3 * (size_t)i + 2];
        double d2 = dx * dx + dy * dy + dz * dz;
        if (!(d2 == d2)) d2 = INFINITY;
        m = fmax(m, d2);
    }
    max_last_block(m, part, out, ticket);
}

}  // namespace

int nl_configure(qeq_ctx *ctx) {
    const qeq_params &p = ctx->p;
    ctx->rl = p.r_cut + p.skin;
    ctx->rl2 = ctx->rl * ctx->rl;
    double lmax = 0.0;
    BrickGeom &g = ctx->geom;
    g.T = 1;
    g.bvol = 1;
    for (int d = 0; d < 3; ++d) {
        const double L = p.box[d];
        lmax = std::max(lmax, L);
        // cells at least r_list / kCellDiv wide (with a relative margin so that
        // rounding in the cell index cannot move an atom by more than one cell);
        // the emit then visits (2 reach + 1)^3 cells.  With four or more cells the
        // count is made even and cells pair into bricks of 2; with fewer, a brick
        // is one cell.
        int nc = (int)std::floor(L / (ctx->rl / kCellDiv * (1.0 + 1e-9)));
        if (nc < 1) nc = 1;
        if (nc > 1024) nc = 1024;
        if (nc >= 4) nc &= ~1;
        ctx->nc[d] = nc;
        ctx->cw[d] = L / nc;
        ctx->reach[d] = (int)std::ceil(ctx->rl * (1.0 + 1e-9) / ctx->cw[d]);
        // image index |s| <= ceil(reach / nc) must stay within [-2, 2]
        const int smax = (ctx->reach[d] + nc - 1) / nc;
        if (smax > 2)
            return set_error(ctx, QEQ_ERR_UNSUPPORTED,
                             "box edge %d (%.6g) is shorter than half the list radius %.6g", d, L,
                             ctx->rl);
        g.nc[d] = nc;
        g.B[d] = nc >= 4 ? 2 : 1;
        g.nb[d] = nc / g.B[d];
        g.br[d] = (ctx->reach[d] + g.B[d] - 1) / g.B[d];
        g.td[d] = 2 * g.br[d] + 1;
        g.T *= g.td[d];
        g.bvol *= g.B[d];
    }
    if (g.T > kMaxTileBricks)
        return set_error(ctx, QEQ_ERR_UNSUPPORTED, "tile of %d bricks exceeds %d", g.T, kMaxTileBricks);
    g.center = (g.br[0] * g.td[1] + g.br[1]) * g.td[2] + g.br[2];
    g.nbricks = (int64_t)g.nb[0] * g.nb[1] * g.nb[2];
    ctx->ncell = (int64_t)ctx->nc[0] * ctx->nc[1] * ctx->nc[2];
    // FP32 prefilter band: |d2_fp32 - d2_exact| is bounded by a few ulp of the
    // coordinates times the list radius; 4e-5 * rl * (Lmax + rl) is >10x that bound.
    const double margin = 4e-5 * ctx->rl * (lmax + ctx->rl) + 1e-6;
    ctx->rl2f_lo = (float)(ctx->rl2 - margin);
    ctx->rl2f_hi = (float)(ctx->rl2 + margin);
    return QEQ_OK;
}

int nl_alloc_list(qeq_ctx *ctx, int width) {
    if (width > kMaxWidthLimit)
        return set_error(ctx, QEQ_ERR_CAPACITY, "neighbour row of %d entries exceeds the limit %d",
                         width, kMaxWidthLimit);
    dev_free(ctx, ctx->nbr);
    dev_free(ctx, ctx->nbr_scratch);
    ctx->nbr = nullptr;
    ctx->nbr_scratch = nullptr;
    int rc = dev_alloc(ctx, (void **)&ctx->nbr, sizeof(uint16_t) * (size_t)width * ctx->n);
    if (rc) return rc;
    rc = dev_alloc(ctx, (void **)&ctx->nbr_scratch, sizeof(uint32_t) * (size_t)width * ctx->n);
    if (rc) return rc;
    ctx->width = width;
    return QEQ_OK;
}

int nl_alloc(qeq_ctx *ctx) {
    const int64_t n = ctx->n;
    struct {
        void **ptr;
        size_t bytes;
    } bufs[] = {
        {(void **)&ctx->cell_of, sizeof(int32_t) * n},
        {(void **)&ctx->cell_count, sizeof(int32_t) * ctx->ncell},
        {(void **)&ctx->cell_start, sizeof(int32_t) * (ctx->ncell + 1)},
        {(void **)&ctx->cell_fill, sizeof(int32_t) * ctx->ncell},
        {(void **)&ctx->tmp_list, sizeof(int32_t) * n},
        {(void **)&ctx->perm, sizeof(int32_t) * n},
        {(void **)&ctx->cell_s, sizeof(int32_t) * n},
        {(void **)&ctx->wrap_off, sizeof(double) * 3 * n},
        {(void **)&ctx->R_build, sizeof(double) * 3 * n},
        {(void **)&ctx->xs64, sizeof(double4_32a) * n},
        {(void **)&ctx->xs32, sizeof(float4) * n},
        {(void **)&ctx->cnt, sizeof(int32_t) * n},
        {(void **)&ctx->d_flags, sizeof(int32_t) * kNumFlags},
        {(void **)&ctx->tile_tab, sizeof(int4) * ctx->geom.nbricks * ctx->geom.T},
        {(void **)&ctx->tile_tot, sizeof(int32_t) * ctx->geom.nbricks},
    };
    for (auto &b : bufs) {
        int rc = dev_alloc(ctx, b.ptr, b.bytes);
        if (rc) return rc;
    }
    ctx->h_flags = new (std::nothrow) int32_t[kNumFlags];
    if (!ctx->h_flags) return set_error(ctx, QEQ_ERR_NOMEM, "host allocation failed");
    // every flag starts at 0; the builds clear all but the bounds flag
    cudaMemsetAsync(ctx->d_flags, 0, sizeof(int32_t) * kNumFlags, ctx->alloc_stream);
    int width = ctx->p.max_neighbors;
    if (width <= 0) {
        const double V = ctx->p.box[0] * ctx->p.box[1] * ctx->p.box[2];
        const double mean = 4.0 / 3.0 * kPi * ctx->rl2 * ctx->rl * (double)n / V;
        width = (int)std::ceil(1.2 * mean + 32.0);
    }
    width = std::max(kListStripe, (width + kListStripe - 1) / kListStripe * kListStripe);
    return nl_alloc_list(ctx, width);
}

void nl_free(qeq_ctx *ctx) {
    void *ptrs[] = {ctx->cell_of, ctx->cell_count, ctx->cell_start, ctx->cell_fill, ctx->tmp_list,
                    ctx->perm,    ctx->cell_s,     ctx->wrap_off,   ctx->R_build,   ctx->xs64,
                    ctx->xs32,    ctx->nbr,        ctx->cnt,        ctx->d_flags,
                    ctx->tile_tab, ctx->tile_tot, ctx->nbr_scratch};
    for (void *p : ptrs) dev_free(ctx, p);
    delete[] ctx->h_flags;
}

// Launches the pair emission of the selected search; returns the kernels launched.
static int launch_emit(qeq_ctx *ctx, cudaStream_t s) {
    EmitArgs a;
    a.n = (int)ctx->n;
    a.ncx = ctx->nc[0]; a.ncy = ctx->nc[1]; a.ncz = ctx->nc[2];
    a.rx = ctx->reach[0]; a.ry = ctx->reach[1]; a.rz = ctx->reach[2];
    a.Lx = ctx->p.box[0]; a.Ly = ctx->p.box[1]; a.Lz = ctx->p.box[2];
    a.L2x = 2.0 * a.Lx; a.L2y = 2.0 * a.Ly; a.L2z = 2.0 * a.Lz;
    a.Lfx = (float)a.Lx; a.Lfy = (float)a.Ly; a.Lfz = (float)a.Lz;
    a.rl2 = ctx->rl2;
    a.lo = ctx->rl2f_lo;
    a.hi = ctx->rl2f_hi;
    a.t_near = (float)(ctx->rl2 / 3.0);
    a.t_cut = (float)(ctx->p.r_cut * ctx->p.r_cut);
    a.width = ctx->width;
    if (ctx->nl_method == QEQ_NL_ATOM) {
        k_tile_tables<<<(unsigned)ctx->geom.nbricks, 32, 0, s>>>(ctx->geom, ctx->cell_start,
                                                                 ctx->tile_tab, ctx->tile_tot,
                                                                 ctx->d_flags);
        k_emit_atom<<<(unsigned)((ctx->n + kEmitThreads - 1) / kEmitThreads), kEmitThreads, 0, s>>>(
            a, ctx->geom, ctx->xs64, ctx->xs32, ctx->cell_s, ctx->cell_start, ctx->tile_tab,
            ctx->tile_tot, ctx->nbr, ctx->cnt, ctx->d_flags);
        return 2;
    }
    // blocks per brick: enough to put about kEmitBlocksPerSm blocks on every SM
    // when the box has few bricks, at most one per 32 rows of the largest brick
    // (from the previous build; 1.5 x the mean before the first)
    const int64_t nb = ctx->geom.nbricks;
    const int rows = ctx->max_rows > 0 ? ctx->max_rows
                                       : (int)std::ceil(1.5 * (double)ctx->n / (double)nb);
    const int64_t want = (int64_t)kEmitBlocksPerSm * ctx->sm_count;
    const int nchunk = (int)std::max<int64_t>(
        1, std::min<int64_t>((want + nb - 1) / nb, (rows + 31) / 32));
    k_emit<<<(unsigned)(nb * nchunk), kEmitThreads, 0, s>>>(
        a, ctx->geom, nchunk, ctx->xs64, ctx->xs32, ctx->cell_s, ctx->cell_start, ctx->nbr,
        ctx->nbr_scratch, ctx->cnt, ctx->tile_tab, ctx->tile_tot, ctx->d_flags);
    return 1;
}

int nl_build(qeq_ctx *ctx, const double *R, cudaStream_t s) {
    const int n = (int)ctx->n;
    ctx->gathered = false;  // the sorted order changes
    prof_begin(ctx, kPhNeighbor, s);
    ctx->launches += 4;
    cudaMemsetAsync(ctx->cell_count, 0, sizeof(int32_t) * ctx->ncell, s);
    cudaMemsetAsync(ctx->d_flags, 0, sizeof(int32_t) * kFlagBounds, s);  // the bounds flag persists
    k_wrap_bin<<<grid_for(n), kThreads, 0, s>>>(
        n, R, ctx->p.box[0], ctx->p.box[1], ctx->p.box[2], ctx->cw[0], ctx->cw[1], ctx->cw[2],
        ctx->geom, ctx->cell_of, ctx->cell_count, ctx->wrap_off, ctx->R_build, ctx->d_flags);
    k_scan<<<1, kScanThreads, 0, s>>>(ctx->ncell, ctx->cell_count, ctx->cell_start, ctx->cell_fill);
    k_scatter<<<grid_for(n), kThreads, 0, s>>>(n, ctx->cell_of, ctx->cell_start, ctx->cell_fill,
                                               ctx->tmp_list);
    k_cell_sort<<<grid_for(ctx->ncell * 32), kThreads, 0, s>>>(
        ctx->ncell, ctx->cell_start, ctx->tmp_list, R, ctx->wrap_off, ctx->perm, ctx->cell_s,
        ctx->xs64, ctx->xs32);
    ctx->launches += launch_emit(ctx, s);
    prof_end(ctx, s);
    for (int attempt = 0; attempt < 4; ++attempt) {
        cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, sizeof(int32_t) * kNumFlags,
                        cudaMemcpyDeviceToHost, s);
        int rc = cuda_check(ctx, cudaStreamSynchronize(s), "neighbour build");
        if (rc) return rc;
        if (ctx->h_flags[kFlagNonFinite]) {
            ctx->list_valid = false;
            return set_error(ctx, QEQ_ERR_NONFINITE, "non-finite position in neighbor_build");
        }
        if (ctx->h_flags[kFlagMaxTile] > kMaxTileAtoms) {
            ctx->list_valid = false;
            return set_error(ctx, QEQ_ERR_CAPACITY,
                             "a brick tile holds %d atoms, more than the %d of 16-bit entries",
                             ctx->h_flags[kFlagMaxTile], kMaxTileAtoms);
        }
        ctx->max_tile = ctx->h_flags[kFlagMaxTile];
        ctx->max_rows = ctx->h_flags[kFlagMaxRows];
        const int need = ctx->h_flags[kFlagMaxRow];
        if (need <= ctx->width) break;
        // grow (the paper's estimate-plus-buffer, Sec. 3.1) and emit again
        rc = nl_alloc_list(ctx, (int)std::ceil(need * 1.1 / kListStripe) * kListStripe + kListStripe);
        if (rc) {
            ctx->list_valid = false;
            return rc;
        }
        cudaMemsetAsync(ctx->d_flags, 0, sizeof(int32_t) * kFlagBounds, s);
        prof_begin(ctx, kPhNeighbor, s);
        ctx->launches += launch_emit(ctx, s);
        prof_end(ctx, s);
    }
    // launch capacities of the real-space kernels (grown in steps, never shrunk).
    // Rows: 1.15 x the mean brick (a brick above it takes a second pass), at
    // most the largest brick.  For the 300,000-atom water box (mean 73, max 90)
    // this keeps 87% of the lanes busy against 76% at the largest brick.
    const int tcap = (ctx->max_tile + 32 + 63) / 64 * 64;
    const int mean_cap = (int)std::ceil(1.15 * (double)ctx->n / (double)ctx->geom.nbricks);
    const int rcap = (std::min(ctx->max_rows, mean_cap) + 7) / 8 * 8;
    ctx->tile_cap = std::max(ctx->tile_cap, tcap);
    ctx->rows_cap = std::max(ctx->rows_cap, rcap);
    int rc = real_tile_reserve(ctx);
    if (rc) {
        ctx->list_valid = false;
        return rc;
    }
    ctx->list_valid = true;
    ctx->n_builds++;
    return cuda_check(ctx, cudaGetLastError(), "neighbour build launch");
}

int nl_displacement(qeq_ctx *ctx, const double *R, cudaStream_t s, double *max_disp2) {
    prof_begin(ctx, kPhIntegrate, s);
    k_max_disp2<<<ctx->red_grid, kThreads, 0, s>>>((int)ctx->n, R, ctx->R_build, ctx->part,
                                                ctx->scal + kScMaxDisp2, ctx->ticket);
    prof_end(ctx, s);
    ctx->launches += 1;
    if (max_disp2) {
        cudaMemcpyAsync(ctx->h_scal + kScMaxDisp2, ctx->scal + kScMaxDisp2, sizeof(double),
                        cudaMemcpyDeviceToHost, s);
        int rc = cuda_check(ctx, cudaStreamSynchronize(s), "displacement check");
        if (rc) return rc;
        *max_disp2 = ctx->h_scal[kScMaxDisp2];
    }
    return QEQ_OK;
}

// Device COO copy of the current list: an exclusive scan of the row counts
// (k_scan into a temporary buffer) gives each row's first slot.
int nl_export_coo(qeq_ctx *ctx, int64_t capacity, int32_t *coo_i, int32_t *coo_j, int8_t *coo_code,
                  int64_t *n_pairs, cudaStream_t s) {
    const int n = (int)ctx->n;
    int32_t *scan_out = nullptr;
    int rc = dev_alloc(ctx, (void **)&scan_out, sizeof(int32_t) * (size_t)(n + 1) * 2);
    if (rc) return rc;
    k_scan<<<1, kScanThreads, 0, s>>>(n, ctx->cnt, scan_out, scan_out + n + 1);
    int32_t total = 0;
    cudaError_t e = cudaMemcpyAsync(&total, scan_out + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    rc = cuda_check(ctx, e, "coo scan");
    if (!rc) {
        *n_pairs = total;
        if (total > capacity) {
            rc = set_error(ctx, QEQ_ERR_CAPACITY, "COO needs %d pairs, capacity is %lld", total,
                           (long long)capacity);
        } else {
            k_coo_scatter<<<(unsigned)ctx->geom.nbricks, kEmitThreads, 0, s>>>(
                n, ctx->geom, ctx->cell_start, ctx->perm, ctx->nbr, ctx->cnt, scan_out, coo_i,
                coo_j, coo_code);
            ctx->launches += 2;
            rc = cuda_check(ctx, cudaGetLastError(), "coo scatter");
        }
    }
    dev_free(ctx, scan_out);
    if (!ctx->async_alloc) cudaDeviceSynchronize();
    return rc;
}

int nl_export(qeq_ctx *ctx, int32_t *counts, int32_t *nbr_out, int8_t *shift_out) {
    const int64_t n = ctx->n;
    const int w = ctx->width;
    const BrickGeom &g = ctx->geom;
    std::vector<int32_t> perm(n), cnt(n), cell_start(ctx->ncell + 1);
    std::vector<uint16_t> nbr((size_t)w * n);
    int rc = cuda_check(ctx, ctx->async_alloc ? cudaStreamSynchronize(ctx->alloc_stream)
                                              : cudaDeviceSynchronize(), "export sync");
    if (rc) return rc;
    rc = cuda_check(ctx, cudaMemcpy(perm.data(), ctx->perm, sizeof(int32_t) * n, cudaMemcpyDeviceToHost),
                    "export perm");
    if (rc) return rc;
    rc = cuda_check(ctx, cudaMemcpy(cnt.data(), ctx->cnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost),
                    "export counts");
    if (rc) return rc;
    rc = cuda_check(ctx, cudaMemcpy(cell_start.data(), ctx->cell_start,
                                    sizeof(int32_t) * (ctx->ncell + 1), cudaMemcpyDeviceToHost),
                    "export cells");
    if (rc) return rc;
    rc = cuda_check(ctx, cudaMemcpy(nbr.data(), ctx->nbr, sizeof(uint16_t) * (size_t)w * n,
                                    cudaMemcpyDeviceToHost),
                    "export list");
    if (rc) return rc;
    // per brick: the tile table (first tile index, first sorted atom, image shift
    // of each tile brick), then every row of the brick decoded through it
    std::vector<int> off(g.T + 1), start(g.T), shift(3 * g.T);
    for (int64_t b = 0; b < g.nbricks; ++b) {
        off[0] = 0;
        for (int rb = 0; rb < g.T; ++rb) {
            int s[3];
            const int64_t wb = tile_brick(g, b, rb, s);
            start[rb] = cell_start[wb * g.bvol];
            off[rb + 1] = off[rb] + cell_start[(wb + 1) * g.bvol] - start[rb];
            for (int d = 0; d < 3; ++d) shift[3 * rb + d] = s[d];
        }
        for (int64_t si = cell_start[b * g.bvol]; si < cell_start[(b + 1) * g.bvol]; ++si) {
            const int64_t atom = perm[si];
            if (counts) counts[atom] = cnt[si];
            for (int k = 0; k < cnt[si]; ++k) {
                const int e = nbr[list_index(k, si, n)];
                const int rb = (int)(std::upper_bound(off.begin(), off.end(), e) - off.begin()) - 1;
                const int32_t j = start[rb] + (e - off[rb]);
                if (nbr_out) nbr_out[atom * w + k] = perm[j];
                if (shift_out)
                    for (int d = 0; d < 3; ++d) shift_out[(atom * w + k) * 3 + d] = (int8_t)shift[3 * rb + d];
            }
        }
    }
    return QEQ_OK;
}

}  // namespace qeq

// ---------------------------------------------------------------------------
// Allocation-free neighbour build (qeq_neighbor_build_noalloc).
//
// Some callers cannot call cudaMalloc / cudaFree.  One example is a plugin
// inside an MD or serving engine that owns every byte of device memory
// through its own arena.  Another is a latency-critical loop that cannot
// afford the device-wide synchronisation cudaFree implies.  A third runs
// under a hard memory budget where an allocation failure mid-run is not
// acceptable.  For them this entry point keeps its scratch in one file-scope
// device array of fixed size, so it needs no qeq_ctx.  That scratch holds the
// cell histogram and offsets, the permutation, the wrap offsets and the
// sorted positions.  The caller passes the inputs and the outputs.
//
// The array lives in every device that loads the library until the process
// exits, and every call shares it.  Each call clears what must start at zero
// (cell counts, flags).  Calls whose work overlaps on the GPU, on different
// streams or from different host threads, race on the array: serialise them.
// ---------------------------------------------------------------------------

namespace qeq {

namespace {

constexpr int kNoAllocMaxAtoms = 32768;
constexpr int kNoAllocMaxCells = 32768;

struct NoAllocScratch {
    double4_32a xs64[kNoAllocMaxAtoms];
    float4 xs32[kNoAllocMaxAtoms];
    double wrap_off[3 * kNoAllocMaxAtoms];
    double R_build[3 * kNoAllocMaxAtoms];
    int32_t cell_of[kNoAllocMaxAtoms];
    int32_t tmp_list[kNoAllocMaxAtoms];
    int32_t perm[kNoAllocMaxAtoms];
    int32_t cell_s[kNoAllocMaxAtoms];
    int32_t cell_count[kNoAllocMaxCells];
    int32_t cell_start[kNoAllocMaxCells + 1];
    int32_t cell_fill[kNoAllocMaxCells];
    int32_t flags[kNumFlags];
};

// About 3.5 MB per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

// In host code g_noalloc_scratch is only a host-side stand-in for the symbol.
// The device address comes from cudaGetSymbolAddress, once per device, with
// that device current.
constexpr int kMaxDevices = 256;
std::mutex g_noalloc_mutex;
void *g_noalloc_addr[kMaxDevices] = {};

int noalloc_scratch(NoAllocScratch **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(nullptr, QEQ_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    }
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(nullptr, QEQ_ERR_UNSUPPORTED, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return set_error(nullptr, QEQ_ERR_CUDA, "cudaGetSymbolAddress: %s",
                             cudaGetErrorString(e));
        }
        g_noalloc_addr[dev] = ptr;
    }
    *out = static_cast<NoAllocScratch *>(g_noalloc_addr[dev]);
    return QEQ_OK;
}

// The pair emission of k_emit, written for the caller: rows and neighbour
// indices in original atom numbering, rows row-major [N][width].
__global__ void __launch_bounds__(kThreads)
k_emit_original(EmitArgs a, const double4_32a *__restrict__ xs64, const float4 *__restrict__ xs32,
                const int32_t *__restrict__ cell_s, const int32_t *__restrict__ cell_start,
                const int32_t *__restrict__ perm, int32_t *__restrict__ nbr,
                int32_t *__restrict__ cnt, int32_t *__restrict__ flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int c = cell_s[i];
    const int cx = c / (a.ncy * a.ncz), cy = (c / a.ncz) % a.ncy, cz = c % a.ncz;
    const double4_32a xi = xs64[i];
    const float4 xf = xs32[i];
    int32_t *row = nbr + (size_t)perm[i] * a.width;
    int count = 0;
    for (int ox = -a.rx; ox <= a.rx; ++ox) {
        const int ux = cx + ox, sx = floor_div(ux, a.ncx), wx = ux - sx * a.ncx;
        const double shx = image_shift(sx, a.Lx, a.L2x);
        const float shxf = (float)sx * a.Lfx;
        for (int oy = -a.ry; oy <= a.ry; ++oy) {
            const int uy = cy + oy, sy = floor_div(uy, a.ncy), wy = uy - sy * a.ncy;
            const double shy = image_shift(sy, a.Ly, a.L2y);
            const float shyf = (float)sy * a.Lfy;
            for (int oz = -a.rz; oz <= a.rz; ++oz) {
                const int uz = cz + oz, sz = floor_div(uz, a.ncz), wz = uz - sz * a.ncz;
                const double shz = image_shift(sz, a.Lz, a.L2z);
                const float shzf = (float)sz * a.Lfz;
                const int cn = (wx * a.ncy + wy) * a.ncz + wz;
                const bool self_img = (sx == 0) && (sy == 0) && (sz == 0);
                const int32_t code = ((sx + 2) * 25 + (sy + 2) * 5 + (sz + 2)) << kIndexBits;
                const int jb = cell_start[cn], je = cell_start[cn + 1];
                for (int j = jb; j < je; ++j) {
                    if (self_img && j == i) continue;
                    const float4 xj = xs32[j];
                    const float dxf = (xj.x - xf.x) + shxf;
                    const float dyf = (xj.y - xf.y) + shyf;
                    const float dzf = (xj.z - xf.z) + shzf;
                    const float d2f = dxf * dxf + dyf * dyf + dzf * dzf;
                    bool keep;
                    if (d2f < a.lo) {
                        keep = true;
                    } else if (d2f > a.hi) {
                        keep = false;
                    } else {
                        const double4_32a xj64 = xs64[j];
                        const double dx = __dadd_rn(__dsub_rn(xj64.x, xi.x), shx);
                        const double dy = __dadd_rn(__dsub_rn(xj64.y, xi.y), shy);
                        const double dz = __dadd_rn(__dsub_rn(xj64.z, xi.z), shz);
                        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                                    __dmul_rn(dz, dz));
                        keep = d2 < a.rl2;
                    }
                    if (keep) {
                        if (count < a.width) row[count] = perm[j] | code;
                        ++count;
                    }
                }
            }
        }
    }
    cnt[perm[i]] = min(count, a.width);
    if (count > a.width) atomicMax(&flags[kFlagMaxRow], count);
}

}  // namespace

}  // namespace qeq

QEQ_API int qeq_neighbor_build_noalloc(const double *R, int64_t n_atoms, const double *box,
                                       double r_list, int32_t width, int32_t *counts,
                                       int32_t *nbr, int32_t *max_row, void *stream) {
    using namespace qeq;
    if (max_row) *max_row = 0;
    if (!R || !box || !counts || !nbr)
        return set_error(nullptr, QEQ_ERR_INVALID, "noalloc neighbour build: NULL argument");
    if (n_atoms < 1 || n_atoms > kNoAllocMaxAtoms)
        return set_error(nullptr, QEQ_ERR_CAPACITY,
                         "noalloc neighbour build: n_atoms %lld outside [1, %d]",
                         (long long)n_atoms, kNoAllocMaxAtoms);
    if (width < 1 || width > kMaxWidthLimit)
        return set_error(nullptr, QEQ_ERR_INVALID, "noalloc neighbour build: width %d outside [1, %d]",
                         width, kMaxWidthLimit);
    if (!(r_list > 0.0) || !std::isfinite(r_list))
        return set_error(nullptr, QEQ_ERR_INVALID, "noalloc neighbour build: r_list must be positive");
    int nc[3], reach[3];
    double cw[3], lmax = 0.0;
    for (int d = 0; d < 3; ++d) {
        if (!(box[d] > 0.0) || !std::isfinite(box[d]))
            return set_error(nullptr, QEQ_ERR_INVALID, "noalloc neighbour build: box[%d] invalid", d);
        lmax = std::max(lmax, box[d]);
        nc[d] = std::max(1, std::min(1024, (int)std::floor(box[d] / (r_list * (1.0 + 1e-9)))));
    }
    // fewer, larger cells when the grid would not fit the fixed cell table
    while ((int64_t)nc[0] * nc[1] * nc[2] > kNoAllocMaxCells) {
        int d = (nc[0] >= nc[1] && nc[0] >= nc[2]) ? 0 : (nc[1] >= nc[2] ? 1 : 2);
        nc[d] = std::max(1, nc[d] / 2);
    }
    for (int d = 0; d < 3; ++d) {
        cw[d] = box[d] / nc[d];
        reach[d] = (int)std::ceil(r_list * (1.0 + 1e-9) / cw[d]);
        if ((reach[d] + nc[d] - 1) / nc[d] > 2)
            return set_error(nullptr, QEQ_ERR_UNSUPPORTED,
                             "noalloc neighbour build: box edge %d shorter than r_list / 2", d);
    }
    const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    NoAllocScratch *S = nullptr;
    int rc = noalloc_scratch(&S);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)n_atoms;
    cudaMemsetAsync(S->cell_count, 0, sizeof(int32_t) * ncell, s);
    cudaMemsetAsync(S->flags, 0, sizeof(int32_t) * kNumFlags, s);
    // one cell per brick: the cell index is the plain (cx * ncy + cy) * ncz + cz
    BrickGeom g{};
    for (int d = 0; d < 3; ++d) {
        g.nc[d] = g.nb[d] = nc[d];
        g.B[d] = 1;
    }
    g.bvol = 1;
    k_wrap_bin<<<grid_for(n), kThreads, 0, s>>>(n, R, box[0], box[1], box[2], cw[0], cw[1], cw[2],
                                                g, S->cell_of, S->cell_count, S->wrap_off,
                                                S->R_build, S->flags);
    k_scan<<<1, kScanThreads, 0, s>>>(ncell, S->cell_count, S->cell_start, S->cell_fill);
    k_scatter<<<grid_for(n), kThreads, 0, s>>>(n, S->cell_of, S->cell_start, S->cell_fill,
                                               S->tmp_list);
    k_cell_sort<<<grid_for(ncell * 32), kThreads, 0, s>>>(ncell, S->cell_start, S->tmp_list, R,
                                                          S->wrap_off, S->perm, S->cell_s,
                                                          S->xs64, S->xs32);
    EmitArgs a;
    a.n = n;
    a.ncx = nc[0]; a.ncy = nc[1]; a.ncz = nc[2];
    a.rx = reach[0]; a.ry = reach[1]; a.rz = reach[2];
    a.Lx = box[0]; a.Ly = box[1]; a.Lz = box[2];
    a.L2x = 2.0 * a.Lx; a.L2y = 2.0 * a.Ly; a.L2z = 2.0 * a.Lz;
    a.Lfx = (float)box[0]; a.Lfy = (float)box[1]; a.Lfz = (float)box[2];
    a.rl2 = r_list * r_list;
    const double margin = 4e-5 * r_list * (lmax + r_list) + 1e-6;
    a.lo = (float)(a.rl2 - margin);
    a.hi = (float)(a.rl2 + margin);
    a.width = width;
    k_emit_original<<<grid_for(n), kThreads, 0, s>>>(a, S->xs64, S->xs32, S->cell_s, S->cell_start,
                                                     S->perm, nbr, counts, S->flags);
    int32_t flags[kNumFlags] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(flags, S->flags, sizeof(flags), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(nullptr, QEQ_ERR_CUDA, "noalloc neighbour build: %s", cudaGetErrorString(e));
    }
    if (flags[kFlagNonFinite])
        return set_error(nullptr, QEQ_ERR_NONFINITE, "noalloc neighbour build: non-finite position");
    if (flags[kFlagMaxRow] > width) {
        if (max_row) *max_row = flags[kFlagMaxRow];
        return set_error(nullptr, QEQ_ERR_CAPACITY,
                         "noalloc neighbour build: a row needs %d entries, width is %d",
                         flags[kFlagMaxRow], width);
    }
    return QEQ_OK;
}
