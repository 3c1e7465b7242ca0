// Periodic Coulomb apply v = Phi q and its field on one GB300.
//
// Phi = real space (Eq. ewald_real over the ELLPACK list, with the
// Gaussian-charge correction) + smooth PME (Alg. 2) + self term (Eq. ewald_self).
// Launch sequence per apply, all on the caller's stream:
//   gather_in   sorted copies (x, y, z, q), sigma and B-spline base/fraction
//   real        one thread per sorted atom over its ELLPACK row (no atomics)
//   spread      one thread per sorted atom, p^3 atomic adds onto the K^3 mesh
//   cuFFT R2C   (library call)
//   influence   Q^ *= G on the half spectrum, plus the mesh energy partial sums
//   cuFFT C2R   (library call; unnormalised, so phi = dE_rec/dQ directly)
//   gather_out  potential and field from the mesh, plus the self term, added to
//               the real-space part and written in original atom order, with
//               energy partial sums
//   finalize    one block per energy component (fixed-order, deterministic)
// FP64 mode runs all of it in double.  FP32_MIXED runs the pair math, the
// spreading, the FFT and the gather in float.  It accumulates rows in float
// chunks of 32 flushed into double, and keeps the energies and outputs in double.
#include <cmath>
#include <cstring>
#include <tuple>
#include <map>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "internal.cuh"

namespace qeq {

namespace {

template <typename T> struct V4;
template <> struct V4<double> { using type = double4_32a; };
template <> struct V4<float> { using type = float4; };
template <typename T> struct C2;
template <> struct C2<double> { using type = double2; };
template <> struct C2<float> { using type = float2; };

// ---------------------------------------------------------------------------
// gather_in: sorted copies of the inputs
// ---------------------------------------------------------------------------

// floor(u) and the fraction u - floor(u) of u < 2^31.  For u >= 0 both come
// from the bits of u (the fraction exact in 64-bit fixed point, then truncated
// to float); a negative u (an atom that left the box through its lower face
// since the list was built) takes the FP64 floor.
__device__ __forceinline__ void split_floor(double u, int &k, float &frac) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(u);
    if (b >> 63) {
        const double fl = floor(u);
        k = (int)fl;
        frac = f64_to_f32_trunc(u - fl);
        return;
    }
    const int e = (int)((b >> 52) & 0x7FF) - 1023;
    if (e < 0) {  // u < 1 (or 0)
        k = 0;
        frac = f64_to_f32_trunc(u);
        return;
    }
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = 52 - e;  // fraction bits (e <= 30)
    k = (int)(m >> sh);
    const unsigned long long f = m & ((1ull << sh) - 1);  // fraction = f 2^-sh
    if (f == 0) {
        frac = 0.0f;
        return;
    }
    const int lz = __clzll(f);                 // the leading one at bit 63 - lz
    const unsigned long long nf = f << lz;      // leading one at bit 63
    const int fe = (63 - lz) - sh;              // fraction = 1.xxx 2^fe
    frac = fe + 127 > 0 ? __int_as_float(((fe + 127) << 23) | (int)((nf >> 40) & 0x7FFFFF)) : 0.0f;
}

template <typename T>
__global__ void k_gather_in(int n, const int32_t *__restrict__ perm, const double *__restrict__ R,
                            const double *__restrict__ w, const double *__restrict__ q,
                            const double *__restrict__ sigma, double sK0, double sK1, double sK2,
                            typename V4<T>::type *__restrict__ xq, T *__restrict__ sg,
                            int4 *__restrict__ sbase, typename V4<T>::type *__restrict__ sfrac,
                            int32_t *__restrict__ smax_bits, float4 *__restrict__ xf,
                            int32_t *__restrict__ flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (smax_bits) {
        // max |sigma| as float bits (non-negative floats order like their bits)
        int32_t b = i < n && QEQ_IN_BOUNDS((unsigned)perm[i] < (unsigned)n, flags, kSiteGatherPerm)
                        ? __float_as_int(f64_to_f32_trunc(sigma[perm[i]])) & 0x7FFFFFFF
                        : 0;
        b = __reduce_max_sync(0xffffffffu, b);
        if ((threadIdx.x & 31) == 0 && b > 0) atomicMax(smax_bits, b);
    }
    if (i >= n) return;
    const int a = perm[i];
    if (!QEQ_IN_BOUNDS((unsigned)a < (unsigned)n, flags, kSiteGatherPerm)) return;
    const double x = R[3 * (size_t)a] + w[3 * (size_t)a];
    const double y = R[3 * (size_t)a + 1] + w[3 * (size_t)a + 1];
    const double z = R[3 * (size_t)a + 2] + w[3 * (size_t)a + 2];
    const double qa = q[a];
    // scaled fractional coordinates u = K x / L (x wrapped into [0, L)), split
    // into floor and fraction
    const double ux = x * sK0, uy = y * sK1, uz = z * sK2;
    if constexpr (std::is_same<T, float>::value) {
        // FP32 copies truncated on the integer pipe (at most 1 ulp, against the
        // half ulp of rounding), the split exact from the bits
        const float qf = f64_to_f32_trunc(qa);
        xq[i] = {f64_to_f32_trunc(x), f64_to_f32_trunc(y), f64_to_f32_trunc(z), qf};
        sg[i] = f64_to_f32_trunc(sigma[a]);
        int kx, ky, kz;
        float fx, fy, fz;
        split_floor(ux, kx, fx);
        split_floor(uy, ky, fy);
        split_floor(uz, kz, fz);
        sbase[i] = make_int4(kx, ky, kz, 0);
        sfrac[i] = {fx, fy, fz, qf};
    } else {
        xq[i] = {(T)x, (T)y, (T)z, (T)qa};
        if (xf) xf[i] = make_float4((float)x, (float)y, (float)z, 0.0f);
        sg[i] = (T)sigma[a];
        const double fx = floor(ux), fy = floor(uy), fz = floor(uz);
        sbase[i] = make_int4((int)fx, (int)fy, (int)fz, 0);
        sfrac[i] = {(T)(ux - fx), (T)(uy - fy), (T)(uz - fz), (T)qa};
    }
}

// Charges only, for an apply at the positions of the previous one: the sorted
// copies keep their positions, sigma and spline bases.
template <typename T>
__global__ void k_gather_q(int n, const int32_t *__restrict__ perm, const double *__restrict__ q,
                           typename V4<T>::type *__restrict__ xq,
                           typename V4<T>::type *__restrict__ sfrac, int32_t *__restrict__ flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (!QEQ_IN_BOUNDS((unsigned)perm[i] < (unsigned)n, flags, kSiteGatherPerm)) return;
    T qa;
    if constexpr (std::is_same<T, float>::value)
        qa = f64_to_f32_trunc(q[perm[i]]);  // as k_gather_in, on the integer pipe
    else
        qa = q[perm[i]];
    xq[i].w = qa;
    sfrac[i].w = qa;
}

// ---------------------------------------------------------------------------
// real space (Eq. ewald_real, Gaussian-charge correction)
// ---------------------------------------------------------------------------

struct RealArgs {
    int n;
    double Lx, Ly, Lz;
    double alpha;
    double rc2;
    double ke;
    // FP32 copies for k_real32, rounded once on the host: a double-to-float
    // conversion in the kernel runs on the FP64 pipe (1/64 rate on GB300), and
    // under register pressure the compiler re-derives such values inside the loop.
    float alpha_f, rc2_f, tspa_f, c1_f, pal_f, Lx_f, Ly_f, Lz_f, ke_f;
    int fg_pieces;  // kept pieces of the FP64 pair-function tables (0: direct erfc path only)
    int gc_pieces;
    float pre_rc2_f;  // FP32 prefilter bound of the FP64 kernel (r_c^2 plus the FP32 error)
};

// FP64 erfc by a piecewise polynomial: [0, kErfcXMax) is cut into kErfcPieces
// equal pieces.  On each piece erfc is the degree-(kErfcCoef - 1) polynomial in
// s in [-1, 1) through the Chebyshev nodes of that piece; the coefficients come
// from the host's long-double erfc (erfc_table()).  Beyond kErfcXMax, where
// erfc < 4e-20, the value and the derivative are 0.  One Horner pass gives
// erfc(x) and d erfc / dx (so no exp is needed).  The relative error is below
// 1e-14, far inside the 1e-10 parity of the FP64 path.
constexpr int kErfcPieces = 256;
constexpr int kErfcCoef = 10;
constexpr double kErfcXMax = 6.5;

__device__ __forceinline__ double erfc_pw(const double *__restrict__ tab, double x, double &dfdx) {
    const double inv_h = kErfcPieces / kErfcXMax;
    if (!(x < kErfcXMax)) {
        dfdx = 0.0;
        return 0.0;
    }
    const double u = x * inv_h;
    const int k = (int)u;
    const double s = 2.0 * (u - (double)k) - 1.0;
    const double *c = tab + k * kErfcCoef;
    double p = c[kErfcCoef - 1], dp = 0.0;
#pragma unroll
    for (int m = kErfcCoef - 2; m >= 0; --m) {
        dp = fma(dp, s, p);
        p = fma(p, s, c[m]);
    }
    dfdx = dp * (2.0 * inv_h);
    return p;
}

// FP64 pair functions by piecewise polynomials.  With
//   F_a(s) = erfc(a sqrt s) / sqrt s,
//   G_a(s) = F_a'(r) / r = 2 dF_a/ds = -(F_a(s) + (2 a / sqrt pi) exp(-a^2 s)) / s,
// a pair at s = r^2 adds q_j F_alpha(s) to the potential and q_j G_alpha(s)
// (r_j - r_i) to the field, and the Gaussian correction erfc(r / gamma) / r is
// F_1(t) / gamma with t = s / gamma^2, its field coefficient G_1(t) / gamma^3.
// Each table covers octaves [2^oct_lo, 2^(oct_lo + octaves)) of its argument,
// octave e (2^e <= s < 2^(e+1)) cut into 2^sub_log2 equal pieces; on each piece
// the two functions are the degree-(ncoef - 1) polynomials in x in [-1, 1)
// through the Chebyshev nodes of the piece, from the host's long-double erfc
// and exp (pw_table()).  The piece and x come from the bits of the argument
// alone: the exponent and the top sub_log2 mantissa bits are the piece, the
// remaining mantissa bits the position in it (x = 2 y - 3 for the double y in
// [1, 2) that holds them), so only the two Horner passes run on the FP64 pipe.
// A piece ends at least 2^(sub_log2 + 1) half-widths from the singularity at 0;
// the Gaussian factor bounds the error at large arguments, so the host measures
// every piece and keeps a table only up to the first one worse than 1e-13
// relative (or 1e-15 of the bare Coulomb term 1 / r, where the function is
// below 1e-2 of it) (pw_valid_pieces()).  Arguments outside the kept pieces
// (r < 0.5 A; t < 1/32) take the direct erfc path.
struct PwShape {
    int oct_lo, sub_log2, ncoef, max_oct;
};
constexpr PwShape kFGShape{-2, 5, 8, 8};   // F_alpha, G_alpha of s in [1/4, 64)
constexpr PwShape kGCShape{-5, 4, 9, 11};  // F_1, G_1 of t in [1/32, 64)
constexpr int kFGMaxPieces = kFGShape.max_oct << kFGShape.sub_log2;
constexpr int kGCMaxPieces = kGCShape.max_oct << kGCShape.sub_log2;
// both tables, at the head of the FP64 kernel's dynamic shared memory
constexpr size_t kFGTableBytes = sizeof(double2) * kFGMaxPieces * kFGShape.ncoef;
constexpr size_t kPwTableBytes = kFGTableBytes + sizeof(double2) * kGCMaxPieces * kGCShape.ncoef;

// Evaluate both functions of a table at arg > 0 (false: outside the npieces kept).
template <int OCT_LO, int SUB, int NC>
__device__ __forceinline__ bool pw_eval(const double2 *tab, unsigned npieces, double arg, double &f,
                                        double &g) {
    const int hi = __double2hiint(arg);
    const unsigned piece = (unsigned)((hi >> (20 - SUB)) - ((1023 + OCT_LO) << SUB));
    if (piece >= npieces) return false;
    const unsigned lo = (unsigned)__double2loint(arg);
    const int hy = 0x3FF00000 | (int)(((unsigned)hi << SUB) & 0x000FFFFFu) | (int)(lo >> (32 - SUB));
    const double x = fma(__hiloint2double(hy, (int)(lo << SUB)), 2.0, -3.0);
    const double2 *c = tab + piece * NC;
    double2 cm = c[NC - 1];
    f = cm.x;
    g = cm.y;
#pragma unroll
    for (int m = NC - 2; m >= 0; --m) {
        cm = c[m];
        f = fma(f, x, cm.x);
        g = fma(g, x, cm.y);
    }
    return true;
}

// Lanes per neighbour row.  kTPR consecutive lanes share one row: lane s takes
// the row's entries s, s + kTPR, ..., which the list stores next to each other
// (kListGroup), and their partial sums are combined with warp shuffles.
constexpr int kTPR = kListLanes;
// One block per brick; its blockDim is kTPR x (largest brick, rounded to warps),
// at most kRealMaxThreads.  Larger bricks take several passes.
constexpr int kRealMaxThreads = 512;
// Resident blocks per SM asked of the FP32 real-space kernel (register cap
// 65536 / (kRealMaxThreads x blocks): three give 40 registers a thread, and
// four 384-thread blocks of the 300,000-atom box fit; two blocks at 54
// registers ran 0.29 ms against 0.24 ms).
#ifndef QEQ_REAL_MIN_BLOCKS
#define QEQ_REAL_MIN_BLOCKS 3
#endif
// Read sigma_j only for pairs inside the row's Gaussian-correction bound.
#ifndef QEQ_REAL_LAZY_SIGMA
#define QEQ_REAL_LAZY_SIGMA 1
#endif
constexpr bool kRealLazySigma = QEQ_REAL_LAZY_SIGMA != 0;

// Tile bytes per atom (position and charge, sigma) and the dynamic shared
// memory the kernels may take: 227 KB per block less their static tables.
// (FP64: double4 position and q, double sigma, and the float4 position copy of
// the FP32 cutoff prefilter.)
constexpr size_t kTile32Bytes = 20, kTile64Bytes = 56;
constexpr size_t kSmemPerBlock = 232448;
constexpr size_t kReal32SmemMax = kSmemPerBlock - 4096;
constexpr size_t kReal64SmemMax = kSmemPerBlock - 4096;  // tables included
// Largest deferred Gaussian-correction queue of the FP64 kernel (entries per lane).
constexpr int kCorrQueueMax = 48;

// Brick spreading: block size and the largest shared-memory window it takes.
constexpr int kSpreadThreads = 128;
constexpr size_t kSpreadSmemMax = 48 * 1024;

int real_block_threads(int max_rows) {
    int t = (kTPR * std::max(1, max_rows) + 31) / 32 * 32;
    return std::min(kRealMaxThreads, std::max(64, t));
}

// Stage the tile of brick blockIdx.x: load its tile table (written by the
// neighbour build), then the warps copy the tile bricks (positions shifted by
// their periodic image, and sigma) into tile[] / tsg[].  Returns the tile size,
// or -1 when it exceeds cap (the whole block then skips the brick and raises
// kFlagTileOverflow).
template <typename T4, typename T>
__device__ __forceinline__ int stage_tile(const BrickGeom &g, const int4 *__restrict__ tile_tab,
                                          const int32_t *__restrict__ tile_tot,
                                          const T4 *__restrict__ xq, const T *__restrict__ sg,
                                          T Lx, T Ly, T Lz, int cap, T4 *tile, T *tsg, int *t_start,
                                          int *t_base, int *t_code, int *t_total,
                                          int32_t *__restrict__ flags) {
    for (int rb = threadIdx.x; rb < g.T; rb += blockDim.x) {
        const int4 e = tile_tab[(int64_t)blockIdx.x * g.T + rb];
        t_start[rb] = e.x;
        t_base[rb] = e.y;
        t_code[rb] = e.z;
    }
    if (threadIdx.x == 0) *t_total = tile_tot[blockIdx.x];
    __syncthreads();
    const int total = *t_total;
    if (total + 1 > cap) {  // the tile plus its sentinel slot
        if (threadIdx.x == 0) atomicExch(&flags[kFlagTileOverflow], 1);
        return -1;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int rb = warp; rb < g.T; rb += nw) {
        const int st = t_start[rb], off = st + t_base[rb];
        const int end = rb + 1 < g.T ? t_start[rb + 1] + t_base[rb + 1] : total;
        const int code = t_code[rb];
        const T sx = (T)(code / 25 - 2) * Lx, sy = (T)((code / 5) % 5 - 2) * Ly,
                sz = (T)(code % 5 - 2) * Lz;
        for (int k = lane; k < end - off; k += 32) {
            T4 x = xq[st + k];
            x.x += sx;
            x.y += sy;
            x.z += sz;
            tile[off + k] = x;
            tsg[off + k] = sg[st + k];
        }
    }
    // sentinel slot: the padding entries of the list point here, far from every
    // atom (r^2 about 3e36 fails the cutoff test in both precisions)
    if (threadIdx.x == 0) {
        T4 far;
        far.x = far.y = far.z = T(1e18);
        far.w = T(0);
        tile[total] = far;
        tsg[total] = T(0);
    }
    __syncthreads();
    return total;
}

// Tile slots of the rows of the block's brick: the brick is the tile's center.
__device__ __forceinline__ void home_rows(const BrickGeom &g, const int *t_start, const int *t_base,
                                          int total, int &i0, int &off, int &nrows) {
    i0 = t_start[g.center];
    off = i0 + t_base[g.center];
    const int end = g.center + 1 < g.T ? t_start[g.center + 1] + t_base[g.center + 1] : total;
    nrows = end - off;
}

// A non-negative double, from its high word, as a float truncated toward zero
// (relative error below 2^-20; 0 below the float range), on the integer pipe.
__device__ __forceinline__ float hi_to_float(int hi) {
    const int b = hi - (896 << 20);  // rebias the exponent from 1023 to 127
    return b > 0 ? __int_as_float(b << 3) : 0.0f;
}
// Gaussian correction of an FP64 pair at r^2 = r2 with gamma^2 = si2 + sj^2: the
// amounts fc = erfc(r / gamma) / r and gcc = (d/dr fc) / r that the pair's
// potential and field coefficient lose.  F_1, G_1 of t = r^2 / gamma^2 from the
// table, else the direct piecewise erfc (exactly 0 beyond r / gamma = kErfcXMax).
__device__ __forceinline__ void gauss_corr64(double r2, double si2, double sj,
                                             const double *__restrict__ erfc_tab,
                                             const double2 *gct, unsigned gpieces, double &fc,
                                             double &gcc) {
    const double g2 = si2 + sj * sj;
    const double ig = rsqrt(g2);
    const double ig2 = ig * ig;
    double f1, g1;
    if (pw_eval<kGCShape.oct_lo, kGCShape.sub_log2, kGCShape.ncoef>(gct, gpieces, r2 * ig2, f1, g1)) {
        fc = ig * f1;
        gcc = ig2 * ig * g1;
    } else {
        const double ir = rsqrt(r2);
        double d2;
        fc = erfc_pw(erfc_tab, (r2 * ir) * ig, d2) * ir;
        gcc = (ig * d2 - fc) * ir * ir;
    }
}

// kErfcXMax^2 with the margin of the FP32 Gaussian-correction test.
constexpr float kGaussTest = (float)(kErfcXMax * kErfcXMax * (1.0 + 1e-5));

// FP64 real space, one block per brick, kTPR lanes per row.  Dynamic shared
// memory holds the two pair-function tables, the tile (double4 positions with
// q, double sigma, float4 positions for the FP32 prefilter; GTILE: in the
// block's slice of a global scratch buffer instead) and the per-lane queues of
// deferred Gaussian corrections; usually one block per SM fits, which keeps the
// FP64 pipe (the bound) about 88% busy.  The piecewise erfc of the direct path
// is read through the read-only cache.  The register cap of two blocks per SM
// (64) leaves the loop without spills.
template <bool FIELD, bool GTILE>
__global__ void __launch_bounds__(kRealMaxThreads, 2)
k_real64(RealArgs a, BrickGeom g, const int4 *__restrict__ tile_tab, const int32_t *__restrict__ tile_tot,
         const uint16_t *__restrict__ nbr, const int32_t *__restrict__ cnt,
         const double4_32a *__restrict__ xq, const double *__restrict__ sg,
         const float4 *__restrict__ xf, const double *__restrict__ erfc_tab,
         const double2 *__restrict__ fg_tab, const double2 *__restrict__ gc_tab, int cap, int qcap,
         unsigned char *__restrict__ gtile, int32_t *__restrict__ flags, double *__restrict__ v_s,
         double *__restrict__ E_s) {
    extern __shared__ __align__(32) unsigned char smem_raw[];
    __shared__ int t_start[kMaxTileBricks], t_base[kMaxTileBricks], t_code[kMaxTileBricks], t_total;
    double2 *fg = (double2 *)smem_raw;
    double2 *gct = (double2 *)(smem_raw + kFGTableBytes);
    unsigned char *base =
        GTILE ? gtile + (size_t)blockIdx.x * cap * kTile64Bytes : smem_raw + kPwTableBytes;
    double4_32a *tile = (double4_32a *)base;
    double *tsg = (double *)(base + (size_t)cap * 32);
    // per-lane queue of deferred Gaussian corrections (slot-major), after the tile
    uint16_t *cq = (uint16_t *)(smem_raw + kPwTableBytes + (GTILE ? 0 : (size_t)cap * kTile64Bytes));
    for (int t = threadIdx.x; t < a.fg_pieces * kFGShape.ncoef; t += blockDim.x) fg[t] = fg_tab[t];
    for (int t = threadIdx.x; t < a.gc_pieces * kGCShape.ncoef; t += blockDim.x) gct[t] = gc_tab[t];
    const int total = stage_tile<double4_32a, double>(g, tile_tab, tile_tot, xq, sg, a.Lx, a.Ly, a.Lz, cap,
                                                     tile, tsg, t_start, t_base, t_code, &t_total,
                                                     flags);
    if (total < 0) return;
    // float copy of the tile positions for the FP32 cutoff prefilter
    float4 *tf = (float4 *)(base + (size_t)cap * 40);
    {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int rb = warp; rb < g.T; rb += nw) {
            const int st = t_start[rb], off = st + t_base[rb];
            const int end = rb + 1 < g.T ? t_start[rb + 1] + t_base[rb + 1] : total;
            const int code = t_code[rb];
            const float sx = (float)(code / 25 - 2) * a.Lx_f, sy = (float)((code / 5) % 5 - 2) * a.Ly_f,
                        sz = (float)(code % 5 - 2) * a.Lz_f;
            for (int k = lane; k < end - off; k += 32) {
                const float4 x = xf[st + k];
                tf[off + k] = make_float4(x.x + sx, x.y + sy, x.z + sz, 0.0f);
            }
        }
        if (threadIdx.x == 0) tf[total] = make_float4(1e18f, 1e18f, 1e18f, 0.0f);
        __syncthreads();
    }
    int i0, offc, nrows;
    home_rows(g, t_start, t_base, total, i0, offc, nrows);
    const double al = a.alpha;
    const unsigned npieces = (unsigned)a.fg_pieces, gpieces = (unsigned)a.gc_pieces;
    const long long rc2_bits = __double_as_longlong(a.rc2);
    const int rpp = blockDim.x / kTPR;
    for (int r0 = 0; r0 < nrows; r0 += rpp) {
        const int r = r0 + threadIdx.x / kTPR, sub = threadIdx.x % kTPR;
        const bool act = r < nrows;
        double v = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
        if (act) {
            const int i = i0 + r;
            const double4_32a xi = tile[offc + r];
            const double si2 = tsg[offc + r] * tsg[offc + r];
            const float si2f = hi_to_float(__double2hiint(si2));
            const float4 xif = tf[offc + r];
            const int c = cnt[i];
            int nq = 0;
            for (int k = sub; k < c; k += kTPR) {
                const int e = nbr[list_index(k, i, a.n)];
                if (!QEQ_IN_BOUNDS(e <= total, flags, kSiteReal64Entry)) continue;
                // FP32 prefilter: pre_rc2_f exceeds r_c^2 by more than the FP32
                // error of r^2, so only pairs that fail the FP64 test are dropped
                const float4 xjf = tf[e];
                const float fx = xjf.x - xif.x, fy = xjf.y - xif.y, fz = xjf.z - xif.z;
                if (!(fmaf(fx, fx, fmaf(fy, fy, fz * fz)) < a.pre_rc2_f)) continue;
                const double4_32a xj = tile[e];
                const double dx = xj.x - xi.x;
                const double dy = xj.y - xi.y;
                const double dz = xj.z - xi.z;
                const double r2 = dx * dx + dy * dy + dz * dz;
                // r2 >= 0, so the cutoff test compares the bit patterns (integer pipe)
                if (!(__double_as_longlong(r2) < rc2_bits)) continue;
                // f = erfc(alpha r) / r, gc = (d/dr f) / r
                double f, gc;
                if (!pw_eval<kFGShape.oct_lo, kFGShape.sub_log2, kFGShape.ncoef>(fg, npieces, r2, f, gc)) {
                    const double ir = rsqrt(r2);
                    double d1;
                    f = erfc_pw(erfc_tab, al * (r2 * ir), d1) * ir;
                    gc = (al * d1 - f) * ir * ir;
                }
                // Gaussian correction.  The test runs in FP32 on values truncated from
                // the high words of r^2 and sigma_j (each at most 2^-20 low) with a
                // 1e-5 margin, so it never drops a pair the FP64 test would keep; a
                // pair it keeps beyond r / gamma = kErfcXMax adds below
                // erfc(6.5) ~ 4e-20 of 1 / r.  About a quarter of the pairs need it,
                // scattered over the lanes, so the lane queues them (the tile slot)
                // and runs them together after the list: the FP64 pipe then works
                // on nearly full warps.
                const int hi = __double2hiint(r2);
                const float sjf = hi_to_float(((const int *)tsg)[2 * e + 1]);
                if (hi_to_float(hi) < kGaussTest * fmaf(sjf, sjf, si2f)) {
                    if (nq < qcap) {
                        cq[nq * blockDim.x + threadIdx.x] = (uint16_t)e;
                        ++nq;
                    } else {
                        double fc, gcc;
                        gauss_corr64(r2, si2, tsg[e], erfc_tab, gct, gpieces, fc, gcc);
                        f -= fc;
                        gc -= gcc;
                    }
                }
                v += xj.w * f;
                if (FIELD) {
                    const double gq = xj.w * gc;
                    ex += gq * dx;
                    ey += gq * dy;
                    ez += gq * dz;
                }
            }
            for (int m = 0; m < nq; ++m) {
                const int e = cq[m * blockDim.x + threadIdx.x];
                const double4_32a xj = tile[e];
                const double dx = xj.x - xi.x;
                const double dy = xj.y - xi.y;
                const double dz = xj.z - xi.z;
                const double r2 = dx * dx + dy * dy + dz * dz;
                double fc, gcc;
                gauss_corr64(r2, si2, tsg[e], erfc_tab, gct, gpieces, fc, gcc);
                v -= xj.w * fc;
                if (FIELD) {
                    const double gq = xj.w * gcc;
                    ex -= gq * dx;
                    ey -= gq * dy;
                    ez -= gq * dz;
                }
            }
        }
#pragma unroll
        for (int o = 1; o < kTPR; o <<= 1) {
            v += __shfl_xor_sync(0xffffffffu, v, o);
            if (FIELD) {
                ex += __shfl_xor_sync(0xffffffffu, ex, o);
                ey += __shfl_xor_sync(0xffffffffu, ey, o);
                ez += __shfl_xor_sync(0xffffffffu, ez, o);
            }
        }
        if (act && sub == 0) {
            const int i = i0 + r;
            v_s[i] = a.ke * v;
            if (FIELD) {
                E_s[3 * (size_t)i] = a.ke * ex;
                E_s[3 * (size_t)i + 1] = a.ke * ey;
                E_s[3 * (size_t)i + 2] = a.ke * ez;
            }
        }
    }
}

// Self-test hook: the FP64 piecewise erfc and its derivative on n device inputs.
__global__ void k_erfc64(int64_t n, const double *__restrict__ tab, const double *__restrict__ x,
                         double *__restrict__ out, double *__restrict__ dout) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        double d;
        out[t] = erfc_pw(tab, x[t], d);
        dout[t] = d;
    }
}

// Self-test hook: the FP64 kernel's pair-function table (which 0: F_alpha,
// G_alpha of s; 1: F_1, G_1 of t) at n device arguments, as the kernel
// evaluates it; in = 0 where the argument is outside the kept pieces.
__global__ void k_pair64_selftest(int64_t n, int which, const double2 *__restrict__ tab,
                                  unsigned npieces, const double *__restrict__ arg,
                                  double *__restrict__ F, double *__restrict__ G,
                                  int32_t *__restrict__ in) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double f = 0.0, g = 0.0;
    const bool ok =
        which == 0 ? pw_eval<kFGShape.oct_lo, kFGShape.sub_log2, kFGShape.ncoef>(tab, npieces, arg[t], f, g)
                   : pw_eval<kGCShape.oct_lo, kGCShape.sub_log2, kGCShape.ncoef>(tab, npieces, arg[t], f, g);
    in[t] = ok ? 1 : 0;
    if (ok) {
        F[t] = f;
        G[t] = g;
    }
}

// erfc(x), x >= 0, in FP32 by Abramowitz & Stegun, Handbook of Mathematical
// Functions, eq. 7.1.26 (Hastings' approximation):
//   erfc(x) = t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2),  t = 1 / (1 + p x),
// with an absolute error of at most 1.5e-7.  t and exp(-x^2) are arguments: the
// field term needs the same exponential, and the callers form t themselves.
constexpr float kAsP = 0.3275911f;
__device__ __forceinline__ float erfc_as7126_t(float t, float ex2) {
    float p = fmaf(t, 1.061405429f, -1.453152027f);
    p = fmaf(t, p, 1.421413741f);
    p = fmaf(t, p, -0.284496736f);
    p = fmaf(t, p, 0.254829592f);
    return t * p * ex2;
}

// Single-instruction approximations of the special-function unit (PTX
// rsqrt / rcp / ex2 .approx.ftz).  The arguments of the real-space kernel are
// never subnormal (r^2 >= 0.1 A^2 between distinct atoms, 1 + p x >= 1, and the
// exponents lie in [-37, 0]), so flushing subnormals changes no result.
// exp(-y) is formed as 2^(-y log2 e) with log2 e folded into a kernel constant.
constexpr float kLog2E = 1.4426950408889634f;
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_ftz(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// erfc(x) with exp(-x^2) passed in, x >= 0 (self-test and Gaussian-correction form).
__device__ __forceinline__ float erfc_as7126(float x, float ex2) {
    return erfc_as7126_t(rcp_ftz(fmaf(kAsP, x, 1.0f)), ex2);
}
__device__ __forceinline__ float exp_neg_sq(float x) { return ex2_ftz(-(x * x) * kLog2E); }

// Kahan-compensated FP32 accumulation of a chunk sum.
__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x) {
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// One FP32 pair term: the erfc(alpha r) / r potential minus the Gaussian-charge
// correction erfc(r / gamma_ij) / r, and (FIELD) the field coefficient, added to
// the running chunk sums.  The correction is evaluated only when r^2 is below
// the row's bound gpre = 25 (sigma_i^2 + max sigma^2) (x 1.0001 against
// rounding), the only pairs where it can be kept; sigma_j is read there only.
// c1 = -alpha^2 log2 e, so exp(-alpha^2 r^2) = 2^(c1 r^2).
template <bool FIELD>
__device__ __forceinline__ void pair32(float dx, float dy, float dz, float qj, const float *sgj,
                                       float si2, float gpre, float pal, float c1, float rc2,
                                       float tspa, float &vf, float &exf, float &eyf, float &ezf) {
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2 < rc2) {
        const float ir = rsqrt_ftz(r2);
        const float r = r2 * ir;
        const float e1 = ex2_ftz(r2 * c1);
        float f = erfc_as7126_t(rcp_ftz(fmaf(pal, r, 1.0f)), e1) * ir;
        float dfr = 0.f;
        if (FIELD) dfr = -fmaf(tspa, e1, f) * ir;
        if (r2 < gpre) {
            const float sj = *sgj;
            const float g2 = fmaf(sj, sj, si2);
            // Gaussian correction; beyond r / gamma = 5 it is below 2e-12 / r and
            // is dropped (FP32 cannot resolve it next to erfc(alpha r) / r)
            if (r2 < 25.f * g2) {
                const float ig = rsqrt_ftz(g2);
                const float x2 = r * ig;
                const float e2 = exp_neg_sq(x2);
                const float fg = erfc_as7126(x2, e2) * ir;
                f -= fg;
                if (FIELD) dfr += fmaf((float)kTwoOverSqrtPi * ig, e2, fg) * ir;
            }
        }
        vf = fmaf(qj, f, vf);
        if (FIELD) {
            const float gq = qj * dfr * ir;
            exf = fmaf(gq, dx, exf);
            eyf = fmaf(gq, dy, eyf);
            ezf = fmaf(gq, dz, ezf);
        }
    }
}


// FP32 real space, one block per brick: the tile (float4 positions with q, and
// sigma) in shared memory (GTILE: in the block's slice of a global scratch
// buffer), kTPR lanes per row, FP32 pair math with one exp per erfc shared with
// the field term, FP32 sums (each lane about r_list^3 rho / 4 terms) and an FP32
// shuffle combine of the lanes; the row's sums, scaled by k_e, go out as one
// float4 (v, E) per sorted atom.  smax_bits holds the float bits of max |sigma|
// over the atoms (written by the gather of the same apply).
template <bool FIELD, bool GTILE>
__global__ void __launch_bounds__(kRealMaxThreads, QEQ_REAL_MIN_BLOCKS)
k_real32(RealArgs a, BrickGeom g, const int4 *__restrict__ tile_tab, const int32_t *__restrict__ tile_tot,
         const uint16_t *__restrict__ nbr, const int32_t *__restrict__ cnt,
         const float4 *__restrict__ xq, const float *__restrict__ sg,
         const int32_t *__restrict__ smax_bits, int cap, unsigned char *__restrict__ gtile,
         int32_t *__restrict__ flags, float4 *__restrict__ vE) {
    extern __shared__ __align__(32) unsigned char smem_raw[];
    __shared__ int t_start[kMaxTileBricks], t_base[kMaxTileBricks], t_code[kMaxTileBricks], t_total;
    unsigned char *base = GTILE ? gtile + (size_t)blockIdx.x * cap * kTile32Bytes : smem_raw;
    float4 *tile = (float4 *)base;
    float *tsg = (float *)(base + (size_t)cap * 16);
    const int total = stage_tile<float4, float>(g, tile_tab, tile_tot, xq, sg, a.Lx_f, a.Ly_f, a.Lz_f, cap,
                                                tile, tsg, t_start, t_base, t_code, &t_total, flags);
    if (total < 0) return;
    int i0, offc, nrows;
    home_rows(g, t_start, t_base, total, i0, offc, nrows);
    const float smax = kRealLazySigma ? __int_as_float(__ldg(smax_bits)) : 0.f;
    const size_t wstep = (size_t)kListStripe / 4 * a.n;  // one stripe further, in 8-byte words
    const int rpp = blockDim.x / kTPR;
    for (int r0 = 0; r0 < nrows; r0 += rpp) {
        const int r = r0 + threadIdx.x / kTPR, sub = threadIdx.x % kTPR;
        const bool act = r < nrows;
        float tv = 0.f, tx = 0.f, ty = 0.f, tz = 0.f;
        if (act) {
            const int i = i0 + r;
            const float4 xi = tile[offc + r];
            const float si = tsg[offc + r];
            const float si2 = si * si;
            // every pair checks sigma_j when max |sigma| is unknown
            const float gpre = kRealLazySigma ? 25.0001f * fmaf(smax, smax, si2) : 3.4e38f;
            const int c = cnt[i];
            // This lane's entries come 4 to an 8-byte word, one word per list
            // stripe; w0 holds the current word and w1 the next, loaded ahead so
            // that the DRAM latency of the list stream overlaps the pair math.
            const int cl = c > sub ? (c - sub + kTPR - 1) / kTPR : 0;
            const uint2 *pw = (const uint2 *)(nbr + list_index(sub, i, a.n));
            uint2 w0 = cl > 0 ? __ldg(pw) : make_uint2(0u, 0u);
            uint2 w1 = cl > 4 ? __ldg(pw + wstep) : make_uint2(0u, 0u);
            for (int t = 0; t < cl; t += 4) {
                const uint2 cur = w0;
                w0 = w1;
                pw += wstep;
                w1 = t + 8 < cl ? __ldg(pw + wstep) : make_uint2(0u, 0u);
                const int ev[4] = {(int)(cur.x & 0xffffu), (int)(cur.x >> 16), (int)(cur.y & 0xffffu),
                                   (int)(cur.y >> 16)};
                // entries past the row's end are padding (the far sentinel slot)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = ev[u];
                    if (!QEQ_IN_BOUNDS(e <= total, flags, kSiteReal32Entry)) continue;
                    const float4 xc = tile[e];
                    pair32<FIELD>(xc.x - xi.x, xc.y - xi.y, xc.z - xi.z, xc.w, tsg + e, si2, gpre,
                                  a.pal_f, a.c1_f, a.rc2_f, a.tspa_f, tv, tx, ty, tz);
                }
            }
        }
#pragma unroll
        for (int o = 1; o < kTPR; o <<= 1) {
            tv += __shfl_xor_sync(0xffffffffu, tv, o);
            if (FIELD) {
                tx += __shfl_xor_sync(0xffffffffu, tx, o);
                ty += __shfl_xor_sync(0xffffffffu, ty, o);
                tz += __shfl_xor_sync(0xffffffffu, tz, o);
            }
        }
        // the row's sums scaled by k_e, in FP32 (one 16-byte store; an FP64
        // epilogue would run on GB300's 1/64-rate FP64 pipe at every row pass)
        if (act && sub == 0) {
            const int i = i0 + r;
            if (FIELD)
                vE[i] = make_float4(a.ke_f * tv, a.ke_f * tx, a.ke_f * ty, a.ke_f * tz);
            else
                reinterpret_cast<float *>(vE)[4 * (size_t)i] = a.ke_f * tv;
        }
    }
}

// Self-test hook: the FP32 erfc of the real-space kernel on n device inputs.
__global__ void k_erfc32(int64_t n, const float *__restrict__ x, float *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        const float xv = x[t];
        out[t] = erfc_as7126(xv, exp_neg_sq(xv));
    }
}

// ---------------------------------------------------------------------------
// PME (Alg. 2)
// ---------------------------------------------------------------------------

// Cardinal B-spline weights M_P(w + j), j = 0..P-1, by the order recursion
// M_n(u) = [u M_{n-1}(u) + (n - u) M_{n-1}(u - 1)] / (n - 1) from M_2, and the
// derivative M_P'(u) = M_{P-1}(u) - M_{P-1}(u - 1).
template <typename T, int P, bool DERIV>
__device__ __forceinline__ void bspline(T w, T (&M)[P], T (&dM)[P]) {
    M[0] = w;
    M[1] = T(1) - w;
#pragma unroll
    for (int j = 2; j < P; ++j) M[j] = T(0);
#pragma unroll
    for (int n = 3; n <= P; ++n) {
        if (DERIV && n == P) {
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const T left = (j < P - 1) ? M[j] : T(0);
                const T right = (j >= 1) ? M[j - 1] : T(0);
                dM[j] = left - right;
            }
        }
        const T inv = T(1) / T(n - 1);
#pragma unroll
        for (int j = n - 1; j >= 0; --j) {
            const T left = (j < n - 1) ? M[j] : T(0);
            const T right = (j >= 1) ? M[j - 1] : T(0);
            M[j] = ((w + T(j)) * left + (T(n) - w - T(j)) * right) * inv;
        }
    }
}

// Vector reduction of two adjacent floats (sm_90+): one L2 atomic for 8 bytes.
// p must be 8-byte aligned.
__device__ __forceinline__ void red_add_v2(float *p, float a, float b) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

__device__ __forceinline__ int wrap_index(int b, int K) {
    int r = b % K;
    return r < 0 ? r + K : r;
}

// One thread per sorted atom; p^3 atomic adds per atom into the global mesh (the
// mesh stays L2 resident; throughput is set by the L2 atomic units).
template <typename T, int P>
__global__ void __launch_bounds__(kThreads)
k_spread(int n, const int4 *__restrict__ sbase, const typename V4<T>::type *__restrict__ sfrac,
         int K0, int K1, int K2, T *__restrict__ mesh) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 b = sbase[i];
    const auto f = sfrac[i];
    T Mx[P], My[P], Mz[P], dummy[P];
    bspline<T, P, false>(f.x, Mx, dummy);
    bspline<T, P, false>(f.y, My, dummy);
    bspline<T, P, false>(f.z, Mz, dummy);
    int iz[P];
#pragma unroll
    for (int c = 0; c < P; ++c) iz[c] = wrap_index(b.z - c, K2);
    // the P z-points base - P + 1 .. base are contiguous unless they wrap
    const int z0 = b.z - (P - 1);
    const bool contiguous = z0 >= 0 && b.z < K2;
#pragma unroll
    for (int a = 0; a < P; ++a) {
        const int ix = wrap_index(b.x - a, K0);
        const T qa = f.w * Mx[a];
#pragma unroll
        for (int bb = 0; bb < P; ++bb) {
            const int iy = wrap_index(b.y - bb, K1);
            const T qab = qa * My[bb];
            T *row = mesh + ((size_t)ix * K1 + iy) * K2;
            if constexpr (std::is_same<T, float>::value && P == 4) {
                if (contiguous) {
                    // two 8-byte vector reductions per row (one when the start is odd)
                    float *p0 = row + z0;
                    if ((((size_t)ix * K1 + iy) * K2 + z0 & 1) == 0) {
                        red_add_v2(p0, qab * Mz[3], qab * Mz[2]);
                        red_add_v2(p0 + 2, qab * Mz[1], qab * Mz[0]);
                    } else {
                        atomicAdd(p0, qab * Mz[3]);
                        red_add_v2(p0 + 1, qab * Mz[2], qab * Mz[1]);
                        atomicAdd(p0 + 3, qab * Mz[0]);
                    }
                    continue;
                }
            }
#pragma unroll
            for (int c = 0; c < P; ++c) atomicAdd(row + iz[c], qab * Mz[c]);
        }
    }
}

// Vector reduction of four adjacent floats (sm_90+): one L2 atomic for 16 bytes.
// p must be 16-byte aligned.
__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
                 "f"(d)
                 : "memory");
}

// Brick-window spreading.  One block per brick: the brick's atoms add their
// p^3 weights into a shared-memory window of the mesh that covers the brick
// plus the spline support, and the block then adds the window into the global
// mesh, four z-points per vector reduction where the row is 16-byte aligned and
// does not wrap.  The window accumulates in 32-bit fixed point: integer shared
// atomics are native, and ran the 300,000-atom spread in 46 us against 66 us
// with float shared atomics (64-bit integers: 101 us).  A contribution
// q Mx My Mz becomes round(scale q Mx My Mz), scale = 2^k the largest power of
// two with scale wmax sum_brick |q| < 2^30, where wmax >= Mx My Mz is the
// largest weight of one mesh point: no window point can overflow.  The sums are
// exact and independent of the atomic order; the resolution is
// wmax sum |q| / 2^30 (about 7e-9 e for a 73-atom water brick with charges of
// 0.3 e).  The window origin of brick (bx, by, bz) is floor(b_d X_d) - (P - 1)
// per axis, X_d = B_d cw_d K_d / L_d; z is rounded down to a multiple of 4.
// An atom whose support leaves the window (possible only through rounding of
// floor(K x / L) at a brick face) adds straight into the global mesh.
struct SpreadWin {
    int K0, K1, K2;
    int E0, E1, E2;      // window extent (E2 a multiple of 4)
    int vec;             // K2 % 4 == 0: vector flush allowed
    float wmax;          // upper bound of one atom's weight at one mesh point
};

template <typename T, int P>
__device__ __forceinline__ void spread_atom_global(const int4 &b, const T (&Mx)[P], const T (&My)[P],
                                                   const T (&Mz)[P], T q, const SpreadWin &w,
                                                   T *__restrict__ mesh) {
    for (int aa = 0; aa < P; ++aa) {
        const int ix = wrap_index(b.x - aa, w.K0);
        for (int bb = 0; bb < P; ++bb) {
            const int iy = wrap_index(b.y - bb, w.K1);
            T *row = mesh + ((size_t)ix * w.K1 + iy) * w.K2;
            for (int c = 0; c < P; ++c) atomicAdd(row + wrap_index(b.z - c, w.K2), q * Mx[aa] * My[bb] * Mz[c]);
        }
    }
}

template <int P>
__global__ void __launch_bounds__(kSpreadThreads)
k_spread_brick(SpreadWin w, BrickGeom g, const int32_t *__restrict__ cell_start,
               const int4 *__restrict__ sbase, const float4 *__restrict__ sfrac,
               float *__restrict__ mesh) {
    extern __shared__ __align__(32) unsigned char smem_raw[];
    int *win = (int *)smem_raw;
    __shared__ float qsum_w[kSpreadThreads / 32];
    const int64_t b = blockIdx.x;
    const int bz = (int)(b % g.nb[2]), by = (int)((b / g.nb[2]) % g.nb[1]);
    const int bx = (int)(b / ((int64_t)g.nb[2] * g.nb[1]));
    // first mesh point of the brick: floor(b K / nb) per axis, in integers (exact;
    // an FP64 multiply and floor would wait on GB300's 1/64-rate FP64 pipe)
    const int lo0 = bx * w.K0 / g.nb[0] - (P - 1), lo1 = by * w.K1 / g.nb[1] - (P - 1);
    const int lo2 = (bz * w.K2 / g.nb[2] - (P - 1)) & ~3;
    const int nwin = w.E0 * w.E1 * w.E2;
    const int a0 = cell_start[b * g.bvol], a1 = cell_start[(b + 1) * g.bvol];
    float qs = 0.f;
    for (int i = a0 + threadIdx.x; i < a1; i += blockDim.x) qs += fabsf(sfrac[i].w);
    for (int t = threadIdx.x; t < nwin; t += blockDim.x) win[t] = 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) qs += __shfl_xor_sync(0xffffffffu, qs, o);
    if ((threadIdx.x & 31) == 0) qsum_w[threadIdx.x >> 5] = qs;
    __syncthreads();
    float qsum = 0.f;
#pragma unroll
    for (int k = 0; k < kSpreadThreads / 32; ++k) qsum += qsum_w[k];
    // scale = 2^(30 - e) with wmax qsum < 2^e (rounded up by 1e-5 relative)
    // frexp from the exponent bits: x = m 2^e2 with m in [0.5, 1)
    const float xq = fmaxf(qsum * w.wmax * 1.00001f, 1e-30f);
    const int e2 = ((__float_as_int(xq) >> 23) & 0xff) - 126;
    const int sh = min(126, 30 - e2);
    const float scale = __int_as_float((127 + sh) << 23);
    const float unscale = __int_as_float((127 - sh) << 23);
    for (int i = a0 + threadIdx.x; i < a1; i += blockDim.x) {
        const int4 bs = sbase[i];
        const float4 f = sfrac[i];
        float Mx[P], My[P], Mz[P], dummy[P];
        bspline<float, P, false>(f.x, Mx, dummy);
        bspline<float, P, false>(f.y, My, dummy);
        bspline<float, P, false>(f.z, Mz, dummy);
        const int lx = bs.x - lo0, ly = bs.y - lo1, lz = bs.z - lo2;
        if (lx < P - 1 || lx >= w.E0 || ly < P - 1 || ly >= w.E1 || lz < P - 1 || lz >= w.E2) {
            spread_atom_global<float, P>(bs, Mx, My, Mz, f.w, w, mesh);
            continue;
        }
        const float qsc = f.w * scale;
#pragma unroll
        for (int aa = 0; aa < P; ++aa) {
            const float qa = qsc * Mx[aa];
#pragma unroll
            for (int bb = 0; bb < P; ++bb) {
                const float qab = qa * My[bb];
                int *row = win + ((lx - aa) * w.E1 + (ly - bb)) * w.E2 + lz;
#pragma unroll
                for (int c = 0; c < P; ++c) atomicAdd(row - c, __float2int_rn(qab * Mz[c]));
            }
        }
    }
    __syncthreads();
    // flush: chunks of 4 z-points of each window row, back to FP32 (x 2^-sh).
    // The chunk index t splits into (row, chunk) and the row into (ix, iy) by FP32
    // reciprocals, exact for indices below 2^22 (the product's error stays below
    // 0.5 / divisor; a window holds at most 12,288 points), and a window index
    // wraps into the mesh with one conditional add or subtract (it lies in
    // [-(P - 1), K + P - 1)): runtime integer divisions and remainders made most
    // of this loop's instructions.
    const int nq = w.E2 / 4;
    const float inv_nq = 1.0f / (float)nq, inv_e1 = 1.0f / (float)w.E1;
    for (int t = threadIdx.x; t < w.E0 * w.E1 * nq; t += blockDim.x) {
        const int row = __float2int_rz(((float)t + 0.5f) * inv_nq);
        const int k = t - row * nq;
        const int ix = __float2int_rz(((float)row + 0.5f) * inv_e1);
        const int iy = row - ix * w.E1;
        const int4 iv = *(const int4 *)(win + (size_t)row * w.E2 + 4 * k);
        if ((iv.x | iv.y | iv.z | iv.w) == 0) continue;
        const float vv[4] = {(float)iv.x * unscale, (float)iv.y * unscale,
                             (float)iv.z * unscale, (float)iv.w * unscale};
        int mx = lo0 + ix, my = lo1 + iy;
        mx += mx < 0 ? w.K0 : (mx >= w.K0 ? -w.K0 : 0);
        my += my < 0 ? w.K1 : (my >= w.K1 ? -w.K1 : 0);
        const int mz = lo2 + 4 * k;
        float *dst = mesh + ((size_t)mx * w.K1 + my) * w.K2;
        if (w.vec && mz >= 0 && mz + 4 <= w.K2) {
            red_add_v4(dst + mz, vv[0], vv[1], vv[2], vv[3]);
            continue;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (vv[c] != 0.f) atomicAdd(dst + wrap_index(mz + c, w.K2), vv[c]);
    }
}

// Q^ *= G on the half spectrum; partial sums of the mesh energy 1/2 sum_full G |Q^|^2,
// where every half-spectrum point stands for itself and its mirror except on the
// planes m3 = 0 and (K3 even) m3 = K3/2.  Grid-stride over the flat half spectrum;
// m3 = t mod K2h is carried incrementally (stride_mod = stride mod K2h), so the
// loop has no integer division.  FP32 mode sums each thread's terms in FP32 with
// compensation; the block partials are FP64.
template <typename T, bool ENERGY>
__global__ void __launch_bounds__(kThreads)
k_influence(int nc, int K2h, int K2, int stride_mod, typename C2<T>::type *__restrict__ meshc,
            const T *__restrict__ G, double *__restrict__ part) {
    const int stride = gridDim.x * blockDim.x;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int m3 = t % K2h;
    T s = T(0), comp = T(0);
    for (; t < nc; t += stride) {
        auto z = meshc[t];
        const T g = G[t];
        if (ENERGY) {
            const T wgt = (m3 == 0 || 2 * m3 == K2) ? T(0.5) : T(1);
            const T term = wgt * g * (z.x * z.x + z.y * z.y);
            if constexpr (std::is_same<T, float>::value) {
                kahan_add(s, comp, term);
            } else {
                s += term;
            }
        }
        z.x *= g;
        z.y *= g;
        meshc[t] = z;
        m3 += stride_mod;
        if (m3 >= K2h) m3 -= K2h;
    }
    if (ENERGY) {
        double vals[1] = {(double)s - (double)comp};
        block_sum<1>(vals);
        if (threadIdx.x == 0) part[blockIdx.x] = vals[0];
    }
}

// Influence multiply without the energy (every MD-step apply): a plain
// elementwise product, one thread per point pair in FP32 (16-byte complex
// loads) or per point in FP64, over the whole grid so that many loads are in
// flight (the grid-stride energy variant above keeps a fixed grid for its
// partials).
__global__ void __launch_bounds__(kThreads) k_influence_mul32(int nc, float4 *__restrict__ meshc,
                                                              const float2 *__restrict__ G) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int npair = nc >> 1;
    if (t < npair) {
        float4 z = meshc[t];
        const float2 g = G[t];
        z.x *= g.x;
        z.y *= g.x;
        z.z *= g.y;
        z.w *= g.y;
        meshc[t] = z;
    } else if (t == npair && (nc & 1)) {
        float2 *zc = (float2 *)meshc + (nc - 1);
        const float g = ((const float *)G)[nc - 1];
        zc->x *= g;
        zc->y *= g;
    }
}

__global__ void __launch_bounds__(kThreads) k_influence_mul64(int nc, double2 *__restrict__ meshc,
                                                              const double *__restrict__ G) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nc) {
        double2 z = meshc[t];
        const double g = G[t];
        z.x *= g;
        z.y *= g;
        meshc[t] = z;
    }
}

struct GatherArgs {
    int n;
    int K0, K1, K2;
    double sx, sy, sz;  // K / L per axis
    double self_coef;   // k_e * (-2 alpha / sqrt(pi))
    double gauss_coef;  // k_e * sqrt(2 / pi) when the Gaussian self-energy is on, else 0
    float sx_f, sy_f, sz_f, self_coef_f, gauss_coef_f;  // FP32 copies (FP32-mixed epilogue)
};


// ENERGY: accumulate the energy partial sums (only when the caller asked for
// the energy parts).  The Gaussian self term k_e sqrt(2/pi) q / sigma takes 1 /
// sigma in FP64 in FP64 mode, and from the sorted FP32 sigma (correctly rounded
// reciprocal, relative error below 6e-8) in FP32-mixed mode: an FP64 divide per
// atom is about 30 operations of GB300's 1/64-rate FP64 pipe, which bounded this
// kernel.
template <typename T, int P, bool FIELD, bool ENERGY>
__global__ void __launch_bounds__(kThreads)
k_gather_out(GatherArgs a, const int32_t *__restrict__ perm, const int4 *__restrict__ sbase,
             const typename V4<T>::type *__restrict__ sfrac, const T *__restrict__ phi,
             const double *__restrict__ v_s, const double *__restrict__ E_s,
             const double *__restrict__ q, const double *__restrict__ sigma,
             const T *__restrict__ sg_sorted, double *__restrict__ v_out, double *__restrict__ E_out,
             double *__restrict__ F_out, double *__restrict__ part) {
    // FP32-mixed: the real-space kernel left (v, E) as one float4 per sorted atom
    const float4 *vE32 = reinterpret_cast<const float4 *>(E_s);
    double e_tot = 0.0, e_real = 0.0, e_self = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        const int4 b = sbase[i];
        const auto f = sfrac[i];
        T Mx[P], My[P], Mz[P], dMx[P], dMy[P], dMz[P];
        bspline<T, P, FIELD>(f.x, Mx, dMx);
        bspline<T, P, FIELD>(f.y, My, dMy);
        bspline<T, P, FIELD>(f.z, Mz, dMz);
        int iz[P];
#pragma unroll
        for (int c = 0; c < P; ++c) iz[c] = wrap_index(b.z - c, a.K2);
        T vr = T(0), gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
        for (int aa = 0; aa < P; ++aa) {
            const int ix = wrap_index(b.x - aa, a.K0);
#pragma unroll
            for (int bb = 0; bb < P; ++bb) {
                const int iy = wrap_index(b.y - bb, a.K1);
                const T *row = phi + ((size_t)ix * a.K1 + iy) * a.K2;
                T sv = T(0), sd = T(0);
#pragma unroll
                for (int c = 0; c < P; ++c) {
                    const T ph = row[iz[c]];
                    sv += Mz[c] * ph;
                    if (FIELD) sd += dMz[c] * ph;
                }
                vr += Mx[aa] * My[bb] * sv;
                if (FIELD) {
                    gx += dMx[aa] * My[bb] * sv;
                    gy += Mx[aa] * dMy[bb] * sv;
                    gz += Mx[aa] * My[bb] * sd;
                }
            }
        }
        const int atom = perm[i];
        if constexpr (std::is_same<T, float>::value && !ENERGY) {
            // FP32-mixed MD-step epilogue, all in FP32: the real-space sums, the
            // mesh part, the self terms and F = q E (with the sorted FP32 charge),
            // each result widened to double on the integer pipe for the store
            const float qf = f.w;
            float scf = a.self_coef_f;
            if (a.gauss_coef_f != 0.f) scf = fmaf(a.gauss_coef_f, __frcp_rn(sg_sorted[i]), scf);
            if (FIELD) {
                const float4 r4 = vE32[i];
                v_out[atom] = f32_to_f64_exact(fmaf(scf, qf, r4.x + vr));
                const float ex = fmaf(-a.sx_f, gx, r4.y);
                const float ey = fmaf(-a.sy_f, gy, r4.z);
                const float ez = fmaf(-a.sz_f, gz, r4.w);
                if (E_out) {
                    E_out[3 * (size_t)atom] = f32_to_f64_exact(ex);
                    E_out[3 * (size_t)atom + 1] = f32_to_f64_exact(ey);
                    E_out[3 * (size_t)atom + 2] = f32_to_f64_exact(ez);
                }
                if (F_out) {
                    F_out[3 * (size_t)atom] = f32_to_f64_exact(qf * ex);
                    F_out[3 * (size_t)atom + 1] = f32_to_f64_exact(qf * ey);
                    F_out[3 * (size_t)atom + 2] = f32_to_f64_exact(qf * ez);
                }
            } else {
                const float vsr = reinterpret_cast<const float *>(vE32)[4 * (size_t)i];
                v_out[atom] = f32_to_f64_exact(fmaf(scf, qf, vsr + vr));
            }
            continue;
        }
        const double qa = q[atom];
        double sc = a.self_coef;
        if (a.gauss_coef != 0.0) {
            if constexpr (std::is_same<T, float>::value)
                sc += a.gauss_coef * (double)__frcp_rn(sg_sorted[i]);
            else
                sc += a.gauss_coef / sigma[atom];
        }
        double vs, esx = 0.0, esy = 0.0, esz = 0.0;
        if constexpr (std::is_same<T, float>::value) {
            if (FIELD) {
                const float4 r4 = vE32[i];
                vs = r4.x;
                esx = r4.y;
                esy = r4.z;
                esz = r4.w;
            } else {
                vs = reinterpret_cast<const float *>(vE32)[4 * (size_t)i];
            }
        } else {
            vs = v_s[i];
            if (FIELD) {
                esx = E_s[3 * (size_t)i];
                esy = E_s[3 * (size_t)i + 1];
                esz = E_s[3 * (size_t)i + 2];
            }
        }
        const double vself = sc * qa;
        const double v = vs + (double)vr + vself;
        v_out[atom] = v;
        if (FIELD) {
            const double Ex = esx - a.sx * (double)gx;
            const double Ey = esy - a.sy * (double)gy;
            const double Ez = esz - a.sz * (double)gz;
            if (E_out) {
                E_out[3 * (size_t)atom] = Ex;
                E_out[3 * (size_t)atom + 1] = Ey;
                E_out[3 * (size_t)atom + 2] = Ez;
            }
            if (F_out) {
                F_out[3 * (size_t)atom] = qa * Ex;
                F_out[3 * (size_t)atom + 1] = qa * Ey;
                F_out[3 * (size_t)atom + 2] = qa * Ez;
            }
        }
        if (ENERGY) {
            e_tot += 0.5 * qa * v;
            e_real += 0.5 * qa * vs;
            e_self += 0.5 * qa * vself;
        }
    }
    if (ENERGY) {
        double vals[3] = {e_tot, e_real, e_self};
        block_sum<3>(vals);
        if (threadIdx.x == 0) {
            part[0 * kRedBlocks + blockIdx.x] = vals[0];
            part[1 * kRedBlocks + blockIdx.x] = vals[1];
            part[3 * kRedBlocks + blockIdx.x] = vals[2];
        }
    }
}

// One block per slot: the sum of the slot's nb block partials, in a fixed order.
__global__ void k_finalize(const double *__restrict__ part, int nb, double *__restrict__ out) {
    double s = 0.0;
    const double *p = part + (size_t)blockIdx.x * kRedBlocks;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) s += p[k];
    double vals[1] = {s};
    block_sum<1>(vals);
    if (threadIdx.x == 0) out[blockIdx.x] = vals[0];
}

// |b(m)|^2 of smooth PME for one axis (K points): b(m) = e^{2 pi i (p-1) m / K} /
// sum_{k=0}^{p-2} M_p(k+1) e^{2 pi i m k / K}; a vanishing denominator (odd p at
// m = K/2) gives 0.  Mk holds M_p(k + 1), k = 0..p-2.
struct SplineInts {
    double Mk[8];
    int p;
};

__global__ void k_bspline_mod2(int K, SplineInts s, double *__restrict__ out) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= K) return;
    double re = 0.0, im = 0.0;
    for (int k = 0; k <= s.p - 2; ++k) {
        double sn, cs;
        sincospi(2.0 * (double)(((long long)m * k) % K) / K, &sn, &cs);
        re += s.Mk[k] * cs;
        im += s.Mk[k] * sn;
    }
    const double d2 = re * re + im * im;
    out[m] = d2 > 1e-10 ? 1.0 / d2 : 0.0;
}

// Influence function G(m) = k_e (4 pi / V) exp(-k^2 / 4 alpha^2) / k^2 * B(m) on
// the half spectrum [K0][K1][K2/2+1], G(0) = 0 (Eq. ewald_rec with the smooth-PME
// B factor), one thread per point, from the per-axis |b|^2 tables b0, b1, b2.
template <typename T>
__global__ void k_influence_table(int K0, int K1, int K2, double Lx, double Ly, double Lz,
                                  double pref, double inv4a2, const double *__restrict__ b0,
                                  const double *__restrict__ b1, const double *__restrict__ b2,
                                  T *__restrict__ G) {
    const int K2h = K2 / 2 + 1;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)K0 * K1 * K2h) return;
    const int m2 = (int)(t % K2h), m1 = (int)((t / K2h) % K1), m0 = (int)(t / ((int64_t)K2h * K1));
    const int c0 = m0 <= K0 / 2 ? m0 : m0 - K0;
    const int c1 = m1 <= K1 / 2 ? m1 : m1 - K1;
    const double kx = 2.0 * kPi * c0 / Lx, ky = 2.0 * kPi * c1 / Ly, kz = 2.0 * kPi * m2 / Lz;
    const double k2 = kx * kx + ky * ky + kz * kz;
    G[t] = k2 > 0.0 ? (T)(pref * exp(-k2 * inv4a2) / k2 * b0[m0] * b1[m1] * b2[m2]) : T(0);
}

// ---------------------------------------------------------------------------
// host-side tables
// ---------------------------------------------------------------------------

// |b(m)|^2 of smooth PME: b(m) = e^{2 pi i (p-1) m / K} / sum_{k=0}^{p-2} M_p(k+1) e^{2 pi i m k / K}.
// A vanishing denominator (odd p at m = K/2) gives 0.
std::vector<double> bspline_mod2(int K, int p) {
    // M_p at the integers 0..p-1 by the same order recursion, evaluated at w = 0
    std::vector<double> M(p, 0.0);
    M[0] = 0.0;
    M[1] = 1.0;
    for (int n = 3; n <= p; ++n) {
        for (int j = n - 1; j >= 0; --j) {
            const double left = (j < n - 1) ? M[j] : 0.0;
            const double right = (j >= 1) ? M[j - 1] : 0.0;
            M[j] = (j * left + (n - j) * right) / (n - 1);
        }
    }
    std::vector<double> out(K);
    for (int m = 0; m < K; ++m) {
        double re = 0.0, im = 0.0;
        for (int k = 0; k <= p - 2; ++k) {
            const double ang = 2.0 * kPi * m * k / K;
            re += M[k + 1] * std::cos(ang);
            im += M[k + 1] * std::sin(ang);
        }
        const double d2 = re * re + im * im;
        out[m] = d2 > 1e-10 ? 1.0 / d2 : 0.0;
    }
    return out;
}

// Coefficients of the piecewise erfc: on piece k, [k h, (k + 1) h) with
// h = kErfcXMax / kErfcPieces, the polynomial in s = 2 (x - k h) / h - 1 that
// interpolates the long-double erfc at the kErfcCoef Chebyshev nodes of the
// piece.  The Vandermonde system in s is solved by Gaussian elimination in long
// double.
std::vector<double> erfc_table() {
    const int D = kErfcCoef;
    std::vector<double> out((size_t)kErfcPieces * D);
    const long double h = (long double)kErfcXMax / kErfcPieces;
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int k = 0; k < kErfcPieces; ++k) {
        long double A[kErfcCoef][kErfcCoef + 1];
        for (int j = 0; j < D; ++j) {
            const long double sj = cosl(pi * (j + 0.5L) / D);
            const long double xj = k * h + (sj + 1.0L) * 0.5L * h;
            long double pw = 1.0L;
            for (int m = 0; m < D; ++m) {
                A[j][m] = pw;
                pw *= sj;
            }
            A[j][D] = erfcl(xj);
        }
        for (int c = 0; c < D; ++c) {
            int best = c;
            for (int r = c + 1; r < D; ++r)
                if (fabsl(A[r][c]) > fabsl(A[best][c])) best = r;
            for (int m = 0; m <= D; ++m) {
                const long double tmp = A[c][m];
                A[c][m] = A[best][m];
                A[best][m] = tmp;
            }
            for (int r = 0; r < D; ++r) {
                if (r == c) continue;
                const long double f = A[r][c] / A[c][c];
                for (int m = c; m <= D; ++m) A[r][m] -= f * A[c][m];
            }
        }
        for (int m = 0; m < D; ++m) out[(size_t)k * D + m] = (double)(A[m][D] / A[m][m]);
    }
    return out;
}

// Piecewise table of F_a and G_a (shape sh, npieces pieces of sh.ncoef
// coefficient pairs, interleaved F, G): piece p covers octave
// e = sh.oct_lo + p / 2^sh.sub_log2, sub-piece j = p mod 2^sh.sub_log2, i.e.
// s = 2^e (1 + (j + (x + 1) / 2) / 2^sh.sub_log2) for x in [-1, 1).  The
// interpolation nodes are the same Chebyshev nodes in x for every piece, so the
// Vandermonde matrix in x is inverted once (Gauss-Jordan with partial pivoting
// in long double) and applied to the long-double F and G at the nodes of each
// piece.
constexpr int kPwMaxCoef = 16;

void pw_functions(long double a, long double s, long double &F, long double &G) {
    const long double pi = 3.141592653589793238462643383279502884L;
    const long double r = sqrtl(s);
    F = erfcl(a * r) / r;
    G = -(F + 2.0L * a / sqrtl(pi) * expl(-a * a * s)) / s;
}

long double pw_arg(const PwShape &sh, int p, long double x) {
    const int S = 1 << sh.sub_log2;
    return ldexpl(1.0L + (p % S + (x + 1.0L) * 0.5L) / S, sh.oct_lo + p / S);
}

std::vector<double> pw_table(double alpha, const PwShape &sh, int npieces) {
    const int D = sh.ncoef;
    const long double pi = 3.141592653589793238462643383279502884L;
    long double xs[kPwMaxCoef], W[kPwMaxCoef][2 * kPwMaxCoef];
    for (int k = 0; k < D; ++k) {
        xs[k] = cosl(pi * (k + 0.5L) / D);
        long double pw = 1.0L;
        for (int m = 0; m < D; ++m) {
            W[k][m] = pw;
            W[k][D + m] = (k == m) ? 1.0L : 0.0L;
            pw *= xs[k];
        }
    }
    for (int c = 0; c < D; ++c) {
        int best = c;
        for (int r = c + 1; r < D; ++r)
            if (fabsl(W[r][c]) > fabsl(W[best][c])) best = r;
        for (int m = 0; m < 2 * D; ++m) {
            const long double tmp = W[c][m];
            W[c][m] = W[best][m];
            W[best][m] = tmp;
        }
        const long double piv = W[c][c];
        for (int m = 0; m < 2 * D; ++m) W[c][m] /= piv;
        for (int r = 0; r < D; ++r) {
            if (r == c) continue;
            const long double f = W[r][c];
            for (int m = 0; m < 2 * D; ++m) W[r][m] -= f * W[c][m];
        }
    }
    // W[.][D..2D) is now the inverse: coefficient m = sum_k inv[m][k] value(x_k)
    std::vector<double> out((size_t)npieces * D * 2);
    for (int p = 0; p < npieces; ++p) {
        long double F[kPwMaxCoef], G[kPwMaxCoef];
        for (int k = 0; k < D; ++k) pw_functions(alpha, pw_arg(sh, p, xs[k]), F[k], G[k]);
        for (int m = 0; m < D; ++m) {
            long double cf = 0.0L, cg = 0.0L;
            for (int k = 0; k < D; ++k) {
                cf += W[m][D + k] * F[k];
                cg += W[m][D + k] * G[k];
            }
            out[((size_t)p * D + m) * 2] = (double)cf;
            out[((size_t)p * D + m) * 2 + 1] = (double)cg;
        }
    }
    return out;
}

// Pieces of a table whose argument stays below smax: the octaves from
// 2^sh.oct_lo up to the one holding the largest argument below smax, at most
// sh.max_oct.
int pw_pieces_for(const PwShape &sh, double smax) {
    if (!(smax > 0.0)) return 0;
    int E = 0;
    const double m = std::frexp(smax, &E);  // smax = m 2^E, m in [0.5, 1)
    const int emax = (m == 0.5) ? E - 2 : E - 1;  // exponent of the largest s < smax
    const int oct = std::max(0, std::min(sh.max_oct, emax - sh.oct_lo + 1));
    return oct << sh.sub_log2;
}

// Leading pieces of a table whose F and G, evaluated by the kernel's Horner
// scheme in double at 33 points of each piece, stay within 1e-13 of the
// long-double functions, relative to the larger of the function and 1e-2 of the
// bare Coulomb term (1 / r for F, 1 / r^3 for G), i.e. within 1e-15 of the bare
// term where the screened one is far below it; the rest takes the direct path.
int pw_valid_pieces(const std::vector<double> &tab, double alpha, const PwShape &sh, int npieces) {
    const int D = sh.ncoef;
    for (int p = 0; p < npieces; ++p) {
        const double *c = tab.data() + (size_t)p * D * 2;
        for (int t = 0; t <= 32; ++t) {
            const double x = -1.0 + t / 16.0 - (t == 32 ? 0x1p-40 : 0.0);
            double f = c[2 * (D - 1)], g = c[2 * (D - 1) + 1];
            for (int m = D - 2; m >= 0; --m) {
                f = std::fma(f, x, c[2 * m]);
                g = std::fma(g, x, c[2 * m + 1]);
            }
            const long double sk = pw_arg(sh, p, x);
            long double F, G;
            pw_functions(alpha, sk, F, G);
            const long double bare = 1.0L / sqrtl(sk);
            const long double fs = std::max(fabsl(F), 1e-2L * bare);
            const long double gs = std::max(fabsl(G), 1e-2L * bare / sk);
            if (fabsl((long double)f - F) > 1e-13L * fs || fabsl((long double)g - G) > 1e-13L * gs)
                return p;
        }
    }
    return npieces;
}

// Process-wide cache of the tables (their host copies live until exit, so the
// uploads need no synchronisation): the coefficients and the kept pieces per
// alpha, shape and size.
const std::vector<double> &pw_cached(double alpha, const PwShape &sh, int np, int *valid) {
    struct Entry {
        std::vector<double> tab;
        int valid;
    };
    static std::mutex mu;
    static std::map<std::tuple<double, int, int>, Entry> cache;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(alpha, sh.oct_lo, np);
    auto it = cache.find(key);
    if (it == cache.end()) {
        Entry en{pw_table(alpha, sh, np), 0};
        en.valid = pw_valid_pieces(en.tab, alpha, sh, np);
        it = cache.emplace(key, std::move(en)).first;
    }
    *valid = it->second.valid;
    return it->second.tab;
}

// The kernel's table evaluation on the host (same bit indexing, same fused
// Horner steps), for the host-only diagnostic.
bool pw_eval_host(const PwShape &sh, const double *tab, int npieces, double arg, double &f,
                  double &g) {
    uint64_t b;
    std::memcpy(&b, &arg, sizeof b);
    const int hi = (int)(uint32_t)(b >> 32);
    const unsigned piece =
        (unsigned)((hi >> (20 - sh.sub_log2)) - ((1023 + sh.oct_lo) << sh.sub_log2));
    if (piece >= (unsigned)npieces) return false;
    const uint32_t lo = (uint32_t)b;
    const uint32_t hy = 0x3FF00000u | (((uint32_t)hi << sh.sub_log2) & 0x000FFFFFu) |
                        (lo >> (32 - sh.sub_log2));
    const uint64_t yb = ((uint64_t)hy << 32) | (uint32_t)(lo << sh.sub_log2);
    double y;
    std::memcpy(&y, &yb, sizeof y);
    const double x = std::fma(y, 2.0, -3.0);
    const int D = sh.ncoef;
    const double *c = tab + (size_t)piece * D * 2;
    f = c[2 * (D - 1)];
    g = c[2 * (D - 1) + 1];
    for (int m = D - 2; m >= 0; --m) {
        f = std::fma(f, x, c[2 * m]);
        g = std::fma(g, x, c[2 * m + 1]);
    }
    return true;
}

// The table a context with this alpha and cutoff^2 smax uses (which 0), or the
// Gaussian-correction table (which 1).
const std::vector<double> &pw_context_table(int which, double alpha, double smax, const PwShape **sh,
                                            int *kept) {
    if (which == 0) {
        *sh = &kFGShape;
        return pw_cached(alpha, kFGShape, pw_pieces_for(kFGShape, smax), kept);
    }
    *sh = &kGCShape;
    return pw_cached(1.0, kGCShape, pw_pieces_for(kGCShape, kErfcXMax * kErfcXMax * (1.0 + 2e-5)), kept);
}

// M_P(P / 2), the peak of the cardinal B-spline of order P, by the same order
// recursion as bspline_mod2 (evaluated at the midpoint).
double bspline_peak(int P) {
    std::vector<double> M(P + 1, 0.0);  // M[j] = M_n(j + f) for the fraction f
    const double f = (P % 2 == 0) ? 0.0 : 0.5;  // P / 2 = j + f
    M[0] = f;
    M[1] = 1.0 - f;
    for (int n = 3; n <= P; ++n) {
        for (int j = n - 1; j >= 0; --j) {
            const double left = (j < n - 1) ? M[j] : 0.0;
            const double right = (j >= 1) ? M[j - 1] : 0.0;
            M[j] = ((f + j) * left + (n - f - j) * right) / (n - 1);
        }
    }
    double peak = 0.0;
    for (int j = 0; j < P; ++j) peak = std::max(peak, M[j]);
    return peak * (1.0 + 1e-6);
}

// Shared-memory window of the brick spreading, or nbytes = 0 when it exceeds
// kSpreadSmemMax (a box of very few bricks against a fine mesh): then the
// one-thread-per-atom global spreading runs instead.
SpreadWin spread_window(const qeq_ctx *ctx, int P, size_t elem, size_t *nbytes) {
    SpreadWin w;
    w.K0 = ctx->K[0];
    w.K1 = ctx->K[1];
    w.K2 = ctx->K[2];
    const BrickGeom &g = ctx->geom;
    const double X[3] = {g.B[0] * ctx->cw[0] * ctx->K[0] / ctx->p.box[0],
                         g.B[1] * ctx->cw[1] * ctx->K[1] / ctx->p.box[1],
                         g.B[2] * ctx->cw[2] * ctx->K[2] / ctx->p.box[2]};
    // base = floor(K x / L) of the brick's atoms lies in [floor(b X), floor((b + 1) X)],
    // floor((b + 1) X) - floor(b X) <= ceil(X), and the support reaches P - 1
    // points below: ceil(X) + P points per axis, up to 3 more below z from the
    // alignment.  An atom that rounding puts outside takes the global path.
    w.E0 = (int)std::ceil(X[0]) + P;
    w.E1 = (int)std::ceil(X[1]) + P;
    w.E2 = ((int)std::ceil(X[2]) + P + 3 + 3) / 4 * 4;
    w.vec = ctx->K[2] % 4 == 0;
    // largest cardinal B-spline value M_P(P / 2), cubed: one atom's largest weight
    w.wmax = (float)std::pow(bspline_peak(P), 3);
    const size_t bytes = elem * w.E0 * w.E1 * w.E2;
    *nbytes = bytes <= kSpreadSmemMax ? bytes : 0;
    return w;
}

template <typename T, int P>
void launch_spread(qeq_ctx *ctx, const int4 *sb, const void *sf, cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
        size_t bytes = 0;
        const SpreadWin w = spread_window(ctx, P, sizeof(int), &bytes);
        if (bytes) {
            k_spread_brick<P><<<(unsigned)ctx->geom.nbricks, kSpreadThreads, bytes, s>>>(
                w, ctx->geom, ctx->cell_start, sb, (const float4 *)sf, (float *)ctx->mesh);
            return;
        }
    }
    k_spread<T, P><<<grid_for(ctx->n), kThreads, 0, s>>>(
        (int)ctx->n, sb, (const typename V4<T>::type *)sf, ctx->K[0], ctx->K[1], ctx->K[2],
        (T *)ctx->mesh);
}

template <typename T, int P, bool FIELD>
void launch_gather(qeq_ctx *ctx, const GatherArgs &ga, const int4 *sb, const void *sf,
                   const double *q, const double *sigma, double *v, double *E, double *F,
                   bool energy, cudaStream_t s) {
    const T *sgs = std::is_same<T, float>::value ? (const T *)ctx->sg32 : (const T *)ctx->sg64;
    if (energy)
        k_gather_out<T, P, FIELD, true><<<ctx->red_grid, kThreads, 0, s>>>(
            ga, ctx->perm, sb, (const typename V4<T>::type *)sf, (const T *)ctx->mesh, ctx->v_s,
            ctx->E_s, q, sigma, sgs, v, E, F, ctx->part);
    else  // no partials: one thread per atom, every atom in flight at once
        k_gather_out<T, P, FIELD, false><<<grid_for(ctx->n), kThreads, 0, s>>>(
            ga, ctx->perm, sb, (const typename V4<T>::type *)sf, (const T *)ctx->mesh, ctx->v_s,
            ctx->E_s, q, sigma, sgs, v, E, F, ctx->part);
}

template <typename T>
void dispatch_spread(qeq_ctx *ctx, const int4 *sb, const void *sf, cudaStream_t s) {
    switch (ctx->p.order) {
        case 4: launch_spread<T, 4>(ctx, sb, sf, s); break;
        case 5: launch_spread<T, 5>(ctx, sb, sf, s); break;
        case 6: launch_spread<T, 6>(ctx, sb, sf, s); break;
        case 7: launch_spread<T, 7>(ctx, sb, sf, s); break;
        default: launch_spread<T, 8>(ctx, sb, sf, s); break;
    }
}

template <typename T, bool FIELD>
void dispatch_gather(qeq_ctx *ctx, const GatherArgs &ga, const int4 *sb, const void *sf,
                     const double *q, const double *sigma, double *v, double *E, double *F,
                     bool energy, cudaStream_t s) {
    switch (ctx->p.order) {
        case 4: launch_gather<T, 4, FIELD>(ctx, ga, sb, sf, q, sigma, v, E, F, energy, s); break;
        case 5: launch_gather<T, 5, FIELD>(ctx, ga, sb, sf, q, sigma, v, E, F, energy, s); break;
        case 6: launch_gather<T, 6, FIELD>(ctx, ga, sb, sf, q, sigma, v, E, F, energy, s); break;
        case 7: launch_gather<T, 7, FIELD>(ctx, ga, sb, sf, q, sigma, v, E, F, energy, s); break;
        default: launch_gather<T, 8, FIELD>(ctx, ga, sb, sf, q, sigma, v, E, F, energy, s); break;
    }
}

// Launch shape of the brick-tiled real-space kernels for the current list: one
// block per brick, kTPR lanes per row of the largest brick, the tile capacity
// ctx->tile_cap (atoms) in shared memory, or in the global tile scratch when it
// does not fit (boxes of a few hundred atoms whose tile repeats the box).
struct RealLaunch {
    int threads;
    int cap;
    int qcap;  // FP64: deferred-correction queue entries per lane
    size_t smem;
    bool gtile;
};

RealLaunch real_launch(const qeq_ctx *ctx, bool f64) {
    RealLaunch L;
    L.threads = real_block_threads(ctx->rows_cap);
    L.cap = ctx->tile_cap;
    const size_t bytes = (size_t)L.cap * (f64 ? kTile64Bytes : kTile32Bytes);
    const size_t tables = f64 ? kPwTableBytes : 0;  // the FP64 pair-function tables
    L.gtile = tables + bytes > (f64 ? kReal64SmemMax : kReal32SmemMax);
    L.smem = tables + (L.gtile ? 0 : bytes);
    L.qcap = 0;
    if (f64) {
        // the correction queue takes what shared memory is left, up to kCorrQueueMax
        const size_t left = kReal64SmemMax - L.smem;
        L.qcap = (int)std::min<size_t>(kCorrQueueMax, left / (sizeof(uint16_t) * L.threads));
        L.smem += (size_t)L.qcap * L.threads * sizeof(uint16_t);
    }
    return L;
}

// Reciprocal-space chain of Alg. 2 up to the mesh potential: clear the mesh,
// spread the charges (a6), forward FFT (a7), influence multiply with the
// optional energy partials (a8), inverse FFT (a9), all on stream sp.  It reads
// only the gathered fractions and charges, so it runs beside the real-space
// kernel.
template <typename T>
int pme_mesh_potential(qeq_ctx *ctx, double *energy4, cudaStream_t sp) {
    constexpr bool f64 = std::is_same<T, double>::value;
    prof_begin(ctx, kPhSpread, sp);
    cudaMemsetAsync(ctx->mesh, 0, sizeof(T) * ctx->mesh_n, sp);
    dispatch_spread<T>(ctx, ctx->sbase, ctx->sfrac, sp);
    prof_end(ctx, sp);
    ctx->launches++;
    cufftResult cr;
    cr = cufftSetStream(ctx->plan_r2c, sp);
    if (cr == CUFFT_SUCCESS) cr = cufftSetStream(ctx->plan_c2r, sp);
    if (cr != CUFFT_SUCCESS) return set_error(ctx, QEQ_ERR_CUFFT, "cufftSetStream failed (%d)", (int)cr);
    prof_begin(ctx, kPhFftFwd, sp);
    if (f64)
        cr = cufftExecD2Z(ctx->plan_r2c, (cufftDoubleReal *)ctx->mesh, (cufftDoubleComplex *)ctx->meshc);
    else
        cr = cufftExecR2C(ctx->plan_r2c, (cufftReal *)ctx->mesh, (cufftComplex *)ctx->meshc);
    prof_end(ctx, sp);
    ctx->fft_execs++;
    if (cr != CUFFT_SUCCESS) return set_error(ctx, QEQ_ERR_CUFFT, "forward FFT failed (%d)", (int)cr);
    prof_begin(ctx, kPhInfluence, sp);
    {
        const int K2h = ctx->K[2] / 2 + 1;
        if (energy4)
            k_influence<T, true><<<ctx->red_grid, kThreads, 0, sp>>>(
                (int)ctx->meshc_n, K2h, ctx->K[2], (ctx->red_grid * kThreads) % K2h,
                (typename C2<T>::type *)ctx->meshc, (const T *)ctx->G, ctx->part + 2 * kRedBlocks);
        else if (f64)
            k_influence_mul64<<<grid_for(ctx->meshc_n), kThreads, 0, sp>>>(
                (int)ctx->meshc_n, (double2 *)ctx->meshc, (const double *)ctx->G);
        else
            k_influence_mul32<<<grid_for(ctx->meshc_n / 2 + 1), kThreads, 0, sp>>>(
                (int)ctx->meshc_n, (float4 *)ctx->meshc, (const float2 *)ctx->G);
    }
    prof_end(ctx, sp);
    ctx->launches++;
    prof_begin(ctx, kPhFftInv, sp);
    if (f64)
        cr = cufftExecZ2D(ctx->plan_c2r, (cufftDoubleComplex *)ctx->meshc, (cufftDoubleReal *)ctx->mesh);
    else
        cr = cufftExecC2R(ctx->plan_c2r, (cufftComplex *)ctx->meshc, (cufftReal *)ctx->mesh);
    prof_end(ctx, sp);
    ctx->fft_execs++;
    if (cr != CUFFT_SUCCESS) return set_error(ctx, QEQ_ERR_CUFFT, "inverse FFT failed (%d)", (int)cr);
    return QEQ_OK;
}

template <typename T>
int apply_t(qeq_ctx *ctx, const double *R, const double *q, const double *sigma, double *v,
            double *E, double *F, double *energy4, bool need_field, bool q_only, cudaStream_t s) {
    const int n = (int)ctx->n;
    using T4 = typename V4<T>::type;
    constexpr bool f64 = std::is_same<T, double>::value;
    T4 *xq = f64 ? (T4 *)ctx->xq64 : (T4 *)ctx->xq32;
    T *sg = f64 ? (T *)ctx->sg64 : (T *)ctx->sg32;
    const qeq_params &p = ctx->p;
    ctx->applies++;
    prof_begin(ctx, kPhGatherIn, s);
    if (q_only) {
        k_gather_q<T><<<grid_for(n), kThreads, 0, s>>>(n, ctx->perm, q, xq, (T4 *)ctx->sfrac,
                                                       ctx->d_flags);
    } else {
        int32_t *smax_bits = (!f64 && kRealLazySigma) ? ctx->d_flags + kFlagSigmaMax : nullptr;
        if (smax_bits) cudaMemsetAsync(smax_bits, 0, sizeof(int32_t), s);
        k_gather_in<T><<<grid_for(n), kThreads, 0, s>>>(
            n, ctx->perm, R, ctx->wrap_off, q, sigma, ctx->K[0] / p.box[0], ctx->K[1] / p.box[1],
            ctx->K[2] / p.box[2], xq, sg, ctx->sbase, (T4 *)ctx->sfrac, smax_bits,
            f64 ? ctx->xf_pre : nullptr, ctx->d_flags);
        ctx->gathered = true;
    }
    prof_end(ctx, s);
    ctx->launches++;

    RealArgs ra;
    ra.n = n;
    ra.Lx = p.box[0]; ra.Ly = p.box[1]; ra.Lz = p.box[2];
    ra.alpha = p.alpha;
    ra.rc2 = p.r_cut * p.r_cut;
    ra.ke = p.k_e;
    ra.alpha_f = (float)ra.alpha;
    ra.rc2_f = (float)ra.rc2;
    ra.tspa_f = (float)(kTwoOverSqrtPi * ra.alpha);
    ra.c1_f = (float)(-ra.alpha * ra.alpha * 1.4426950408889634);
    ra.pal_f = (float)(0.3275911 * ra.alpha);
    ra.ke_f = (float)ra.ke;
    ra.Lx_f = (float)ra.Lx;
    ra.Ly_f = (float)ra.Ly;
    ra.Lz_f = (float)ra.Lz;
    ra.fg_pieces = ctx->fg_pieces;
    ra.gc_pieces = ctx->gc_pieces;
    {
        // tile coordinates lie within 3 box lengths of 0, so each FP32 coordinate
        // difference is off by at most 4.8e-7 L_max and r^2 by far less than
        // 4e-6 r_list L_max + 1e-5 r_c^2
        const double Lm = std::max(ra.Lx, std::max(ra.Ly, ra.Lz));
        ra.pre_rc2_f = (float)(ra.rc2 * (1.0 + 1e-5) + 4e-6 * ctx->rl * Lm);
    }
    // The mesh chain goes first, on the context's high-priority side stream
    // (forked here, joined before the combining gather), so that its short,
    // latency-bound kernels fill the issue slots the real-space kernel leaves;
    // profiled passes keep one stream so that each phase is timed alone.
    const bool pme = p.recip != QEQ_RECIP_EWALD;
    cudaStream_t sp = s;
    if (pme) {
        if (!ctx->prof.on && ctx->pme_stream) {
            sp = ctx->pme_stream;
            cudaEventRecord(ctx->pme_fork, s);
            cudaStreamWaitEvent(sp, ctx->pme_fork, 0);
        }
        const int rc = pme_mesh_potential<T>(ctx, energy4, sp);
        if (sp != s) {
            cudaEventRecord(ctx->pme_join, sp);
            if (rc) cudaStreamWaitEvent(s, ctx->pme_join, 0);
        }
        if (rc) return rc;
    }
    prof_begin(ctx, kPhReal, s);
    {
        const RealLaunch L = real_launch(ctx, f64);
        const dim3 grid((unsigned)ctx->geom.nbricks);
        int32_t *fl = ctx->d_flags;
        unsigned char *gt = ctx->tile_scratch;
        if (f64) {
            auto *x4 = (const double4_32a *)xq;
            auto *s1 = (const double *)sg;
            if (need_field && !L.gtile)
                k_real64<true, false><<<grid, L.threads, L.smem, s>>>(ra, ctx->geom, ctx->tile_tab, ctx->tile_tot, ctx->nbr, ctx->cnt, x4, s1, ctx->xf_pre, ctx->erfc_tab64, (const double2 *)ctx->fg_tab64, (const double2 *)ctx->gc_tab64, L.cap, L.qcap, gt, fl, ctx->v_s, ctx->E_s);
            else if (need_field)
                k_real64<true, true><<<grid, L.threads, L.smem, s>>>(ra, ctx->geom, ctx->tile_tab, ctx->tile_tot, ctx->nbr, ctx->cnt, x4, s1, ctx->xf_pre, ctx->erfc_tab64, (const double2 *)ctx->fg_tab64, (const double2 *)ctx->gc_tab64, L.cap, L.qcap, gt, fl, ctx->v_s, ctx->E_s);
            else if (!L.gtile)
                k_real64<false, false><<<grid, L.threads, L.smem, s>>>(ra, ctx->geom, ctx->tile_tab, ctx->tile_tot, ctx->nbr, ctx->cnt, x4, s1, ctx->xf_pre, ctx->erfc_tab64, (const double2 *)ctx->fg_tab64, (const double2 *)ctx->gc_tab64, L.cap, L.qcap, gt, fl, ctx->v_s, ctx->E_s);
            else
                k_real64<false, true><<<grid, L.threads, L.smem, s>>>(ra, ctx->geom, ctx->tile_tab, ctx->tile_tot, ctx->nbr, ctx->cnt, x4, s1, ctx->xf_pre, ctx->erfc_tab64, (const double2 *)ctx->fg_tab64, (const double2 *)ctx->gc_tab64, L.cap, L.qcap, gt, fl, ctx->v_s, ctx->E_s);
        } else {
            auto *x4 = (const float4 *)xq;
            auto *s1 = (const float *)sg;
            const int32_t *sm = ctx->d_flags + kFlagSigmaMax;
            // FP32 partial sums in the E_s buffer (24 bytes per atom hold the 16)
            auto *vE32 = (float4 *)ctx->E_s;
            if (need_field && !L.gtile)
                k_real32<true, false><<<grid, L.threads, L.smem, s>>>(ra, ctx->geom, ctx->tile_tab, ctx->tile_tot, ctx->nbr, ctx->cnt, x4, s1, sm, L.cap, gt, fl, vE32);
            else if (need_field)
                k_real32<true, true><<<grid, L.threads, 0, s>>>(ra, ctx->geom, ctx->tile_tab, ctx->tile_tot, ctx->nbr, ctx->cnt, x4, s1, sm, L.cap, gt, fl, vE32);
            else if (!L.gtile)
                k_real32<false, false><<<grid, L.threads, L.smem, s>>>(ra, ctx->geom, ctx->tile_tab, ctx->tile_tot, ctx->nbr, ctx->cnt, x4, s1, sm, L.cap, gt, fl, vE32);
            else
                k_real32<false, true><<<grid, L.threads, 0, s>>>(ra, ctx->geom, ctx->tile_tab, ctx->tile_tot, ctx->nbr, ctx->cnt, x4, s1, sm, L.cap, gt, fl, vE32);
        }
    }

    prof_end(ctx, s);
    ctx->launches++;
    if (!pme) {
        int rc = ewald_recip_and_combine(ctx, q, sigma, v, E, F, need_field, s);
        if (rc) return rc;
        if (energy4) {
            k_finalize<<<4, kThreads, 0, s>>>(ctx->part, ctx->red_grid, energy4);
            ctx->launches++;
        }
        return cuda_check(ctx, cudaGetLastError(), "coulomb apply launch");
    }
    if (sp != s) cudaStreamWaitEvent(s, ctx->pme_join, 0);
    GatherArgs ga;
    ga.n = n;
    ga.K0 = ctx->K[0]; ga.K1 = ctx->K[1]; ga.K2 = ctx->K[2];
    ga.sx = ctx->K[0] / p.box[0];
    ga.sy = ctx->K[1] / p.box[1];
    ga.sz = ctx->K[2] / p.box[2];
    ga.self_coef = p.k_e * (-kTwoOverSqrtPi * p.alpha);
    ga.gauss_coef = p.gaussian_self ? p.k_e * kSqrtTwoOverPi : 0.0;
    ga.sx_f = (float)ga.sx;
    ga.sy_f = (float)ga.sy;
    ga.sz_f = (float)ga.sz;
    ga.self_coef_f = (float)ga.self_coef;
    ga.gauss_coef_f = (float)ga.gauss_coef;
    prof_begin(ctx, kPhGatherOut, s);
    const bool energy = energy4 != nullptr;
    if (need_field)
        dispatch_gather<T, true>(ctx, ga, ctx->sbase, ctx->sfrac, q, sigma, v, E, F, energy, s);
    else
        dispatch_gather<T, false>(ctx, ga, ctx->sbase, ctx->sfrac, q, sigma, v, nullptr, nullptr,
                                  energy, s);
    prof_end(ctx, s);
    ctx->launches++;
    if (energy4) {
        k_finalize<<<4, kThreads, 0, s>>>(ctx->part, ctx->red_grid, energy4);
        ctx->launches++;
    }
    return cuda_check(ctx, cudaGetLastError(), "coulomb apply launch");
}

}  // namespace

void launch_finalize(const qeq_ctx *ctx, const double *part, int nslots, double *out, cudaStream_t s) {
    k_finalize<<<nslots, kThreads, 0, s>>>(part, ctx->red_grid, out);
}

// Process-wide pool of mesh side streams (high-priority, non-blocking) and
// their fork / join events, per device: a context takes one at creation and
// returns it at destruction, so per-request contexts create no streams.  A
// returned stream may still hold its last owner's queued work; the next
// owner's work queues behind it, and each owner reaches its stream only
// through its own fork and join events.
namespace {
struct SideStream {
    int device;
    cudaStream_t s;
    cudaEvent_t fork, join;
};
std::mutex g_side_mu;
std::vector<SideStream> g_side_free;
}  // namespace

cudaError_t side_acquire(int device, cudaStream_t *s, cudaEvent_t *fork, cudaEvent_t *join) {
    {
        std::lock_guard<std::mutex> lock(g_side_mu);
        for (size_t k = 0; k < g_side_free.size(); ++k)
            if (g_side_free[k].device == device) {
                *s = g_side_free[k].s;
                *fork = g_side_free[k].fork;
                *join = g_side_free[k].join;
                g_side_free.erase(g_side_free.begin() + (std::ptrdiff_t)k);
                return cudaSuccess;
            }
    }
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(s, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(join, cudaEventDisableTiming);
    return e;
}

void side_release(int device, cudaStream_t s, cudaEvent_t fork, cudaEvent_t join) {
    if (!s || !fork || !join) {  // a partly created set (creation failed): destroy it
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (s) cudaStreamDestroy(s);
        return;
    }
    std::lock_guard<std::mutex> lock(g_side_mu);
    g_side_free.push_back({device, s, fork, join});
}

int coulomb_alloc(qeq_ctx *ctx) {
    const qeq_params &p = ctx->p;
    const int64_t n = ctx->n;
    for (int d = 0; d < 3; ++d) ctx->K[d] = p.mesh[d];
    const int K2h = ctx->K[2] / 2 + 1;
    ctx->mesh_n = (int64_t)ctx->K[0] * ctx->K[1] * ctx->K[2];
    ctx->meshc_n = (int64_t)ctx->K[0] * ctx->K[1] * K2h;
    const size_t rs = ctx->fp32 ? sizeof(float) : sizeof(double);
    struct {
        void **ptr;
        size_t bytes;
    } bufs[] = {
        {(void **)&ctx->v_s, sizeof(double) * n},
        {(void **)&ctx->E_s, sizeof(double) * 3 * n},
        {(void **)&ctx->sbase, sizeof(int4) * n},
        {(void **)&ctx->sfrac, 4 * rs * n},
        {ctx->fp32 ? (void **)&ctx->xq32 : (void **)&ctx->xq64, 4 * rs * n},
        {ctx->fp32 ? (void **)&ctx->sg32 : (void **)&ctx->sg64, rs * n},
        {(void **)&ctx->xf_pre, ctx->fp32 ? 0 : sizeof(float4) * n},
        {&ctx->mesh, rs * ctx->mesh_n},
        {&ctx->meshc, 2 * rs * ctx->meshc_n},
        {&ctx->G, rs * ctx->meshc_n},
        {(void **)&ctx->part, sizeof(double) * kMaxRedSlots * kRedBlocks},
        {(void **)&ctx->scal, sizeof(double) * kNumScal},
        {(void **)&ctx->energy4, sizeof(double) * 4},
        {(void **)&ctx->ticket, sizeof(unsigned int) * 4},
    };
    for (auto &b : bufs) {
        int rc = dev_alloc(ctx, b.ptr, b.bytes);
        if (rc) return rc;
    }
    ctx->h_scal = new (std::nothrow) double[kNumScal];
    if (!ctx->h_scal) return set_error(ctx, QEQ_ERR_NOMEM, "host allocation failed");
    cudaMemsetAsync(ctx->scal, 0, sizeof(double) * kNumScal, ctx->alloc_stream);
    cudaMemsetAsync(ctx->part, 0, sizeof(double) * kMaxRedSlots * kRedBlocks, ctx->alloc_stream);
    cudaMemsetAsync(ctx->ticket, 0, sizeof(unsigned int) * 4, ctx->alloc_stream);

    // influence function on the device: per-axis |b|^2 (into the reduction
    // partials, free until the first apply), then G on the half spectrum
    {
        SplineInts si{};
        si.p = p.order;
        {
            std::vector<double> M(p.order, 0.0);  // M_p at the integers by the order recursion
            M[1] = 1.0;
            for (int nn = 3; nn <= p.order; ++nn)
                for (int j = nn - 1; j >= 0; --j) {
                    const double left = (j < nn - 1) ? M[j] : 0.0;
                    const double right = (j >= 1) ? M[j - 1] : 0.0;
                    M[j] = (j * left + (nn - j) * right) / (nn - 1);
                }
            for (int k = 0; k + 1 < p.order; ++k) si.Mk[k] = M[k + 1];
        }
        double *bm = ctx->part;  // K0 + K1 + K2 <= 3 * 4096 < kMaxRedSlots * kRedBlocks
        cudaStream_t as = ctx->alloc_stream;
        k_bspline_mod2<<<grid_for(ctx->K[0]), kThreads, 0, as>>>(ctx->K[0], si, bm);
        k_bspline_mod2<<<grid_for(ctx->K[1]), kThreads, 0, as>>>(ctx->K[1], si, bm + ctx->K[0]);
        k_bspline_mod2<<<grid_for(ctx->K[2]), kThreads, 0, as>>>(ctx->K[2], si, bm + ctx->K[0] + ctx->K[1]);
        const double V = p.box[0] * p.box[1] * p.box[2];
        const double pref = p.k_e * 4.0 * kPi / V;
        const double inv4a2 = 1.0 / (4.0 * p.alpha * p.alpha);
        if (ctx->fp32)
            k_influence_table<float><<<grid_for(ctx->meshc_n), kThreads, 0, as>>>(
                ctx->K[0], ctx->K[1], ctx->K[2], p.box[0], p.box[1], p.box[2], pref, inv4a2, bm,
                bm + ctx->K[0], bm + ctx->K[0] + ctx->K[1], (float *)ctx->G);
        else
            k_influence_table<double><<<grid_for(ctx->meshc_n), kThreads, 0, as>>>(
                ctx->K[0], ctx->K[1], ctx->K[2], p.box[0], p.box[1], p.box[2], pref, inv4a2, bm,
                bm + ctx->K[0], bm + ctx->K[0] + ctx->K[1], (double *)ctx->G);
        cudaMemsetAsync(ctx->part, 0, sizeof(double) * (ctx->K[0] + ctx->K[1] + ctx->K[2]), as);
        int rcg = cuda_check(ctx, cudaGetLastError(), "influence table");
        if (rcg) return rcg;
    }
    cudaError_t e = cudaSuccess;
    int rc = QEQ_OK;
    if (p.recip != QEQ_RECIP_EWALD) {
        e = side_acquire(ctx->device, &ctx->pme_stream, &ctx->pme_fork, &ctx->pme_join);
        rc = cuda_check(ctx, e, "mesh side stream");
        if (rc) return rc;
    }

    if (p.recip == QEQ_RECIP_EWALD) {
        rc = ewald_alloc(ctx);
        if (rc) return rc;
    }

    // dynamic shared memory of the tiled real-space kernels (up to 227 KB a block)
    {
        cudaError_t ea = cudaFuncSetAttribute(k_real32<true, false>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kReal32SmemMax);
        if (ea == cudaSuccess)
            ea = cudaFuncSetAttribute(k_real32<false, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kReal32SmemMax);
        if (ea == cudaSuccess)
            ea = cudaFuncSetAttribute(k_real64<true, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kReal64SmemMax);
        if (ea == cudaSuccess)
            ea = cudaFuncSetAttribute(k_real64<false, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kReal64SmemMax);
        if (ea == cudaSuccess)
            ea = cudaFuncSetAttribute(k_real64<true, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kReal64SmemMax);
        if (ea == cudaSuccess)
            ea = cudaFuncSetAttribute(k_real64<false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kReal64SmemMax);
        const int rca = cuda_check(ctx, ea, "real-space shared memory attribute");
        if (rca) return rca;
    }

    // piecewise erfc table of the FP64 real-space kernel (computed once per process;
    // the host copy lives until exit, so the upload needs no synchronisation)
    {
        static std::once_flag once;
        static std::vector<double> tab;
        std::call_once(once, [] { tab = erfc_table(); });
        rc = dev_alloc(ctx, (void **)&ctx->erfc_tab64, sizeof(double) * tab.size());
        if (rc) return rc;
        e = cudaMemcpyAsync(ctx->erfc_tab64, tab.data(), sizeof(double) * tab.size(),
                            cudaMemcpyHostToDevice, ctx->alloc_stream);
        rc = cuda_check(ctx, e, "erfc table upload");
        if (rc) return rc;
    }

    // pair-function tables of the FP64 real-space kernel: F_alpha, G_alpha of
    // r^2 < r_c^2, and F_1, G_1 of r^2 / gamma^2 below the Gaussian-correction bound
    if (!ctx->fp32) {
        struct {
            double **dev;
            int *pieces;
        } tabs[2] = {{&ctx->fg_tab64, &ctx->fg_pieces}, {&ctx->gc_tab64, &ctx->gc_pieces}};
        for (int which = 0; which < 2; ++which) {
            auto &t = tabs[which];
            const PwShape *sh = nullptr;
            int valid = 0;
            const std::vector<double> &tab = pw_context_table(which, p.alpha, p.r_cut * p.r_cut, &sh, &valid);
            *t.pieces = valid;
            if (valid == 0) continue;
            rc = dev_alloc(ctx, (void **)t.dev, sizeof(double) * tab.size());
            if (rc) return rc;
            e = cudaMemcpyAsync(*t.dev, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice,
                                ctx->alloc_stream);
            rc = cuda_check(ctx, e, "pair-function table upload");
            if (rc) return rc;
        }
    }

    // cuFFT plans (from the plan pool) with a work area from this library's
    // allocator (no allocation inside cuFFT)
    size_t ws1 = 0, ws2 = 0;
    const cufftType t1 = ctx->fp32 ? CUFFT_R2C : CUFFT_D2Z, t2 = ctx->fp32 ? CUFFT_C2R : CUFFT_Z2D;
    cufftResult cr = plan_acquire(ctx->device, ctx->K, t1, &ctx->plan_r2c, &ws1);
    if (cr != CUFFT_SUCCESS) return set_error(ctx, QEQ_ERR_CUFFT, "cuFFT plan failed (%d)", (int)cr);
    cr = plan_acquire(ctx->device, ctx->K, t2, &ctx->plan_c2r, &ws2);
    if (cr != CUFFT_SUCCESS) {
        plan_release(ctx->device, ctx->K, t1, ctx->plan_r2c, ws1);
        return set_error(ctx, QEQ_ERR_CUFFT, "cuFFT plan failed (%d)", (int)cr);
    }
    ctx->have_plans = true;
    ctx->plan_ws[0] = ws1;
    ctx->plan_ws[1] = ws2;
    rc = dev_alloc(ctx, &ctx->fft_work, ws1 > ws2 ? ws1 : ws2);
    if (rc) return rc;
    cr = cufftSetWorkArea(ctx->plan_r2c, ctx->fft_work);
    if (cr == CUFFT_SUCCESS) cr = cufftSetWorkArea(ctx->plan_c2r, ctx->fft_work);
    if (cr != CUFFT_SUCCESS) return set_error(ctx, QEQ_ERR_CUFFT, "cufftSetWorkArea failed (%d)", (int)cr);
    return QEQ_OK;
}

// cuFFT plan pool.  Planning a 3D FFT costs milliseconds, which dominated the
// creation of short-lived contexts (the serving loop creates one per request).
// A destroyed context returns its plans here instead of destroying them, and a
// new context with the same device, mesh and transform takes them back.  A
// plan is held by one context at a time; its stream and work area are set by
// the holder.  At most kMaxPooledPlans idle plans are kept per key.
namespace {
struct PlanKey {
    int dev, K0, K1, K2, type;
    bool operator<(const PlanKey &o) const {
        return std::tie(dev, K0, K1, K2, type) < std::tie(o.dev, o.K0, o.K1, o.K2, o.type);
    }
};
constexpr size_t kMaxPooledPlans = 32;
std::mutex g_plan_mutex;
std::map<PlanKey, std::vector<std::pair<cufftHandle, size_t>>> g_plan_pool;
}  // namespace

cufftResult plan_acquire(int dev, const int K[3], cufftType type, cufftHandle *out, size_t *ws) {
    const PlanKey key{dev, K[0], K[1], K[2], (int)type};
    {
        std::lock_guard<std::mutex> lock(g_plan_mutex);
        auto it = g_plan_pool.find(key);
        if (it != g_plan_pool.end() && !it->second.empty()) {
            *out = it->second.back().first;
            *ws = it->second.back().second;
            it->second.pop_back();
            return CUFFT_SUCCESS;
        }
    }
    cufftHandle h = 0;
    cufftResult cr = cufftCreate(&h);
    if (cr != CUFFT_SUCCESS) return cr;
    cr = cufftSetAutoAllocation(h, 0);
    if (cr == CUFFT_SUCCESS) cr = cufftMakePlan3d(h, K[0], K[1], K[2], type, ws);
    if (cr != CUFFT_SUCCESS) {
        cufftDestroy(h);
        return cr;
    }
    *out = h;
    return CUFFT_SUCCESS;
}

void plan_release(int dev, const int K[3], cufftType type, cufftHandle h, size_t ws) {
    const PlanKey key{dev, K[0], K[1], K[2], (int)type};
    std::lock_guard<std::mutex> lock(g_plan_mutex);
    auto &v = g_plan_pool[key];
    if (v.size() < kMaxPooledPlans) {
        v.emplace_back(h, ws);
        return;
    }
    cufftDestroy(h);
}

int real_tile_reserve(qeq_ctx *ctx) {
    const RealLaunch L = real_launch(ctx, !ctx->fp32);
    if (!L.gtile) return QEQ_OK;
    const size_t need = (size_t)ctx->geom.nbricks * L.cap * (ctx->fp32 ? kTile32Bytes : kTile64Bytes);
    if (need <= ctx->tile_scratch_bytes) return QEQ_OK;
    dev_free(ctx, ctx->tile_scratch);
    ctx->tile_scratch = nullptr;
    ctx->tile_scratch_bytes = 0;
    const int rc = dev_alloc(ctx, (void **)&ctx->tile_scratch, need);
    if (rc) return rc;
    ctx->tile_scratch_bytes = need;
    return QEQ_OK;
}

void coulomb_free(qeq_ctx *ctx) {
    if (ctx->have_plans) {
        plan_release(ctx->device, ctx->K, ctx->fp32 ? CUFFT_R2C : CUFFT_D2Z, ctx->plan_r2c,
                     ctx->plan_ws[0]);
        plan_release(ctx->device, ctx->K, ctx->fp32 ? CUFFT_C2R : CUFFT_Z2D, ctx->plan_c2r,
                     ctx->plan_ws[1]);
    }
    void *ptrs[] = {ctx->v_s,  ctx->E_s,  ctx->sbase, ctx->sfrac, ctx->xq32, ctx->xq64,
                    ctx->sg32, ctx->sg64, ctx->mesh,  ctx->meshc, ctx->G,    ctx->part,
                    ctx->scal, ctx->energy4, ctx->fft_work, ctx->erfc_tab64, ctx->fg_tab64, ctx->gc_tab64, ctx->xf_pre, ctx->tile_scratch,
                    ctx->ticket};
    for (void *p : ptrs) dev_free(ctx, p);
    if (ctx->pme_stream) side_release(ctx->device, ctx->pme_stream, ctx->pme_fork, ctx->pme_join);
    ctx->pme_fork = ctx->pme_join = nullptr;
    ctx->pme_stream = nullptr;
    ewald_free(ctx);
    delete[] ctx->h_scal;
}

int erfc32_selftest(const float *x, float *out, int64_t n, cudaStream_t s) {
    k_erfc32<<<grid_for(n), kThreads, 0, s>>>(n, x, out);
    return cudaGetLastError() == cudaSuccess ? QEQ_OK : QEQ_ERR_CUDA;
}

int erfc64_selftest(qeq_ctx *ctx, const double *x, double *out, double *dout, int64_t n,
                    cudaStream_t s) {
    k_erfc64<<<grid_for(n), kThreads, 0, s>>>(n, ctx->erfc_tab64, x, out, dout);
    return cuda_check(ctx, cudaGetLastError(), "erfc64 selftest");
}

int pair_table_eval_host(int which, double alpha, double smax, int64_t n, const double *arg,
                         double *F, double *G, int32_t *in, int32_t *kept) {
    const PwShape *sh = nullptr;
    int valid = 0;
    const std::vector<double> &tab = pw_context_table(which, alpha, smax, &sh, &valid);
    *kept = valid;
    for (int64_t k = 0; k < n; ++k) {
        double f, g;
        const bool ok = pw_eval_host(*sh, tab.data(), valid, arg[k], f, g);
        in[k] = ok ? 1 : 0;
        if (ok) {
            F[k] = f;
            G[k] = g;
        }
    }
    return QEQ_OK;
}

int pair64_selftest(qeq_ctx *ctx, int which, const double *arg, double *F, double *G, int32_t *in,
                    int64_t n, cudaStream_t s) {
    if (ctx->fp32) return set_error(ctx, QEQ_ERR_INVALID, "no FP64 pair tables in FP32-mixed mode");
    const double2 *tab = (const double2 *)(which == 0 ? ctx->fg_tab64 : ctx->gc_tab64);
    const unsigned np = (unsigned)(which == 0 ? ctx->fg_pieces : ctx->gc_pieces);
    k_pair64_selftest<<<grid_for(n), kThreads, 0, s>>>(n, which, tab, np, arg, F, G, in);
    return cuda_check(ctx, cudaGetLastError(), "pair table selftest");
}

int coulomb_apply_impl(qeq_ctx *ctx, const double *R, const double *q, const double *sigma,
                       double *v, double *E, double *F, double *energy4, bool need_field,
                       cudaStream_t s, bool same_R) {
    if (!ctx->list_valid) return set_error(ctx, QEQ_ERR_NOLIST, "coulomb_apply before neighbor_build");
    const bool q_only = same_R && ctx->gathered;
    if (ctx->fp32) return apply_t<float>(ctx, R, q, sigma, v, E, F, energy4, need_field, q_only, s);
    return apply_t<double>(ctx, R, q, sigma, v, E, F, energy4, need_field, q_only, s);
}

}  // namespace qeq
