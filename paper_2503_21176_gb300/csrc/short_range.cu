// Built-in short-range stand-in V_short (QEQ_SHORT_WATER), FP64.
//
// The paper's V_short is a trained HIP-NN model (Sec. 4).  It is replaced here
// by plain flexible-water terms, with atoms ordered O, H, H per molecule:
//   1/2 k_b (|r_OH| - r_0)^2 per O-H bond, 1/2 k_theta (theta - theta_0)^2 per
//   molecule, 4 eps [(s / r)^12 - (s / r)^6] per O-O pair inside r_cut.
// r_0 = 0.9572 A and theta_0 = 104.52 deg are the workload geometry.  k_b,
// k_theta, eps and s are the SPC/Fw values (Wu, Tepper & Voth, J. Chem. Phys.
// 124, 024503 (2006)) converted from kcal/mol to eV.
// Intramolecular terms: one thread per molecule (minimum image).  Lennard-Jones:
// one thread per sorted O atom over its ELLPACK row (both directions of a pair
// are visited, so the energy takes 1/2), with the current positions and the
// images of the list.
#include "internal.cuh"

namespace qeq {

namespace {

constexpr double kKcal = 0.0433641;
constexpr double kKBond = 1059.162 * kKcal;
constexpr double kR0 = 0.9572;
constexpr double kKAngle = 75.90 * kKcal;
constexpr double kTheta0 = 104.52 * kPi / 180.0;
constexpr double kLjEps = 0.1554 * kKcal;
constexpr double kLjSigma = 3.165492;

__device__ __forceinline__ double min_image(double d, double L) { return d - L * rint(d / L); }

__global__ void k_water_intra(int n_mol, const double *__restrict__ R, double Lx, double Ly,
                              double Lz, double *__restrict__ F, double *__restrict__ part) {
    double e = 0.0;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n_mol; m += gridDim.x * blockDim.x) {
        const double *o = R + 9 * (size_t)m;
        double a[3], b[3];
        const double L[3] = {Lx, Ly, Lz};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            a[d] = min_image(o[3 + d] - o[d], L[d]);
            b[d] = min_image(o[6 + d] - o[d], L[d]);
        }
        const double ra = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        const double rb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
        e += 0.5 * kKBond * ((ra - kR0) * (ra - kR0) + (rb - kR0) * (rb - kR0));
        double cos_t = (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) / (ra * rb);
        cos_t = fmin(1.0, fmax(-1.0, cos_t));
        const double theta = acos(cos_t);
        e += 0.5 * kKAngle * (theta - kTheta0) * (theta - kTheta0);
        const double sin_t = sqrt(fmax(1.0 - cos_t * cos_t, 1e-300));
        const double pref = kKAngle * (theta - kTheta0) / sin_t;
        double fh1[3], fh2[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double fa = -kKBond * (ra - kR0) * a[d] / ra;
            const double fb = -kKBond * (rb - kR0) * b[d] / rb;
            const double ga = pref * (b[d] / (ra * rb) - cos_t * a[d] / (ra * ra));
            const double gb = pref * (a[d] / (ra * rb) - cos_t * b[d] / (rb * rb));
            fh1[d] = fa + ga;
            fh2[d] = fb + gb;
        }
        double *f = F + 9 * (size_t)m;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            f[d] = -(fh1[d] + fh2[d]);
            f[3 + d] = fh1[d];
            f[6 + d] = fh2[d];
        }
    }
    double vals[1] = {e};
    block_sum<1>(vals);
    if (threadIdx.x == 0) part[blockIdx.x] = vals[0];
}

// O-O Lennard-Jones over the list, one block per brick: sorted atom i is an O
// when perm[i] % 3 == 0; an entry e of row i is decoded through the brick's tile
// table into the sorted atom j and its image shift.
__global__ void __launch_bounds__(kThreads)
k_water_lj(int n, BrickGeom g, const int32_t *__restrict__ cell_start,
           const int32_t *__restrict__ perm, const uint16_t *__restrict__ nbr,
           const int32_t *__restrict__ cnt, const double *__restrict__ R,
           const double *__restrict__ wrap_off, double Lx, double Ly, double Lz, double rc2,
           double *__restrict__ F, double *__restrict__ part) {
    __shared__ int t_start[kMaxTileBricks], t_base[kMaxTileBricks], t_code[kMaxTileBricks], t_total;
    double e = 0.0;
    const double s6 = kLjSigma * kLjSigma * kLjSigma * kLjSigma * kLjSigma * kLjSigma;
    for (int64_t b = blockIdx.x; b < g.nbricks; b += gridDim.x) {
        __syncthreads();
        if (threadIdx.x < 32) tile_table(g, b, cell_start, t_start, t_base, t_code, &t_total);
        __syncthreads();
        const int i0 = t_start[g.center], i1 = cell_start[(b + 1) * g.bvol];
        for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const int ai = perm[i];
            if (ai % 3 != 0) continue;
            const double xi = R[3 * (size_t)ai] + wrap_off[3 * (size_t)ai];
            const double yi = R[3 * (size_t)ai + 1] + wrap_off[3 * (size_t)ai + 1];
            const double zi = R[3 * (size_t)ai + 2] + wrap_off[3 * (size_t)ai + 2];
            double fx = 0.0, fy = 0.0, fz = 0.0;
            const int c = cnt[i];
            for (int k = 0; k < c; ++k) {
                const int en = nbr[list_index(k, i, n)];
                const int rb = tile_locate(en, g.T, t_start, t_base);
                const int aj = perm[en - t_base[rb]];
                if (aj % 3 != 0) continue;
                const int code = t_code[rb];
                const double dx = (R[3 * (size_t)aj] + wrap_off[3 * (size_t)aj] - xi) + (code / 25 - 2) * Lx;
                const double dy = (R[3 * (size_t)aj + 1] + wrap_off[3 * (size_t)aj + 1] - yi) +
                                  ((code / 5) % 5 - 2) * Ly;
                const double dz = (R[3 * (size_t)aj + 2] + wrap_off[3 * (size_t)aj + 2] - zi) +
                                  (code % 5 - 2) * Lz;
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < rc2)) continue;
                const double inv6 = s6 / (r2 * r2 * r2);
                e += 0.5 * 4.0 * kLjEps * (inv6 * inv6 - inv6);
                const double gg = 4.0 * kLjEps * (-12.0 * inv6 * inv6 + 6.0 * inv6) / r2;
                fx += gg * dx;
                fy += gg * dy;
                fz += gg * dz;
            }
            F[3 * (size_t)ai] += fx;
            F[3 * (size_t)ai + 1] += fy;
            F[3 * (size_t)ai + 2] += fz;
        }
    }
    double vals[1] = {e};
    block_sum<1>(vals);
    if (threadIdx.x == 0) part[kRedBlocks + blockIdx.x] = vals[0];
}

}  // namespace

// F_short (device [N][3]) and its energy into e_slot[0..1] (device: intramolecular,
// Lennard-Jones), all on stream s.
int short_range_forces(qeq_ctx *ctx, const double *R, const double *, double *F_short,
                       double *e_slot, cudaStream_t s) {
    const int n = (int)ctx->n;
    const qeq_params &p = ctx->p;
    k_water_intra<<<ctx->red_grid, kThreads, 0, s>>>(n / 3, R, p.box[0], p.box[1], p.box[2], F_short,
                                                  ctx->part);
    k_water_lj<<<ctx->red_grid, kThreads, 0, s>>>(n, ctx->geom, ctx->cell_start, ctx->perm, ctx->nbr,
                                               ctx->cnt, R, ctx->wrap_off, p.box[0], p.box[1],
                                               p.box[2], p.r_cut * p.r_cut, F_short, ctx->part);
    launch_finalize(ctx, ctx->part, 2, e_slot, s);
    ctx->launches += 3;
    return cuda_check(ctx, cudaGetLastError(), "short-range launch");
}

int short_range_eval(qeq_ctx *ctx, const double *R, const double *mass, double *e_slot,
                     cudaStream_t s) {
    if (ctx->short_fn) {
        cudaMemsetAsync(e_slot, 0, 2 * sizeof(double), s);
        const int rc = ctx->short_fn(ctx->short_user, ctx->n, R, ctx->F_short, e_slot, (void *)s);
        if (rc) return set_error(ctx, QEQ_ERR_INVALID, "short-range callback returned %d", rc);
        return cuda_check(ctx, cudaGetLastError(), "short-range callback");
    }
    if (ctx->p.short_range == QEQ_SHORT_WATER)
        return short_range_forces(ctx, R, mass, ctx->F_short, e_slot, s);
    cudaMemsetAsync(e_slot, 0, 2 * sizeof(double), s);
    return QEQ_OK;
}


}  // namespace qeq
