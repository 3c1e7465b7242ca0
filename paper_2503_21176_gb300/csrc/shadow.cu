// Shadow XL-BOMD step for the charge-equilibration model (Sec. 3.5), FP64 on the GPU.
//
// evaluate(R, n):
//   v[n], E[n]    = apply(n)                              (one Coulomb apply)
//   lambda, q[n]  from Eq. diag_linear_qeq in closed form:
//                 lambda = -(Q_tot + sum (chi + v) / u) / sum 1 / u,
//                 q = -(chi + v + lambda) / u
//   f = q - n;    Phi f, E[f] = apply(f)                  (second apply)
//   F = q o E[n] + n o E[f] (+ short range)
//   Krylov:       w_1 = f / |f|, r_k = J w_k with
//                 J x = -(Phi x + mu) / u - x, mu = -(sum Phi x / u) / sum 1 / u;
//                 w_{k+1} = r_k Gram-Schmidt-orthonormalised against w_1..w_k
//                 (one potential-only apply per extra vector);
//                 O = R^T R, c = O^{-1} R^T f, Kf = W c
//   energies      shadow energy (Eq. qeq_energy at q[n]), lambda, sum q, |f|
// advance: velocity-Verlet half kick + drift, dissipative Verlet update of the
//   n history (constants of Niklasson et al., J. Chem. Phys. 130, 214109 (2009)),
//   neighbour rebuild when an atom moved more than skin / 2.
// finish: second half kick and kinetic energy.
// Every reduction writes one partial per block of a fixed grid, and a
// one-block finalize sums them in fixed order, so a step is deterministic apart
// from the floating-point atomics of the PME spread.
#include <cmath>

#include "internal.cuh"

namespace qeq {

namespace {

// scalar slots (ctx->scal)
constexpr int S_LAM = 32;   // S1 = sum (chi + v) / u, S2 = sum 1 / u
constexpr int S_CHG = 34;   // sum f^2, sum q chi, sum u q^2 / 2, sum q v, sum n v, sum q
constexpr int S_MU = 40;    // sum (Phi w) / u
constexpr int S_DOT = 41;   // Gram-Schmidt dot
constexpr int S_OM = 48;    // O (kMaxRank^2, row-major) then g = R^T f (kMaxRank)
constexpr int S_KE = 120;   // kinetic energy
constexpr int S_RES = 121;  // relative least-squares residual |R c - f| / |f| of the kernel update
constexpr int S_SHORT = 126;  // short-range energy: intramolecular, Lennard-Jones
// Scalars derived once by the last block of the reduction that produces them
// (an FP64 divide or square root in every thread would occupy GB300's 1/64-rate
// FP64 pipe for each of the grid's 77,824 threads).
constexpr int S_LAMV = 122;  // lambda = -(Q_tot + S1) / S2
constexpr int S_INVF = 123;  // 1 / |f|  (0 for f = 0)
constexpr int S_MUV = 124;   // mu = -sum (Phi w) / u / S2
constexpr int S_INVN = 125;  // 1 / |x| of the last normalising dot

// 1 / x for positive normal x without an FP64 divide: an FP32 reciprocal of x
// (truncated to float on the integer pipe) refined by two Newton-Raphson steps
// y <- y + y (1 - x y) in FP64.  Each step squares the relative error, so the
// seed's 2^-22 becomes about 2^-88: the result is within an ulp or so of 1 / x.
__device__ __forceinline__ double recip_nr(double x) {
    const float xf = f64_to_f32_trunc(x);
    float yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(xf));
    double y = f32_to_f64_exact(yf);
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

__global__ void k_lambda_part(int n, double q_tot, const double *__restrict__ chi,
                              const double *__restrict__ u, const double *__restrict__ v,
                              double *__restrict__ inv_u, double *__restrict__ part,
                              double *__restrict__ out, double *__restrict__ scal,
                              unsigned int *__restrict__ ticket) {
    pdl_begin();
    double s1 = 0.0, s2 = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double iu = recip_nr(u[i]);
        inv_u[i] = iu;
        s1 += (chi[i] + v[i]) * iu;
        s2 += iu;
    }
    double vals[2] = {s1, s2};
    block_sum<2>(vals);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = vals[0];
        part[kRedBlocks + blockIdx.x] = vals[1];
    }
    if (finalize_last_block<2>(part, out, ticket) && threadIdx.x == 0)
        scal[S_LAMV] = -(q_tot + out[0]) / out[1];
}

__global__ void k_charges(int n, double q_tot, const double *__restrict__ chi,
                          const double *__restrict__ u, const double *__restrict__ inv_u,
                          const double *__restrict__ v,
                          const double *__restrict__ nn, const double *__restrict__ scal,
                          double *__restrict__ q, double *__restrict__ f, double *__restrict__ part,
                          double *__restrict__ out, unsigned int *__restrict__ ticket) {
    pdl_begin();
    const double lam = scal[S_LAMV];
    double a[6] = {0, 0, 0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double qi = -(chi[i] + v[i] + lam) * inv_u[i];
        const double fi = qi - nn[i];
        q[i] = qi;
        f[i] = fi;
        a[0] += fi * fi;
        a[1] += qi * chi[i];
        a[2] += 0.5 * u[i] * qi * qi;
        a[3] += qi * v[i];
        a[4] += nn[i] * v[i];
        a[5] += qi;
    }
    block_sum<6>(a);
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) part[k * kRedBlocks + blockIdx.x] = a[k];
    if (finalize_last_block<6>(part, out, ticket) && threadIdx.x == 0) {
        const double nf = sqrt(out[0]);
        out[S_INVF - S_CHG] = nf > 0.0 ? 1.0 / nf : 0.0;
    }
}

// F = q E[n] + n E[f] (+ F_short); w_1 = f / |f|; Phi w_1 = Phi f / |f| (in place);
// partial sum of (Phi w_1) / u for mu.
__global__ void k_forces_w1(int n, const double *__restrict__ q, const double *__restrict__ nn,
                            const double *__restrict__ En, const double *__restrict__ Ef,
                            const double *__restrict__ Fs, const double *__restrict__ f,
                            const double *__restrict__ inv_u, const double *__restrict__ scal,
                            double *__restrict__ F, double *__restrict__ w1,
                            double *__restrict__ phi, double *__restrict__ part,
                            double *__restrict__ out, unsigned int *__restrict__ ticket) {
    pdl_begin();
    const double inv = scal[S_INVF];
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double Fi = q[i] * En[3 * (size_t)i + d] + nn[i] * Ef[3 * (size_t)i + d];
            if (Fs) Fi += Fs[3 * (size_t)i + d];
            F[3 * (size_t)i + d] = Fi;
        }
        w1[i] = f[i] * inv;
        const double pw = phi[i] * inv;
        phi[i] = pw;
        s += pw * inv_u[i];
    }
    double vals[1] = {s};
    block_sum<1>(vals);
    if (threadIdx.x == 0) part[blockIdx.x] = vals[0];
    if (finalize_last_block<1>(part, out, ticket) && threadIdx.x == 0)
        out[S_MUV - S_MU] = -out[0] / out[S_LAM + 1 - S_MU];
}

__global__ void k_mu_part(int n, const double *__restrict__ phi, const double *__restrict__ inv_u,
                          double *__restrict__ part, double *__restrict__ out,
                          unsigned int *__restrict__ ticket) {
    pdl_begin();
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        s += phi[i] * inv_u[i];
    double vals[1] = {s};
    block_sum<1>(vals);
    if (threadIdx.x == 0) part[blockIdx.x] = vals[0];
    if (finalize_last_block<1>(part, out, ticket) && threadIdx.x == 0)
        out[S_MUV - S_MU] = -out[0] / out[S_LAM + 1 - S_MU];
}

// r = J w = -(Phi w + mu) / u - w with mu = -(sum Phi w / u) / sum 1 / u.
// When wnext is given, also start the next basis vector: wnext = r and the
// partial of <w0, r>, the first modified Gram-Schmidt projection.
__global__ void k_jacobian(int n, const double *__restrict__ phi, const double *__restrict__ w,
                           const double *__restrict__ inv_u, const double *__restrict__ scal,
                           double *__restrict__ r, double *__restrict__ wnext,
                           const double *__restrict__ w0, double *__restrict__ part,
                           double *__restrict__ out, unsigned int *__restrict__ ticket) {
    pdl_begin();
    const double mu = scal[S_MUV];
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double ri = -(phi[i] + mu) * inv_u[i] - w[i];
        r[i] = ri;
        if (wnext) {
            wnext[i] = ri;
            s += w0[i] * ri;
        }
    }
    if (wnext) {
        double vals[1] = {s};
        block_sum<1>(vals);
        if (threadIdx.x == 0) part[blockIdx.x] = vals[0];
        finalize_last_block<1>(part, out, ticket);
    }
}

// x -= scal[S_DOT] * y, then partial of <z, x> (z may alias x for the norm)
__global__ void k_axpy_dot(int n, const double *__restrict__ scal, const double *__restrict__ y,
                           double *x, const double *z, bool norm, double *__restrict__ part,
                           double *__restrict__ out, unsigned int *__restrict__ ticket) {
    pdl_begin();
    const double a = scal[S_DOT];
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double xi = x[i] - a * y[i];
        x[i] = xi;
        s += z[i] * xi;
    }
    double vals[1] = {s};
    block_sum<1>(vals);
    if (threadIdx.x == 0) part[blockIdx.x] = vals[0];
    // norm: out is |x|^2, and the last block derives 1 / |x| for k_normalize
    if (finalize_last_block<1>(part, out, ticket) && norm && threadIdx.x == 0) {
        const double nv = sqrt(out[0]);
        out[S_INVN - S_DOT] = nv > 0.0 ? 1.0 / nv : 0.0;
    }
}

__global__ void k_normalize(int n, const double *__restrict__ scal, double *__restrict__ x) {
    pdl_begin();
    const double inv = scal[S_INVN];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x[i] *= inv;
}

// One block: sum the partials of O = R^T R and g = R^T f in fixed order, solve
// O c = g (m x m) by Gaussian elimination with partial pivoting (singular
// directions get c = 0), and write c, the residual estimate and the energies.
// The partials of other blocks of the same launch are read through L2 (ldcg).
__device__ __forceinline__ void normal_solve_block(int m, double q_tot, int applies,
                                                   const double *__restrict__ part, int nb,
                                                   double *__restrict__ scal,
                                                   double *__restrict__ energies) {
    __shared__ double sums[kMaxRank * (kMaxRank + 1) / 2 + kMaxRank];
    const int nO = m * (m + 1) / 2;
    // one warp per slot, lanes over the block partials in a fixed order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = warp; k < nO + m; k += nw) {
        double acc = 0.0;
        const double *p = part + (size_t)k * kRedBlocks;
        for (int b = lane; b < nb; b += 32) acc += __ldcg(p + b);
        acc = warp_sum(acc);
        if (lane == 0) sums[k] = acc;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double A[kMaxRank][kMaxRank + 1];
    int k = 0;
    for (int a = 0; a < m; ++a)
        for (int b = a; b < m; ++b) {
            A[a][b] = sums[k];
            A[b][a] = sums[k];
            ++k;
        }
    for (int a = 0; a < m; ++a) A[a][m] = sums[nO + a];
    double scale = 0.0;
    for (int a = 0; a < m; ++a) scale = fmax(scale, fabs(A[a][a]));
    const double tiny = scale * 1e-300;
    int piv_ok[kMaxRank];
    for (int c = 0; c < m; ++c) {
        int best = c;
        for (int r = c + 1; r < m; ++r)
            if (fabs(A[r][c]) > fabs(A[best][c])) best = r;
        if (best != c)
            for (int j = 0; j <= m; ++j) {
                const double t = A[c][j];
                A[c][j] = A[best][j];
                A[best][j] = t;
            }
        piv_ok[c] = fabs(A[c][c]) > tiny && A[c][c] != 0.0;
        if (!piv_ok[c]) continue;
        for (int r = c + 1; r < m; ++r) {
            const double fct = A[r][c] / A[c][c];
            for (int j = c; j <= m; ++j) A[r][j] -= fct * A[c][j];
        }
    }
    double x[kMaxRank];
    for (int c = m - 1; c >= 0; --c) {
        if (!piv_ok[c]) {
            x[c] = 0.0;
            continue;
        }
        double acc = A[c][m];
        for (int j = c + 1; j < m; ++j) acc -= A[c][j] * x[j];
        x[c] = acc / A[c][c];
    }
    for (int a = 0; a < m; ++a) scal[S_OM + kMaxRank * kMaxRank + a] = x[a];
    // |R c - f|^2 = |f|^2 - c . R^T f at the least-squares solution
    double cg = 0.0;
    for (int a = 0; a < m; ++a) cg += x[a] * sums[nO + a];
    const double f2 = scal[S_CHG];
    scal[S_RES] = f2 > 0.0 ? sqrt(fmax(f2 - cg, 0.0) / f2) : 0.0;
    const double lam = -(q_tot + scal[S_LAM]) / scal[S_LAM + 1];
    const double e_short = scal[S_SHORT] + scal[S_SHORT + 1];
    energies[1] = scal[S_CHG + 1] + scal[S_CHG + 2] + scal[S_CHG + 3] - 0.5 * scal[S_CHG + 4] + e_short;
    energies[3] = e_short;
    energies[4] = lam;
    energies[5] = scal[S_CHG + 5];
    energies[6] = sqrt(scal[S_CHG]);
    energies[7] = (double)applies;
}

// partials of O_ab = <R_a, R_b> (a <= b) and g_a = <R_a, f>; the rank M is a
// template parameter so that the accumulators stay in registers.
template <int M>
__global__ void k_normal_part(int n, const double *__restrict__ Rb, const double *__restrict__ f,
                              double *__restrict__ part, double q_tot, int applies,
                              double *__restrict__ scal, double *__restrict__ energies,
                              unsigned int *__restrict__ ticket) {
    pdl_begin();
    constexpr int nO = M * (M + 1) / 2;
    double acc[nO + M];
#pragma unroll
    for (int k = 0; k < nO + M; ++k) acc[k] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double r[M];
#pragma unroll
        for (int a = 0; a < M; ++a) r[a] = Rb[(size_t)a * n + i];
        const double fi = f[i];
        int k = 0;
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = a; b < M; ++b) acc[k++] += r[a] * r[b];
#pragma unroll
        for (int a = 0; a < M; ++a) acc[nO + a] += r[a] * fi;
    }
    block_sum<nO + M>(acc);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < nO + M; ++k) part[k * kRedBlocks + blockIdx.x] = acc[k];
    // the last block to arrive solves the normal equations
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    normal_solve_block(M, q_tot, applies, part, (int)gridDim.x, scal, energies);
    if (threadIdx.x == 0) *ticket = 0u;
}

void launch_normal_part(bool pdl, int grid, int m, int n, const double *Rb, const double *f,
                        double *part, double q_tot, int applies, double *scal, double *energies,
                        unsigned int *ticket, cudaStream_t s) {
#define QEQ_NP_ARGS n, Rb, f, part, q_tot, applies, scal, energies, ticket
    switch (m) {
        case 1: launch_pdl(pdl, k_normal_part<1>, grid, kThreads, 0, s, QEQ_NP_ARGS); break;
        case 2: launch_pdl(pdl, k_normal_part<2>, grid, kThreads, 0, s, QEQ_NP_ARGS); break;
        case 3: launch_pdl(pdl, k_normal_part<3>, grid, kThreads, 0, s, QEQ_NP_ARGS); break;
        case 4: launch_pdl(pdl, k_normal_part<4>, grid, kThreads, 0, s, QEQ_NP_ARGS); break;
        case 5: launch_pdl(pdl, k_normal_part<5>, grid, kThreads, 0, s, QEQ_NP_ARGS); break;
        case 6: launch_pdl(pdl, k_normal_part<6>, grid, kThreads, 0, s, QEQ_NP_ARGS); break;
        case 7: launch_pdl(pdl, k_normal_part<7>, grid, kThreads, 0, s, QEQ_NP_ARGS); break;
        default: launch_pdl(pdl, k_normal_part<8>, grid, kThreads, 0, s, QEQ_NP_ARGS); break;
    }
#undef QEQ_NP_ARGS
}


// partial of |R c - f|^2 for the current c (rank m): the least-squares residual of
// the kernel update, computed directly (the normal-equation identity
// |f|^2 - c.R^T f cancels catastrophically once the residual is small)
__global__ void k_ls_residual(int n, int m, const double *__restrict__ Rb,
                              const double *__restrict__ f, const double *__restrict__ scal,
                              double *__restrict__ part, double *__restrict__ out,
                              unsigned int *__restrict__ ticket) {
    pdl_begin();
    const double *c = scal + S_OM + kMaxRank * kMaxRank;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double r = -f[i];
        for (int a = 0; a < m; ++a) r += c[a] * Rb[(size_t)a * n + i];
        acc += r * r;
    }
    double vals[1] = {acc};
    block_sum<1>(vals);
    if (threadIdx.x == 0) part[blockIdx.x] = vals[0];
    finalize_last_block<1>(part, out, ticket);
}

struct Dissipation {
    double kappa, alpha;
    double c[kMaxHist];
    // the update's coefficients of n_{t-k} with 2 n_t - n_{t-1} folded in:
    // w_0 = 2 + alpha c_0, w_1 = alpha c_1 - 1, w_k = alpha c_k (k >= 2)
    double w[kMaxHist];
    int kd;
};

Dissipation dissipation(int kd) {
    // Niklasson et al., J. Chem. Phys. 130, 214109 (2009), Table I
    Dissipation d{};
    d.kd = kd;
    static const double c3[] = {-2, 3, 0, -1};
    static const double c4[] = {-3, 6, -2, -2, 1};
    static const double c5[] = {-6, 14, -8, -3, 4, -1};
    static const double c6[] = {-14, 36, -27, -2, 12, -6, 1};
    static const double c7[] = {-36, 99, -88, 11, 32, -25, 8, -1};
    const double *c = nullptr;
    switch (kd) {
        case 3: d.kappa = 1.69; d.alpha = 150e-3; c = c3; break;
        case 4: d.kappa = 1.75; d.alpha = 57e-3; c = c4; break;
        case 5: d.kappa = 1.82; d.alpha = 18e-3; c = c5; break;
        case 6: d.kappa = 1.84; d.alpha = 5.5e-3; c = c6; break;
        default: d.kappa = 1.86; d.alpha = 1.6e-3; c = c7; break;
    }
    for (int k = 0; k <= kd; ++k) {
        d.c[k] = c[k];
        d.w[k] = d.alpha * c[k] + (k == 0 ? 2.0 : (k == 1 ? -1.0 : 0.0));
    }
    return d;
}

// |x| as a float truncated toward zero (at most 2^-23 low) on the integer pipe,
// +inf from 2^100 up and for infinities and NaNs: the skin check's
// displacement components.
__device__ __forceinline__ float disp_f32(double x) {
    const int hi = __double2hiint(x) & 0x7fffffff;
    const unsigned lo = (unsigned)__double2loint(x);
    const int ex = (hi >> 20) - 1023 + 127;
    if (ex <= 0) return 0.0f;
    if (ex >= 227) return __int_as_float(0x7f800000);
    return __int_as_float((ex << 23) | ((hi & 0xFFFFF) << 3) | (int)(lo >> 29));
}

// Half kick + drift of R; n_{t+1} = 2 n_t - n_{t-1} - kappa Kf + alpha sum_k c_k n_{t-k}
// (with the folded coefficients w); history shifted in place (each thread owns
// one atom's column).  half_kick = dt / (2 m) is written for the finish.  The
// same pass finds the largest squared displacement since the last neighbour
// build (the skin check) into *max_d2: the FP64 differences truncated to FP32 and
// the FP32 sum scaled by 1 + 2^-20, so it is never below the exact value and a
// rebuild is never late (GB300 runs FP64 at 1/64 of the FP32 rate).
__global__ void k_advance(int n, double dt, double half_dt, double mass_unit, Dissipation dis,
                          const double *__restrict__ mass, const double *__restrict__ F,
                          const double *__restrict__ Kf, double *__restrict__ R,
                          double *__restrict__ V, double *__restrict__ hist,
                          double *__restrict__ half_kick, const double *__restrict__ R0,
                          double *__restrict__ part, double *__restrict__ max_d2,
                          unsigned int *__restrict__ ticket) {
    pdl_begin();
    float mx = 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double hk = half_dt * recip_nr(mass[i] * mass_unit);
        half_kick[i] = hk;
        float d2 = 0.0f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double vi = fma(F[3 * (size_t)i + d], hk, V[3 * (size_t)i + d]);
            V[3 * (size_t)i + d] = vi;
            const double r = fma(dt, vi, R[3 * (size_t)i + d]);
            R[3 * (size_t)i + d] = r;
            const float dd = disp_f32(r - R0[3 * (size_t)i + d]);
            d2 = fmaf(dd, dd, d2);
        }
        mx = fmaxf(mx, d2 * (1.0f + 0x1p-20f));
        double h[kMaxHist];
        for (int k = 0; k <= dis.kd; ++k) h[k] = hist[(size_t)k * n + i];
        double nn = -dis.kappa * Kf[i];
        for (int k = 0; k <= dis.kd; ++k) nn = fma(dis.w[k], h[k], nn);
        for (int k = dis.kd; k >= 1; --k) hist[(size_t)k * n + i] = h[k - 1];
        hist[i] = nn;
    }
    max_last_block(f32_to_f64_exact(mx), part, max_d2, ticket);
}

// optional second half kick, then partial of the kinetic energy; with kf_rank > 0
// also the kernel update Kf = W c of the evaluation (c from the normal equations)
__global__ void k_finish(int n, double half_mass_unit, bool kick,
                         const double *__restrict__ mass, const double *__restrict__ half_kick,
                         const double *__restrict__ F, double *__restrict__ V, int kf_rank,
                         const double *__restrict__ Wb, double *__restrict__ Kf,
                         double *__restrict__ part, double *__restrict__ scal,
                         double *__restrict__ energies, unsigned int *__restrict__ ticket) {
    pdl_begin();
    const double *c = scal + S_OM + kMaxRank * kMaxRank;
    double ke = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (kf_rank > 0) {
            double kfi = 0.0;
            for (int a = 0; a < kf_rank; ++a) kfi += c[a] * Wb[(size_t)a * n + i];
            Kf[i] = kfi;
        }
        double v2 = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double vi = V[3 * (size_t)i + d];
            if (kick) {
                vi = fma(F[3 * (size_t)i + d], half_kick[i], vi);
                V[3 * (size_t)i + d] = vi;
            }
            v2 = fma(vi, vi, v2);
        }
        ke = fma(half_mass_unit * mass[i], v2, ke);
    }
    double vals[1] = {ke};
    block_sum<1>(vals);
    if (threadIdx.x == 0) part[blockIdx.x] = vals[0];
    // the last block also writes the kinetic and total energies
    if (finalize_last_block<1>(part, scal + S_KE, ticket) && threadIdx.x == 0) {
        energies[0] = scal[S_KE];
        energies[2] = scal[S_KE] + energies[1];
    }
}

}  // namespace

int shadow_alloc(qeq_ctx *ctx) {
    const int64_t n = ctx->n;
    const int m = ctx->p.krylov_rank;
    struct {
        void **ptr;
        size_t bytes;
    } bufs[] = {
        {(void **)&ctx->v_n, sizeof(double) * n},
        {(void **)&ctx->E_n, sizeof(double) * 3 * n},
        {(void **)&ctx->phi, sizeof(double) * n},
        {(void **)&ctx->E_f, sizeof(double) * 3 * n},
        {(void **)&ctx->fvec, sizeof(double) * n},
        {(void **)&ctx->Wb, sizeof(double) * (size_t)m * n},
        {(void **)&ctx->Rb, sizeof(double) * (size_t)m * n},
        {(void **)&ctx->inv_u, sizeof(double) * n},
        {(void **)&ctx->half_kick, sizeof(double) * n},
    };
    for (auto &b : bufs) {
        int rc = dev_alloc(ctx, b.ptr, b.bytes);
        if (rc) return rc;
    }
    // every context holds the short-range force buffer, so that registering a user
    // model later (qeq_set_short_range) never allocates or orders a new buffer
    int rc = dev_alloc(ctx, (void **)&ctx->F_short, sizeof(double) * 3 * n);
    if (rc) return rc;
    return QEQ_OK;
}

void shadow_free(qeq_ctx *ctx) {
    void *ptrs[] = {ctx->v_n, ctx->E_n, ctx->phi, ctx->E_f, ctx->fvec, ctx->Wb,
                    ctx->Rb,  ctx->F_short, ctx->inv_u, ctx->half_kick};
    for (void *p : ptrs) dev_free(ctx, p);
}

int short_range_forces(qeq_ctx *ctx, const double *R, const double *mass, double *F_short,
                       double *e_short_slot, cudaStream_t s);

int shadow_evaluate(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, cudaStream_t s) {
    const int n = (int)ctx->n;
    const int m = ctx->p.krylov_rank;
    const double *u = prm->eta;
    double *nn = st->n_hist;  // n(t) is history slot 0
    double *part = ctx->part;
    double *scal = ctx->scal;
    const int G = ctx->red_grid;
    unsigned int *tk = ctx->ticket;
    auto fin = [&]() { ctx->launches += 1; };  // a reducing kernel (its last block finalizes)

    // short-range stand-in (or zero)
    prof_begin(ctx, kPhShadow, s);
    {
        int rc = short_range_eval(ctx, st->R, prm->mass, scal + S_SHORT, s);
        if (rc) return rc;
    }
    prof_end(ctx, s);

    // 1. v[n], E[n]
    int rc = coulomb_apply_impl(ctx, st->R, nn, prm->sigma, ctx->v_n, ctx->E_n, nullptr, nullptr,
                                true, s);
    if (rc) return rc;
    // 2. lambda and q[n] (Eq. diag_linear_qeq); 1/u kept for the rest of the evaluation
    prof_begin(ctx, kPhShadow, s);
    launch_pdl(ctx->pdl, k_lambda_part, G, kThreads, 0, s, n, ctx->p.q_tot, prm->chi, u, ctx->v_n, ctx->inv_u,
               part, scal + S_LAM, scal, tk);
    fin();
    launch_pdl(ctx->pdl, k_charges, G, kThreads, 0, s, n, ctx->p.q_tot, prm->chi, u, ctx->inv_u, ctx->v_n, nn,
               scal, st->q, ctx->fvec, part, scal + S_CHG, tk);
    fin();
    prof_end(ctx, s);
    // 3. Phi f, E[f]
    rc = coulomb_apply_impl(ctx, st->R, ctx->fvec, prm->sigma, ctx->phi, ctx->E_f, nullptr, nullptr,
                            true, s, true);
    if (rc) return rc;
    // 4. forces, w_1, r_1 (and, when m > 1, the start of w_2)
    const bool adaptive = ctx->p.krylov_tol > 0.0;
    prof_begin(ctx, kPhShadow, s);
    launch_pdl(ctx->pdl, k_forces_w1, G, kThreads, 0, s, n, st->q, nn, ctx->E_n, ctx->E_f,
               has_short(ctx) ? ctx->F_short : nullptr, ctx->fvec, ctx->inv_u, scal, st->F, ctx->Wb,
               ctx->phi, part, scal + S_MU, tk);
    fin();
    launch_pdl(ctx->pdl, k_jacobian, G, kThreads, 0, s, n, ctx->phi, ctx->Wb, ctx->inv_u, scal, ctx->Rb,
               m > 1 ? ctx->Wb + (size_t)n : nullptr, ctx->Wb, part, scal + S_DOT, tk);
    ctx->launches++;
    prof_end(ctx, s);
    // normal equations, m x m solve and energies for rank k; with a tolerance, the
    // host reads the least-squares residual and stops adding vectors when it is met
    auto solve_rank = [&](int k, bool *done) -> int {
        const int nO = k * (k + 1) / 2;
        prof_begin(ctx, kPhShadow, s);
        launch_normal_part(ctx->pdl, ctx->red_grid, k, n, ctx->Rb, ctx->fvec, part, ctx->p.q_tot, k + 1, scal,
                           st->energies, tk, s);
        ctx->launches += 1;
        prof_end(ctx, s);
        (void)nO;
        *done = true;
        if (!adaptive || k == m) return QEQ_OK;
        launch_pdl(ctx->pdl, k_ls_residual, G, kThreads, 0, s, n, k, ctx->Rb, ctx->fvec, scal, part,
                   scal + S_RES, tk);
        fin();
        double hv[2] = {0.0, 0.0};  // |R c - f|^2 and |f|^2
        cudaError_t e = cudaMemcpyAsync(&hv[0], scal + S_RES, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&hv[1], scal + S_CHG, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        int rc2 = cuda_check(ctx, e, "krylov residual");
        if (rc2) return rc2;
        *done = !(hv[0] > ctx->p.krylov_tol * ctx->p.krylov_tol * hv[1]);
        return QEQ_OK;
    };
    int m_used = 1;
    bool done = !adaptive && m > 1 ? false : true;
    if (adaptive) {
        rc = solve_rank(1, &done);
        if (rc) return rc;
    }
    // 5. further Krylov vectors: w_k starts as r_{k-1} with <w_0, w_k> already reduced
    for (int k = 1; k < m && !(adaptive && done); ++k) {
        double *Wk = ctx->Wb + (size_t)k * n;
        prof_begin(ctx, kPhShadow, s);
        // modified Gram-Schmidt: Wk -= <w_j, Wk> w_j for j = 0..k-1, then normalise
        for (int j = 0; j < k; ++j) {
            const double *wj = ctx->Wb + (size_t)j * n;
            const double *znext = (j + 1 < k) ? ctx->Wb + (size_t)(j + 1) * n : Wk;
            launch_pdl(ctx->pdl, k_axpy_dot, G, kThreads, 0, s, n, scal, wj, Wk, znext, j + 1 == k, part,
                       scal + S_DOT, tk);
            fin();
        }
        launch_pdl(ctx->pdl, k_normalize, G, kThreads, 0, s, n, scal, Wk);
        ctx->launches++;
        prof_end(ctx, s);
        rc = coulomb_apply_impl(ctx, st->R, Wk, prm->sigma, ctx->phi, nullptr, nullptr, nullptr,
                                false, s, true);
        if (rc) return rc;
        prof_begin(ctx, kPhShadow, s);
        launch_pdl(ctx->pdl, k_mu_part, G, kThreads, 0, s, n, ctx->phi, ctx->inv_u, part, scal + S_MU, tk);
        fin();
        const bool more = k + 1 < m;
        launch_pdl(ctx->pdl, k_jacobian, G, kThreads, 0, s, n, ctx->phi, Wk, ctx->inv_u, scal,
                   ctx->Rb + (size_t)k * n, more ? ctx->Wb + (size_t)(k + 1) * n : nullptr, ctx->Wb,
                   part, scal + S_DOT, tk);
        ctx->launches++;
        prof_end(ctx, s);
        m_used = k + 1;
        if (adaptive) {
            rc = solve_rank(m_used, &done);
            if (rc) return rc;
        }
    }
    if (!adaptive) {
        m_used = m;
        rc = solve_rank(m, &done);
        if (rc) return rc;
    }
    // 6. Kf = W c is formed by the finish kernel that follows every evaluation
    ctx->kf_rank = m_used;
    return cuda_check(ctx, cudaGetLastError(), "shadow evaluate launch");
}

int shadow_advance_queue(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, cudaStream_t s) {
    const int n = (int)ctx->n;
    prof_begin(ctx, kPhIntegrate, s);
    launch_pdl(ctx->pdl, k_advance, ctx->red_grid, kThreads, 0, s, n, ctx->p.dt, 0.5 * ctx->p.dt,
               ctx->p.mass_unit, dissipation(ctx->p.dissipation_k), prm->mass, st->F, st->Kf, st->R,
               st->V, st->n_hist, ctx->half_kick, ctx->R_build, ctx->part, ctx->scal + kScMaxDisp2,
               ctx->ticket);
    prof_end(ctx, s);
    ctx->launches++;
    return cuda_check(ctx, cudaGetLastError(), "advance launch");
}

int shadow_advance(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, cudaStream_t s) {
    int rc = shadow_advance_queue(ctx, prm, st, s);
    if (rc) return rc;
    cudaMemcpyAsync(ctx->h_scal + kScMaxDisp2, ctx->scal + kScMaxDisp2, sizeof(double),
                    cudaMemcpyDeviceToHost, s);
    rc = cuda_check(ctx, cudaStreamSynchronize(s), "displacement check");
    if (rc) return rc;
    const double d2 = ctx->h_scal[kScMaxDisp2];
    const double half = 0.5 * ctx->p.skin;
    if (!(d2 <= half * half)) {
        rc = nl_build(ctx, st->R, s);
        if (rc) return rc;
    }
    return QEQ_OK;
}

int shadow_finish(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, bool kick,
                  cudaStream_t s, bool kf) {
    const int n = (int)ctx->n;
    prof_begin(ctx, kPhIntegrate, s);
    const int rank = kf && st->Kf ? ctx->kf_rank : 0;
    launch_pdl(ctx->pdl, k_finish, ctx->red_grid, kThreads, 0, s, n, 0.5 * ctx->p.mass_unit, kick, prm->mass,
               ctx->half_kick, st->F, st->V, rank, ctx->Wb, st->Kf, ctx->part, ctx->scal,
               st->energies, ctx->ticket);
    prof_end(ctx, s);
    ctx->launches += 1;
    return cuda_check(ctx, cudaGetLastError(), "shadow finish launch");
}

}  // namespace qeq
