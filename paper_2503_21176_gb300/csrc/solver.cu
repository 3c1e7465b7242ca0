// Regular QEq by GMRES and regular Born-Oppenheimer MD (Sec. 3.4, Sec. 4.1).
//
// The bordered system of Eq. linear_qeq,
//     [diag(u) + Phi   1] [q     ]   [-chi ]
//     [1^T             0] [lambda] = [Q_tot],
// is solved by restarted GMRES with a right Jacobi preconditioner
// M = diag(u_i + g_i, 1), where g_i = k_e sqrt(2/pi) / sigma_i is the Gaussian
// self-energy when that term is on (the dominant part of Phi_ii), else 0.
// Right preconditioning keeps the monitored residual the true one,
// ||b - A z|| / ||b||.  That is the paper's tolerance.  Each Arnoldi vector
// costs one potential-only Coulomb apply.  Vectors have N + 1 entries, the
// last one being lambda.  Orthogonalisation is classical Gram-Schmidt done
// twice, each pass one multi-dot kernel plus one update kernel.  The
// (m + 1) x m Hessenberg least-squares problem is reduced by Givens rotations
// on the host from one small device-to-host copy per iteration.
//
// The regular BO-MD step: velocity-Verlet half kick and drift, a neighbour
// rebuild when due, a solve warm-started from the previous charges, one apply
// with the field for F = q o E (+ short range), and the second half kick.  The
// potential energy is sum q chi + 1/2 sum u q^2 + 1/2 q.Phi q (+ short range)
// at the approximate charges.
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace qeq {

namespace {

constexpr int kMaxDots = kMaxGmresRestart;  // Gram-Schmidt against at most this many vectors

// y = A x for x = [xq; xl]:  y_q = u o xq + Phi xq + xl,  y_l = sum xq.
// phi holds Phi xq.  The partial of sum xq goes to part slot 0.
__global__ void k_bordered_apply(int n, const double *__restrict__ u, const double *__restrict__ phi,
                                 const double *__restrict__ x, double *__restrict__ y,
                                 double *__restrict__ part) {
    const double xl = x[n];
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        y[i] = u[i] * x[i] + phi[i] + xl;
        s += x[i];
    }
    double vals[1] = {s};
    block_sum<1>(vals);
    if (threadIdx.x == 0) part[blockIdx.x] = vals[0];
}

// last entry of y from the finalized sum
__global__ void k_set_last(int n, const double *__restrict__ src, double *__restrict__ y) {
    if (threadIdx.x == 0 && blockIdx.x == 0) y[n] = src[0];
}

// z = M^{-1} x (q part divided by d, lambda unchanged)
__global__ void k_precond(int n, const double *__restrict__ dinv, const double *__restrict__ x,
                          double *__restrict__ z) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x)
        z[i] = i < n ? x[i] * dinv[i] : x[i];
}

// partials of <V_k, w> for k < nv over n + 1 entries (slot k), and of <w, w> (slot nv)
__global__ void k_multi_dot(int n1, int nv, const double *__restrict__ V, const double *__restrict__ w,
                            double *__restrict__ part) {
    for (int k = 0; k <= nv; ++k) {
        const double *a = k < nv ? V + (size_t)k * n1 : w;
        double s = 0.0;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += gridDim.x * blockDim.x)
            s += a[i] * w[i];
        double vals[1] = {s};
        block_sum<1>(vals);
        if (threadIdx.x == 0) part[(size_t)k * kRedBlocks + blockIdx.x] = vals[0];
    }
}

// w -= sum_k h_k V_k
__global__ void k_subtract(int n1, int nv, const double *__restrict__ V, const double *__restrict__ h,
                           double *__restrict__ w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += gridDim.x * blockDim.x) {
        double s = w[i];
        for (int k = 0; k < nv; ++k) s -= h[k] * V[(size_t)k * n1 + i];
        w[i] = s;
    }
}

// y = a * x   (n1 entries)
__global__ void k_scale(int n1, double a, const double *__restrict__ x, double *__restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += gridDim.x * blockDim.x)
        y[i] = a * x[i];
}

// r = b - Az with b = [-chi; q_tot]
__global__ void k_residual(int n, double q_tot, const double *__restrict__ chi,
                           const double *__restrict__ Az, double *__restrict__ r) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x)
        r[i] = (i < n ? -chi[i] : q_tot) - Az[i];
}

// z += M^{-1} (sum_k y_k V_k)
__global__ void k_update_solution(int n, int nv, const double *__restrict__ V,
                                  const double *__restrict__ y, const double *__restrict__ dinv,
                                  double *__restrict__ z) {
    const int n1 = n + 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nv; ++k) s += y[k] * V[(size_t)k * n1 + i];
        z[i] += i < n ? s * dinv[i] : s;
    }
}

__global__ void k_jacobi(int n, const double *__restrict__ u, const double *__restrict__ sigma,
                         double gauss_coef, double *__restrict__ dinv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d = u[i];
        if (gauss_coef != 0.0 && sigma[i] > 0.0) d += gauss_coef / sigma[i];
        dinv[i] = 1.0 / d;
    }
}

// q part of z into q, and the energy partials: sum q chi, sum u q^2 / 2, sum q v / 2, sum q
__global__ void k_bo_energy_part(int n, const double *__restrict__ q, const double *__restrict__ chi,
                                 const double *__restrict__ u, const double *__restrict__ v,
                                 double *__restrict__ part) {
    double a[4] = {0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        a[0] += q[i] * chi[i];
        a[1] += 0.5 * u[i] * q[i] * q[i];
        a[2] += 0.5 * q[i] * v[i];
        a[3] += q[i];
    }
    block_sum<4>(a);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) part[(size_t)k * kRedBlocks + blockIdx.x] = a[k];
}

__global__ void k_bo_forces(int n, const double *__restrict__ q, const double *__restrict__ E,
                            const double *__restrict__ Fs, double *__restrict__ F) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double f = q[i] * E[3 * (size_t)i + d];
            if (Fs) f += Fs[3 * (size_t)i + d];
            F[3 * (size_t)i + d] = f;
        }
}

// energies: 1 potential (BO energy + short), 3 short, 4 lambda, 5 sum q, 6 rel residual, 7 applies
__global__ void k_bo_energies(const double *__restrict__ sums, const double *__restrict__ e_short2,
                              double lambda, double relres, double applies,
                              double *__restrict__ energies) {
    const double es = e_short2[0] + e_short2[1];
    energies[1] = sums[0] + sums[1] + sums[2] + es;
    energies[3] = es;
    energies[4] = lambda;
    energies[5] = sums[3];
    energies[6] = relres;
    energies[7] = applies;
}

}  // namespace

int short_range_forces(qeq_ctx *ctx, const double *R, const double *mass, double *F_short,
                       double *e_slot, cudaStream_t s);

int solver_alloc(qeq_ctx *ctx, int restart) {
    if (ctx->gm_restart >= restart && ctx->gmV) return QEQ_OK;
    dev_free(ctx, ctx->gmV);
    dev_free(ctx, ctx->gmW);
    dev_free(ctx, ctx->gmZ);
    dev_free(ctx, ctx->gmDinv);
    dev_free(ctx, ctx->gmH);
    ctx->gmV = ctx->gmW = ctx->gmZ = ctx->gmDinv = ctx->gmH = nullptr;
    const size_t n1 = (size_t)ctx->n + 1;
    int rc = dev_alloc(ctx, (void **)&ctx->gmV, sizeof(double) * n1 * (restart + 1));
    if (!rc) rc = dev_alloc(ctx, (void **)&ctx->gmW, sizeof(double) * n1 * 2);
    if (!rc) rc = dev_alloc(ctx, (void **)&ctx->gmZ, sizeof(double) * n1);
    if (!rc) rc = dev_alloc(ctx, (void **)&ctx->gmDinv, sizeof(double) * n1);
    if (!rc) rc = dev_alloc(ctx, (void **)&ctx->gmH, sizeof(double) * (kMaxDots + 4) * 2);
    if (rc) return rc;
    ctx->gm_restart = restart;
    return QEQ_OK;
}

void solver_free(qeq_ctx *ctx) {
    dev_free(ctx, ctx->gmV);
    dev_free(ctx, ctx->gmW);
    dev_free(ctx, ctx->gmZ);
    dev_free(ctx, ctx->gmDinv);
    dev_free(ctx, ctx->gmH);
    dev_free(ctx, ctx->gmSol);
}

namespace {

// Orthogonalise w against V_0..V_{nv-1}, classical Gram-Schmidt twice.
// On return h[k] is the sum of both passes' coefficients and norm = |w|.
int cgs2(qeq_ctx *ctx, int n1, int nv, double *w, std::vector<double> &h, double &norm,
         cudaStream_t s) {
    double *part = ctx->part;
    double *dh = ctx->gmH;  // pass 1 at [0, nv), pass 2 at [kMaxDots + 2, ...), |w|^2 at the end
    const int off2 = kMaxDots + 2;
    for (int pass = 0; pass < 2; ++pass) {
        double *dst = dh + (pass == 0 ? 0 : off2);
        k_multi_dot<<<ctx->red_grid, kThreads, 0, s>>>(n1, nv, ctx->gmV, w, part);
        launch_finalize(ctx, part, nv, dst, s);
        k_subtract<<<ctx->red_grid, kThreads, 0, s>>>(n1, nv, ctx->gmV, dst, w);
        ctx->launches += 3;
    }
    k_multi_dot<<<ctx->red_grid, kThreads, 0, s>>>(n1, 0, ctx->gmV, w, part);
    launch_finalize(ctx, part, 1, dh + 2 * off2, s);
    ctx->launches += 2;
    std::vector<double> hb(2 * off2 + 1);
    cudaError_t e = cudaMemcpyAsync(hb.data(), dh, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int rc = cuda_check(ctx, e, "gmres orthogonalise");
    if (rc) return rc;
    h.assign(nv, 0.0);
    for (int k = 0; k < nv; ++k) h[k] = hb[k] + hb[off2 + k];
    norm = std::sqrt(std::max(0.0, hb[2 * off2]));
    return QEQ_OK;
}

// y = A M^{-1} x  (one potential-only Coulomb apply)
int precond_apply(qeq_ctx *ctx, const double *R, const double *u, const double *sigma,
                  const double *x, double *y, cudaStream_t s, bool same_R) {
    const int n = (int)ctx->n;
    double *z = ctx->gmZ;
    k_precond<<<ctx->red_grid, kThreads, 0, s>>>(n, ctx->gmDinv, x, z);
    ctx->launches++;
    int rc = coulomb_apply_impl(ctx, R, z, sigma, ctx->phi, nullptr, nullptr, nullptr, false, s,
                                same_R);
    if (rc) return rc;
    k_bordered_apply<<<ctx->red_grid, kThreads, 0, s>>>(n, u, ctx->phi, z, y, ctx->part);
    launch_finalize(ctx, ctx->part, 1, ctx->gmH + 2 * (kMaxDots + 2) + 1, s);
    k_set_last<<<1, 32, 0, s>>>(n, ctx->gmH + 2 * (kMaxDots + 2) + 1, y);
    ctx->launches += 3;
    return QEQ_OK;
}

// A x without preconditioning (x in gmZ already as a plain vector)
int plain_apply(qeq_ctx *ctx, const double *R, const double *u, const double *sigma,
                const double *x, double *y, cudaStream_t s, bool same_R) {
    const int n = (int)ctx->n;
    int rc = coulomb_apply_impl(ctx, R, x, sigma, ctx->phi, nullptr, nullptr, nullptr, false, s,
                                same_R);
    if (rc) return rc;
    k_bordered_apply<<<ctx->red_grid, kThreads, 0, s>>>(n, u, ctx->phi, x, y, ctx->part);
    launch_finalize(ctx, ctx->part, 1, ctx->gmH + 2 * (kMaxDots + 2) + 1, s);
    k_set_last<<<1, 32, 0, s>>>(n, ctx->gmH + 2 * (kMaxDots + 2) + 1, y);
    ctx->launches += 3;
    return QEQ_OK;
}

double host_norm(qeq_ctx *ctx, const double *x, int n1, cudaStream_t s, int *rc) {
    k_multi_dot<<<ctx->red_grid, kThreads, 0, s>>>(n1, 0, ctx->gmV, x, ctx->part);
    launch_finalize(ctx, ctx->part, 1, ctx->gmH, s);
    ctx->launches += 2;
    double v = 0.0;
    cudaError_t e = cudaMemcpyAsync(&v, ctx->gmH, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *rc = cuda_check(ctx, e, "gmres norm");
    return std::sqrt(std::max(0.0, v));
}

}  // namespace

// Solve the bordered QEq system; z (device, N + 1) holds the initial guess
// [q; lambda] on entry and the solution on exit.
int gmres_solve(qeq_ctx *ctx, const double *R, const double *chi, const double *u,
                const double *sigma, double *z, double tol, int max_iter, int restart,
                bool final_check, qeq_solve_info *info, cudaStream_t s) {
    const int n = (int)ctx->n;
    const int n1 = n + 1;
    restart = std::max(1, std::min(restart, kMaxDots));
    int rc = solver_alloc(ctx, restart);
    if (rc) return rc;
    const qeq_params &p = ctx->p;
    k_jacobi<<<ctx->red_grid, kThreads, 0, s>>>(n, u, sigma, p.gaussian_self ? p.k_e * kSqrtTwoOverPi : 0.0,
                                             ctx->gmDinv);
    ctx->launches++;
    double *w = ctx->gmW;       // A z, then the residual / Arnoldi work vector
    double *bvec = ctx->gmW + n1;
    // |b| with b = [-chi; q_tot]  (residual of A z = 0)
    cudaMemsetAsync(w, 0, sizeof(double) * n1, s);
    k_residual<<<ctx->red_grid, kThreads, 0, s>>>(n, p.q_tot, chi, w, bvec);
    ctx->launches++;
    double bnorm = host_norm(ctx, bvec, n1, s, &rc);
    if (rc) return rc;
    if (!(bnorm > 0.0)) bnorm = 1.0;
    int iters = 0, applies = 0;
    double relres = 1.0;
    std::vector<double> H((size_t)(restart + 1) * restart), cs(restart), sn(restart), g(restart + 1), h;
    while (true) {
        // r = b - A z
        rc = plain_apply(ctx, R, u, sigma, z, w, s, applies > 0);
        if (rc) return rc;
        ++applies;
        k_residual<<<ctx->red_grid, kThreads, 0, s>>>(n, p.q_tot, chi, w, w);
        ctx->launches++;
        const double beta = host_norm(ctx, w, n1, s, &rc);
        if (rc) return rc;
        relres = beta / bnorm;
        if (relres <= tol || iters >= max_iter || !(beta > 0.0)) break;
        k_scale<<<ctx->red_grid, kThreads, 0, s>>>(n1, 1.0 / beta, w, ctx->gmV);
        ctx->launches++;
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0;
        for (; j < restart && iters < max_iter; ++j) {
            double *vj = ctx->gmV + (size_t)j * n1;
            double *vnext = ctx->gmV + (size_t)(j + 1) * n1;
            rc = precond_apply(ctx, R, u, sigma, vj, vnext, s, applies > 0);
            if (rc) return rc;
            ++applies;
            ++iters;
            double hn;
            rc = cgs2(ctx, n1, j + 1, vnext, h, hn, s);
            if (rc) return rc;
            for (int k = 0; k <= j; ++k) H[(size_t)k * restart + j] = h[k];
            H[(size_t)(j + 1) * restart + j] = hn;
            if (hn > 0.0) {
                k_scale<<<ctx->red_grid, kThreads, 0, s>>>(n1, 1.0 / hn, vnext, vnext);
                ctx->launches++;
            }
            // apply the previous rotations to column j, then a new one
            for (int k = 0; k < j; ++k) {
                const double a = H[(size_t)k * restart + j], b = H[(size_t)(k + 1) * restart + j];
                H[(size_t)k * restart + j] = cs[k] * a + sn[k] * b;
                H[(size_t)(k + 1) * restart + j] = -sn[k] * a + cs[k] * b;
            }
            const double a = H[(size_t)j * restart + j], b = H[(size_t)(j + 1) * restart + j];
            const double rr = std::hypot(a, b);
            cs[j] = rr > 0.0 ? a / rr : 1.0;
            sn[j] = rr > 0.0 ? b / rr : 0.0;
            H[(size_t)j * restart + j] = rr;
            H[(size_t)(j + 1) * restart + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            relres = std::fabs(g[j + 1]) / bnorm;
            if (relres <= tol || !(hn > 0.0)) {
                ++j;
                break;
            }
        }
        // y = H^{-1} g (upper triangular j x j), z += M^{-1} V y
        std::vector<double> y(j, 0.0);
        for (int r = j - 1; r >= 0; --r) {
            double acc = g[r];
            for (int c = r + 1; c < j; ++c) acc -= H[(size_t)r * restart + c] * y[c];
            const double d = H[(size_t)r * restart + r];
            y[r] = d != 0.0 ? acc / d : 0.0;
        }
        cudaError_t e = cudaMemcpyAsync(ctx->gmH, y.data(), sizeof(double) * std::max(1, j),
                                        cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        rc = cuda_check(ctx, e, "gmres update");
        if (rc) return rc;
        k_update_solution<<<ctx->red_grid, kThreads, 0, s>>>(n, j, ctx->gmV, ctx->gmH, ctx->gmDinv, z);
        ctx->launches++;
        if ((relres <= tol || iters >= max_iter) && !final_check) break;
        if (relres <= tol || iters >= max_iter) {
            // true residual of the final iterate (one more apply)
            rc = plain_apply(ctx, R, u, sigma, z, w, s, applies > 0);
            if (rc) return rc;
            ++applies;
            k_residual<<<ctx->red_grid, kThreads, 0, s>>>(n, p.q_tot, chi, w, w);
            ctx->launches++;
            relres = host_norm(ctx, w, n1, s, &rc) / bnorm;
            if (rc) return rc;
            break;
        }
    }
    if (info) {
        info->iterations = iters;
        info->applies = applies;
        info->rel_residual = relres;
        double lam = 0.0;
        cudaMemcpyAsync(&lam, z + n, sizeof(double), cudaMemcpyDeviceToHost, s);
        rc = cuda_check(ctx, cudaStreamSynchronize(s), "gmres lambda");
        if (rc) return rc;
        info->lambda = lam;
    }
    return QEQ_OK;
}

namespace {

// Velocity-Verlet half kick and drift; dt / (2 m mass_unit) kept for the second kick.
__global__ void k_kick_drift(int n, double dt, double mass_unit, const double *__restrict__ mass,
                             const double *__restrict__ F, double *__restrict__ R,
                             double *__restrict__ V, double *__restrict__ half_kick) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double hk = 0.5 * dt / (mass[i] * mass_unit);
        half_kick[i] = hk;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double vi = fma(F[3 * (size_t)i + d], hk, V[3 * (size_t)i + d]);
            V[3 * (size_t)i + d] = vi;
            R[3 * (size_t)i + d] += dt * vi;
        }
    }
}

}  // namespace

int bomd_advance(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, cudaStream_t s) {
    const int n = (int)ctx->n;
    prof_begin(ctx, kPhIntegrate, s);
    k_kick_drift<<<ctx->red_grid, kThreads, 0, s>>>(n, ctx->p.dt, ctx->p.mass_unit, prm->mass, st->F,
                                                 st->R, st->V, ctx->half_kick);
    prof_end(ctx, s);
    ctx->launches++;
    double d2 = 0.0;
    int rc = nl_displacement(ctx, st->R, s, &d2);
    if (rc) return rc;
    const double half = 0.5 * ctx->p.skin;
    if (!(d2 <= half * half)) return nl_build(ctx, st->R, s);
    return QEQ_OK;
}

// One BO evaluation at the current positions: solve (warm start from st->q),
// forces F = q o E (+ short range) and energies.  st->q holds N entries; the
// solver's N + 1 vector lives in ctx->gmSol.
int bomd_evaluate(qeq_ctx *ctx, const qeq_md_params *prm, qeq_md_state *st, double tol,
                  int max_iter, qeq_solve_info *info, cudaStream_t s) {
    const int n = (int)ctx->n;
    int rc = solver_alloc(ctx, 40);
    if (rc) return rc;
    if (!ctx->gmSol) {
        rc = dev_alloc(ctx, (void **)&ctx->gmSol, sizeof(double) * (n + 1));
        if (rc) return rc;
        cudaMemsetAsync(ctx->gmSol, 0, sizeof(double) * (n + 1), s);
    }
    cudaMemcpyAsync(ctx->gmSol, st->q, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    qeq_solve_info local{};
    // the force apply below evaluates the final charges, so GMRES skips its own check
    rc = gmres_solve(ctx, st->R, prm->chi, prm->eta, prm->sigma, ctx->gmSol, tol, max_iter, 40,
                     false, &local, s);
    if (rc) return rc;
    cudaMemcpyAsync(st->q, ctx->gmSol, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    double *scal = ctx->scal;
    rc = short_range_eval(ctx, st->R, prm->mass, scal + 126, s);
    if (rc) return rc;
    // the solve applied the operator at these positions already
    rc = coulomb_apply_impl(ctx, st->R, st->q, prm->sigma, ctx->v_n, ctx->E_n, nullptr, nullptr,
                            true, s, true);
    if (rc) return rc;
    local.applies += 1;
    k_bo_forces<<<ctx->red_grid, kThreads, 0, s>>>(
        n, st->q, ctx->E_n, has_short(ctx) ? ctx->F_short : nullptr, st->F);
    k_bo_energy_part<<<ctx->red_grid, kThreads, 0, s>>>(n, st->q, prm->chi, prm->eta, ctx->v_n, ctx->part);
    launch_finalize(ctx, ctx->part, 4, scal + 128, s);
    k_bo_energies<<<1, 1, 0, s>>>(scal + 128, scal + 126, local.lambda, local.rel_residual,
                                  (double)local.applies, st->energies);
    ctx->launches += 5;
    if (info) *info = local;
    return cuda_check(ctx, cudaGetLastError(), "bomd evaluate launch");
}

}  // namespace qeq
