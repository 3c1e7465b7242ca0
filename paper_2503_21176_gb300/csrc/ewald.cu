// Regular Ewald reciprocal sum with explicit k-vectors (Sec. 3.2, Eq. ewald_rec and
// its derivative forms), FP64, as the alternative to smooth PME (recip = QEQ_RECIP_EWALD).
//
// The k-vectors of the half space m1 > 0, or m1 = 0 and m2 > 0, or m1 = m2 = 0 and
// m3 > 0, with |k| <= k_cut are tabulated at create time.  Each table entry carries
// g(k) = 2 k_e (4 pi / V) exp(-k^2 / 4 alpha^2) / k^2, the factor 2 standing for -k.
// Per apply:
//   sfac_partial  blocks over (k tile, atom chunk): S(k) partial sums with the atoms
//                 of the chunk staged through shared memory
//   sfac_reduce   S(k) = sum over chunks in fixed order, and the energy partials
//                 1/2 g |S|^2
//   ewald_out     one thread per sorted atom, k-vectors and S staged through shared
//                 memory: v_i = sum_k g Re(e^{-i k.r_i} S(k)) and
//                 E_i = sum_k g k [sin(k.r_i) Re S - cos(k.r_i) Im S].  Fused with the
//                 real-space part, the self term, F = q E, the scatter back to the
//                 original order and the energy partials (like the PME gather).
// The paper builds the M = R K^T blocks on the fly in on-chip memory instead of
// materialising the N x k matrix (Sec. 3.2); the staging here does the same.
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace qeq {

namespace {

constexpr int kChunkAtoms = 1024;  // atoms per structure-factor chunk

__global__ void __launch_bounds__(kThreads)
k_sfac_partial(int n, int nk, const double4_32a *__restrict__ kv, const double4_32a *__restrict__ xq,
               double2 *__restrict__ partial) {
    __shared__ double4_32a atoms[kThreads];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int a0 = blockIdx.y * kChunkAtoms, a1 = min(n, a0 + kChunkAtoms);
    double4_32a kk = make_double4_32a(0, 0, 0, 0);
    if (k < nk) kk = kv[k];
    double sr = 0.0, si = 0.0;
    for (int t0 = a0; t0 < a1; t0 += kThreads) {
        const int a = t0 + threadIdx.x;
        atoms[threadIdx.x] = a < a1 ? xq[a] : make_double4_32a(0, 0, 0, 0);
        __syncthreads();
        const int m = min(kThreads, a1 - t0);
        if (k < nk) {
            for (int t = 0; t < m; ++t) {
                const double4_32a r = atoms[t];
                double s, c;
                sincos(kk.x * r.x + kk.y * r.y + kk.z * r.z, &s, &c);
                sr += r.w * c;
                si += r.w * s;
            }
        }
        __syncthreads();
    }
    if (k < nk) partial[(size_t)blockIdx.y * nk + k] = make_double2(sr, si);
}

__global__ void k_sfac_reduce(int nk, int nchunk, const double4_32a *__restrict__ kv,
                              const double2 *__restrict__ partial, double2 *__restrict__ S,
                              double *__restrict__ part) {
    double e = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nk; k += gridDim.x * blockDim.x) {
        double sr = 0.0, si = 0.0;
        for (int c = 0; c < nchunk; ++c) {
            const double2 p = partial[(size_t)c * nk + k];
            sr += p.x;
            si += p.y;
        }
        S[k] = make_double2(sr, si);
        e += 0.5 * kv[k].w * (sr * sr + si * si);
    }
    double vals[1] = {e};
    block_sum<1>(vals);
    if (threadIdx.x == 0) part[blockIdx.x] = vals[0];
}

struct EwaldOutArgs {
    int n, nk;
    double self_coef, gauss_coef;
};

template <bool FIELD>
__global__ void __launch_bounds__(kThreads)
k_ewald_out(EwaldOutArgs a, const int32_t *__restrict__ perm, const double4_32a *__restrict__ xq,
            const double4_32a *__restrict__ kv, const double2 *__restrict__ S,
            const double *__restrict__ v_s, const double *__restrict__ E_s,
            const double *__restrict__ q, const double *__restrict__ sigma,
            double *__restrict__ v_out, double *__restrict__ E_out, double *__restrict__ F_out,
            double *__restrict__ part) {
    __shared__ double4_32a ks[kThreads];
    __shared__ double2 ss[kThreads];
    double e_tot = 0.0, e_real = 0.0, e_self = 0.0;
    const int stride = gridDim.x * blockDim.x;
    const int rounds = (a.n + stride - 1) / stride;
    for (int rd = 0; rd < rounds; ++rd) {
        const int i = rd * stride + blockIdx.x * blockDim.x + threadIdx.x;
        const bool act = i < a.n;
        double4_32a r = make_double4_32a(0, 0, 0, 0);
        if (act) r = xq[i];
        double v = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
        for (int t0 = 0; t0 < a.nk; t0 += kThreads) {
            const int kk = t0 + threadIdx.x;
            if (kk < a.nk) {
                ks[threadIdx.x] = kv[kk];
                ss[threadIdx.x] = S[kk];
            }
            __syncthreads();
            const int m = min(kThreads, a.nk - t0);
            if (act) {
                for (int t = 0; t < m; ++t) {
                    const double4_32a k4 = ks[t];
                    const double2 s2 = ss[t];
                    double sn, cs;
                    sincos(k4.x * r.x + k4.y * r.y + k4.z * r.z, &sn, &cs);
                    v += k4.w * (cs * s2.x + sn * s2.y);
                    if (FIELD) {
                        const double wgt = k4.w * (sn * s2.x - cs * s2.y);
                        ex += wgt * k4.x;
                        ey += wgt * k4.y;
                        ez += wgt * k4.z;
                    }
                }
            }
            __syncthreads();
        }
        if (act) {
            const int atom = perm[i];
            const double qa = q[atom];
            double sc = a.self_coef;
            if (a.gauss_coef != 0.0) sc += a.gauss_coef / sigma[atom];
            const double vs = v_s[i];
            const double vself = sc * qa;
            const double vt = vs + v + vself;
            v_out[atom] = vt;
            if (FIELD) {
                const double Ex = E_s[3 * (size_t)i] + ex;
                const double Ey = E_s[3 * (size_t)i + 1] + ey;
                const double Ez = E_s[3 * (size_t)i + 2] + ez;
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
            e_tot += 0.5 * qa * vt;
            e_real += 0.5 * qa * vs;
            e_self += 0.5 * qa * vself;
        }
    }
    double vals[3] = {e_tot, e_real, e_self};
    block_sum<3>(vals);
    if (threadIdx.x == 0) {
        part[0 * kRedBlocks + blockIdx.x] = vals[0];
        part[1 * kRedBlocks + blockIdx.x] = vals[1];
        part[3 * kRedBlocks + blockIdx.x] = vals[2];
    }
}

}  // namespace

int ewald_alloc(qeq_ctx *ctx) {
    const qeq_params &p = ctx->p;
    double kc = p.k_cut;
    if (!(kc > 0.0)) kc = 2.0 * p.alpha * std::sqrt(-std::log(1e-16));  // exp(-k^2/4a^2) < 1e-16
    const double V = p.box[0] * p.box[1] * p.box[2];
    int mmax[3];
    for (int d = 0; d < 3; ++d) mmax[d] = (int)std::floor(kc * p.box[d] / (2.0 * kPi)) + 1;
    std::vector<double> tab;
    for (int m1 = 0; m1 <= mmax[0]; ++m1)
        for (int m2 = -mmax[1]; m2 <= mmax[1]; ++m2)
            for (int m3 = -mmax[2]; m3 <= mmax[2]; ++m3) {
                if (m1 == 0 && (m2 < 0 || (m2 == 0 && m3 <= 0))) continue;
                const double kx = 2.0 * kPi * m1 / p.box[0];
                const double ky = 2.0 * kPi * m2 / p.box[1];
                const double kz = 2.0 * kPi * m3 / p.box[2];
                const double k2 = kx * kx + ky * ky + kz * kz;
                if (k2 > kc * kc) continue;
                const double g = 2.0 * p.k_e * (4.0 * kPi / V) * std::exp(-k2 / (4.0 * p.alpha * p.alpha)) / k2;
                tab.insert(tab.end(), {kx, ky, kz, g});
            }
    ctx->ewald_nk = (int)(tab.size() / 4);
    if (ctx->ewald_nk == 0) tab.assign(4, 0.0);
    ctx->ewald_nchunk = (int)((ctx->n + kChunkAtoms - 1) / kChunkAtoms);
    const size_t nk = std::max(1, ctx->ewald_nk);
    int rc = dev_alloc(ctx, (void **)&ctx->ewald_k, sizeof(double4_32a) * nk);
    if (!rc) rc = dev_alloc(ctx, (void **)&ctx->ewald_S, sizeof(double2) * nk);
    if (!rc) rc = dev_alloc(ctx, (void **)&ctx->ewald_partial, sizeof(double2) * nk * ctx->ewald_nchunk);
    if (!rc) rc = dev_alloc(ctx, (void **)&ctx->xq64, sizeof(double4_32a) * ctx->n);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(ctx->ewald_k, tab.data(), sizeof(double) * tab.size(),
                                    cudaMemcpyHostToDevice, ctx->alloc_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->alloc_stream);
    return cuda_check(ctx, e, "ewald k-vector upload");
}

void ewald_free(qeq_ctx *ctx) {
    dev_free(ctx, ctx->ewald_k);
    dev_free(ctx, ctx->ewald_S);
    dev_free(ctx, ctx->ewald_partial);
}

// Reciprocal part by the k-sum plus the combine step; the sorted inputs (xq64, v_s, E_s)
// are already in place.
int ewald_recip_and_combine(qeq_ctx *ctx, const double *q, const double *sigma, double *v,
                            double *E, double *F, bool need_field, cudaStream_t s) {
    const int n = (int)ctx->n, nk = ctx->ewald_nk;
    const qeq_params &p = ctx->p;
    prof_begin(ctx, kPhSpread, s);
    if (nk > 0) {
        dim3 grid((nk + kThreads - 1) / kThreads, ctx->ewald_nchunk);
        k_sfac_partial<<<grid, kThreads, 0, s>>>(n, nk, (const double4_32a *)ctx->ewald_k, ctx->xq64,
                                                 (double2 *)ctx->ewald_partial);
        k_sfac_reduce<<<ctx->red_grid, kThreads, 0, s>>>(nk, ctx->ewald_nchunk,
                                                      (const double4_32a *)ctx->ewald_k,
                                                      (const double2 *)ctx->ewald_partial,
                                                      (double2 *)ctx->ewald_S, ctx->part + 2 * kRedBlocks);
    } else {
        cudaMemsetAsync(ctx->part + 2 * kRedBlocks, 0, sizeof(double) * kRedBlocks, s);
    }
    prof_end(ctx, s);
    EwaldOutArgs a;
    a.n = n;
    a.nk = nk;
    a.self_coef = p.k_e * (-kTwoOverSqrtPi * p.alpha);
    a.gauss_coef = p.gaussian_self ? p.k_e * kSqrtTwoOverPi : 0.0;
    prof_begin(ctx, kPhGatherOut, s);
    if (need_field)
        k_ewald_out<true><<<ctx->red_grid, kThreads, 0, s>>>(a, ctx->perm, ctx->xq64,
                                                          (const double4_32a *)ctx->ewald_k,
                                                          (const double2 *)ctx->ewald_S, ctx->v_s,
                                                          ctx->E_s, q, sigma, v, E, F, ctx->part);
    else
        k_ewald_out<false><<<ctx->red_grid, kThreads, 0, s>>>(a, ctx->perm, ctx->xq64,
                                                           (const double4_32a *)ctx->ewald_k,
                                                           (const double2 *)ctx->ewald_S, ctx->v_s,
                                                           ctx->E_s, q, sigma, v, nullptr, nullptr,
                                                           ctx->part);
    prof_end(ctx, s);
    ctx->launches += 3;
    return cuda_check(ctx, cudaGetLastError(), "ewald launch");
}

}  // namespace qeq
