/*
 * CPU reference loops of the oracle (test infrastructure; FP64 throughout).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
 * file.  It shares no code with the CUDA library.  Every loop is the plain
 * definition of the quantity it computes, with no blocking or fusion.
 * Compile with -ffp-contract=off so that no multiply-add is fused.  The
 * neighbour-pair decision depends on that for its exact operation order.
 *
 * Units: lengths in Angstrom, charges in e.  The pair kernels return
 * potential-per-unit-k_e; the Python side multiplies by k_e.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_TWO_OVER_SQRT_PI 1.12837916709551257390

/*
 * Real-space pair function of Eq. (ewald_real) with the Gaussian-charge
 * correction: f(r) = [erfc(alpha r) - erfc(r / gamma)] / r.  Point charges have
 * gamma = 0, and then the correction term is zero.  *g returns f'(r) / r, so
 * that the field at i due to charge q_j at displacement d = r_j - r_i is
 * q_j * g * d.
 */
static void pair_fg(double r, double alpha, double gamma, double *f, double *g)
{
    double ea = erfc(alpha * r);
    double fa = ea / r;
    double dfa = -(fa + OR_TWO_OVER_SQRT_PI * alpha * exp(-alpha * alpha * r * r)) / r;
    double fv = fa, df = dfa;
    if (gamma > 0.0) {
        double eg = erfc(r / gamma);
        double fgam = eg / r;
        double dfg = -(fgam + OR_TWO_OVER_SQRT_PI / gamma * exp(-(r * r) / (gamma * gamma))) / r;
        fv -= fgam;
        df -= dfg;
    }
    *f = fv;
    *g = df / r;
}

/* ---------------------------------------------------------------------- */
/* Brute-force neighbour pairs (Alg. 1 behaviour, exact set semantics).     */
/* ---------------------------------------------------------------------- */

/*
 * Inputs are the wrapped positions xw (N x 3).  A pair (i, j, s) is kept when
 * the image displacement d = (xw_j - xw_i) + s * L is shorter than r_list.  It is
 * kept for every integer image vector s with |s_d| <= smax_d, except the pair
 * with itself (i == j, s == 0).
 * d2 = (dx*dx + dy*dy) + dz*dz, compared with r_list*r_list (strict <).
 * Rows are emitted in ascending (j, sx, sy, sz) order.
 * Pass 1: counts[i].  Pass 2 (jout != NULL): fill from offsets[i].
 */
static void pairs_row(int64_t i, int64_t n, const double *xw, const double *box, double rl2,
                      const int32_t *smax, int64_t *count, int32_t *jout, int8_t *sout)
{
    int64_t c = 0;
    const double xi = xw[3 * i], yi = xw[3 * i + 1], zi = xw[3 * i + 2];
    for (int64_t j = 0; j < n; ++j) {
        const double bx = xw[3 * j] - xi, by = xw[3 * j + 1] - yi, bz = xw[3 * j + 2] - zi;
        for (int sx = -smax[0]; sx <= smax[0]; ++sx) {
            const double dx = bx + (double)sx * box[0];
            for (int sy = -smax[1]; sy <= smax[1]; ++sy) {
                const double dy = by + (double)sy * box[1];
                for (int sz = -smax[2]; sz <= smax[2]; ++sz) {
                    if (j == i && sx == 0 && sy == 0 && sz == 0) continue;
                    const double dz = bz + (double)sz * box[2];
                    const double d2 = (dx * dx + dy * dy) + dz * dz;
                    if (d2 < rl2) {
                        if (jout) {
                            jout[c] = (int32_t)j;
                            sout[3 * c] = (int8_t)sx;
                            sout[3 * c + 1] = (int8_t)sy;
                            sout[3 * c + 2] = (int8_t)sz;
                        }
                        ++c;
                    }
                }
            }
        }
    }
    *count = c;
}

int or_pairs_count(int64_t n, const double *xw, const double *box, double r_list,
                   const int32_t *smax, int64_t *counts)
{
    const double rl2 = r_list * r_list;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i)
        pairs_row(i, n, xw, box, rl2, smax, &counts[i], NULL, NULL);
    return 0;
}

int or_pairs_fill(int64_t n, const double *xw, const double *box, double r_list,
                  const int32_t *smax, const int64_t *offsets, int32_t *jout, int8_t *sout)
{
    const double rl2 = r_list * r_list;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c;
        pairs_row(i, n, xw, box, rl2, smax, &c, jout + offsets[i], sout + 3 * offsets[i]);
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Real-space sum, brute force over all atoms and images.                   */
/* ---------------------------------------------------------------------- */

/*
 * For each requested row i: v_i = sum_{j, s: (j,s) != (i,0), |d| < r_c} q_j f(|d|),
 * E_i = sum q_j g(|d|) d, with d = r_j - r_i + s * L.  Positions need not be
 * wrapped.  For each j the images scanned are the ones around the minimum image
 * whose distance can be below r_c.  rows == NULL means all rows, in order.
 */
int or_realspace_brute(int64_t n, const double *x, const double *q, const double *sigma,
                       const double *box, double alpha, double r_c, int64_t n_rows,
                       const int64_t *rows, double *v_out, double *E_out)
{
    const double rc2 = r_c * r_c;
    int smax[3];
    for (int d = 0; d < 3; ++d) smax[d] = (int)ceil(r_c / box[d]) + 1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < n_rows; ++t) {
        const int64_t i = rows ? rows[t] : t;
        double v = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double gamma = sqrt(sigma[i] * sigma[i] + sigma[j] * sigma[j]);
            double b[3];
            int s0[3];
            for (int d = 0; d < 3; ++d) {
                b[d] = x[3 * j + d] - x[3 * i + d];
                s0[d] = -(int)floor(b[d] / box[d] + 0.5);
            }
            for (int sx = s0[0] - smax[0]; sx <= s0[0] + smax[0]; ++sx)
                for (int sy = s0[1] - smax[1]; sy <= s0[1] + smax[1]; ++sy)
                    for (int sz = s0[2] - smax[2]; sz <= s0[2] + smax[2]; ++sz) {
                        if (j == i && sx == 0 && sy == 0 && sz == 0) continue;
                        const double dx = b[0] + sx * box[0];
                        const double dy = b[1] + sy * box[1];
                        const double dz = b[2] + sz * box[2];
                        const double r2 = dx * dx + dy * dy + dz * dz;
                        if (!(r2 < rc2)) continue;
                        double f, g;
                        pair_fg(sqrt(r2), alpha, gamma, &f, &g);
                        v += q[j] * f;
                        ex += q[j] * g * dx;
                        ey += q[j] * g * dy;
                        ez += q[j] * g * dz;
                    }
        }
        v_out[t] = v;
        E_out[3 * t] = ex;
        E_out[3 * t + 1] = ey;
        E_out[3 * t + 2] = ez;
    }
    return 0;
}

/*
 * Dense real-space matrix: out[i*n + j] = sum over images s with
 * (j,s) != (i,0) and |d| < r_c of f(|d|).  Small N only.
 */
int or_realspace_matrix(int64_t n, const double *x, const double *sigma, const double *box,
                        double alpha, double r_c, double *out)
{
    const double rc2 = r_c * r_c;
    int smax[3];
    for (int d = 0; d < 3; ++d) smax[d] = (int)ceil(r_c / box[d]) + 1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            const double gamma = sqrt(sigma[i] * sigma[i] + sigma[j] * sigma[j]);
            double b[3];
            int s0[3];
            for (int d = 0; d < 3; ++d) {
                b[d] = x[3 * j + d] - x[3 * i + d];
                s0[d] = -(int)floor(b[d] / box[d] + 0.5);
            }
            double acc = 0.0;
            for (int sx = s0[0] - smax[0]; sx <= s0[0] + smax[0]; ++sx)
                for (int sy = s0[1] - smax[1]; sy <= s0[1] + smax[1]; ++sy)
                    for (int sz = s0[2] - smax[2]; sz <= s0[2] + smax[2]; ++sz) {
                        if (j == i && sx == 0 && sy == 0 && sz == 0) continue;
                        const double dx = b[0] + sx * box[0];
                        const double dy = b[1] + sy * box[1];
                        const double dz = b[2] + sz * box[2];
                        const double r2 = dx * dx + dy * dy + dz * dz;
                        if (!(r2 < rc2)) continue;
                        double f, g;
                        pair_fg(sqrt(r2), alpha, gamma, &f, &g);
                        acc += f;
                    }
            out[i * n + j] = acc;
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Real-space sum through a cell list (same result, for large N).           */
/* ---------------------------------------------------------------------- */

/*
 * Cells of edge >= r_c / reach per dimension.  Every atom of every cell image
 * within `reach` cells is tested, so each (j, image) is visited exactly once
 * even when the box holds fewer than 2 * reach + 1 cells.
 */
int or_realspace_cells(int64_t n, const double *x, const double *q, const double *sigma,
                       const double *box, double alpha, double r_c, double *v_out, double *E_out)
{
    const double rc2 = r_c * r_c;
    int nc[3], reach[3];
    double cw[3];
    for (int d = 0; d < 3; ++d) {
        nc[d] = (int)floor(box[d] / r_c);
        if (nc[d] < 1) nc[d] = 1;
        cw[d] = box[d] / nc[d];
        reach[d] = (int)ceil(r_c / cw[d]);
    }
    const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    double *xw = (double *)malloc(sizeof(double) * 3 * n);
    int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * n);
    int64_t *start = (int64_t *)calloc(ncell + 1, sizeof(int64_t));
    int64_t *fillp = (int64_t *)malloc(sizeof(int64_t) * ncell);
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * n);
    if (!xw || !cell || !start || !fillp || !order) {
        free(xw); free(cell); free(start); free(fillp); free(order);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) {
        int c3[3];
        for (int d = 0; d < 3; ++d) {
            double w = x[3 * i + d] - box[d] * floor(x[3 * i + d] / box[d]);
            xw[3 * i + d] = w;
            int c = (int)floor(w / cw[d]);
            if (c < 0) c = 0;
            if (c >= nc[d]) c = nc[d] - 1;
            c3[d] = c;
        }
        cell[i] = ((int64_t)c3[0] * nc[1] + c3[1]) * nc[2] + c3[2];
        start[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    for (int64_t c = 0; c < ncell; ++c) fillp[c] = start[c];
    for (int64_t i = 0; i < n; ++i) order[fillp[cell[i]]++] = i;

#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        const int64_t ci = cell[i];
        const int c0[3] = {(int)(ci / ((int64_t)nc[1] * nc[2])), (int)((ci / nc[2]) % nc[1]),
                           (int)(ci % nc[2])};
        double v = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
        for (int ox = -reach[0]; ox <= reach[0]; ++ox)
            for (int oy = -reach[1]; oy <= reach[1]; ++oy)
                for (int oz = -reach[2]; oz <= reach[2]; ++oz) {
                    const int u[3] = {c0[0] + ox, c0[1] + oy, c0[2] + oz};
                    int w[3];
                    double sh[3];
                    for (int d = 0; d < 3; ++d) {
                        int s = (int)floor((double)u[d] / nc[d]);
                        w[d] = u[d] - s * nc[d];
                        sh[d] = s * box[d];
                    }
                    const int64_t cn = ((int64_t)w[0] * nc[1] + w[1]) * nc[2] + w[2];
                    for (int64_t t = start[cn]; t < start[cn + 1]; ++t) {
                        const int64_t j = order[t];
                        const double dx = xw[3 * j] + sh[0] - xw[3 * i];
                        const double dy = xw[3 * j + 1] + sh[1] - xw[3 * i + 1];
                        const double dz = xw[3 * j + 2] + sh[2] - xw[3 * i + 2];
                        const double r2 = dx * dx + dy * dy + dz * dz;
                        if (j == i && sh[0] == 0.0 && sh[1] == 0.0 && sh[2] == 0.0) continue;
                        if (!(r2 < rc2)) continue;
                        const double gamma = sqrt(sigma[i] * sigma[i] + sigma[j] * sigma[j]);
                        double f, g;
                        pair_fg(sqrt(r2), alpha, gamma, &f, &g);
                        v += q[j] * f;
                        ex += q[j] * g * dx;
                        ey += q[j] * g * dy;
                        ez += q[j] * g * dz;
                    }
                }
        v_out[i] = v;
        E_out[3 * i] = ex;
        E_out[3 * i + 1] = ey;
        E_out[3 * i + 2] = ez;
    }
    free(xw); free(cell); free(start); free(fillp); free(order);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Explicit k-vector reciprocal sum (Eq. ewald_rec and its derivatives).    */
/* ---------------------------------------------------------------------- */

/*
 * k = 2 pi (m1/Lx, m2/Ly, m3/Lz) over the half space of integer m != 0 with
 * |k| <= k_cut.  Each vector stands for itself and -k.
 *   g(k) = (4 pi / V) exp(-k^2 / 4 alpha^2) / k^2,  S(k) = sum_j q_j e^{i k.r_j}
 *   E_rec = 1/2 sum_{k != 0} g |S|^2
 *   v_i   = sum_{k != 0} g Re(e^{-i k.r_i} S)
 *   E_i   = -grad_i v_i = sum_{k != 0} g k [sin(k.r_i) Re S - cos(k.r_i) Im S]
 * Both halves of the k-space are included by doubling the half-space terms.
 */
static int64_t kvec_list(const double *box, double k_cut, double **kout)
{
    int mmax[3];
    for (int d = 0; d < 3; ++d) mmax[d] = (int)floor(k_cut * box[d] / (2.0 * OR_PI)) + 1;
    int64_t cap = (int64_t)(2 * mmax[0] + 1) * (2 * mmax[1] + 1) * (2 * mmax[2] + 1);
    double *k = (double *)malloc(sizeof(double) * 3 * cap);
    if (!k) return -1;
    int64_t nk = 0;
    const double kc2 = k_cut * k_cut;
    for (int m1 = 0; m1 <= mmax[0]; ++m1)
        for (int m2 = -mmax[1]; m2 <= mmax[1]; ++m2)
            for (int m3 = -mmax[2]; m3 <= mmax[2]; ++m3) {
                if (m1 == 0 && (m2 < 0 || (m2 == 0 && m3 <= 0))) continue;
                const double kx = 2.0 * OR_PI * m1 / box[0];
                const double ky = 2.0 * OR_PI * m2 / box[1];
                const double kz = 2.0 * OR_PI * m3 / box[2];
                const double k2 = kx * kx + ky * ky + kz * kz;
                if (k2 > kc2) continue;
                k[3 * nk] = kx;
                k[3 * nk + 1] = ky;
                k[3 * nk + 2] = kz;
                ++nk;
            }
    *kout = k;
    return nk;
}

int or_ewald_kspace(int64_t n, const double *x, const double *q, const double *box, double alpha,
                    double k_cut, double *v_out, double *E_out, double *energy_out)
{
    double *k = NULL;
    const int64_t nk = kvec_list(box, k_cut, &k);
    if (nk < 0) return -1;
    const double V = box[0] * box[1] * box[2];
    double *g = (double *)malloc(sizeof(double) * (nk > 0 ? nk : 1));
    double *sre = (double *)malloc(sizeof(double) * (nk > 0 ? nk : 1));
    double *sim = (double *)malloc(sizeof(double) * (nk > 0 ? nk : 1));
    if (!g || !sre || !sim) {
        free(k); free(g); free(sre); free(sim);
        return -1;
    }
    double energy = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : energy)
    for (int64_t t = 0; t < nk; ++t) {
        const double kx = k[3 * t], ky = k[3 * t + 1], kz = k[3 * t + 2];
        const double k2 = kx * kx + ky * ky + kz * kz;
        g[t] = 2.0 * (4.0 * OR_PI / V) * exp(-k2 / (4.0 * alpha * alpha)) / k2; /* x2: +-k */
        double a = 0.0, b = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double ph = kx * x[3 * j] + ky * x[3 * j + 1] + kz * x[3 * j + 2];
            a += q[j] * cos(ph);
            b += q[j] * sin(ph);
        }
        sre[t] = a;
        sim[t] = b;
        energy += 0.5 * g[t] * (a * a + b * b);
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double v = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
        for (int64_t t = 0; t < nk; ++t) {
            const double kx = k[3 * t], ky = k[3 * t + 1], kz = k[3 * t + 2];
            const double ph = kx * x[3 * i] + ky * x[3 * i + 1] + kz * x[3 * i + 2];
            const double c = cos(ph), s = sin(ph);
            v += g[t] * (c * sre[t] + s * sim[t]);
            const double w = g[t] * (s * sre[t] - c * sim[t]);
            ex += w * kx;
            ey += w * ky;
            ez += w * kz;
        }
        v_out[i] = v;
        E_out[3 * i] = ex;
        E_out[3 * i + 1] = ey;
        E_out[3 * i + 2] = ez;
    }
    *energy_out = energy;
    free(k); free(g); free(sre); free(sim);
    return (int)(nk > 0x7fffffff ? 0x7fffffff : nk);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
