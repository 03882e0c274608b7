/*
 * msm_oracle.c -- plain, slow, FP64 CPU oracle for the multilevel summation
 * method (MSM), velocity Verlet and parareal.
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the
 * benchmark's CPU-baseline leg call it; the product library never links,
 * loads or calls anything here, and nothing here includes product headers.
 *
 * Build with -ffp-contract=off: every a*b+c below rounds twice, as written.
 * OpenMP (optional) only splits loops whose iterations write disjoint
 * outputs; every sum is formed by one thread in a fixed order, so results are
 * bit-identical for any thread count.
 *
 * What each function follows (Pazurikova & Matyska, "Parallel-in-time method
 * for calculation of long-range electrostatic interactions"):
 *   orc_gamma, orc_dgamma ... Sec. 3, the C^2 Taylor smoothing gamma(rho)
 *   orc_gstar, orc_gk ....... Sec. 3, kernel splitting 1/r = g* + g^0 + ... + g^{l-1}
 *   orc_Phi, orc_dPhi ....... Sec. 3, nodal basis phi^k_mu = Phi(.)Phi(.)Phi(.);
 *                             Phi = cubic C1 numerical Hermite (Sec. 3, p = 3)
 *   orc_short_range ......... Sec. 3, u_i^short = sum_j g*(r_i, r_j) q_j (step 1)
 *   orc_anterpolate ......... Sec. 3, anterpolation q^0_mu = sum_j phi^0_mu(r_j) q_j
 *   orc_restrict ............ Sec. 3, restriction q^{k+1}_mu = sum_nu phi^{k+1}_mu(r^k_nu) q^k_nu
 *   orc_lattice_cutoff ...... Sec. 3, u^{k,cut}_mu = sum_nu g^k(r^k_mu, r^k_nu) q^k_nu
 *   orc_top_level ........... Sec. 3, u^{l-1}_mu = sum_nu g^{l-1}(r_mu, r_nu) q_nu
 *   orc_prolongate .......... Sec. 3, u^k = u^{k,cut} + sum_nu phi^{k+1}_nu(r^k_mu) u^{k+1}_nu
 *   orc_interpolate ......... Sec. 3, u_i^long = sum_mu phi^0_mu(r_i) u^0_mu (+ gradient)
 *   orc_msm ................. Sec. 3 example steps 1-9, U_i = k_e (u^short + u^long)
 *   orc_direct .............. Sec. 2, eq. (coulomb), read as sum over i<j
 *   orc_cutoff .............. Sec. 5, the coarse propagator's electrostatics:
 *                             simple cutoff (Coulomb's law for pairs within a)
 *                             or Wolf summation (damped, shifted, neutralised)
 *   orc_md_run .............. Sec. 2, F = -dU/dr and velocity Verlet; with
 *                             mts > 1 the multiple-time-step impulse method
 *                             (Sec. 3: the MSM suits one), grid part as the
 *                             slow force (orc_model_forces_split)
 *   orc_parareal ............ Sec. 4, lambda^{k+1}_{n+1} = G(lambda^{k+1}_n)
 *                                       + F(lambda^k_n) - G(lambda^k_n)
 *   orc_parareal_window ..... Sec. 4, the same recurrence over a sliding
 *                             computational window of at most W slices
 *   orc_project_rigid ....... water completion: corrected parareal states
 *                             projected back onto the rigid constraints
 * Readings of points the paper leaves open (self-interaction, open boundaries,
 * grid extents, the force formula, exclusions, parareal order) are stated
 * beside the code that takes them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ERANGE -2
#define ORC_ENOMEM -3
#define ORC_ENOCONV -6

/* ------------------------------------------------------------------------ */
/* Smoothing and kernels (Sec. 3)                                            */
/* ------------------------------------------------------------------------ */

/* gamma(rho): 15/8 - 5/4 rho^2 + 3/8 rho^4 below 1, 1/rho from 1 on. */
double orc_gamma(double rho)
{
    if (rho < 1.0) {
        double r2 = rho * rho;
        return 15.0 / 8.0 - (5.0 / 4.0) * r2 + (3.0 / 8.0) * r2 * r2;
    }
    return 1.0 / rho;
}

/* d gamma / d rho. */
double orc_dgamma(double rho)
{
    if (rho < 1.0)
        return -(5.0 / 2.0) * rho + (3.0 / 2.0) * rho * rho * rho;
    return -1.0 / (rho * rho);
}

/* g*(r) = 1/r - gamma(r/a)/a; identically zero from r = a on (gamma = 1/rho there). */
double orc_gstar(double r, double a)
{
    if (r >= a) return 0.0;
    return 1.0 / r - orc_gamma(r / a) / a;
}

/* d g*(r) / dr = -1/r^2 - gamma'(r/a)/a^2 (zero from r = a on). */
double orc_dgstar(double r, double a)
{
    if (r >= a) return 0.0;
    return -1.0 / (r * r) - orc_dgamma(r / a) / (a * a);
}

/* Level kernel.  For k < l-1:
 *   g^k(r) = gamma(r / 2^k a) / (2^k a) - gamma(r / 2^{k+1} a) / (2^{k+1} a),
 * which is identically zero from r = 2^{k+1} a on (both terms are 1/r there).
 * For the top level k = l-1: g^{l-1}(r) = gamma(r / 2^{l-1} a) / (2^{l-1} a). */
double orc_gk(double r, double a, int k, int l)
{
    double ak = ldexp(a, k);
    if (k == l - 1) return orc_gamma(r / ak) / ak;
    double ak1 = ldexp(a, k + 1);
    if (r >= ak1) return 0.0;
    return orc_gamma(r / ak) / ak - orc_gamma(r / ak1) / ak1;
}

/* Cubic C1 numerical Hermite nodal basis (support |t| < 2):
 *   Phi(t) = (1-|t|)(1+|t|-3/2 t^2)    for |t| <= 1
 *          = -1/2 (|t|-1)(2-|t|)^2     for 1 <= |t| <= 2
 *          = 0                          otherwise. */
double orc_Phi(double t)
{
    double s = fabs(t);
    if (s <= 1.0) return (1.0 - s) * (1.0 + s - 1.5 * s * s);
    if (s <= 2.0) return -0.5 * (s - 1.0) * (2.0 - s) * (2.0 - s);
    return 0.0;
}

/* dPhi/dt: -5|t| + 9/2 t^2 on |t| <= 1, -1/2 (2-|t|)(4-3|t|) on 1..2, odd in t. */
double orc_dPhi(double t)
{
    double s = fabs(t), d;
    if (s <= 1.0) d = -5.0 * s + 4.5 * s * s;
    else if (s <= 2.0) d = -0.5 * (2.0 - s) * (4.0 - 3.0 * s);
    else d = 0.0;
    return t < 0.0 ? -d : d;
}

/* ------------------------------------------------------------------------ */
/* Grid geometry (reading: open boundaries, Sec. 3 leaves them unstated)     */
/* ------------------------------------------------------------------------ */

static int64_t floordiv(int64_t a, int64_t b) { int64_t q = a / b; if ((a % b != 0) && ((a < 0) != (b < 0))) q--; return q; }

/* Per-axis index ranges of every level.  Level 0 covers every point whose
 * basis function touches an atom inside [x0, x0+L): mu in [-1, floor(L/h)+2].
 * Level k+1 covers every point with a non-zero restriction weight from level
 * k: mu in [ceil((lo-3)/2), floor((hi+3)/2)].  lo and hi are (l x 3) arrays. */
int orc_grid_dims(const double *box, double h, int l, int64_t *lo, int64_t *hi)
{
    if (l < 1 || !(h > 0)) return ORC_EINVAL;
    for (int d = 0; d < 3; d++) {
        double L = box[3 + d];
        if (!(L > 0)) return ORC_EINVAL;
        lo[d] = -1;
        hi[d] = (int64_t)floor(L / h) + 2;
    }
    for (int k = 1; k < l; k++)
        for (int d = 0; d < 3; d++) {
            lo[3 * k + d] = -floordiv(-(lo[3 * (k - 1) + d] - 3), 2);
            hi[3 * k + d] = floordiv(hi[3 * (k - 1) + d] + 3, 2);
        }
    return ORC_OK;
}

typedef struct { int64_t lo[3], n[3]; } glevel;

static glevel mk_level(const int64_t *lo, const int64_t *hi, int k)
{
    glevel g;
    for (int d = 0; d < 3; d++) { g.lo[d] = lo[3 * k + d]; g.n[d] = hi[3 * k + d] - lo[3 * k + d] + 1; }
    return g;
}
static int64_t gsize(const glevel *g) { return g->n[0] * g->n[1] * g->n[2]; }
static int64_t gidx(const glevel *g, int64_t mx, int64_t my, int64_t mz)
{
    return (mx - g->lo[0]) + g->n[0] * ((my - g->lo[1]) + g->n[1] * (mz - g->lo[2]));
}

/* ------------------------------------------------------------------------ */
/* Binning (bit-exact contract for the cell lists)                           */
/* ------------------------------------------------------------------------ */

/* Finest-grid cell of every atom: t = (x - x0) * (1/h) with 1/h rounded once
 * to FP64 (IEEE subtract, IEEE multiply, no contraction), c = floor(t).
 * Valid atoms have t >= 0 and c <= floor(L/h) on every axis.
 * key = (cz * ny + cy) * nx + cx with n = floor(L/h) + 1 cells per axis.
 * perm = atoms ordered by (key, original index): a textbook stable counting
 * sort.  cell_start has n_cells + 1 entries.  Returns ORC_EINVAL for a
 * non-finite coordinate and ORC_ERANGE for an atom outside the box. */
int orc_bin(int64_t n, const double *pos, const double *box, double h,
            int64_t *cell, int64_t *key, int64_t *perm, int64_t *cell_start)
{
    int64_t nc[3];
    for (int d = 0; d < 3; d++) nc[d] = (int64_t)floor(box[3 + d] / h) + 1;
    int64_t ncells = nc[0] * nc[1] * nc[2];
    double inv_h = 1.0 / h;
    for (int64_t i = 0; i < n; i++) {
        int64_t c[3];
        for (int d = 0; d < 3; d++) {
            double x = pos[3 * i + d];
            if (!isfinite(x)) return ORC_EINVAL;
            double t = (x - box[d]) * inv_h;
            if (!(t >= 0.0)) return ORC_ERANGE;
            double f = floor(t);
            if (f > (double)(nc[d] - 1)) return ORC_ERANGE;
            c[d] = (int64_t)f;
            if (cell) cell[3 * i + d] = c[d];
        }
        key[i] = (c[2] * nc[1] + c[1]) * nc[0] + c[0];
    }
    if (perm && cell_start) {
        int64_t *cnt = calloc((size_t)ncells + 1, sizeof(int64_t));
        if (!cnt) return ORC_ENOMEM;
        for (int64_t i = 0; i < n; i++) cnt[key[i] + 1]++;
        for (int64_t c = 0; c < ncells; c++) cnt[c + 1] += cnt[c];
        memcpy(cell_start, cnt, sizeof(int64_t) * (size_t)(ncells + 1));
        for (int64_t i = 0; i < n; i++) perm[cnt[key[i]]++] = i;   /* ascending i: stable */
        free(cnt);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Short-range part (Sec. 3, step 1)                                         */
/* ------------------------------------------------------------------------ */

/* All pairs, for tiny systems: phi_s[i] = sum_{j != i} q_j g*(r_ij),
 * f_s[i] = -q_i sum_{j != i} q_j g*'(r_ij) (r_i - r_j)/r_ij. */
void orc_short_range_brute(int64_t n, const double *pos, const double *q, double a,
                           double *phi_s, double *f_s)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        double p = 0, fx = 0, fy = 0, fz = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1], dz = pos[3 * i + 2] - pos[3 * j + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (r >= a) continue;
            p += q[j] * orc_gstar(r, a);
            double s = -q[i] * q[j] * orc_dgstar(r, a) / r;
            fx += s * dx; fy += s * dy; fz += s * dz;
        }
        phi_s[i] = p;
        f_s[3 * i] = fx; f_s[3 * i + 1] = fy; f_s[3 * i + 2] = fz;
    }
}

/* Same sum, with candidate pairs found through bins of edge >= a (27 bins
 * around each atom contain every j with r_ij < a).  If targets != NULL only
 * the n_t listed atoms are evaluated; outputs are then indexed 0..n_t-1. */
int orc_short_range(int64_t n, const double *pos, const double *q, double a, const double *box,
                    int64_t n_t, const int64_t *targets, double *phi_s, double *f_s)
{
    int64_t nb[3]; double eb[3];
    for (int d = 0; d < 3; d++) {
        nb[d] = (int64_t)floor(box[3 + d] / a);
        if (nb[d] < 1) nb[d] = 1;
        eb[d] = box[3 + d] / (double)nb[d];
    }
    int64_t nbin = nb[0] * nb[1] * nb[2];
    int64_t *bin = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *start = calloc((size_t)nbin + 1, sizeof(int64_t));
    int64_t *list = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!bin || !start || !list) { free(bin); free(start); free(list); return ORC_ENOMEM; }
    for (int64_t i = 0; i < n; i++) {
        int64_t c[3];
        for (int d = 0; d < 3; d++) {
            int64_t v = (int64_t)floor((pos[3 * i + d] - box[d]) / eb[d]);
            c[d] = v < 0 ? 0 : (v >= nb[d] ? nb[d] - 1 : v);
        }
        bin[i] = (c[2] * nb[1] + c[1]) * nb[0] + c[0];
        start[bin[i] + 1]++;
    }
    for (int64_t b = 0; b < nbin; b++) start[b + 1] += start[b];
    {
        int64_t *fill = malloc(sizeof(int64_t) * (size_t)nbin);
        if (!fill) { free(bin); free(start); free(list); return ORC_ENOMEM; }
        memcpy(fill, start, sizeof(int64_t) * (size_t)nbin);
        for (int64_t i = 0; i < n; i++) list[fill[bin[i]]++] = i;
        free(fill);
    }
    int64_t m = targets ? n_t : n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < m; t++) {
        int64_t i = targets ? targets[t] : t;
        int64_t bx = bin[i] % nb[0], by = (bin[i] / nb[0]) % nb[1], bz = bin[i] / (nb[0] * nb[1]);
        double p = 0, fx = 0, fy = 0, fz = 0;
        for (int64_t z = bz - 1; z <= bz + 1; z++) {
            if (z < 0 || z >= nb[2]) continue;
            for (int64_t y = by - 1; y <= by + 1; y++) {
                if (y < 0 || y >= nb[1]) continue;
                for (int64_t x = bx - 1; x <= bx + 1; x++) {
                    if (x < 0 || x >= nb[0]) continue;
                    int64_t b = (z * nb[1] + y) * nb[0] + x;
                    for (int64_t s = start[b]; s < start[b + 1]; s++) {
                        int64_t j = list[s];
                        if (j == i) continue;
                        double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1], dz = pos[3 * i + 2] - pos[3 * j + 2];
                        double r = sqrt(dx * dx + dy * dy + dz * dz);
                        if (r >= a) continue;
                        p += q[j] * orc_gstar(r, a);
                        double sc = -q[i] * q[j] * orc_dgstar(r, a) / r;
                        fx += sc * dx; fy += sc * dy; fz += sc * dz;
                    }
                }
            }
        }
        phi_s[t] = p;
        f_s[3 * t] = fx; f_s[3 * t + 1] = fy; f_s[3 * t + 2] = fz;
    }
    free(bin); free(start); free(list);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Grid transfers and grid sums (Sec. 3, long-range steps)                   */
/* ------------------------------------------------------------------------ */

/* Anterpolation: q^0_mu = sum_j phi^0_mu(r_j) q_j, phi^0_mu(r) =
 * Phi((x - x_mu)/h) Phi((y - y_mu)/h) Phi((z - z_mu)/h), x_mu = x0 + mu h.
 * With t = (x - x0)/h the argument is t - mu; the support is
 * mu = floor(t)-1 .. floor(t)+2 on each axis. */
int orc_anterpolate(const int64_t *lo, const int64_t *hi, double h, const double *box,
                    int64_t n, const double *pos, const double *q, double *q0)
{
    glevel g = mk_level(lo, hi, 0);
    memset(q0, 0, sizeof(double) * (size_t)gsize(&g));
    for (int64_t j = 0; j < n; j++) {
        double t[3]; int64_t c[3];
        for (int d = 0; d < 3; d++) { t[d] = (pos[3 * j + d] - box[d]) / h; c[d] = (int64_t)floor(t[d]); }
        for (int64_t mz = c[2] - 1; mz <= c[2] + 2; mz++)
            for (int64_t my = c[1] - 1; my <= c[1] + 2; my++)
                for (int64_t mx = c[0] - 1; mx <= c[0] + 2; mx++) {
                    if (mx < g.lo[0] || my < g.lo[1] || mz < g.lo[2] ||
                        mx >= g.lo[0] + g.n[0] || my >= g.lo[1] + g.n[1] || mz >= g.lo[2] + g.n[2])
                        return ORC_ERANGE;
                    double w = orc_Phi(t[0] - (double)mx) * orc_Phi(t[1] - (double)my) * orc_Phi(t[2] - (double)mz);
                    q0[gidx(&g, mx, my, mz)] += w * q[j];
                }
    }
    return ORC_OK;
}

/* Restriction k -> k+1: q^{k+1}_mu = sum_nu phi^{k+1}_mu(r^k_nu) q^k_nu.
 * Level-k point nu sits at x0 + nu 2^k h and level-(k+1) point mu at
 * x0 + mu 2^{k+1} h, so the basis argument is (nu 2^k h - mu 2^{k+1} h)/(2^{k+1} h)
 * = nu/2 - mu; Phi vanishes for |nu/2 - mu| >= 2, i.e. outside nu in [2mu-3, 2mu+3]. */
void orc_restrict(const int64_t *lo, const int64_t *hi, int k, const double *qk, double *qk1)
{
    glevel f = mk_level(lo, hi, k), c = mk_level(lo, hi, k + 1);
#pragma omp parallel for schedule(static)
    for (int64_t idx = 0; idx < gsize(&c); idx++) {
        int64_t mx = c.lo[0] + idx % c.n[0], my = c.lo[1] + (idx / c.n[0]) % c.n[1], mz = c.lo[2] + idx / (c.n[0] * c.n[1]);
        double s = 0;
        for (int64_t nz = 2 * mz - 3; nz <= 2 * mz + 3; nz++) {
            if (nz < f.lo[2] || nz >= f.lo[2] + f.n[2]) continue;
            for (int64_t ny = 2 * my - 3; ny <= 2 * my + 3; ny++) {
                if (ny < f.lo[1] || ny >= f.lo[1] + f.n[1]) continue;
                for (int64_t nx = 2 * mx - 3; nx <= 2 * mx + 3; nx++) {
                    if (nx < f.lo[0] || nx >= f.lo[0] + f.n[0]) continue;
                    double w = orc_Phi(0.5 * (double)nx - (double)mx) * orc_Phi(0.5 * (double)ny - (double)my) *
                               orc_Phi(0.5 * (double)nz - (double)mz);
                    s += w * qk[gidx(&f, nx, ny, nz)];
                }
            }
        }
        qk1[idx] = s;
    }
}

/* Lattice cutoff on level k < l-1: u^{k,cut}_mu = sum_nu g^k(|r_mu - r_nu|) q^k_nu,
 * |r_mu - r_nu| = 2^k h |mu - nu|.  g^k vanishes from 2^{k+1} a on, i.e. for
 * |mu - nu| >= 2a/h, so only nu within R = ceil(2a/h) per axis can contribute. */
void orc_lattice_cutoff(const int64_t *lo, const int64_t *hi, int k, int l, double a, double h,
                        const double *qk, double *ucut)
{
    glevel g = mk_level(lo, hi, k);
    double hk = ldexp(h, k);
    int64_t R = (int64_t)ceil(2.0 * a / h);
#pragma omp parallel for schedule(static)
    for (int64_t idx = 0; idx < gsize(&g); idx++) {
        int64_t mx = g.lo[0] + idx % g.n[0], my = g.lo[1] + (idx / g.n[0]) % g.n[1], mz = g.lo[2] + idx / (g.n[0] * g.n[1]);
        double s = 0;
        for (int64_t nz = mz - R; nz <= mz + R; nz++) {
            if (nz < g.lo[2] || nz >= g.lo[2] + g.n[2]) continue;
            for (int64_t ny = my - R; ny <= my + R; ny++) {
                if (ny < g.lo[1] || ny >= g.lo[1] + g.n[1]) continue;
                for (int64_t nx = mx - R; nx <= mx + R; nx++) {
                    if (nx < g.lo[0] || nx >= g.lo[0] + g.n[0]) continue;
                    double dx = (double)(mx - nx) * hk, dy = (double)(my - ny) * hk, dz = (double)(mz - nz) * hk;
                    double r = sqrt(dx * dx + dy * dy + dz * dz);
                    s += orc_gk(r, a, k, l) * qk[gidx(&g, nx, ny, nz)];
                }
            }
        }
        ucut[idx] = s;
    }
}

/* Top level: u^{l-1}_mu = sum over all nu (nu = mu included; g^{l-1}(0) =
 * gamma(0)/(2^{l-1} a) is finite) of g^{l-1}(|r_mu - r_nu|) q^{l-1}_nu. */
void orc_top_level(const int64_t *lo, const int64_t *hi, int l, double a, double h,
                   const double *qt, double *ut)
{
    int k = l - 1;
    glevel g = mk_level(lo, hi, k);
    double hk = ldexp(h, k);
    int64_t m = gsize(&g);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; i++) {
        int64_t mx = i % g.n[0], my = (i / g.n[0]) % g.n[1], mz = i / (g.n[0] * g.n[1]);
        double s = 0;
        for (int64_t j = 0; j < m; j++) {
            int64_t nx = j % g.n[0], ny = (j / g.n[0]) % g.n[1], nz = j / (g.n[0] * g.n[1]);
            double dx = (double)(mx - nx) * hk, dy = (double)(my - ny) * hk, dz = (double)(mz - nz) * hk;
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            s += orc_gk(r, a, k, l) * qt[j];
        }
        ut[i] = s;
    }
}

/* Prolongation k+1 -> k: u^k_mu = u^{k,cut}_mu + sum_nu phi^{k+1}_nu(r^k_mu) u^{k+1}_nu,
 * basis argument mu/2 - nu, non-zero for nu in [(mu-3)/2, (mu+3)/2]. */
void orc_prolongate(const int64_t *lo, const int64_t *hi, int k, const double *ucut,
                    const double *uk1, double *uk)
{
    glevel f = mk_level(lo, hi, k), c = mk_level(lo, hi, k + 1);
#pragma omp parallel for schedule(static)
    for (int64_t idx = 0; idx < gsize(&f); idx++) {
        int64_t mx = f.lo[0] + idx % f.n[0], my = f.lo[1] + (idx / f.n[0]) % f.n[1], mz = f.lo[2] + idx / (f.n[0] * f.n[1]);
        double s = 0;
        for (int64_t nz = floordiv(mz - 3, 2); nz <= floordiv(mz + 3, 2) + 1; nz++) {
            if (nz < c.lo[2] || nz >= c.lo[2] + c.n[2]) continue;
            for (int64_t ny = floordiv(my - 3, 2); ny <= floordiv(my + 3, 2) + 1; ny++) {
                if (ny < c.lo[1] || ny >= c.lo[1] + c.n[1]) continue;
                for (int64_t nx = floordiv(mx - 3, 2); nx <= floordiv(mx + 3, 2) + 1; nx++) {
                    if (nx < c.lo[0] || nx >= c.lo[0] + c.n[0]) continue;
                    double w = orc_Phi(0.5 * (double)mx - (double)nx) * orc_Phi(0.5 * (double)my - (double)ny) *
                               orc_Phi(0.5 * (double)mz - (double)nz);
                    s += w * uk1[gidx(&c, nx, ny, nz)];
                }
            }
        }
        uk[idx] = ucut[idx] + s;
    }
}

/* Interpolation: phi_L[i] = sum_mu phi^0_mu(r_i) u^0_mu and its gradient
 * grad_L[i] = sum_mu grad phi^0_mu(r_i) u^0_mu (d/dx of Phi((x - x_mu)/h) is
 * Phi'((x - x_mu)/h)/h). */
void orc_interpolate(const int64_t *lo, const int64_t *hi, double h, const double *box,
                     int64_t n, const double *pos, const double *u0, double *phi_l, double *grad_l)
{
    glevel g = mk_level(lo, hi, 0);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double t[3]; int64_t c[3];
        for (int d = 0; d < 3; d++) { t[d] = (pos[3 * i + d] - box[d]) / h; c[d] = (int64_t)floor(t[d]); }
        double p = 0, gx = 0, gy = 0, gz = 0;
        for (int64_t mz = c[2] - 1; mz <= c[2] + 2; mz++)
            for (int64_t my = c[1] - 1; my <= c[1] + 2; my++)
                for (int64_t mx = c[0] - 1; mx <= c[0] + 2; mx++) {
                    double u = u0[gidx(&g, mx, my, mz)];
                    double px = orc_Phi(t[0] - (double)mx), py = orc_Phi(t[1] - (double)my), pz = orc_Phi(t[2] - (double)mz);
                    double dx = orc_dPhi(t[0] - (double)mx) / h, dy = orc_dPhi(t[1] - (double)my) / h,
                           dz = orc_dPhi(t[2] - (double)mz) / h;
                    p += px * py * pz * u;
                    gx += dx * py * pz * u;
                    gy += px * dy * pz * u;
                    gz += px * py * dz * u;
                }
        phi_l[i] = p;
        grad_l[3 * i] = gx; grad_l[3 * i + 1] = gy; grad_l[3 * i + 2] = gz;
    }
}

/* ------------------------------------------------------------------------ */
/* Whole MSM evaluation                                                      */
/* ------------------------------------------------------------------------ */

/* Optional per-stage outputs: every non-NULL pointer receives a copy of the
 * named quantity (grids for all levels concatenated level 0 first). */
typedef struct {
    double *phi_short;   /* n      */
    double *f_short;     /* n*3    */
    double *phi_long;    /* n      */
    double *grad_long;   /* n*3    */
    double *qgrid;       /* sum_k |level k|: q^k                   */
    double *ucut;        /* sum_{k<l-1} |level k|: u^{k,cut}        */
    double *ugrid;       /* sum_k |level k|: u^k (u^{l-1} = top)   */
} orc_stage_out;

/* One MSM energy/force evaluation, following the worked example of Sec. 3:
 *   1. short range   2. anterpolation   3-4. restriction + lattice cutoff
 *   5. top level     6-7. prolongation  8. interpolation  9. totals.
 * Readings:
 *   - self-interaction: the grid part contains each atom's own smooth
 *     potential; since g* + sum_k g^k = 1/r and g* ~ 1/r - gamma(0)/a at
 *     r -> 0, the exact self term is q_i gamma(0)/a (gamma(0) = 15/8), which
 *     is subtracted from phi_i (no force: it does not depend on r_i);
 *   - phi_i = k_e (u_i^short + u_i^long - q_i gamma(0)/a), U = 1/2 sum_i q_i phi_i
 *     (the paper's double sum counts each pair twice);
 *   - F_i = -dU/dr_i = k_e (f_short_i - q_i grad u^long(r_i)), exact because
 *     every interpolation operator I^k is symmetric in its two arguments.
 * prm = {a, h, k_e}.  Returns ORC_ERANGE if an atom lies outside the box. */
int orc_msm(const double *prm, int l, int64_t n, const double *pos, const double *q, const double *box,
            double *energy, double *forces, double *pot, orc_stage_out *st)
{
    double a = prm[0], h = prm[1], ke = prm[2];
    if (l < 1 || l > 16 || !(a > 0) || !(h > 0)) return ORC_EINVAL;
    int64_t lo[48], hi[48];
    int rc = orc_grid_dims(box, h, l, lo, hi);
    if (rc) return rc;
    {
        int64_t *key = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        if (!key) return ORC_ENOMEM;
        rc = orc_bin(n, pos, box, h, NULL, key, NULL, NULL);
        free(key);
        if (rc) return rc;
    }
    int64_t off[17], tot = 0;
    for (int k = 0; k < l; k++) { glevel g = mk_level(lo, hi, k); off[k] = tot; tot += gsize(&g); }
    off[l] = tot;
    double *qg = calloc((size_t)tot, sizeof(double));
    double *ug = calloc((size_t)tot, sizeof(double));
    double *uc = calloc((size_t)tot, sizeof(double));
    double *ps = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *fs = malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *pl = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *gl = malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!qg || !ug || !uc || !ps || !fs || !pl || !gl) { rc = ORC_ENOMEM; goto done; }

    rc = orc_short_range(n, pos, q, a, box, 0, NULL, ps, fs);                       /* step 1 */
    if (rc) goto done;
    rc = orc_anterpolate(lo, hi, h, box, n, pos, q, qg + off[0]);                   /* step 2 */
    if (rc) goto done;
    for (int k = 0; k + 1 < l; k++) {                                               /* steps 3-4 */
        orc_restrict(lo, hi, k, qg + off[k], qg + off[k + 1]);
        orc_lattice_cutoff(lo, hi, k, l, a, h, qg + off[k], uc + off[k]);
    }
    orc_top_level(lo, hi, l, a, h, qg + off[l - 1], ug + off[l - 1]);               /* step 5 */
    for (int k = l - 2; k >= 0; k--)                                                /* steps 6-7 */
        orc_prolongate(lo, hi, k, uc + off[k], ug + off[k + 1], ug + off[k]);
    orc_interpolate(lo, hi, h, box, n, pos, ug + off[0], pl, gl);                   /* step 8 */

    {                                                                               /* step 9 */
        double self = orc_gamma(0.0) / a, U = 0;
        for (int64_t i = 0; i < n; i++) {
            double phi = ke * (ps[i] + pl[i] - q[i] * self);
            if (pot) pot[i] = phi;
            U += q[i] * phi;
            if (forces)
                for (int d = 0; d < 3; d++) forces[3 * i + d] = ke * (fs[3 * i + d] - q[i] * gl[3 * i + d]);
        }
        if (energy) *energy = 0.5 * U;
    }
    if (st) {
        if (st->phi_short) memcpy(st->phi_short, ps, sizeof(double) * (size_t)n);
        if (st->f_short) memcpy(st->f_short, fs, sizeof(double) * 3 * (size_t)n);
        if (st->phi_long) memcpy(st->phi_long, pl, sizeof(double) * (size_t)n);
        if (st->grad_long) memcpy(st->grad_long, gl, sizeof(double) * 3 * (size_t)n);
        if (st->qgrid) memcpy(st->qgrid, qg, sizeof(double) * (size_t)tot);
        if (st->ucut) memcpy(st->ucut, uc, sizeof(double) * (size_t)(l > 1 ? off[l - 1] : 0));
        if (st->ugrid) memcpy(st->ugrid, ug, sizeof(double) * (size_t)tot);
    }
done:
    free(qg); free(ug); free(uc); free(ps); free(fs); free(pl); free(gl);
    return rc;
}

/* Sec. 2, eq. (coulomb), read as U = sum_{i<j} q_i q_j / r_ij (the printed
 * double sum counts every pair twice and includes i = j).  phi_i =
 * k_e sum_{j != i} q_j / r_ij, F_i = k_e q_i sum_{j != i} q_j (r_i - r_j)/r_ij^3. */
void orc_direct(int64_t n, const double *pos, const double *q, double ke,
                double *energy, double *forces, double *pot)
{
    double *phi = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        double p = 0, fx = 0, fy = 0, fz = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1], dz = pos[3 * i + 2] - pos[3 * j + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            p += q[j] / r;
            double s = q[i] * q[j] / (r * r * r);
            fx += s * dx; fy += s * dy; fz += s * dz;
        }
        phi[i] = ke * p;
        if (forces) { forces[3 * i] = ke * fx; forces[3 * i + 1] = ke * fy; forces[3 * i + 2] = ke * fz; }
    }
    double U = 0;
    for (int64_t i = 0; i < n; i++) { U += q[i] * phi[i]; if (pot) pot[i] = phi[i]; }
    if (energy) *energy = 0.5 * U;
    free(phi);
}

/* ------------------------------------------------------------------------ */
/* Cutoff electrostatics for the coarse propagator (Sec. 5)                  */
/* ------------------------------------------------------------------------ */

#define ORC_METHOD_MSM 0
#define ORC_METHOD_CUTOFF 1
#define ORC_METHOD_WOLF 2
#define ORC_PI 3.14159265358979323846

/* Sec. 5 lists the coarse approximations G the paper weighs and keeps two:
 *   method 1, simple cutoff: Coulomb's law between the pairs closer than the
 *     cutoff a, nothing beyond (the paper's chosen G):
 *       U = 1/2 sum_i sum_{j != i, r_ij < a} k_e q_i q_j / r_ij;
 *   method 2, Wolf summation (Wolf, Keblinski, Phillpot & Eggebrecht 1999,
 *     the paper's proposed later G): the pair term damped by erfc, shifted to
 *     zero at a, and the charge-neutralisation self term,
 *       U = 1/2 sum_i sum_{j != i, r_ij < a} k_e q_i q_j [erfc(alpha r)/r - erfc(alpha a)/a]
 *           - k_e [erfc(alpha a)/(2a) + alpha/sqrt(pi)] sum_i q_i^2.
 * Potentials phi_i = dU/dq_i (so U = 1/2 sum q_i phi_i), forces the exact
 * gradient F_i = -dU/dr_i (the shift is constant inside a).  Pairs inside one
 * rigid triple (atoms 3m..3m+2, m < n_mol) are skipped: with no grid there is
 * no smooth part to remove.  Brute force over all pairs, FP64. */
int orc_cutoff(int method, double a, double alpha, double ke, int64_t n, int64_t n_mol, const double *pos,
               const double *q, double *energy, double *forces, double *pot)
{
    if ((method != ORC_METHOD_CUTOFF && method != ORC_METHOD_WOLF) || !(a > 0) || !(alpha >= 0)) return ORC_EINVAL;
    const int wolf = method == ORC_METHOD_WOLF;
    const double shift = wolf ? erfc(alpha * a) / a : 0.0;
    const double selfc = wolf ? erfc(alpha * a) / a + 2.0 * alpha / sqrt(ORC_PI) : 0.0;
    double *phi = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!phi) return ORC_ENOMEM;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        const int64_t mi = i < 3 * n_mol ? i / 3 : -1 - i;
        double p = 0, fx = 0, fy = 0, fz = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            if (j < 3 * n_mol && j / 3 == mi) continue;
            double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1], dz = pos[3 * i + 2] - pos[3 * j + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (!(r < a)) continue;
            double g, mdg;                               /* pair term and -d/dr of it */
            if (wolf) {
                g = erfc(alpha * r) / r - shift;
                mdg = erfc(alpha * r) / (r * r) + 2.0 * alpha / sqrt(ORC_PI) * exp(-alpha * alpha * r * r) / r;
            } else {
                g = 1.0 / r;
                mdg = 1.0 / (r * r);
            }
            p += q[j] * g;
            double s = q[i] * q[j] * mdg / r;
            fx += s * dx; fy += s * dy; fz += s * dz;
        }
        phi[i] = ke * (p - selfc * q[i]);
        if (forces) { forces[3 * i] = ke * fx; forces[3 * i + 1] = ke * fy; forces[3 * i + 2] = ke * fz; }
    }
    double U = 0;
    for (int64_t i = 0; i < n; i++) { U += q[i] * phi[i]; if (pot) pot[i] = phi[i]; }
    if (energy) *energy = 0.5 * U;
    free(phi);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Model completion for rigid 3-site water (outside the paper)               */
/* ------------------------------------------------------------------------ */

/* The paper's MD loop (Sec. 2) integrates U_all, of which it treats only the
 * Coulomb part.  Bare point charges collapse within femtoseconds, so water
 * workloads add, outside the paper:
 *   - exclusion of the three intramolecular pairs of each (O, H, H) triple:
 *     the MSM sum contains g*(r) + (grid approximation of gamma(r/a)/a) for
 *     them, and the exact 1/r = g* + gamma(r/a)/a is subtracted, leaving only
 *     the grid's interpolation error of the smooth part;
 *   - a Lennard-Jones 12-6 interaction between flagged sites within the
 *     cutoff a, shifted so it is zero at a;
 *   - rigid O-H and H-H distances, imposed by SHAKE/RATTLE;
 *   - a harmonic flat-bottom wall keeping atoms inside the open domain (the
 *     paper states no boundary conditions): an atom closer than wall_w to a
 *     face of the box gets 1/2 wall_k (wall_w - distance)^2 (wall_k = 0: off).
 * The electrostatics is the MSM (method 0) or, for a coarse propagator, one
 * of the cutoff methods of orc_cutoff (1 simple cutoff, 2 Wolf summation with
 * damping wolf_alpha), which skip the intramolecular pairs instead of
 * subtracting them.
 * mdp = {a, h, k_e, lj_sigma, lj_epsilon, d_oh, d_hh, wall_k, wall_w, method, wolf_alpha, mts}
 * (mts: the multiple-time-step factor of md_steps). */
typedef struct {
    double a, h, ke, sigma, eps, d_oh, d_hh, wall_k, wall_w, alpha;
    int method;
    int mts;            /* fast steps per slow step (<= 1: plain velocity Verlet) */
    int l;
    int64_t n, n_mol;
    const double *q, *m;
    const unsigned char *lj;
    const double *box;
} orc_model;

static void model_from(orc_model *md, const double *mdp, int l, int64_t n, int64_t n_mol,
                       const double *q, const double *m, const unsigned char *lj, const double *box)
{
    md->a = mdp[0]; md->h = mdp[1]; md->ke = mdp[2]; md->sigma = mdp[3]; md->eps = mdp[4];
    md->d_oh = mdp[5]; md->d_hh = mdp[6]; md->wall_k = mdp[7]; md->wall_w = mdp[8];
    md->method = (int)mdp[9]; md->alpha = mdp[10]; md->mts = (int)mdp[11];
    md->l = l; md->n = n; md->n_mol = n_mol;
    md->q = q; md->m = m; md->lj = lj; md->box = box;
}

/* The water completion's Lennard-Jones and wall terms, added to *dU_out and F. */
static int add_lj_wall(const orc_model *md, const double *x, double *dU_out, double *F)
{
    int64_t n = md->n;
    double dU = *dU_out;            /* continues the caller's sum in its order */
    /* Lennard-Jones between flagged sites within a (all pairs of flagged sites) */
    if (md->lj && md->eps != 0.0) {
        double s2 = md->sigma * md->sigma, a2 = md->a * md->a;
        double sa6 = (s2 / a2) * (s2 / a2) * (s2 / a2);
        double eshift = 4.0 * md->eps * (sa6 * sa6 - sa6);
        int64_t nl = 0;
        int64_t *idx = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        double *fl = calloc(3 * (size_t)(n > 0 ? n : 1), sizeof(double));
        double *el = calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        if (!idx || !fl || !el) { free(idx); free(fl); free(el); return ORC_ENOMEM; }
        for (int64_t i = 0; i < n; i++) if (md->lj[i]) idx[nl++] = i;
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t u = 0; u < nl; u++) {
            int64_t i = idx[u];
            double e = 0, fx = 0, fy = 0, fz = 0;
            for (int64_t w = 0; w < nl; w++) {
                int64_t j = idx[w];
                if (j == i) continue;
                double dx = x[3 * i] - x[3 * j], dy = x[3 * i + 1] - x[3 * j + 1], dz = x[3 * i + 2] - x[3 * j + 2];
                double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 >= a2) continue;
                double sr6 = (s2 / r2) * (s2 / r2) * (s2 / r2);
                e += 4.0 * md->eps * (sr6 * sr6 - sr6) - eshift;
                double s = 24.0 * md->eps * (2.0 * sr6 * sr6 - sr6) / r2;
                fx += s * dx; fy += s * dy; fz += s * dz;
            }
            el[i] = e; fl[3 * i] = fx; fl[3 * i + 1] = fy; fl[3 * i + 2] = fz;
        }
        for (int64_t u = 0; u < nl; u++) {
            int64_t i = idx[u];
            dU += 0.5 * el[i];
            F[3 * i] += fl[3 * i]; F[3 * i + 1] += fl[3 * i + 1]; F[3 * i + 2] += fl[3 * i + 2];
        }
        free(idx); free(fl); free(el);
    }
    /* flat-bottom wall on each face of the box */
    if (md->wall_k > 0.0) {
        for (int64_t i = 0; i < n; i++)
            for (int d = 0; d < 3; d++) {
                double dist_lo = x[3 * i + d] - md->box[d];
                double dist_hi = (md->box[d] + md->box[3 + d]) - x[3 * i + d];
                if (dist_lo < md->wall_w) {
                    double pen = md->wall_w - dist_lo;
                    dU += 0.5 * md->wall_k * pen * pen;
                    F[3 * i + d] += md->wall_k * pen;
                }
                if (dist_hi < md->wall_w) {
                    double pen = md->wall_w - dist_hi;
                    dU += 0.5 * md->wall_k * pen * pen;
                    F[3 * i + d] -= md->wall_k * pen;
                }
            }
    }
    *dU_out = dU;
    return ORC_OK;
}

static int model_forces(const orc_model *md, const double *x, double *U, double *F, double *pot)
{
    double prm[3] = {md->a, md->h, md->ke};
    int64_t n = md->n;
    double *phi = pot ? pot : malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!phi) return ORC_ENOMEM;
    int rc;
    if (md->method == ORC_METHOD_MSM) {
        rc = orc_msm(prm, md->l, n, x, md->q, md->box, U, F, phi, NULL);
    } else {
        /* the cutoff methods need no grid, but atoms must still lie in the open
         * domain (the binning contract, the same for every method) */
        int64_t *key = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        if (!key) { if (!pot) free(phi); return ORC_ENOMEM; }
        rc = orc_bin(n, x, md->box, md->h, NULL, key, NULL, NULL);
        free(key);
        if (rc == ORC_OK) rc = orc_cutoff(md->method, md->a, md->alpha, md->ke, n, md->n_mol, x, md->q, U, F, phi);
    }
    if (rc) { if (!pot) free(phi); return rc; }
    double dU = 0;
    /* intramolecular exclusions (MSM only: the cutoff methods skipped these pairs):
     * subtract k_e q_i q_j / r for (O,H1), (O,H2), (H1,H2) */
    for (int64_t mo = 0; md->method == ORC_METHOD_MSM && mo < md->n_mol; mo++) {
        static const int pi[3] = {0, 0, 1}, pj[3] = {1, 2, 2};
        for (int c = 0; c < 3; c++) {
            int64_t i = 3 * mo + pi[c], j = 3 * mo + pj[c];
            double dx = x[3 * i] - x[3 * j], dy = x[3 * i + 1] - x[3 * j + 1], dz = x[3 * i + 2] - x[3 * j + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double e = md->ke * md->q[i] * md->q[j] / r;
            dU -= e;
            phi[i] -= md->ke * md->q[j] / r;
            phi[j] -= md->ke * md->q[i] / r;
            double s = e / (r * r);
            F[3 * i] -= s * dx; F[3 * i + 1] -= s * dy; F[3 * i + 2] -= s * dz;
            F[3 * j] += s * dx; F[3 * j + 1] += s * dy; F[3 * j + 2] += s * dz;
        }
    }
    rc = add_lj_wall(md, x, &dU, F);
    if (rc) { if (!pot) free(phi); return rc; }
    *U += dU;
    if (!pot) free(phi);
    return ORC_OK;
}

/* The forces of the model split for multiple time stepping.  Sec. 3 notes that
 * the MSM uses a multiple-time-step integrator well: its short-range part g*
 * changes on the time scale of the atoms' collisions, its grid part is smooth
 * and changes slowly.  Reading: the fast part Ff is the short-range g* sum over
 * the non-excluded pairs, the Lennard-Jones term and the wall; the slow part Fs
 * is the grid part -k_e q_i grad u^long(r_i) minus the smooth part
 * k_e q_i q_j gamma(r/a)/a of each excluded pair (which the grids carry and the
 * exclusion removes).  U is the whole energy, as model_forces gives it, and Us
 * its slow part 1/2 sum_i q_i k_e (u_i^long - q_i gamma(0)/a) minus the
 * excluded pairs' smooth energies.  MSM method only. */
static int model_forces_split(const orc_model *md, const double *x, double *U, double *Us, double *Ff, double *Fs)
{
    int64_t n = md->n;
    size_t nn = (size_t)(n > 0 ? n : 1);
    double prm[3] = {md->a, md->h, md->ke};
    double ke = md->ke, a = md->a;
    double *ps = malloc(sizeof(double) * nn), *fs = malloc(sizeof(double) * 3 * nn);
    double *pl = malloc(sizeof(double) * nn), *gl = malloc(sizeof(double) * 3 * nn);
    if (!ps || !fs || !pl || !gl) { free(ps); free(fs); free(pl); free(gl); return ORC_ENOMEM; }
    orc_stage_out st = {ps, fs, pl, gl, NULL, NULL, NULL};
    int rc = orc_msm(prm, md->l, n, x, md->q, md->box, NULL, NULL, NULL, &st);
    if (rc) { free(ps); free(fs); free(pl); free(gl); return rc; }
    double self = orc_gamma(0.0) / a, u = 0, us = 0;
    for (int64_t i = 0; i < n; i++) {
        double qi = md->q[i];
        u += qi * (ke * (ps[i] + pl[i] - qi * self));
        us += qi * (ke * (pl[i] - qi * self));
        for (int d = 0; d < 3; d++) {
            Ff[3 * i + d] = ke * fs[3 * i + d];
            Fs[3 * i + d] = -ke * qi * gl[3 * i + d];
        }
    }
    double dU = 0.5 * u, dUs = 0.5 * us;
    /* exclusions: 1/r = g*(r) + gamma(r/a)/a; the g* part leaves the fast
     * forces, the smooth part the slow ones, the whole 1/r the energy */
    for (int64_t mo = 0; mo < md->n_mol; mo++) {
        static const int pi[3] = {0, 0, 1}, pj[3] = {1, 2, 2};
        for (int c = 0; c < 3; c++) {
            int64_t i = 3 * mo + pi[c], j = 3 * mo + pj[c];
            double dx = x[3 * i] - x[3 * j], dy = x[3 * i + 1] - x[3 * j + 1], dz = x[3 * i + 2] - x[3 * j + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double qq = ke * md->q[i] * md->q[j];
            dU -= qq / r;
            dUs -= qq * orc_gamma(r / a) / a;
            /* removing energy e(r) adds e'(r) (r_i - r_j)/r to F_i */
            double sf = qq * orc_dgstar(r, a) / r, ss = qq * orc_dgamma(r / a) / (a * a) / r;
            Ff[3 * i] += sf * dx; Ff[3 * i + 1] += sf * dy; Ff[3 * i + 2] += sf * dz;
            Ff[3 * j] -= sf * dx; Ff[3 * j + 1] -= sf * dy; Ff[3 * j + 2] -= sf * dz;
            Fs[3 * i] += ss * dx; Fs[3 * i + 1] += ss * dy; Fs[3 * i + 2] += ss * dz;
            Fs[3 * j] -= ss * dx; Fs[3 * j + 1] -= ss * dy; Fs[3 * j + 2] -= ss * dz;
        }
    }
    free(ps); free(fs); free(pl); free(gl);
    rc = add_lj_wall(md, x, &dU, Ff);
    if (rc) return rc;
    *U = dU;
    *Us = dUs;
    return ORC_OK;
}

/* The split forces of the model (see model_forces_split): U, Us, Ff, Fs. */
int orc_model_forces_split(const double *mdp, int l, int64_t n, int64_t n_mol, const double *x, const double *q,
                           const unsigned char *lj, const double *box, double *energy, double *energy_slow,
                           double *f_fast, double *f_slow)
{
    orc_model md;
    model_from(&md, mdp, l, n, n_mol, q, NULL, lj, box);
    if (md.method != ORC_METHOD_MSM) return ORC_EINVAL;
    return model_forces_split(&md, x, energy, energy_slow, f_fast, f_slow);
}

/* Energy and forces of the water model (MSM + exclusions + LJ). */
int orc_model_forces(const double *mdp, int l, int64_t n, int64_t n_mol, const double *x, const double *q,
                     const unsigned char *lj, const double *box, double *energy, double *forces, double *pot)
{
    orc_model md;
    model_from(&md, mdp, l, n, n_mol, q, NULL, lj, box);
    return model_forces(&md, x, energy, forces, pot);
}

/* SHAKE (Ryckaert, Ciccotti & Berendsen 1977): move the unconstrained new
 * positions xn along the old bond vectors until |xn_i - xn_j| = d for the
 * three bonds of every triple, one bond at a time, repeated until all hold to
 * a relative 1e-12 in d^2.  vh receives the matching velocity change. */
static int shake(const orc_model *md, const double *xo, double *xn, double *vh, double dt)
{
    static const int pi[3] = {0, 0, 1}, pj[3] = {1, 2, 2};
    const double d2[3] = {md->d_oh * md->d_oh, md->d_oh * md->d_oh, md->d_hh * md->d_hh};
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t mo = 0; mo < md->n_mol; mo++) {
        int it, ok = 0;
        for (it = 0; it < 1000 && !ok; it++) {
            ok = 1;
            for (int c = 0; c < 3; c++) {
                int64_t i = 3 * mo + pi[c], j = 3 * mo + pj[c];
                double rn[3], ro[3], rn2 = 0, dot = 0;
                for (int d = 0; d < 3; d++) { rn[d] = xn[3 * i + d] - xn[3 * j + d]; rn2 += rn[d] * rn[d]; }
                double diff = d2[c] - rn2;
                if (fabs(diff) <= 1e-12 * d2[c]) continue;
                ok = 0;
                for (int d = 0; d < 3; d++) { ro[d] = xo[3 * i + d] - xo[3 * j + d]; dot += ro[d] * rn[d]; }
                double wi = 1.0 / md->m[i], wj = 1.0 / md->m[j];
                double g = diff / (2.0 * dot * (wi + wj));
                for (int d = 0; d < 3; d++) {
                    xn[3 * i + d] += g * wi * ro[d]; xn[3 * j + d] -= g * wj * ro[d];
                    vh[3 * i + d] += g * wi * ro[d] / dt; vh[3 * j + d] -= g * wj * ro[d] / dt;
                }
            }
        }
        if (!ok) bad += 1;
    }
    return bad ? ORC_ENOCONV : ORC_OK;
}

/* RATTLE velocity stage (Andersen 1983): remove the velocity component along
 * each bond, (v_i - v_j).(x_i - x_j) = 0, one bond at a time, repeated until
 * every |(v_i - v_j).(x_i - x_j)| <= 1e-14 nm^2/ps. */
static int rattle_v(const orc_model *md, const double *x, double *v)
{
    static const int pi[3] = {0, 0, 1}, pj[3] = {1, 2, 2};
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t mo = 0; mo < md->n_mol; mo++) {
        int it, ok = 0;
        for (it = 0; it < 1000 && !ok; it++) {
            ok = 1;
            for (int c = 0; c < 3; c++) {
                int64_t i = 3 * mo + pi[c], j = 3 * mo + pj[c];
                double r[3], r2 = 0, rv = 0;
                for (int d = 0; d < 3; d++) {
                    r[d] = x[3 * i + d] - x[3 * j + d];
                    r2 += r[d] * r[d];
                    rv += r[d] * (v[3 * i + d] - v[3 * j + d]);
                }
                if (fabs(rv) <= 1e-14) continue;
                ok = 0;
                double wi = 1.0 / md->m[i], wj = 1.0 / md->m[j];
                double k = rv / (r2 * (wi + wj));
                for (int d = 0; d < 3; d++) { v[3 * i + d] -= k * wi * r[d]; v[3 * j + d] += k * wj * r[d]; }
            }
        }
        if (!ok) bad += 1;
    }
    return bad ? ORC_ENOCONV : ORC_OK;
}

static double kinetic(int64_t n, const double *m, const double *v)
{
    double K = 0;
    for (int64_t i = 0; i < n; i++) K += 0.5 * m[i] * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
    return K;
}

static int md_steps_mts(const orc_model *md, double *x, double *v, double dt, int n_steps, double *uk);

static int md_steps(const orc_model *md, double *x, double *v, double dt, int n_steps, double *uk)
{
    if (md->mts > 1) return md_steps_mts(md, x, v, dt, n_steps, uk);
    int64_t n = md->n;
    double *F = malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *xo = malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!F || !xo) { free(F); free(xo); return ORC_ENOMEM; }
    double U;
    int rc = model_forces(md, x, &U, F, NULL);
    if (rc) goto out;
    if (uk) { uk[0] = U; uk[1] = kinetic(n, md->m, v); }
    for (int s = 0; s < n_steps; s++) {
        memcpy(xo, x, sizeof(double) * 3 * (size_t)n);
        for (int64_t i = 0; i < n; i++)                       /* half kick, drift */
            for (int d = 0; d < 3; d++) {
                v[3 * i + d] += 0.5 * dt * F[3 * i + d] / md->m[i];
                x[3 * i + d] += dt * v[3 * i + d];
            }
        rc = shake(md, xo, x, v, dt);
        if (rc) goto out;
        rc = model_forces(md, x, &U, F, NULL);                 /* forces at the new positions */
        if (rc) goto out;
        for (int64_t i = 0; i < n; i++)                        /* second half kick */
            for (int d = 0; d < 3; d++) v[3 * i + d] += 0.5 * dt * F[3 * i + d] / md->m[i];
        rc = rattle_v(md, x, v);
        if (rc) goto out;
        if (uk) { uk[2 * (s + 1)] = U; uk[2 * (s + 1) + 1] = kinetic(n, md->m, v); }
    }
out:
    free(F); free(xo);
    return rc;
}

/* Multiple time stepping (Sec. 3: the MSM suits a multiple-time-step
 * integrator), as the impulse method (Grubmueller et al. 1991; Tuckerman,
 * Berne & Martyna 1992, "r-RESPA") restated with SHAKE/RATTLE: an outer step
 * of k = mts fast steps of dt.  The slow force Fs acts as two impulses of
 * k dt/2, at the start and the end of the outer step, each folded into the
 * adjacent half kick of the fast velocity Verlet step, which then uses
 * Ff + k Fs (a RATTLE half step with that force); the inner half kicks use Ff
 * alone.  Fs is evaluated at the end of each outer step only.  n_steps must
 * be a multiple of k.  uk records (U, K) after every step, U being the fast
 * energy at the current positions plus the slow energy of the last slow
 * evaluation (at the ends of outer steps: the whole energy). */
static int md_steps_mts(const orc_model *md, double *x, double *v, double dt, int n_steps, double *uk)
{
    int64_t n = md->n;
    const int k = md->mts;
    if (md->method != ORC_METHOD_MSM || n_steps % k != 0) return ORC_EINVAL;
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *Ff = malloc(sizeof(double) * 3 * nn), *Fs = malloc(sizeof(double) * 3 * nn);
    double *Gs = malloc(sizeof(double) * 3 * nn), *xo = malloc(sizeof(double) * 3 * nn);
    if (!Ff || !Fs || !Gs || !xo) { free(Ff); free(Fs); free(Gs); free(xo); return ORC_ENOMEM; }
    double U, Us, Ut, Ust;
    int rc = model_forces_split(md, x, &U, &Us, Ff, Fs);
    if (rc) goto out;
    if (uk) { uk[0] = U; uk[1] = kinetic(n, md->m, v); }
    for (int s = 0; s < n_steps; s++) {
        const int first = s % k == 0, last = s % k == k - 1;
        memcpy(xo, x, sizeof(double) * 3 * (size_t)n);
        for (int64_t i = 0; i < n; i++)                       /* half kick (+ slow impulse), drift */
            for (int d = 0; d < 3; d++) {
                double f = first ? Ff[3 * i + d] + (double)k * Fs[3 * i + d] : Ff[3 * i + d];
                v[3 * i + d] += 0.5 * dt * f / md->m[i];
                x[3 * i + d] += dt * v[3 * i + d];
            }
        rc = shake(md, xo, x, v, dt);
        if (rc) goto out;
        /* the oracle evaluates both parts every step and keeps the slow one only at
         * the ends of outer steps */
        rc = model_forces_split(md, x, &Ut, &Ust, Ff, Gs);
        if (rc) goto out;
        if (last) { memcpy(Fs, Gs, sizeof(double) * 3 * (size_t)n); U = Ut; Us = Ust; }
        else U = (Ut - Ust) + Us;
        for (int64_t i = 0; i < n; i++)                        /* second half kick (+ slow impulse) */
            for (int d = 0; d < 3; d++) {
                double f = last ? Ff[3 * i + d] + (double)k * Fs[3 * i + d] : Ff[3 * i + d];
                v[3 * i + d] += 0.5 * dt * f / md->m[i];
            }
        rc = rattle_v(md, x, v);
        if (rc) goto out;
        if (uk) { uk[2 * (s + 1)] = U; uk[2 * (s + 1) + 1] = kinetic(n, md->m, v); }
    }
out:
    free(Ff); free(Fs); free(Gs); free(xo);
    return rc;
}

/* Velocity Verlet (Sec. 2: forces F = -dU/dr, then move the atoms) with
 * SHAKE/RATTLE for the rigid triples.  x, v are updated in place.  uk, if
 * non-NULL, receives (U, K) before the first step and after each step. */
int orc_md_run(const double *mdp, int l, int64_t n, int64_t n_mol, double *x, double *v,
               const double *q, const double *m, const unsigned char *lj, const double *box,
               double dt, int n_steps, double *uk)
{
    orc_model md;
    model_from(&md, mdp, l, n, n_mol, q, m, lj, box);
    return md_steps(&md, x, v, dt, n_steps, uk);
}

/* Parareal (Sec. 4).  State lambda = (x, v).  Slice n maps lambda_n at T_n to
 * lambda_{n+1} (0-based; lambda_0 = state0 is exact in every iteration).
 *   init:      lambda^0_{n+1} = G(lambda^0_n), sequentially;
 *   iteration: f_n = F(lambda^k_n) for all n (independent), then sequentially
 *              lambda^{k+1}_{n+1} = f_n + (G(lambda^{k+1}_n) - G(lambda^k_n))
 *              (this evaluation order: when lambda^{k+1}_n equals lambda^k_n
 *              bitwise the bracket is exactly 0 and slice n+1 equals F);
 *   stop when max_{n,i,d} |x^{k+1} - x^k| <= tol, or after max_iter iterations.
 * slices_x/v: (n_slices+1) * n * 3, slot 0 holds state0 on entry.
 * gp/fp: {mdp (12 values), dt, steps, levels}. */
/* Parareal's correction F + (G_new - G_old) adds positions of rigid molecules
 * taken from different trajectories, so the corrected molecules need not have
 * the rigid bond lengths; a grossly distorted one would start the next coarse
 * propagation outside SHAKE's reach.  Reading for the water completion (the
 * paper has no constraints): every molecule whose squared bond lengths miss
 * the rigid ones by more than 10x the SHAKE tolerance (1e-11 relative) is
 * projected back -- positions by SHAKE iterations along the molecule's own
 * current bond vectors with inverse-mass weights, until every bond is within
 * 1e-12 relative, then velocities by the RATTLE velocity stage.  Molecules
 * within the threshold are left untouched, bit for bit, so states the fine
 * propagator produced pass through unchanged. */
static int project_rigid(const orc_model *md, double *x, double *v)
{
    static const int pi[3] = {0, 0, 1}, pj[3] = {1, 2, 2};
    const double d2[3] = {md->d_oh * md->d_oh, md->d_oh * md->d_oh, md->d_hh * md->d_hh};
    int bad = 0;
    for (int64_t mo = 0; mo < md->n_mol; mo++) {
        int off = 0;
        for (int c = 0; c < 3; c++) {
            int64_t i = 3 * mo + pi[c], j = 3 * mo + pj[c];
            double r2 = 0;
            for (int d = 0; d < 3; d++) { double t = x[3 * i + d] - x[3 * j + d]; r2 += t * t; }
            if (fabs(d2[c] - r2) > 1e-11 * d2[c]) off = 1;
        }
        if (!off) continue;
        int it, ok = 0;
        for (it = 0; it < 1000 && !ok; it++) {
            ok = 1;
            for (int c = 0; c < 3; c++) {
                int64_t i = 3 * mo + pi[c], j = 3 * mo + pj[c];
                double r[3], r2 = 0;
                for (int d = 0; d < 3; d++) { r[d] = x[3 * i + d] - x[3 * j + d]; r2 += r[d] * r[d]; }
                double diff = d2[c] - r2;
                if (fabs(diff) <= 1e-12 * d2[c]) continue;
                ok = 0;
                double wi = 1.0 / md->m[i], wj = 1.0 / md->m[j];
                double g = diff / (2.0 * r2 * (wi + wj));
                for (int d = 0; d < 3; d++) { x[3 * i + d] += g * wi * r[d]; x[3 * j + d] -= g * wj * r[d]; }
            }
        }
        if (!ok) { bad += 1; continue; }
        for (it = 0, ok = 0; it < 1000 && !ok; it++) {
            ok = 1;
            for (int c = 0; c < 3; c++) {
                int64_t i = 3 * mo + pi[c], j = 3 * mo + pj[c];
                double r[3], r2 = 0, rv = 0;
                for (int d = 0; d < 3; d++) {
                    r[d] = x[3 * i + d] - x[3 * j + d];
                    r2 += r[d] * r[d];
                    rv += r[d] * (v[3 * i + d] - v[3 * j + d]);
                }
                if (fabs(rv) <= 1e-14) continue;
                ok = 0;
                double wi = 1.0 / md->m[i], wj = 1.0 / md->m[j];
                double k = rv / (r2 * (wi + wj));
                for (int d = 0; d < 3; d++) { v[3 * i + d] -= k * wi * r[d]; v[3 * j + d] += k * wj * r[d]; }
            }
        }
        if (!ok) bad += 1;
    }
    return bad ? ORC_ENOCONV : ORC_OK;
}

/* The projection alone, for its tests: n_mol leading triples of x, v (in place). */
int orc_project_rigid(int64_t n, int64_t n_mol, const double *m, double d_oh, double d_hh, double *x, double *v)
{
    orc_model md;
    memset(&md, 0, sizeof md);
    md.n = n; md.n_mol = n_mol; md.m = m; md.d_oh = d_oh; md.d_hh = d_hh;
    return project_rigid(&md, x, v);
}

int orc_parareal(const double *gp, const double *fp, int64_t n, int64_t n_mol,
                 const double *q, const double *m, const unsigned char *lj, const double *box,
                 int n_slices, int max_iter, double tol, double *slices_x, double *slices_v,
                 int *iters_done, double *last_dx)
{
    orc_model G, F;
    model_from(&G, gp, (int)gp[14], n, n_mol, q, m, lj, box);
    model_from(&F, fp, (int)fp[14], n, n_mol, q, m, lj, box);
    double dtG = gp[12], dtF = fp[12];
    int sG = (int)gp[13], sF = (int)fp[13];
    size_t sz = 3 * (size_t)n;
    int rc = ORC_OK;
    double *gold_x = malloc(sizeof(double) * sz * (size_t)n_slices), *gold_v = malloc(sizeof(double) * sz * (size_t)n_slices);
    double *f_x = malloc(sizeof(double) * sz * (size_t)n_slices), *f_v = malloc(sizeof(double) * sz * (size_t)n_slices);
    double *nx = malloc(sizeof(double) * sz * (size_t)(n_slices + 1)), *nv = malloc(sizeof(double) * sz * (size_t)(n_slices + 1));
    double *tx = malloc(sizeof(double) * sz), *tv = malloc(sizeof(double) * sz);
    if (!gold_x || !gold_v || !f_x || !f_v || !nx || !nv || !tx || !tv) { rc = ORC_ENOMEM; goto out; }
    for (int s = 0; s < n_slices; s++) {                                   /* init row */
        memcpy(tx, slices_x + sz * s, sizeof(double) * sz);
        memcpy(tv, slices_v + sz * s, sizeof(double) * sz);
        if ((rc = md_steps(&G, tx, tv, dtG, sG, NULL))) goto out;
        memcpy(gold_x + sz * s, tx, sizeof(double) * sz); memcpy(gold_v + sz * s, tv, sizeof(double) * sz);
        memcpy(slices_x + sz * (s + 1), tx, sizeof(double) * sz); memcpy(slices_v + sz * (s + 1), tv, sizeof(double) * sz);
    }
    *iters_done = 0;
    *last_dx = INFINITY;
    for (int k = 0; k < max_iter; k++) {
        for (int s = 0; s < n_slices; s++) {                               /* f_n = F(lambda^k_n) */
            memcpy(f_x + sz * s, slices_x + sz * s, sizeof(double) * sz);
            memcpy(f_v + sz * s, slices_v + sz * s, sizeof(double) * sz);
            if ((rc = md_steps(&F, f_x + sz * s, f_v + sz * s, dtF, sF, NULL))) goto out;
        }
        memcpy(nx, slices_x, sizeof(double) * sz);
        memcpy(nv, slices_v, sizeof(double) * sz);
        for (int s = 0; s < n_slices; s++) {                               /* sequential correction */
            memcpy(tx, nx + sz * s, sizeof(double) * sz);
            memcpy(tv, nv + sz * s, sizeof(double) * sz);
            /* a coarse propagation that breaks down on a corrected state means the
             * iteration diverged: stop with the last complete iterate in slices_x/v */
            if (md_steps(&G, tx, tv, dtG, sG, NULL)) { rc = ORC_ENOCONV; goto out; }
            for (size_t e = 0; e < sz; e++) {
                nx[sz * (s + 1) + e] = f_x[sz * s + e] + (tx[e] - gold_x[sz * s + e]);
                nv[sz * (s + 1) + e] = f_v[sz * s + e] + (tv[e] - gold_v[sz * s + e]);
            }
            if ((rc = project_rigid(&F, nx + sz * (s + 1), nv + sz * (s + 1)))) goto out;
            memcpy(gold_x + sz * s, tx, sizeof(double) * sz); memcpy(gold_v + sz * s, tv, sizeof(double) * sz);
        }
        double dx = 0;
        for (size_t e = 0; e < sz * (size_t)(n_slices + 1); e++) { double t = fabs(nx[e] - slices_x[e]); if (t > dx) dx = t; }
        memcpy(slices_x, nx, sizeof(double) * sz * (size_t)(n_slices + 1));
        memcpy(slices_v, nv, sizeof(double) * sz * (size_t)(n_slices + 1));
        *iters_done = k + 1;
        *last_dx = dx;
        if (dx <= tol) break;
    }
    if (*last_dx > tol) rc = ORC_ENOCONV;
out:
    free(gold_x); free(gold_v); free(f_x); free(f_v); free(nx); free(nv); free(tx); free(tv);
    return rc;
}

/* Parareal over a sliding computational window (Sec. 4: the iteration runs on
 * a window of T_W time points; Sec. 6.1 sizes the window).  The paper states
 * the window but not how it moves; reading: the window holds slices [b, e),
 * e - b <= W.  Each iteration applies the recurrence of orc_parareal to the
 * window (F of every window slice from the current iterate, then the
 * sequential correction sweep from the window's first state lambda_b, which
 * is final).  A slice n is converged when max |x^{k+1}_{n+1} - x^k_{n+1}| <=
 * tol; b advances past slice b (its end F(lambda_b) is exact once computed)
 * and past the converged slices that follow it, and the window is refilled up
 * to W slices, the new slices' first iterate being the coarse propagation G
 * from the last state of the window.  Stops when b reaches n_slices or after
 * max_iter iterations.  With W = n_slices and tol = 0 the iterates equal
 * orc_parareal's bit for bit (which needs one more iteration to see that the
 * last slice no longer changes); with W = 1 it is the serial fine run.
 * slices_x/v: (n_slices+1) * n * 3, slot 0 = state0 on entry; on return the
 * converged slice ends are final and the rest the last iterate.
 * *iters_done counts iterations, *last_dx is the largest change of the last one. */
int orc_parareal_window(const double *gp, const double *fp, int64_t n, int64_t n_mol,
                        const double *q, const double *m, const unsigned char *lj, const double *box,
                        int n_slices, int window, int max_iter, double tol, double *slices_x, double *slices_v,
                        int *iters_done, double *last_dx)
{
    if (window < 1 || n_slices < 1) return ORC_EINVAL;
    orc_model G, F;
    model_from(&G, gp, (int)gp[14], n, n_mol, q, m, lj, box);
    model_from(&F, fp, (int)fp[14], n, n_mol, q, m, lj, box);
    double dtG = gp[12], dtF = fp[12];
    int sG = (int)gp[13], sF = (int)fp[13];
    const size_t sz = 3 * (size_t)n, ns = (size_t)n_slices;
    int rc = ORC_OK;
    /* per slice n: its coarse propagation of the current iterate (gold), its fine one (f) */
    double *gold_x = malloc(sizeof(double) * sz * ns), *gold_v = malloc(sizeof(double) * sz * ns);
    double *f_x = malloc(sizeof(double) * sz * ns), *f_v = malloc(sizeof(double) * sz * ns);
    double *tx = malloc(sizeof(double) * sz), *tv = malloc(sizeof(double) * sz);
    double *nx = malloc(sizeof(double) * sz), *nv = malloc(sizeof(double) * sz);
    double *dxs = malloc(sizeof(double) * ns);
    if (!gold_x || !gold_v || !f_x || !f_v || !tx || !tv || !nx || !nv || !dxs) { rc = ORC_ENOMEM; goto out; }
    int b = 0, e = 0;
    *iters_done = 0;
    *last_dx = INFINITY;
    for (int k = 0; b < n_slices && k < max_iter; k++) {
        /* fill the window: first iterates of the new slices by G, in order */
        int e_new = b + window < n_slices ? b + window : n_slices;
        for (int s = e; s < e_new; s++) {
            memcpy(tx, slices_x + sz * s, sizeof(double) * sz);
            memcpy(tv, slices_v + sz * s, sizeof(double) * sz);
            if (md_steps(&G, tx, tv, dtG, sG, NULL)) { rc = ORC_ENOCONV; goto out; }
            memcpy(gold_x + sz * s, tx, sizeof(double) * sz); memcpy(gold_v + sz * s, tv, sizeof(double) * sz);
            memcpy(slices_x + sz * (s + 1), tx, sizeof(double) * sz);
            memcpy(slices_v + sz * (s + 1), tv, sizeof(double) * sz);
        }
        e = e_new;
        for (int s = b; s < e; s++) {                                      /* f_n = F(lambda^k_n) */
            memcpy(f_x + sz * s, slices_x + sz * s, sizeof(double) * sz);
            memcpy(f_v + sz * s, slices_v + sz * s, sizeof(double) * sz);
            if ((rc = md_steps(&F, f_x + sz * s, f_v + sz * s, dtF, sF, NULL))) goto out;
        }
        /* sequential correction over the window, from its final first state */
        memcpy(nx, slices_x + sz * b, sizeof(double) * sz);
        memcpy(nv, slices_v + sz * b, sizeof(double) * sz);
        double dmax = 0;
        for (int s = b; s < e; s++) {
            memcpy(tx, nx, sizeof(double) * sz);
            memcpy(tv, nv, sizeof(double) * sz);
            if (md_steps(&G, tx, tv, dtG, sG, NULL)) { rc = ORC_ENOCONV; goto out; }
            for (size_t c = 0; c < sz; c++) {
                nx[c] = f_x[sz * s + c] + (tx[c] - gold_x[sz * s + c]);
                nv[c] = f_v[sz * s + c] + (tv[c] - gold_v[sz * s + c]);
            }
            if ((rc = project_rigid(&F, nx, nv))) goto out;
            double d = 0;
            for (size_t c = 0; c < sz; c++) { double t = fabs(nx[c] - slices_x[sz * (s + 1) + c]); if (t > d) d = t; }
            dxs[s] = d;
            if (d > dmax) dmax = d;
            memcpy(gold_x + sz * s, tx, sizeof(double) * sz); memcpy(gold_v + sz * s, tv, sizeof(double) * sz);
            memcpy(slices_x + sz * (s + 1), nx, sizeof(double) * sz);
            memcpy(slices_v + sz * (s + 1), nv, sizeof(double) * sz);
        }
        *iters_done = k + 1;
        *last_dx = dmax;
        b++;                                   /* slice b's end F(lambda_b) is exact: final */
        while (b < e && dxs[b] <= tol) b++;    /* and the converged slices that follow it */
    }
    if (b < n_slices) rc = ORC_ENOCONV;
out:
    free(gold_x); free(gold_v); free(f_x); free(f_v); free(tx); free(tv); free(nx); free(nv); free(dxs);
    return rc;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the OpenMP loops from now on (results do not depend on it). */
void orc_set_num_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}
