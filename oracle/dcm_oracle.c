/*
 * dcm_oracle.c -- plain FP64 CPU oracle of the dynamic cutoff method.
 *
 * TEST INFRASTRUCTURE ONLY (see dcm_oracle.h).  Written from the thesis's
 * equations and algorithms; nothing here is shared with the CUDA library.
 * Compile with -ffp-contract=off so that no expression is fused.
 *
 * Parity pins (tests/test_oracle_*.py) tie every routine here to something
 * other than itself: closed-form LJ facts, Eq. 8 identities, brute force,
 * Newton's third law in the static limit, hand-solved Godunov values,
 * binomial coefficients, the global optimum of Eq. 14 on bimodal data, and
 * an independent ODE integration for the integrator.
 */
#include "dcm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

int orc_set_threads(int nthreads)
{
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
    g_threads = nthreads;
#else
    g_threads = 1;
#endif
    return g_threads;
}

int orc_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------------ */
/* Eq. 4 */
void orc_lj(double r, double eps, double sigma, double *V, double *fr)
{
    double s = sigma / r;
    double s2 = s * s;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    if (V) *V = 4.0 * eps * (s12 - s6);
    /* -V'(r)/r = 24 eps (2 (sigma/r)^12 - (sigma/r)^6) / r^2 */
    if (fr) *fr = 24.0 * eps * (2.0 * s12 - s6) / (r * r);
}

/* Eq. 7 with the constants of Eq. 8 */
double orc_cutoff(double d, double rc_min, double rc_max, double alpha)
{
    if (d <= 0.0) return rc_max;
    if (d >= rc_max) return rc_min;
    double a = (rc_max - rc_min) / (pow(2.0, alpha * rc_max) - 1.0);
    double b = rc_min - a;
    return a * pow(2.0, alpha * (rc_max - d)) + b;
}

void orc_class_thresholds(double rc_min, double rc_max, double alpha, int K,
                          double *thr)
{
    if (K < 3) return;
    double a = (rc_max - rc_min) / (pow(2.0, alpha * rc_max) - 1.0);
    double b = rc_min - a;
    for (int k = 1; k <= K - 2; ++k) {
        double r = rc_min + (rc_max - rc_min) * (double)k / (double)(K - 1);
        /* invert Eq. 7: d = rc_max - log2((r - b)/a) / alpha */
        thr[k - 1] = rc_max - log2((r - b) / a) / alpha;
    }
}

/* Section 3.1, Fig. 12: the "linear" cutoff function, read as the straight
 * line from (0, rc_max) to (rc_max, rc_min), with the same outer cases as
 * Eq. 7 */
double orc_cutoff_linear(double d, double rc_min, double rc_max)
{
    if (d <= 0.0) return rc_max;
    if (d >= rc_max) return rc_min;
    return rc_max - (rc_max - rc_min) * d / rc_max;
}

/* class edges of the linear function: d(r_k) = (rc_max - r_k) rc_max / (rc_max - rc_min) */
void orc_class_thresholds_linear(double rc_min, double rc_max, int K, double *thr)
{
    if (K < 3) return;
    for (int k = 1; k <= K - 2; ++k) {
        double r = rc_min + (rc_max - rc_min) * (double)k / (double)(K - 1);
        thr[k - 1] = (rc_max - r) * rc_max / (rc_max - rc_min);
    }
}

int orc_cutoff_class(double d, double rc_max, int K, const double *thr)
{
    if (d >= rc_max) return 0;
    int c = 1;
    for (int k = 0; k < K - 2; ++k)
        if (d < thr[k]) c++;
    return c;
}

/* ------------------------------------------------------------------------ */
void orc_grid_dims(const double L[3], double b, int dims[3])
{
    for (int a = 0; a < 3; ++a) {
        int n = (int)floor(L[a] / b);
        dims[a] = n < 3 ? 3 : n;
    }
}

void orc_cell_dims(const double L[3], double c, int nc[3])
{
    for (int a = 0; a < 3; ++a) {
        int n = (int)floor(L[a] / c);
        nc[a] = n < 1 ? 1 : n;
    }
}

int orc_bin_index(double x, int n, double L)
{
    double inv = (double)n / L;
    int k = (int)floor(x * inv);
    if (k > n - 1) k = n - 1;
    if (k < 0) k = 0;
    return k;
}

double orc_wrap(double x, double L)
{
    if (x < 0.0) x += L;
    if (x >= L) x -= L;
    return x;
}

static inline double min_image(double dx, double L)
{
    if (dx > 0.5 * L) return dx - L;
    if (dx < -0.5 * L) return dx + L;
    return dx;
}

/* ------------------------------------------------------------------------ */
/* link cells (Section 2.2.1): counting sort by cell, ascending id */
void orc_cell_list(int64_t n, const double *x, const double L[3], const int nc[3],
                   int32_t *cell_of, int32_t *cell_start, int32_t *sorted_id)
{
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int32_t *cursor = (int32_t *)calloc((size_t)ncell + 1, sizeof(int32_t));
    for (int64_t c = 0; c <= ncell; ++c) cell_start[c] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int cx = orc_bin_index(x[3 * i + 0], nc[0], L[0]);
        int cy = orc_bin_index(x[3 * i + 1], nc[1], L[1]);
        int cz = orc_bin_index(x[3 * i + 2], nc[2], L[2]);
        int32_t c = (int32_t)(cx + (int64_t)nc[0] * (cy + (int64_t)nc[1] * cz));
        cell_of[i] = c;
        cell_start[c + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
    for (int64_t i = 0; i < n; ++i) {
        int32_t c = cell_of[i];
        sorted_id[cell_start[c] + cursor[c]] = (int32_t)i;
        cursor[c]++;
    }
    free(cursor);
}

/* one pair of Algorithm 3.2: adds the contribution of j to particle i */
static inline int dcm_pair(const double *x, int64_t i, int64_t j, double rci2,
                           const double L[3], double eps, double sigma,
                           double fi[3], double *pei, double viri[6])
{
    double dx = min_image(x[3 * i + 0] - x[3 * j + 0], L[0]);
    double dy = min_image(x[3 * i + 1] - x[3 * j + 1], L[1]);
    double dz = min_image(x[3 * i + 2] - x[3 * j + 2], L[2]);
    double r2 = dx * dx + dy * dy + dz * dz;
    if (!(r2 < rci2)) return 0; /* Algorithm 3.2: |r_ij| < r_c[i] */
    double V, fr;
    orc_lj(sqrt(r2), eps, sigma, &V, &fr);
    double fx = fr * dx, fy = fr * dy, fz = fr * dz;
    fi[0] += fx;
    fi[1] += fy;
    fi[2] += fz;
    *pei += 0.5 * V;
    viri[0] += 0.5 * dx * fx;
    viri[1] += 0.5 * dy * fy;
    viri[2] += 0.5 * dz * fz;
    viri[3] += 0.5 * dx * fy;
    viri[4] += 0.5 * dx * fz;
    viri[5] += 0.5 * dy * fz;
    return 1;
}

static int box_ok(const double *rc, int64_t n, const double L[3])
{
    double lmin = L[0];
    if (L[1] < lmin) lmin = L[1];
    if (L[2] < lmin) lmin = L[2];
    for (int64_t i = 0; i < n; ++i)
        if (!(rc[i] < 0.5 * lmin)) return 0;
    return 1;
}

static void finish_outputs(int64_t n, const double *fbuf, const double *pebuf,
                           const double *virbuf, const int32_t *npbuf, double *f,
                           double *pe, double *vir, int32_t *npair)
{
    memcpy(f, fbuf, sizeof(double) * 3 * (size_t)n);
    if (pe) memcpy(pe, pebuf, sizeof(double) * (size_t)n);
    if (npair) memcpy(npair, npbuf, sizeof(int32_t) * (size_t)n);
    if (vir) {
        for (int a = 0; a < 6; ++a) vir[a] = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int a = 0; a < 6; ++a) vir[a] += virbuf[6 * i + a];
    }
}

/* Algorithm 3.2 over the link-cell stencil.  For particle i the cells
 * within s = ceil(rc[i]/c) along each axis are visited (all cells once if
 * 2s+1 >= n); inside them every j != i is tested with the pair rule. */
int orc_forces(int64_t n, const double *x, const double *rc, const double L[3],
               const int nc[3], double eps, double sigma, double *f, double *pe,
               double *vir, int32_t *npair)
{
    if (!box_ok(rc, n, L)) return -1;
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int32_t *cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *start = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncell + 1));
    int32_t *sid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *fbuf = (double *)calloc((size_t)(3 * n + 1), sizeof(double));
    double *pebuf = (double *)calloc((size_t)(n + 1), sizeof(double));
    double *virbuf = (double *)calloc((size_t)(6 * n + 1), sizeof(double));
    int32_t *npbuf = (int32_t *)calloc((size_t)(n + 1), sizeof(int32_t));
    orc_cell_list(n, x, L, nc, cell_of, start, sid);

#pragma omp parallel for schedule(dynamic, 20) num_threads(g_threads)
    for (int64_t i = 0; i < n; ++i) {
        int ci[3], s[3], lo[3], cnt[3];
        int32_t c = cell_of[i];
        ci[0] = (int)(c % nc[0]);
        ci[1] = (int)((c / nc[0]) % nc[1]);
        ci[2] = (int)(c / ((int64_t)nc[0] * nc[1]));
        for (int a = 0; a < 3; ++a) {
            double edge = L[a] / (double)nc[a];
            s[a] = (int)ceil(rc[i] / edge);
            if (2 * s[a] + 1 >= nc[a]) {
                lo[a] = 0;
                cnt[a] = nc[a];
            } else {
                lo[a] = ci[a] - s[a];
                cnt[a] = 2 * s[a] + 1;
            }
        }
        double fi[3] = {0.0, 0.0, 0.0}, pei = 0.0, viri[6] = {0, 0, 0, 0, 0, 0};
        int32_t np = 0;
        double rci2 = rc[i] * rc[i];
        for (int kz = 0; kz < cnt[2]; ++kz) {
            int cz = ((lo[2] + kz) % nc[2] + nc[2]) % nc[2];
            for (int ky = 0; ky < cnt[1]; ++ky) {
                int cy = ((lo[1] + ky) % nc[1] + nc[1]) % nc[1];
                for (int kx = 0; kx < cnt[0]; ++kx) {
                    int cx = ((lo[0] + kx) % nc[0] + nc[0]) % nc[0];
                    int64_t cj = cx + (int64_t)nc[0] * (cy + (int64_t)nc[1] * cz);
                    for (int32_t k = start[cj]; k < start[cj + 1]; ++k) {
                        int64_t j = sid[k];
                        if (j == i) continue;
                        np += dcm_pair(x, i, j, rci2, L, eps, sigma, fi, &pei, viri);
                    }
                }
            }
        }
        for (int a = 0; a < 3; ++a) fbuf[3 * i + a] = fi[a];
        pebuf[i] = pei;
        for (int a = 0; a < 6; ++a) virbuf[6 * i + a] = viri[a];
        npbuf[i] = np;
    }
    finish_outputs(n, fbuf, pebuf, virbuf, npbuf, f, pe, vir, npair);
    free(cell_of);
    free(start);
    free(sid);
    free(fbuf);
    free(pebuf);
    free(virbuf);
    free(npbuf);
    return 0;
}

int orc_forces_brute(int64_t n, const double *x, const double *rc,
                     const double L[3], double eps, double sigma, double *f,
                     double *pe, double *vir, int32_t *npair)
{
    if (!box_ok(rc, n, L)) return -1;
    double *fbuf = (double *)calloc((size_t)(3 * n + 1), sizeof(double));
    double *pebuf = (double *)calloc((size_t)(n + 1), sizeof(double));
    double *virbuf = (double *)calloc((size_t)(6 * n + 1), sizeof(double));
    int32_t *npbuf = (int32_t *)calloc((size_t)(n + 1), sizeof(int32_t));
#pragma omp parallel for schedule(dynamic, 20) num_threads(g_threads)
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0}, pei = 0.0, viri[6] = {0, 0, 0, 0, 0, 0};
        int32_t np = 0;
        double rci2 = rc[i] * rc[i];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            np += dcm_pair(x, i, j, rci2, L, eps, sigma, fi, &pei, viri);
        }
        for (int a = 0; a < 3; ++a) fbuf[3 * i + a] = fi[a];
        pebuf[i] = pei;
        for (int a = 0; a < 6; ++a) virbuf[6 * i + a] = viri[a];
        npbuf[i] = np;
    }
    finish_outputs(n, fbuf, pebuf, virbuf, npbuf, f, pe, vir, npair);
    free(fbuf);
    free(pebuf);
    free(virbuf);
    free(npbuf);
    return 0;
}

/* Algorithm 2.1: every pair once (i < j), force added to both (Newton 3) */
int orc_forces_static_half(int64_t n, const double *x, double rc,
                           const double L[3], double eps, double sigma,
                           double *f, double *pe)
{
    double lmin = L[0] < L[1] ? L[0] : L[1];
    if (L[2] < lmin) lmin = L[2];
    if (!(rc < 0.5 * lmin)) return -1;
    for (int64_t i = 0; i < 3 * n; ++i) f[i] = 0.0;
    if (pe)
        for (int64_t i = 0; i < n; ++i) pe[i] = 0.0;
    double rc2 = rc * rc;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            double dx = min_image(x[3 * i + 0] - x[3 * j + 0], L[0]);
            double dy = min_image(x[3 * i + 1] - x[3 * j + 1], L[1]);
            double dz = min_image(x[3 * i + 2] - x[3 * j + 2], L[2]);
            double r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < rc2)) continue;
            double V, fr;
            orc_lj(sqrt(r2), eps, sigma, &V, &fr);
            f[3 * i + 0] += fr * dx;
            f[3 * i + 1] += fr * dy;
            f[3 * i + 2] += fr * dz;
            f[3 * j + 0] -= fr * dx;
            f[3 * j + 1] -= fr * dy;
            f[3 * j + 2] -= fr * dz;
            if (pe) {
                pe[i] += 0.5 * V;
                pe[j] += 0.5 * V;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. 9: b_ijk = number of particles in box (i,j,k) */
void orc_density(int64_t n, const double *x, const double L[3], const int dims[3],
                 int32_t *B)
{
    int64_t nv = (int64_t)dims[0] * dims[1] * dims[2];
    for (int64_t v = 0; v < nv; ++v) B[v] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int gx = orc_bin_index(x[3 * i + 0], dims[0], L[0]);
        int gy = orc_bin_index(x[3 * i + 1], dims[1], L[1]);
        int gz = orc_bin_index(x[3 * i + 2], dims[2], L[2]);
        B[gx + (int64_t)dims[0] * (gy + (int64_t)dims[1] * gz)] += 1;
    }
}

static inline int64_t wrapi(int64_t k, int64_t n) { return ((k % n) + n) % n; }

void orc_smooth(const int dims[3], const int32_t *B, int order, double *Bs)
{
    int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    int64_t nv = nx * ny * nz;
    if (order <= 0) {
        for (int64_t v = 0; v < nv; ++v) Bs[v] = (double)B[v];
        return;
    }
    /* binomial weights by Pascal's rule */
    double *w = (double *)calloc((size_t)order + 1, sizeof(double));
    w[0] = 1.0;
    for (int r = 1; r <= order; ++r)
        for (int k = r; k >= 1; --k) w[k] = w[k] + w[k - 1];
    int half = order / 2;
    double *t1 = (double *)malloc(sizeof(double) * (size_t)nv);
    double *t2 = (double *)malloc(sizeof(double) * (size_t)nv);
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                double s = 0.0;
                for (int k = 0; k <= order; ++k)
                    s += w[k] * (double)B[wrapi(x + k - half, nx) + nx * (y + ny * z)];
                t1[x + nx * (y + ny * z)] = s;
            }
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                double s = 0.0;
                for (int k = 0; k <= order; ++k)
                    s += w[k] * t1[x + nx * (wrapi(y + k - half, ny) + ny * z)];
                t2[x + nx * (y + ny * z)] = s;
            }
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                double s = 0.0;
                for (int k = 0; k <= order; ++k)
                    s += w[k] * t2[x + nx * (y + ny * wrapi(z + k - half, nz))];
                Bs[x + nx * (y + ny * z)] = s;
            }
    free(w);
    free(t1);
    free(t2);
}

/* Eq. 14 with K = 2, Lloyd iterations (Section 4.1) */
int orc_kmeans(int64_t nvox, const double *Bs, int max_iter, uint8_t *S,
               double *c_l_out, double *c_v_out)
{
    double cl = Bs[0], cv = Bs[0];
    for (int64_t v = 1; v < nvox; ++v) {
        if (Bs[v] > cl) cl = Bs[v];
        if (Bs[v] < cv) cv = Bs[v];
    }
    uint8_t *prev = (uint8_t *)malloc((size_t)nvox);
    int have_prev = 0;
    int it = 0;
    while (it < max_iter) {
        double t = (cl + cv) * 0.5;
        for (int64_t v = 0; v < nvox; ++v) S[v] = (Bs[v] >= t) ? 0 : 1;
        it++;
        if (have_prev && memcmp(prev, S, (size_t)nvox) == 0) break;
        double sl = 0.0, sv = 0.0;
        int64_t nl = 0, nvap = 0;
        for (int64_t v = 0; v < nvox; ++v) {
            if (S[v] == 0) {
                sl += Bs[v];
                nl++;
            } else {
                sv += Bs[v];
                nvap++;
            }
        }
        if (nl > 0) cl = sl / (double)nl;
        if (nvap > 0) cv = sv / (double)nvap;
        memcpy(prev, S, (size_t)nvox);
        have_prev = 1;
    }
    free(prev);
    if (c_l_out) *c_l_out = cl;
    if (c_v_out) *c_v_out = cv;
    return it;
}

/* Eq. 13: two-phase piecewise-constant Mumford-Shah segmentation, with the
 * densities (c_l, c_v) fixed.  Readings: the integrand pairing is taken as
 * liquid with rho_l, vapor with rho_v (as printed it is swapped); the
 * perimeter is the number of grid faces between a liquid and a vapor voxel
 * (periodic, unit face area: the anisotropic perimeter of the voxel set);
 * the thesis cites its solver and does not give it, so the minimiser is
 * computed by the convex relaxation of Chan, Esedoglu and Nikolova:
 *   min over u in [0,1]^V of  sum_v u_v r_v + nu sum_faces |u_a - u_b|,
 *   r_v = (rho_v - c_l)^2 - (rho_v - c_v)^2  (u = 1: liquid),
 * whose thresholded minimisers are exact minimisers of Eq. 13 for this
 * perimeter (discrete coarea formula).  It is solved by the first-order
 * primal-dual iteration of Chambolle and Pock with one dual variable per
 * face (|p| <= nu), step sizes tau = sigma = 0.99 / sqrt(12) (the method
 * converges for tau sigma |grad|^2 < 1, and |grad|^2 = 12 for periodic
 * forward differences in 3D, reached by the checkerboard mode), u starting
 * at 1/2, a fixed number of iterations; labels: liquid (s = 0) where
 * u > 1/2.  After a fixed number of iterations the relaxed u is converged
 * only approximately; its threshold is an exact minimiser of Eq. 13 once u
 * is converged.  Precision: the thesis fixes none for the segmentation, and
 * the labels are a threshold decision, so the iteration runs in single
 * precision (u, u-bar, the duals, the step sizes and nu as float; the data
 * term r is formed in double and rounded once to float), every operation a
 * separately rounded float operation in the order written here. */
double orc_ms_energy(const int dims[3], const double *rho, double c_l, double c_v, double nu,
                     const uint8_t *S)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    double e = 0.0;
    int64_t faces = 0;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t v = x + nx * (y + ny * z);
                const double c = S[v] == 0 ? c_l : c_v;
                e += (rho[v] - c) * (rho[v] - c);
                const int64_t up[3] = {((x + 1) % nx) + nx * (y + ny * z),
                                       x + nx * (((y + 1) % ny) + ny * z),
                                       x + nx * (y + ny * ((z + 1) % nz))};
                const int64_t n[3] = {nx, ny, nz};
                for (int a = 0; a < 3; ++a)
                    if (n[a] > 1 && S[up[a]] != S[v]) faces++;
            }
    return e + nu * (double)faces;
}

void orc_ms_segment(const int dims[3], const double *rho, double c_l, double c_v, double nu,
                    int iters, uint8_t *S, double *u_out)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    const int64_t nv = nx * ny * nz;
    const int64_t n[3] = {nx, ny, nz};
    const float tau = (float)(0.99 / sqrt(12.0)), sigma = tau, nuf = (float)nu;
    float *u = (float *)malloc(sizeof(float) * (size_t)(nv > 0 ? nv : 1));
    float *ub = (float *)malloc(sizeof(float) * (size_t)(nv > 0 ? nv : 1));
    float *r = (float *)malloc(sizeof(float) * (size_t)(nv > 0 ? nv : 1));
    float *p = (float *)calloc((size_t)(3 * (nv > 0 ? nv : 1)), sizeof(float));
    for (int64_t v = 0; v < nv; ++v) {
        u[v] = 0.5f;
        ub[v] = 0.5f;
        r[v] = (float)((rho[v] - c_l) * (rho[v] - c_l) - (rho[v] - c_v) * (rho[v] - c_v));
    }
    for (int it = 0; it < iters; ++it) {
        /* dual ascent on the faces: p_a(v) on the face between v and v + e_a */
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    const int64_t v = x + nx * (y + ny * z);
                    const int64_t up[3] = {((x + 1) % nx) + nx * (y + ny * z),
                                           x + nx * (((y + 1) % ny) + ny * z),
                                           x + nx * (y + ny * ((z + 1) % nz))};
                    for (int a = 0; a < 3; ++a) {
                        float q = n[a] > 1 ? p[3 * v + a] + sigma * (ub[up[a]] - ub[v]) : 0.0f;
                        if (q > nuf) q = nuf;
                        if (q < -nuf) q = -nuf;
                        p[3 * v + a] = q;
                    }
                }
        /* primal descent: u -= tau (grad^T p + r), clipped to [0, 1]; then
         * the extrapolation ub = 2 u_new - u_old */
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    const int64_t v = x + nx * (y + ny * z);
                    const int64_t dn[3] = {((x + nx - 1) % nx) + nx * (y + ny * z),
                                           x + nx * (((y + ny - 1) % ny) + ny * z),
                                           x + nx * (y + ny * ((z + nz - 1) % nz))};
                    /* grad^T p at v: inflow from the lower faces minus outflow */
                    float gtp = 0.0f;
                    for (int a = 0; a < 3; ++a) gtp += p[3 * dn[a] + a] - p[3 * v + a];
                    float un = u[v] - tau * (gtp + r[v]);
                    if (un < 0.0f) un = 0.0f;
                    if (un > 1.0f) un = 1.0f;
                    ub[v] = 2.0f * un - u[v];
                    u[v] = un;
                }
    }
    for (int64_t v = 0; v < nv; ++v) {
        S[v] = u[v] > 0.5f ? 0 : 1;
        if (u_out) u_out[v] = (double)u[v];
    }
    free(u);
    free(ub);
    free(r);
    free(p);
}

/* Eq. 13 over the densities too: alternate the segmentation with fixed
 * densities and the densities as the means of rho over each phase (the
 * minimisers of the data terms for fixed sets), from the K-means centres
 * (Eq. 14), until the labels repeat or max_outer rounds.  A phase left
 * empty keeps its density.  Returns the rounds. */
int orc_ms_alternate(const int dims[3], const double *rho, double nu, int iters, int max_outer,
                     uint8_t *S, double *c_l_io, double *c_v_io)
{
    const int64_t nv = (int64_t)dims[0] * dims[1] * dims[2];
    uint8_t *prev = (uint8_t *)malloc((size_t)(nv > 0 ? nv : 1));
    double cl = *c_l_io, cv = *c_v_io;
    int round = 0;
    while (round < max_outer) {
        orc_ms_segment(dims, rho, cl, cv, nu, iters, S, NULL);
        round++;
        if (round > 1 && memcmp(prev, S, (size_t)nv) == 0) break;
        double sl = 0.0, sv = 0.0;
        int64_t nl = 0, nvap = 0;
        for (int64_t v = 0; v < nv; ++v) {
            if (S[v] == 0) {
                sl += rho[v];
                nl++;
            } else {
                sv += rho[v];
                nvap++;
            }
        }
        if (nl > 0) cl = sl / (double)nl;
        if (nvap > 0) cv = sv / (double)nvap;
        memcpy(prev, S, (size_t)nv);
    }
    free(prev);
    *c_l_io = cl;
    *c_v_io = cv;
    return round;
}

/* Eq. 13 as the segmentation step of the interface detection: on the
 * smoothed density image of the detection, rho_v = Bs_v * inv_scale (the
 * number density, inv_scale = 1 / (2^(3 order) V) for voxel volume V and
 * smoothing order `order`), starting from the labels in S (the K-means
 * labelling).  Each round takes the phase means of the current labels,
 * c = (sum of Bs over the phase / its voxels) * inv_scale, with the sums
 * exact (integers below 2^53), segments with those densities fixed
 * (orc_ms_segment), and stops once the labels repeat, or after max_outer
 * rounds.  A labelling with an empty phase is left as it is (no interface).
 * S is updated in place; returns the rounds. */
int orc_ms_detect(const int dims[3], const double *Bs, double inv_scale, double nu, int iters,
                  int max_outer, uint8_t *S)
{
    const int64_t nv = (int64_t)dims[0] * dims[1] * dims[2];
    double *rho = (double *)malloc(sizeof(double) * (size_t)(nv > 0 ? nv : 1));
    uint8_t *prev = (uint8_t *)malloc((size_t)(nv > 0 ? nv : 1));
    for (int64_t v = 0; v < nv; ++v) rho[v] = Bs[v] * inv_scale;
    int round = 0;
    while (round < max_outer) {
        double sl = 0.0, sv = 0.0;
        int64_t nl = 0, nvap = 0;
        for (int64_t v = 0; v < nv; ++v) {
            if (S[v] == 0) {
                sl += Bs[v];
                nl++;
            } else {
                sv += Bs[v];
                nvap++;
            }
        }
        if (nl == 0 || nvap == 0) break;
        const double cl = (sl / (double)nl) * inv_scale;
        const double cv = (sv / (double)nvap) * inv_scale;
        memcpy(prev, S, (size_t)nv);
        orc_ms_segment(dims, rho, cl, cv, nu, iters, S, NULL);
        round++;
        if (memcmp(prev, S, (size_t)nv) == 0) break;
    }
    free(rho);
    free(prev);
    return round;
}

/* Section 4.2, Algorithm 4.1: connected-component labelling of one phase.
 * The thesis gives the 2D row-major pass and says the 3D extension with
 * periodic boundaries is direct; the reading here:
 *   - connectivity: the 6 face neighbours (the thesis does not say);
 *   - pass: z, then y, then x innermost (row-major, x fastest as in the
 *     grid layout); a voxel of the phase looks at its already-visited face
 *     neighbours inside the grid (-x, -y, -z; no wrap during the pass):
 *     none labelled -> a new label; otherwise the smallest of their labels,
 *     and all of their labels are marked equivalent;
 *   - periodic boundaries: afterwards, every pair of voxels of the phase on
 *     opposite faces (0 and n-1 along an axis) marks its labels equivalent;
 *   - merge: equivalent labels are merged (union-find over the provisional
 *     labels, linking the larger root under the smaller), and the merged
 *     labels renumbered 0, 1, ... in order of first appearance in the pass.
 * label[v] = component of v, or -1 for voxels of the other phase.  Returns
 * the number of components. */
static int64_t uf_find(int64_t *par, int64_t a)
{
    while (par[a] != a) a = par[a];
    return a;
}

static void uf_union(int64_t *par, int64_t a, int64_t b)
{
    a = uf_find(par, a);
    b = uf_find(par, b);
    if (a == b) return;
    if (a < b) par[b] = a;
    else par[a] = b;
}

int64_t orc_label_components(const int dims[3], const uint8_t *S, int phase, int32_t *label)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    const int64_t nv = nx * ny * nz;
    int64_t *prov = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nv > 0 ? nv : 1));
    int64_t *par = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nv > 0 ? nv : 1));
    int64_t next = 0;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t v = x + nx * (y + ny * z);
                prov[v] = -1;
                if (S[v] != phase) continue;
                int64_t nb[3];
                int m = 0;
                if (x > 0 && S[v - 1] == phase) nb[m++] = prov[v - 1];
                if (y > 0 && S[v - nx] == phase) nb[m++] = prov[v - nx];
                if (z > 0 && S[v - nx * ny] == phase) nb[m++] = prov[v - nx * ny];
                if (m == 0) {
                    par[next] = next;
                    prov[v] = next++;
                } else {
                    int64_t lo = nb[0];
                    for (int q = 1; q < m; ++q)
                        if (nb[q] < lo) lo = nb[q];
                    prov[v] = lo;
                    for (int q = 0; q < m; ++q) uf_union(par, lo, nb[q]);
                }
            }
    /* periodic faces */
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y) {
            const int64_t a = nx * (y + ny * z), b = a + nx - 1;
            if (nx > 1 && S[a] == phase && S[b] == phase) uf_union(par, prov[a], prov[b]);
        }
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t x = 0; x < nx; ++x) {
            const int64_t a = x + nx * ny * z, b = a + nx * (ny - 1);
            if (ny > 1 && S[a] == phase && S[b] == phase) uf_union(par, prov[a], prov[b]);
        }
    for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x) {
            const int64_t a = x + nx * y, b = a + nx * ny * (nz - 1);
            if (nz > 1 && S[a] == phase && S[b] == phase) uf_union(par, prov[a], prov[b]);
        }
    /* merge and renumber in order of first appearance */
    int64_t *num = (int64_t *)malloc(sizeof(int64_t) * (size_t)(next > 0 ? next : 1));
    for (int64_t l = 0; l < next; ++l) num[l] = -1;
    int64_t ncomp = 0;
    for (int64_t v = 0; v < nv; ++v) {
        if (prov[v] < 0) {
            label[v] = -1;
            continue;
        }
        const int64_t r = uf_find(par, prov[v]);
        if (num[r] < 0) num[r] = ncomp++;
        label[v] = (int32_t)num[r];
    }
    free(num);
    free(par);
    free(prov);
    return ncomp;
}

/* Section 4.2 (Fig. 20-21): removal of small connected components.  The
 * outline removes the small components of the liquid phase and then those
 * of the vapor phase; the reading here: the liquid components (s = 0) of
 * fewer than min_voxels voxels become vapor, then the vapor components
 * (s = 1) of the resulting grid with fewer than min_voxels voxels become
 * liquid (the thesis's example removes every component smaller than 5).
 * min_voxels <= 0: nothing changes.  Returns the number of voxels whose
 * phase changed. */
int64_t orc_remove_small_components(const int dims[3], uint8_t *S, int min_voxels)
{
    if (min_voxels <= 0) return 0;
    const int64_t nv = (int64_t)dims[0] * dims[1] * dims[2];
    int32_t *label = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    int64_t flipped = 0;
    for (int phase = 0; phase <= 1; ++phase) {
        const int64_t nc = orc_label_components(dims, S, phase, label);
        int64_t *size = (int64_t *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(int64_t));
        for (int64_t v = 0; v < nv; ++v)
            if (label[v] >= 0) size[label[v]]++;
        for (int64_t v = 0; v < nv; ++v)
            if (label[v] >= 0 && size[label[v]] < min_voxels) {
                S[v] = (uint8_t)(1 - phase);
                flipped++;
            }
        free(size);
    }
    free(label);
    return flipped;
}

/* Eq. 16-18 generalised to three axes and per-axis spacing h_k: the
 * solution d of sum_k ((d - a_k)^+ / h_k)^2 = 1, found by growing the active
 * set in ascending a (ties broken by axis order). */
double orc_godunov(const double a_in[3], const double h_in[3])
{
    double a[3] = {a_in[0], a_in[1], a_in[2]};
    double h[3] = {h_in[0], h_in[1], h_in[2]};
    /* stable insertion sort by a */
    for (int i = 1; i < 3; ++i) {
        double ka = a[i], kh = h[i];
        int j = i - 1;
        while (j >= 0 && a[j] > ka) {
            a[j + 1] = a[j];
            h[j + 1] = h[j];
            j--;
        }
        a[j + 1] = ka;
        h[j + 1] = kh;
    }
    if (isinf(a[0])) return INFINITY;
    double d2 = a[1] - a[0];
    double d3 = a[2] - a[0];
    double e = h[0];
    if (e <= d2) return a[0] + e;
    double w1 = 1.0 / (h[0] * h[0]);
    double w2 = 1.0 / (h[1] * h[1]);
    double w3 = 1.0 / (h[2] * h[2]);
    double wd2 = w2 * d2;
    double A = w1 + w2;
    double B = wd2;
    double C = wd2 * d2 - 1.0;
    double disc = B * B - A * C;
    if (disc < 0.0) disc = 0.0;
    e = (B + sqrt(disc)) / A;
    if (e <= d3) return a[0] + e;
    double wd3 = w3 * d3;
    A = w1 + w2 + w3;
    B = wd2 + wd3;
    C = (wd2 * d2 + wd3 * d3) - 1.0;
    disc = B * B - A * C;
    if (disc < 0.0) disc = 0.0;
    e = (B + sqrt(disc)) / A;
    return a[0] + e;
}

static inline void nbr_minima(const int dims[3], const double *D, int64_t x,
                              int64_t y, int64_t z, double a[3])
{
    int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    double m0 = D[wrapi(x - 1, nx) + nx * (y + ny * z)];
    double m1 = D[wrapi(x + 1, nx) + nx * (y + ny * z)];
    a[0] = m0 < m1 ? m0 : m1;
    m0 = D[x + nx * (wrapi(y - 1, ny) + ny * z)];
    m1 = D[x + nx * (wrapi(y + 1, ny) + ny * z)];
    a[1] = m0 < m1 ? m0 : m1;
    m0 = D[x + nx * (y + ny * wrapi(z - 1, nz))];
    m1 = D[x + nx * (y + ny * wrapi(z + 1, nz))];
    a[2] = m0 < m1 ? m0 : m1;
}

/* Algorithm 4.2 in 3D with PBC, repeated until a round of 8 sweeps changes
 * nothing, then the cap */
int orc_fsm(const int dims[3], const double h[3], const uint8_t *S, double cap,
            double *D)
{
    int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    int64_t nv = nx * ny * nz;
    for (int64_t v = 0; v < nv; ++v) D[v] = (S[v] == 1) ? 0.0 : INFINITY;
    int rounds = 0;
    int changed = 1;
    while (changed && rounds < 100000) {
        changed = 0;
        rounds++;
        for (int dir = 0; dir < 8; ++dir) {
            int sx = (dir & 1) ? -1 : 1, sy = (dir & 2) ? -1 : 1, sz = (dir & 4) ? -1 : 1;
            for (int64_t kz = 0; kz < nz; ++kz) {
                int64_t z = sz > 0 ? kz : nz - 1 - kz;
                for (int64_t ky = 0; ky < ny; ++ky) {
                    int64_t y = sy > 0 ? ky : ny - 1 - ky;
                    for (int64_t kx = 0; kx < nx; ++kx) {
                        int64_t x = sx > 0 ? kx : nx - 1 - kx;
                        int64_t v = x + nx * (y + ny * z);
                        if (S[v] == 1) continue;
                        double a[3];
                        nbr_minima(dims, D, x, y, z, a);
                        double dbar = orc_godunov(a, h);
                        if (dbar < D[v]) { /* Eq. 19 */
                            D[v] = dbar;
                            changed = 1;
                        }
                    }
                }
            }
        }
    }
    if (cap > 0.0)
        for (int64_t v = 0; v < nv; ++v)
            if (D[v] > cap) D[v] = cap;
    return rounds;
}

/* Algorithm 4.3 */
int orc_cfsm(const int dims[3], const double h[3], const uint8_t *S,
             double r_grid, int iter_max, double eps, double *D)
{
    int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    int64_t nv = nx * ny * nz;
    int64_t *Q = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    int64_t *Qn = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    uint8_t *inq = (uint8_t *)calloc((size_t)nv, 1);
    int64_t nq = 0;
    /* initialize: D = 0 on vapor, +inf on liquid; Q = liquid boxes with a
     * vapor face neighbour (the interfacial boxes) */
    for (int64_t v = 0; v < nv; ++v) D[v] = (S[v] == 1) ? 0.0 : INFINITY;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                int64_t v = x + nx * (y + ny * z);
                if (S[v] == 1) continue;
                int64_t nb[6] = {wrapi(x - 1, nx) + nx * (y + ny * z),
                                 wrapi(x + 1, nx) + nx * (y + ny * z),
                                 x + nx * (wrapi(y - 1, ny) + ny * z),
                                 x + nx * (wrapi(y + 1, ny) + ny * z),
                                 x + nx * (y + ny * wrapi(z - 1, nz)),
                                 x + nx * (y + ny * wrapi(z + 1, nz))};
                for (int k = 0; k < 6; ++k)
                    if (S[nb[k]] == 1) {
                        Q[nq++] = v;
                        break;
                    }
            }
    int result = -1;
    for (int iter = 0; iter < iter_max; ++iter) {
        double de = 0.0;
        int64_t nqn = 0;
        for (int64_t q = 0; q < nq; ++q) {
            int64_t v = Q[q];
            int64_t x = v % nx, y = (v / nx) % ny, z = v / (nx * ny);
            double a[3];
            nbr_minima(dims, D, x, y, z, a);
            double dbar = orc_godunov(a, h);
            double dnew = dbar < D[v] ? dbar : D[v]; /* local FSM with Eq. 19 */
            if (dnew <= r_grid) {
                double ch = fabs(D[v] - dnew);
                if (isinf(D[v])) ch = INFINITY;
                if (ch > de) de = ch;
                D[v] = dnew;
                int64_t nb[6] = {wrapi(x - 1, nx) + nx * (y + ny * z),
                                 wrapi(x + 1, nx) + nx * (y + ny * z),
                                 x + nx * (wrapi(y - 1, ny) + ny * z),
                                 x + nx * (wrapi(y + 1, ny) + ny * z),
                                 x + nx * (y + ny * wrapi(z - 1, nz)),
                                 x + nx * (y + ny * wrapi(z + 1, nz))};
                for (int k = 0; k < 6; ++k) {
                    int64_t u = nb[k];
                    if (S[u] == 1 || inq[u]) continue;
                    inq[u] = 1;
                    Qn[nqn++] = u;
                }
            }
        }
        for (int64_t q = 0; q < nqn; ++q) inq[Qn[q]] = 0;
        int64_t *tq = Q;
        Q = Qn;
        Qn = tq;
        nq = nqn;
        int stop = (eps > 0.0) ? (de < eps) : (de == 0.0);
        if (stop) {
            result = iter + 1;
            break;
        }
    }
    for (int64_t v = 0; v < nv; ++v)
        if (D[v] > r_grid) D[v] = r_grid;
    free(Q);
    free(Qn);
    free(inq);
    return result;
}

/* ------------------------------------------------------------------------ */
static inline double lerp(double a, double b, double t) { return a + t * (b - a); }

/* Algorithm 3.1: lower-left-front box of the particle relative to the box
 * centres, then x, y, z linear interpolations */
void orc_particle_distance(int64_t n, const double *x, const double L[3],
                           const int dims[3], const double *D, double *d)
{
    int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    for (int64_t i = 0; i < n; ++i) {
        int64_t i0[3], i1[3];
        double t[3];
        for (int a = 0; a < 3; ++a) {
            double inv = (double)dims[a] / L[a];
            double g = x[3 * i + a] * inv - 0.5;
            double fl = floor(g);
            t[a] = g - fl;
            i0[a] = wrapi((int64_t)fl, dims[a]);
            i1[a] = wrapi((int64_t)fl + 1, dims[a]);
        }
#define DV(X, Y, Z) D[(X) + nx * ((Y) + ny * (Z))]
        double c00 = lerp(DV(i0[0], i0[1], i0[2]), DV(i1[0], i0[1], i0[2]), t[0]);
        double c10 = lerp(DV(i0[0], i1[1], i0[2]), DV(i1[0], i1[1], i0[2]), t[0]);
        double c01 = lerp(DV(i0[0], i0[1], i1[2]), DV(i1[0], i0[1], i1[2]), t[0]);
        double c11 = lerp(DV(i0[0], i1[1], i1[2]), DV(i1[0], i1[1], i1[2]), t[0]);
#undef DV
        double c0 = lerp(c00, c10, t[1]);
        double c1 = lerp(c01, c11, t[1]);
        d[i] = lerp(c0, c1, t[2]);
        (void)nz;
    }
}

int orc_detect(int64_t n, const double *x, const double L[3],
               const orc_detect_params *p, int dims_out[3], int32_t *B_out,
               double *Bs_out, uint8_t *S_out, double *D_out, double *d,
               double *rc, uint8_t *cls)
{
    int dims[3];
    orc_grid_dims(L, p->voxel, dims);
    int64_t nv = (int64_t)dims[0] * dims[1] * dims[2];
    int32_t *B = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    double *Bs = (double *)malloc(sizeof(double) * (size_t)nv);
    uint8_t *S = (uint8_t *)malloc((size_t)nv);
    double *D = (double *)malloc(sizeof(double) * (size_t)nv);
    orc_density(n, x, L, dims, B);
    orc_smooth(dims, B, p->smooth_order, Bs);
    orc_kmeans(nv, Bs, p->kmeans_max_iter > 0 ? p->kmeans_max_iter : 100, S, NULL, NULL);
    if (p->segmentation == 1) {
        const double V = (L[0] / dims[0]) * (L[1] / dims[1]) * (L[2] / dims[2]);
        const double inv_scale = 1.0 / ldexp(V, 3 * (p->smooth_order > 0 ? p->smooth_order : 0));
        orc_ms_detect(dims, Bs, inv_scale, p->ms_nu, p->ms_iters > 0 ? p->ms_iters : 50,
                      p->ms_outer > 0 ? p->ms_outer : 1, S);
    }
    orc_remove_small_components(dims, S, p->min_component_voxels);
    double h[3] = {L[0] / dims[0], L[1] / dims[1], L[2] / dims[2]};
    double hmax = h[0];
    if (h[1] > hmax) hmax = h[1];
    if (h[2] > hmax) hmax = h[2];
    double r_grid = p->rc_max + hmax;
    int dmax = dims[0];
    if (dims[1] > dmax) dmax = dims[1];
    if (dims[2] > dmax) dmax = dims[2];
    int iter_max = p->cfsm_iter_max > 0 ? p->cfsm_iter_max : 4 * dmax;
    int it = orc_cfsm(dims, h, S, r_grid, iter_max, p->cfsm_eps, D);
    orc_particle_distance(n, x, L, dims, D, d);
    int K = p->n_classes < 2 ? 2 : p->n_classes;
    double thr[16];
    const int lin = p->cutoff_fn == 1 && p->rc_max > p->rc_min;
    if (lin)
        orc_class_thresholds_linear(p->rc_min, p->rc_max, K, thr);
    else
        orc_class_thresholds(p->rc_min, p->rc_max, p->alpha, K, thr);
    for (int64_t i = 0; i < n; ++i) {
        rc[i] = lin ? orc_cutoff_linear(d[i], p->rc_min, p->rc_max)
                    : orc_cutoff(d[i], p->rc_min, p->rc_max, p->alpha);
        if (cls) cls[i] = (uint8_t)orc_cutoff_class(d[i], p->rc_max, K, thr);
    }
    if (dims_out) memcpy(dims_out, dims, sizeof(dims));
    if (B_out) memcpy(B_out, B, sizeof(int32_t) * (size_t)nv);
    if (Bs_out) memcpy(Bs_out, Bs, sizeof(double) * (size_t)nv);
    if (S_out) memcpy(S_out, S, (size_t)nv);
    if (D_out) memcpy(D_out, D, sizeof(double) * (size_t)nv);
    free(B);
    free(Bs);
    free(S);
    free(D);
    return it;
}

/* ------------------------------------------------------------------------ */
static double kinetic(int64_t n, const double *v, double m)
{
    double s = 0.0;
    for (int64_t i = 0; i < 3 * n; ++i) s += v[i] * v[i];
    return 0.5 * m * s;
}

static double potential(int64_t n, const double *pe)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += pe[i];
    return s;
}

/* Eq. 1-2 integrated by velocity Verlet, with interface detection every
 * detect_every steps and r_c held between detections */
int orc_run(int64_t n, double *x, double *v, const double L[3],
            const orc_run_params *p, int64_t step0, int64_t nsteps, double *f,
            double *rc, double *epot, double *ekin)
{
    int nc[3];
    orc_cell_dims(L, p->cell_min, nc);
    double *d = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *pe = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < 3 * n; ++i) x[i] = orc_wrap(x[i], L[i % 3]);
    orc_detect(n, x, L, &p->det, NULL, NULL, NULL, NULL, NULL, d, rc, NULL);
    int rcode = orc_forces(n, x, rc, L, nc, p->eps, p->sigma, f, pe, NULL, NULL);
    if (rcode) goto done;
    if (epot) epot[0] = potential(n, pe);
    if (ekin) ekin[0] = kinetic(n, v, p->mass);
    double hdt = 0.5 * p->dt / p->mass;
    for (int64_t s = 1; s <= nsteps; ++s) {
        for (int64_t i = 0; i < 3 * n; ++i) {
            v[i] = v[i] + hdt * f[i];
            x[i] = orc_wrap(x[i] + p->dt * v[i], L[i % 3]);
        }
        if (p->detect_every > 0 && (step0 + s) % p->detect_every == 0)
            orc_detect(n, x, L, &p->det, NULL, NULL, NULL, NULL, NULL, d, rc, NULL);
        rcode = orc_forces(n, x, rc, L, nc, p->eps, p->sigma, f, pe, NULL, NULL);
        if (rcode) goto done;
        for (int64_t i = 0; i < 3 * n; ++i) v[i] = v[i] + hdt * f[i];
        if (epot) epot[s] = potential(n, pe);
        if (ekin) ekin[s] = kinetic(n, v, p->mass);
    }
done:
    free(d);
    free(pe);
    return rcode;
}
