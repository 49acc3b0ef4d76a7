/*
 * dcm_oracle.h -- plain, slow FP64 CPU oracle for the dynamic cutoff method
 * (DCM) of Springer, "A Scalable, Linear-Time Dynamic Cutoff Algorithm for
 * Molecular Simulations of Interfacial Systems" (arxiv 1502.03234).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no source,
 * header, table or constant with the CUDA library; the CUDA library never
 * loads it.
 *
 * Every routine is a direct statement of one passage of the thesis (cited
 * per function), in FP64, in the order the thesis gives, with no blocking,
 * fusion or reordering.  Where the thesis is silent or ambiguous the reading
 * is stated next to the routine.
 *
 * Conventions shared by all routines (the geometry both sides must agree on
 * bit-for-bit, stated here so the definitions can be checked by eye):
 *   - positions are AoS x[3*i+a], a = 0,1,2; the box is orthorhombic with
 *     origin 0 and periodic in x, y, z;
 *   - a bin of edge L/n (link cell, voxel) holding coordinate x has index
 *     min(n-1, floor(x * (n / L)))   (one IEEE multiply, no FMA);
 *   - minimum image of a difference dx: if dx > L/2 then dx - L,
 *     else if dx < -L/2 then dx + L;
 *   - r^2 = dx*dx + dy*dy + dz*dz evaluated left to right, no FMA.
 * The library is compiled with -ffp-contract=off.
 */
#ifndef DCM_ORACLE_H
#define DCM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* threads used by the loops over particles (OpenMP, schedule(dynamic,20)
 * as in the thesis's Algorithm 5.1); 1 = serial.  Returns the count set. */
int orc_set_threads(int nthreads);
int orc_get_threads(void);

/* ---- Eq. 4: Lennard-Jones pair ------------------------------------------
 * V(r) = 4 eps ((sigma/r)^12 - (sigma/r)^6).  *fr receives the radial factor
 * such that the force on i from j is  F_i<-j = fr * (x_i - x_j)
 * (fr = -V'(r)/r).  Truncated, not shifted (Section 3.2 never shifts). */
void orc_lj(double r, double eps, double sigma, double *V, double *fr);

/* ---- Eq. 7-8: exponential cutoff function -------------------------------
 * r_c(d) = rc_max for d <= 0; a*2^(alpha*(rc_max-d)) + b for 0 < d < rc_max;
 * rc_min for d >= rc_max, with a = (rc_max-rc_min)/(2^(alpha rc_max)-1),
 * b = rc_min - a. */
double orc_cutoff(double d, double rc_min, double rc_max, double alpha);

/* Class thresholds for the load-balancing classes (not in the thesis; a
 * partition of the Eq. 7 range).  Class 0: d >= rc_max (r_c = rc_min);
 * class K-1: d <= 0 (r_c = rc_max); classes 1..K-2 split the open range by
 * the cutoff value, with edges r_k = rc_min + k (rc_max-rc_min)/(K-1),
 * k = 1..K-2, mapped to distances by inverting Eq. 7.  thr[k-1] = d(r_k),
 * descending.  Class of d in (0, rc_max): 1 + #{k : d < thr[k-1]}. */
void orc_class_thresholds(double rc_min, double rc_max, double alpha, int K,
                          double *thr /* K-2 entries */);
int orc_cutoff_class(double d, double rc_max, int K, const double *thr);

/* ---- Section 3.1, Fig. 12: linear cutoff function -------------------------
 * r_c(d) = rc_max for d <= 0; rc_max - (rc_max-rc_min) d / rc_max for
 * 0 < d < rc_max; rc_min for d >= rc_max (a reading of the figure: the
 * thesis draws it and gives no formula).  Class edges as above, from
 * inverting this line. */
double orc_cutoff_linear(double d, double rc_min, double rc_max);
void orc_class_thresholds_linear(double rc_min, double rc_max, int K, double *thr);

/* ---- bins ---------------------------------------------------------------*/
/* Eq. 10 with the reading N_x = max(3, floor(L_x / b)). */
void orc_grid_dims(const double L[3], double b, int dims[3]);
/* link cells: n = max(1, floor(L / c)) */
void orc_cell_dims(const double L[3], double c, int nc[3]);
int orc_bin_index(double x, int n, double L);

/* ---- link-cell list (Section 2.2.1) ----------------------------------------
 * cell_of[i] = cell index (x fastest); cell_start[nc+1] prefix offsets;
 * sorted_id[] particle ids grouped by cell, ascending id within a cell. */
void orc_cell_list(int64_t n, const double *x, const double L[3], const int nc[3],
                   int32_t *cell_of, int32_t *cell_start, int32_t *sorted_id);

/* ---- Algorithm 3.2: DCM force over the link-cell stencil -------------------
 * F_i = sum over j != i with |r_ij| < rc[i] of F_LJ(r_ij); no Newton-3; the
 * particle i only ever receives its own force.  pe[i] = 1/2 sum_j V(r_ij)
 * (nullable); vir[6] = 1/2 sum_i sum_j (r_ij)_a (F_i<-j)_b for ab = xx, yy,
 * zz, xy, xz, yz (nullable); npair[i] = number of contributing j (nullable).
 * Returns 0, or -1 if rc_max >= min(L)/2 (minimum image would be ambiguous). */
int orc_forces(int64_t n, const double *x, const double *rc, const double L[3],
               const int nc[3], double eps, double sigma, double *f, double *pe,
               double *vir, int32_t *npair);

/* Same sum by O(N^2) brute force over all j (the definition, no cells). */
int orc_forces_brute(int64_t n, const double *x, const double *rc,
                     const double L[3], double eps, double sigma, double *f,
                     double *pe, double *vir, int32_t *npair);

/* Algorithm 2.1: static half-list force with Newton's third law, pair rule
 * |r_ij| < rc (all pairs i<j found by brute force).  Used to pin the static
 * limit rc_min == rc_max of DCM. */
int orc_forces_static_half(int64_t n, const double *x, double rc,
                           const double L[3], double eps, double sigma,
                           double *f, double *pe);

/* ---- Eq. 9: density image ---------------------------------------------------*/
void orc_density(int64_t n, const double *x, const double L[3], const int dims[3],
                 int32_t *B);

/* ---- smoothing (not in the thesis; replaces the perimeter term) ------------
 * Three periodic 1D passes (x, then y, then z) with the integer binomial
 * weights C(order, k), k = 0..order, centred.  order 0 copies B.  The result
 * is an exact integer held in FP64. */
void orc_smooth(const int dims[3], const int32_t *B, int order, double *Bs);

/* ---- Eq. 11-14: two-class K-means segmentation -------------------------------
 * Lloyd iterations from c_l = max, c_v = min (the thesis's naive estimates);
 * a voxel is liquid (s = 0) iff value >= (c_l + c_v)/2, else vapor (s = 1).
 * Stops when the assignment no longer changes, at most max_iter passes.
 * Returns the number of assignment passes. */
int orc_kmeans(int64_t nvox, const double *Bs, int max_iter, uint8_t *S,
               double *c_l, double *c_v);

/* ---- Eq. 13: two-phase piecewise-constant Mumford-Shah ------------------------
 * orc_ms_energy: Eq. 13 of labels S (0 liquid, 1 vapor) on the image rho with
 * fixed densities c_l, c_v: sum over liquid voxels of (rho - c_l)^2, over
 * vapor voxels of (rho - c_v)^2, plus nu times the number of periodic grid
 * faces between a liquid and a vapor voxel.  orc_ms_segment: its minimiser
 * by the convex relaxation (Chan-Esedoglu-Nikolova) solved with `iters`
 * Chambolle-Pock iterations from u = 1/2; S = 0 where u > 1/2; u_out
 * (nullable) receives the relaxed solution. */
double orc_ms_energy(const int dims[3], const double *rho, double c_l, double c_v, double nu,
                     const uint8_t *S);
void orc_ms_segment(const int dims[3], const double *rho, double c_l, double c_v, double nu,
                    int iters, uint8_t *S, double *u_out);
/* Eq. 13 over the densities as well: segmentation with fixed densities and
 * densities as the phase means, alternated from *c_l_io, *c_v_io (the K-means
 * centres) until the labels repeat or max_outer rounds; the final densities
 * are written back.  Returns the rounds. */
/* Eq. 13 as the detection's segmentation step: on rho = Bs * inv_scale from
 * the labels in S (updated in place), rounds of exact phase means and
 * segmentation until the labels repeat or max_outer rounds; returns the
 * rounds (see dcm_oracle.c). */
int orc_ms_detect(const int dims[3], const double *Bs, double inv_scale, double nu, int iters,
                  int max_outer, uint8_t *S);
int orc_ms_alternate(const int dims[3], const double *rho, double nu, int iters, int max_outer,
                     uint8_t *S, double *c_l_io, double *c_v_io);

/* ---- Section 4.2, Algorithm 4.1: small connected components ------------------
 * orc_label_components: components of the voxels with S == phase, face
 * (6-) connectivity across the periodic faces, by the row-major two-pass
 * labelling of Algorithm 4.1; label[v] = 0, 1, ... in order of first
 * appearance (x fastest), -1 for the other phase.  Returns the count.
 * orc_remove_small_components: liquid components of fewer than min_voxels
 * voxels become vapor, then vapor components (of that result) of fewer than
 * min_voxels become liquid; <= 0: none.  Returns the voxels changed. */
int64_t orc_label_components(const int dims[3], const uint8_t *S, int phase, int32_t *label);
int64_t orc_remove_small_components(const int dims[3], uint8_t *S, int min_voxels);

/* ---- Eq. 15-19: Godunov upwind local solve ------------------------------------
 * Returns the Eq. 19 candidate dbar for a voxel whose per-axis neighbour
 * minima are a[3] (Eq. 17) with spacings h[3]; +inf if all a are +inf. */
double orc_godunov(const double a[3], const double h[3]);

/* Algorithm 4.2 in 3D with periodic boundaries: D = 0 on vapor (S == 1),
 * +inf on liquid, then rounds of the 2^3 alternating Gauss-Seidel sweeps
 * until a round changes nothing; finally D = min(D, cap) (cap <= 0: none).
 * Returns the number of rounds. */
int orc_fsm(const int dims[3], const double h[3], const uint8_t *S, double cap,
            double *D);

/* Algorithm 4.3 (cutoff-based FSM): queue of interfacial boxes, local solve,
 * update only when d_new <= r_grid, stop when the largest change is < eps
 * (eps == 0 read as: no value changed) or after iter_max passes; voxels never
 * reached take the value r_grid.  Returns passes, or -1 if iter_max was hit. */
int orc_cfsm(const int dims[3], const double h[3], const uint8_t *S,
             double r_grid, int iter_max, double eps, double *D);

/* ---- Algorithm 3.1: trilinear particle-interface distance ------------------*/
void orc_particle_distance(int64_t n, const double *x, const double L[3],
                           const int dims[3], const double *D, double *d);

/* ---- full interface detection (Fig. 14 order) ---------------------------------
 * density -> smoothing -> K-means labels -> [Eq. 13 segmentation from them,
 * when segmentation == 1] -> [small-component removal, when
 * min_component_voxels > 0] -> CFSM distance (cap r_grid =
 * rc_max + max h) -> particle distance -> cutoff (Eq. 7) -> class.  All
 * output arrays are nullable except d/rc/cls.  Returns CFSM passes (or -1). */
typedef struct {
    double rc_min, rc_max, alpha;
    double voxel;
    int smooth_order;
    int kmeans_max_iter;
    int cfsm_iter_max; /* <= 0: 4 * max(dims) */
    double cfsm_eps;
    int n_classes;
    int min_component_voxels; /* Section 4.2; <= 0: no removal */
    int cutoff_fn;            /* 0: exponential (Eq. 7), 1: linear (Fig. 12) */
    int segmentation;         /* 0: K-means labels (Eq. 11-14); 1: then Eq. 13 (orc_ms_detect) */
    int ms_iters;             /* Eq. 13: primal-dual iterations per round; <= 0: 50 */
    int ms_outer;             /* Eq. 13: rounds of segmentation and phase means; <= 0: 1 */
    double ms_nu;             /* Eq. 13: perimeter weight (number-density units) */
} orc_detect_params;

int orc_detect(int64_t n, const double *x, const double L[3],
               const orc_detect_params *p, int dims_out[3], int32_t *B,
               double *Bs, uint8_t *S, double *D, double *d, double *rc,
               uint8_t *cls);

/* ---- Eq. 1-2: velocity Verlet with the DCM cadence --------------------------
 * Setup (once): detect, force.  Each step s = step0+1 .. step0+nsteps:
 *   v += dt/2 F/m; x += dt v; wrap; if s % detect_every == 0: detect;
 *   force; v += dt/2 F/m.
 * x, v updated in place; f receives the last forces; rc the cutoffs in use;
 * epot/ekin per step (nullable, nsteps+1 entries incl. the initial state). */
typedef struct {
    orc_detect_params det;
    double dt, mass, eps, sigma;
    double cell_min;
    int detect_every;
} orc_run_params;

int orc_run(int64_t n, double *x, double *v, const double L[3],
            const orc_run_params *p, int64_t step0, int64_t nsteps, double *f,
            double *rc, double *epot, double *ekin);

/* wrap one coordinate into [0, L) */
double orc_wrap(double x, double L);

#ifdef __cplusplus
}
#endif
#endif
