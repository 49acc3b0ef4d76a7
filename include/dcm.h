/*
 * dcm.h -- C ABI of the GB300 (sm_103a) dynamic cutoff method library
 * (libdcm.so).
 *
 * Method: Springer, "A Scalable, Linear-Time Dynamic Cutoff Algorithm for
 * Molecular Simulations of Interfacial Systems" (arxiv 1502.03234).  Each
 * Lennard-Jones particle i carries its own cutoff r_c[i], set from its
 * distance to the liquid/vapor interface (Eq. 7-8); the interface is found
 * on a voxel grid (Section 4) and the forces are summed over a full
 * neighbourhood without Newton's third law (Algorithm 3.2).
 *
 * Conventions for every entry point:
 *   - Return value: DCM_OK (0) or a DCM_ERR_* code; no exception or signal
 *     crosses the ABI.  dcm_last_error() returns a message for the calling
 *     thread's most recent failure.
 *   - Positions/velocities/forces cross the ABI as AoS double[3*N]
 *     (x0,y0,z0,x1,...), in the caller's particle order ("id order").
 *     Arrays passed in are copied, never retained.
 *   - mem = DCM_HOST: host pointers; the call returns when the copy is done.
 *     mem = DCM_DEVICE: device pointers (e.g. a torch CUDA tensor's
 *     data_ptr); the copy is enqueued on the handle's stream.
 *   - Work is enqueued on the CUDA stream given to dcm_create (the library
 *     makes its own non-blocking stream when given NULL).  Only dcm_get_*,
 *     dcm_energy_virial, dcm_sync and the DCM_HOST copies block the host.
 *   - The library owns all device memory it allocates; everything is
 *     allocated by dcm_create, nothing inside dcm_step.
 *   - Units are reduced LJ units unless the parameters say otherwise.
 *   - The box is orthorhombic with origin 0, periodic in x, y and z; every
 *     cutoff must stay below half the shortest edge minus one link cell
 *     (DCM_ERR_BOX_TOO_SMALL otherwise).
 *   - One handle is used by one host thread at a time.
 */
#ifndef DCM_H
#define DCM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DCM_ABI_VERSION 1

enum dcm_status {
    DCM_OK = 0,
    DCM_ERR_ARG = 1,            /* invalid argument or parameter */
    DCM_ERR_OOM = 2,            /* device allocation failed */
    DCM_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    DCM_ERR_BOX_TOO_SMALL = 4,  /* rc_max + link cell >= half the shortest edge */
    DCM_ERR_NOT_CONVERGED = 5,  /* CFSM or K-means hit its iteration cap */
    DCM_ERR_DEVICE_CHECK = 6,   /* a device-side check failed (non-finite
                                   position, particle moved more than a box
                                   edge in one step, bounded wait expired) */
    DCM_ERR_CANCELLED = 7,      /* work stopped by a cancel request */
    DCM_ERR_STATE = 8           /* call out of order (e.g. no state set) */
};

enum { DCM_FP64 = 0,   /* FP64 pair distances, forces and accumulation */
       DCM_MIXED = 1   /* FP32 pair distances and forces for pairs beyond
                          1.5 sigma; closer pairs in double-float (2 x FP32)
                          arithmetic from the exact displacement; exact
                          fixed-point sums of the lane partials; FP64 state,
                          integration and reductions.  Per-particle forces
                          meet |F - F_FP64| <= 1e-6 + 1e-5 |F| for liquid
                          states with link cells up to about 2 sigma. */
};
enum { DCM_HOST = 0, DCM_DEVICE = 1 };
enum { DCM_CUTOFF_EXP = 0, DCM_CUTOFF_LINEAR = 1 };
enum { DCM_SEG_KMEANS = 0, DCM_SEG_MUMFORD_SHAH = 1 };

#define DCM_MAX_CLASSES 8

typedef struct {
    double lx, ly, lz;
} dcm_box;

typedef struct {
    /* Eq. 7-8: cutoff function; rc_min == rc_max is the static cutoff */
    double rc_min, rc_max, alpha;          /* alpha < 0; thesis uses -0.5 */
    /* Eq. 1-2, Eq. 4 */
    double dt, mass, eps, sigma;
    /* Eq. 10: target voxel edge b; N_x = max(3, floor(L_x / b)) */
    double voxel;
    /* binomial smoothing order (even, 0..16; 8 -> sigma = sqrt(2) voxels) */
    int32_t smooth_order;
    /* interface detection every detect_every steps (thesis: every other
       step); 0 = never re-detect inside dcm_step */
    int32_t detect_every;
    int32_t kmeans_max_iter;               /* Eq. 14 Lloyd passes, <= 0: 100 */
    int32_t cfsm_iter_max;                 /* Algorithm 4.3, <= 0: 4*max(N) */
    double cfsm_eps;                       /* Algorithm 4.3 stop; 0: exact */
    int32_t precision;                     /* DCM_FP64 or DCM_MIXED */
    int32_t n_classes;                     /* cutoff classes, 2..8 */
    double cell_min;                       /* link-cell edge target; <= 0: auto */
    /* Verlet-list skin r_s in sigma (Section 2.2.1, Algorithm 3.3).  0: walk
       the link cells directly every step.  > 0: each particle keeps a list
       of every j within its list radius R_i (r_c[i] + skin, see
       list_margin), rebuilt (with a fresh cell sort) once some particle's
       displacement since the build plus the largest displacement reaches
       its headroom R_i - r_c[i](t), or when the list storage would
       overflow (that step falls back to the direct walk).  Requires at most
       2^24 particles per handle, a stencil of at most 7 cells in y and z,
       and list storage (n x min((4/3) pi (r_c,max + skin)^3,
       4 pi (r_c,min + skin)^3) entries) below 2^31 entries; dcm_create
       returns DCM_ERR_ARG otherwise. */
    double skin;
    /* Verlet lists built by the warp walk (DCM_MIXED): each
       particle's entry capacity is list_density x (4/3) pi R^3 + 8,
       rounded up to a multiple of 8, for its list radius R; <= 0: 1.0 per
       sigma^3.  A list that would overflow leaves that step's forces to the
       direct walk and raises the density by 25 % for the next build (per
       handle: system 0's value). */
    float list_density;
    /* With detected cutoffs, each list radius is the cutoff the particle
       would get if its interface distance fell by list_margin sigma, plus
       the skin, so that the jitter of the detected interface does not force
       a rebuild at every detection.  0: 1 sigma; < 0: no margin (per
       handle: system 0's value). */
    float list_margin;
    /* Adaptive skins (skin_time > 0): instead of skin/2 for every
       particle, particle i's share of a pair's skin is the distance it
       would cover in skin_time at constant acceleration,
       skin_time |v_i| + skin_time^2 |F_i| / (2 m), clamped to
       [skin_floor, skin/2] at the build, and the pair (i, j) is listed while
       it is closer than i's anticipated cutoff plus both shares.  Slow,
       weakly pushed particles then carry short lists and fast or strongly
       pushed ones do not force early rebuilds; skin still bounds every
       pair's skin.  skin_time = 0: uniform shares. */
    float skin_time;
    float skin_floor;
    /* Section 4.2 (Fig. 20-21): after the segmentation, liquid components
       of fewer than this many voxels become vapor, then vapor components
       (of that result) of fewer than this many become liquid, before the
       distance pass.  Components are 6-connected across the periodic
       faces.  0 (default): no removal.  Per system. */
    int32_t min_component_voxels;
    /* Cutoff function of particle i's distance to the interface:
       DCM_CUTOFF_EXP (default) is Eq. 7-8 with alpha; DCM_CUTOFF_LINEAR is
       the straight line of Section 3.1 / Fig. 12 from (0, rc_max) to
       (rc_max, rc_min), with Eq. 7's outer cases.  Per system. */
    int32_t cutoff_fn;
    /* Segmentation of the density image (Section 4.1).  DCM_SEG_KMEANS
       (default): two-class K-means on the smoothed density (Eq. 11-14).
       DCM_SEG_MUMFORD_SHAH: from those labels, Eq. 13 on the smoothed
       number density rho = Bs / (2^(3 smooth_order) V) with perimeter weight
       ms_nu (the thesis's 0.005 by default): rounds of exact phase means and
       ms_iters primal-dual iterations of its convex relaxation (Chan,
       Esedoglu, Nikolova; Chambolle-Pock, tau = sigma = 0.99/sqrt(12)), until
       the labels repeat or ms_outer rounds (1 by default: the K-means
       densities, then Eq. 13, as in Section 4.1; more rounds alternate the
       densities and the segmentation).  Per handle (system 0's; every
       system of an ensemble must agree). */
    int32_t segmentation;
    int32_t ms_iters;                      /* <= 0: 50 */
    int32_t ms_outer;                      /* <= 0: 1 */
    double ms_nu;                          /* >= 0; default 0.005 */
} dcm_params;

/* Force walk variants (dcm_tuning.walk).  DCM_WALK_WARP: one warp per
 * particle over its flattened candidate list, and with Verlet lists the
 * list force with list_lanes lanes per particle; DCM_MIXED always runs
 * these kernels (dcm_set_tuning refuses DCM_WALK_LANES for it with
 * DCM_ERR_ARG).  DCM_WALK_LANES: lanes[] lanes per particle walk its
 * stencil rows; DCM_FP64 always runs this walk, whatever is set. */
enum { DCM_WALK_WARP = 0, DCM_WALK_LANES = 1 };

/* Shape of the CUDA graph of one step (dcm_tuning.step_graph).  With the
 * warp Verlet-list kernels, DCM_GRAPH_BRANCHED (default) puts the work of a
 * list rebuild and the list force in conditional nodes on the rebuild
 * decision, so a step launches only the kernels it needs; DCM_GRAPH_FLAT
 * launches every kernel every step and each returns at once when it is not
 * its step (same results; profilers that cannot trace kernels inside
 * conditional graphs see every kernel). */
enum { DCM_GRAPH_BRANCHED = 0, DCM_GRAPH_FLAT = 1 };

/* Launch shape of the force kernel (the autotuner's output; see
 * dcm_set_tuning).  lanes[] and block apply to DCM_WALK_LANES. */
typedef struct {
    int32_t lanes[DCM_MAX_CLASSES];        /* lanes per particle: 1..32, pow2 */
    int32_t block;                         /* threads per block: 64..256 */
    int32_t walk;                          /* DCM_WALK_WARP (default) or DCM_WALK_LANES */
    int32_t list_lanes;                    /* warp walk + Verlet lists: lanes per particle of
                                              the list force, 4, 8, 16 or 32 (0: 8) */
    int32_t step_graph;                    /* DCM_GRAPH_BRANCHED or DCM_GRAPH_FLAT */
    int32_t list_lanes_class[DCM_MAX_CLASSES]; /* all 0 (default): list_lanes for every
                                              particle, in sorted-slot order.  Otherwise the
                                              list force runs class by class (heaviest
                                              first) with list_lanes_class[q] lanes (4, 8,
                                              16 or 32) per particle of cutoff class q, for
                                              every q < n_classes (Section 5.1's per-class
                                              schedule) */
    int32_t reserved[4];
} dcm_tuning;

typedef struct {
    int64_t step;                          /* global step counter */
    int64_t pairs;                         /* in-cutoff pairs, last force call */
    int32_t kmeans_iters;                  /* last detection */
    int32_t cfsm_iters;                    /* last detection */
    int32_t class_count[DCM_MAX_CLASSES];  /* particles per class */
    int32_t grid[3];                       /* voxel grid N_x, N_y, N_z */
    int32_t cells[3];                      /* link-cell grid */
    double c_liquid, c_vapor;              /* Eq. 14 cluster centres */
    int64_t guard_rechecks;                /* MIXED: FP64 re-decided pairs */
    int32_t kernels_plain;                 /* kernels one step launches (with
                                              Verlet lists: a step that rebuilds
                                              them) */
    int32_t kernels_detect;                /* ... in a step with detection */
    int64_t list_builds;                   /* Verlet-list builds so far */
    int64_t list_entries;                  /* entries of the current lists */
    int32_t kernels_plain_reuse;           /* kernels of a step that reuses its
                                              Verlet lists (= kernels_plain
                                              without lists) */
    int32_t kernels_detect_reuse;          /* ... in a step with detection */
    int64_t cc_flipped;                    /* voxels the small-component removal
                                              changed in the last detection */
    int64_t refined;                       /* MIXED: particles whose forces the last
                                              force pass evaluated again in
                                              double-float (net force below
                                              0.5 epsilon/sigma) */
} dcm_stats;

/* Phases of one step, in order, for dcm_get_phase_times. */
enum { DCM_PHASE_KICK_DRIFT = 0, DCM_PHASE_DETECT = 1, DCM_PHASE_BIN = 2,
       DCM_PHASE_FORCE = 3, DCM_PHASE_KICK = 4, DCM_NUM_PHASES = 5 };

typedef struct dcm_handle dcm_handle;

/* Fills the thesis defaults: rc 3/6, alpha -0.5, dt 0.005, m = eps = sigma
 * = 1, voxel 1, smoothing order 8, detect_every 2, FP64, 4 classes. */
void dcm_default_params(dcm_params *p);

/* Device memory.  A handle owns every device buffer it uses.  It allocates
 * them when it is created (and a few on first use: small-component removal
 * buffers; dcm_ms_segment's scratch, released before it returns), never
 * during a step, in the stream order of its stream: with
 * cudaMallocAsync / cudaFreeAsync from the device's default memory pool,
 * or, after dcm_set_allocator, with the caller's functions (for example a
 * framework's caching allocator), called as alloc(bytes, stream, ctx) ->
 * device pointer (NULL: out of memory) and release(ptr, stream, ctx) with
 * the handle's stream.  The setting is process-wide and taken by each
 * handle when it is created (handles keep theirs); both NULL restores the
 * default.  Errors: DCM_ERR_ARG when only one function is given. */
typedef void *(*dcm_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*dcm_release_fn)(void *ptr, void *stream, void *ctx);
int dcm_set_allocator(dcm_alloc_fn alloc, dcm_release_fn release, void *ctx);

/* Creates a single-system handle for n particles in box.  stream is a
 * cudaStream_t (NULL: the library creates one).  Allocates every device
 * buffer of the system.  Errors: DCM_ERR_ARG (n < 1, bad parameters),
 * DCM_ERR_BOX_TOO_SMALL, DCM_ERR_OOM, DCM_ERR_CUDA. */
int dcm_create(const dcm_box *box, int64_t n, const dcm_params *p,
               void *stream, dcm_handle **out);
int dcm_destroy(dcm_handle *h);

/* Copies positions (wrapped into the box) and velocities (NULL: zero) in.
 * Resets the step counter and marks cutoffs and forces stale. */
int dcm_set_state(dcm_handle *h, const double *x, const double *v, int mem);
/* Replaces the state of a running system (a host-side update inside a run:
 * a thermostat, a constraint, the host's copy handed back): positions
 * (wrapped into the box) and velocities (NULL: zero) in; the step counter,
 * the cutoffs of the last detection (refreshed at the next detection step,
 * Eq. 7 on the cadence of detect_every) and the Verlet lists are kept.  The
 * forces are recomputed from the new positions before the next step, and the
 * lists are rebuilt then only if the skin criterion (Algorithm 3.3, the
 * library's per-particle reuse test) finds that a particle moved beyond its
 * share since the last build.  Before the first force evaluation it acts as
 * dcm_set_state without resetting the step counter.  Single-system handles.
 * Errors: as dcm_set_state. */
int dcm_update_state(dcm_handle *h, const double *x, const double *v, int mem);
/* Copies positions, velocities and forces out; each pointer nullable. */
int dcm_get_state(dcm_handle *h, double *x, double *v, double *f, int mem);
int dcm_set_step(dcm_handle *h, int64_t step);

/* Supplies per-particle cutoffs directly (double[N], id order), bypassing
 * interface detection until the next dcm_detect_interface or detection
 * step.  Each must lie in [rc_min, rc_max]. */
int dcm_set_cutoffs(dcm_handle *h, const double *rc, int mem);

/* Section 4 + Algorithm 3.1 + Eq. 7: density image (Eq. 9), binomial
 * smoothing, two-class K-means labels (Eq. 11-14), CFSM distance
 * (Algorithm 4.3, band r_c,max + h), trilinear particle distance, cutoff
 * and class of every particle.  Enqueued; DCM_ERR_NOT_CONVERGED is
 * reported by the next dcm_sync if CFSM hit its cap. */
int dcm_detect_interface(dcm_handle *h);

/* Link-cell counting sort + Algorithm 3.2 with the cutoffs in use (detects
 * first if no cutoffs exist yet).  Enqueued. */
int dcm_compute_forces(dcm_handle *h);

/* nsteps of velocity Verlet (Eq. 1-2) with detection every detect_every
 * steps and r_c held in between; the loop runs from a CUDA graph with no
 * host round trip.  Enqueued. */
int dcm_step(dcm_handle *h, int64_t nsteps);

/* PE = 1/2 sum_i sum_{j: r_ij < r_c[i]} V(r_ij), KE = 1/2 m sum v^2,
 * w = 1/2 sum_i sum_j (r_ij)_a (F_i<-j)_b for ab = xx yy zz xy xz yz, at the
 * current positions and cutoffs (deterministic FP64 reduction).  Blocks. */
int dcm_energy_virial(dcm_handle *h, double *pe, double *ke, double w[6]);

/* Diagnostics (host pointers, blocking, each nullable). */
int dcm_get_grid(dcm_handle *h, int32_t dims[3], int32_t *counts,
                 double *smoothed, uint8_t *labels, double *dist);
int dcm_get_cutoffs(dcm_handle *h, double *d, double *rc, uint8_t *cls);
int dcm_get_cells(dcm_handle *h, int32_t nc[3], int32_t *cell_start,
                  int32_t *sorted_id);
int dcm_get_pair_counts(dcm_handle *h, int32_t *npair);
int dcm_get_stats(dcm_handle *h, dcm_stats *s);

/* Force-kernel launch shape per cutoff class (see dcm_tuning). */
int dcm_set_tuning(dcm_handle *h, const dcm_tuning *t);
int dcm_get_tuning(dcm_handle *h, dcm_tuning *t);

/* Phase timing: with on != 0 the step graphs record a CUDA event between
 * phases (a few microseconds of overhead); dcm_get_phase_times waits for
 * the stream and returns the device milliseconds of each phase of the
 * most recent step (DCM_PHASE_*; 0 for a phase the step skipped). */
int dcm_set_timing(dcm_handle *h, int on);
int dcm_get_phase_times(dcm_handle *h, float ms[DCM_NUM_PHASES]);

/* ---- ensembles: many independent systems in one handle --------------------
 * Batched form of the same method (no counterpart in the thesis, which runs
 * one system per MPI job): count systems of their own box, size and
 * parameters share one handle; every kernel of a step covers all of them
 * and the force kernel is a single persistent launch draining one work
 * queue over every system and cutoff class, so small systems fill the GPU
 * together.  Precision, detect_every, n_classes and smooth_order must be
 * the same for all systems.  Particles of system k occupy the slots
 * [first, first + count) of the concatenated arrays that dcm_set_state,
 * dcm_get_state, dcm_set_cutoffs, dcm_get_cutoffs and dcm_get_pair_counts
 * use; dcm_energy_virial returns the sums over all systems; dcm_get_grid and
 * dcm_get_cells describe system 0.  dcm_create is the count = 1 case. */
int dcm_ensemble_create(int count, const dcm_box *boxes, const int64_t *n,
                        const dcm_params *params, void *stream, dcm_handle **out);
int dcm_system_count(const dcm_handle *h);
int dcm_system_range(const dcm_handle *h, int k, int64_t *first, int64_t *count);
/* state of system k alone (AoS double[3*count]); set marks cutoffs and
 * forces of the whole handle stale */
int dcm_ensemble_set_state(dcm_handle *h, int k, const double *x, const double *v,
                           int mem);
int dcm_ensemble_get_state(dcm_handle *h, int k, double *x, double *v, double *f,
                           int mem);
int dcm_ensemble_energy_virial(dcm_handle *h, int k, double *pe, double *ke,
                               double w[6]);

/* Section 4.2 on a caller's label grid (diagnostics and tests): labels is
 * system 0's voxel grid in the layout of dcm_get_grid (x fastest; 0 liquid,
 * 1 vapor; other values belong to neither phase and stay), host or device
 * (mem), rewritten in place with the liquid components of fewer than
 * min_voxels voxels made vapor and then the vapor components of fewer than
 * min_voxels made liquid (min_voxels 0: unchanged).  flipped (nullable)
 * receives the voxels changed.  Uses the handle's stream and synchronises;
 * allocates the component forests on first use when the handle was created
 * without min_component_voxels.  The handle's own labels are untouched.
 * Errors: DCM_ERR_ARG, DCM_ERR_STATE (during stream capture), DCM_ERR_OOM,
 * DCM_ERR_CUDA, DCM_ERR_DEVICE_CHECK (a union ran out of attempts). */
int dcm_remove_small_components(dcm_handle *h, uint8_t *labels, int32_t min_voxels, int mem,
                                int64_t *flipped);

/* Eq. 13 (two-phase piecewise-constant Mumford-Shah) with fixed densities
 * on an image of system 0's voxel grid (diagnostics and tests; the detection
 * itself labels by K-means): rho (double[nvox], layout of dcm_get_grid, host
 * or device per mem) is segmented by minimising
 *   sum_liquid (rho - c_l)^2 + sum_vapor (rho - c_v)^2 + nu x (number of
 *   periodic grid faces between a liquid and a vapor voxel)
 * through the convex relaxation of Chan, Esedoglu and Nikolova, solved by
 * `iters` Chambolle-Pock iterations (tau 1/4, sigma 1/3) from u = 1/2;
 * labels (uint8[nvox]) = 0 where the relaxed u > 1/2, else 1; u_out
 * (nullable, double[nvox]) receives u.  FP64 in a fixed operation order.
 * Allocates and frees its scratch (7 doubles per voxel) and synchronises.
 * Errors: DCM_ERR_ARG (null pointers, nu < 0, iters < 0), DCM_ERR_STATE
 * (during stream capture), DCM_ERR_OOM, DCM_ERR_CUDA. */
int dcm_ms_segment(dcm_handle *h, const double *rho, double c_l, double c_v, double nu,
                   int32_t iters, uint8_t *labels, double *u_out, int mem);

/* Waits for the handle's stream; returns the sticky device error, if any. */
int dcm_sync(dcm_handle *h);
/* Failure-detection self-check (no counterpart in the thesis): launches the
 * library's bounded grid barrier with one block that never arrives.  The
 * waiting block gives up after its poll limit (well under a second), flags
 * the device error and returns, so the call returns DCM_ERR_DEVICE_CHECK
 * and the handle stays usable.  Any other result means waits are not
 * bounded. */
int dcm_check_bounded_wait(dcm_handle *h);

/* Measurement aid (no counterpart in the thesis): the FP32 FMA throughput of
 * the current device, from 8 independent chains of iters dependent FMAs per
 * thread on every SM, timed by CUDA events on a stream of its own.
 *   iters   chain length (>= 1; ~1e5 gives a launch of tens of ms)
 *   tflops  out: 2 * FMAs / time, in TFLOP/s
 *   ms      out (may be NULL): the timed launch's duration
 * Errors: DCM_ERR_ARG, DCM_ERR_CUDA. */
int dcm_fp32_peak(int32_t iters, double *tflops, double *ms);

/* ---- allocation-free link-cell sort ------------------------------------------
 * The thesis has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory when they need a cell list -- a host
 * application whose memory pool owns the whole device and forbids
 * allocations outside it, or a latency-bound loop that cannot afford
 * cudaMalloc/cudaFree (both synchronise the device).  It returns the same
 * cell list as the handle-based path (dcm_get_cells): cells of edge L/nc,
 * cell index = min(nc-1, floor(x * nc/L)) per axis, x fastest, particles of
 * a cell in ascending index.
 *
 *   x          device, AoS double[3*n], positions already wrapped into the box
 *   n          1 .. DCM_NOALLOC_MAX_PARTICLES
 *   box, nc    box edges and cells per axis; nc[0]*nc[1]*nc[2] must not
 *              exceed DCM_NOALLOC_MAX_CELLS
 *   cell_start device int32[ncell + 1], written (exclusive prefix of counts)
 *   sorted_id  device int32[n], written (particle indices in cell order)
 *   stream     cudaStream_t the work is enqueued on (NULL: legacy stream)
 *
 * It calls no cudaMalloc, cudaFree or allocating library routine: its scratch
 * (per-cell counts, per-particle slots, scan sums) is one fixed device array
 * of DCM_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current; make that first
 * call before any stream capture.  All calls share the array and it keeps the
 * last call's contents (the counts are cleared at the start of each call), so
 * calls that overlap on the GPU -- on different streams or devices' shared
 * contexts without ordering between them -- race and must be serialised by
 * the caller.  Errors: DCM_ERR_ARG for a null pointer, a non-positive edge or
 * cell count, or sizes beyond the maxima (nothing is launched); DCM_ERR_CUDA
 * if the set-up or a launch fails.  Returns after enqueueing the work. */
#define DCM_NOALLOC_MAX_PARTICLES (1 << 19)
#define DCM_NOALLOC_MAX_CELLS (1 << 20)
#define DCM_NOALLOC_SCRATCH_BYTES \
    (4 * (DCM_NOALLOC_MAX_CELLS + DCM_NOALLOC_MAX_PARTICLES + (DCM_NOALLOC_MAX_CELLS + 2047) / 2048))
int dcm_cell_sort_noalloc(const double *x, int64_t n, const dcm_box *box,
                          const int32_t nc[3], int32_t *cell_start,
                          int32_t *sorted_id, void *stream);

/* Total device bytes the handle holds. */
int64_t dcm_device_bytes(const dcm_handle *h);
/* Device bytes dcm_create would allocate for this system. */
int64_t dcm_estimate_bytes(const dcm_box *box, int64_t n, const dcm_params *p);

const char *dcm_last_error(void);
int dcm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DCM_H */
