// dcm_internal.cuh -- internal declarations of libdcm (sm_103a).
//
// A handle holds M >= 1 independent systems (M = 1 from dcm_create, M =
// count from dcm_ensemble_create).  Every kernel works on all systems at
// once: per-system arrays are concatenated and each element finds its
// system from the offset tables (p_off over particles, c_off over link
// cells, v_off over voxels) of the device system table.
//
// Device data layout (all in HBM, allocated once at creation; N, Nc, Nv are
// totals over the systems):
//   state     x, v, f : double SoA [3][N] in the caller's particle order
//   cutoffs   d, rc   : double [N];  cls : uint8 [N]   (id order)
//   link cells        : cell_of[N], slot[N] (id order); cell_count[Nc],
//                       cell_start[Nc+1], sorted_id[N]; sp4[N] float4
//                       (cell-relative x,y,z in FP32 on the grid qpos, cell
//                       x index), MIXED: spl4[N] float4 (the FP32 remainders
//                       of the cell-relative x,y,z) and FP64: spd[N]
//                       double4_32a (absolute x,y,z), all in cell order;
//                       MIXED: rq[N] float4 (r_c^2 and its guard band, culling
//                       radius) and pk[N] int4 (id, cell y, cell z) in cell order
//   voxel grid        : B int32, sm1/sm2 uint32 (smoothing passes), Bs double,
//                       S uint8, D0/D1 double (CFSM ping-pong), stamp int32,
//                       four frontier lists int32 [Nv]
//   per-particle      : npair int32, pe double, vir double [6][N]
// Cells and voxels are indexed x fastest: c = cx + nx*(cy + ny*cz).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dcm.h"

#define DCM_CHECK_CUDA(call)                                                   \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) return dcm::fail_cuda(e_, #call, __FILE__, __LINE__); \
    } while (0)

namespace dcm {

// sticky device error bits (dcm_sync maps them to status codes)
enum : int {
    DEV_ERR_NONFINITE = 1,       // non-finite position or velocity
    DEV_ERR_JUMP = 2,            // moved more than a box edge in one step
    DEV_ERR_BARRIER = 4,         // a bounded grid barrier gave up
    DEV_ERR_CFSM_CAP = 8,        // CFSM hit iter_max
    DEV_ERR_DENSITY = 16,        // voxel count too large for exact smoothing
    DEV_ERR_CANCEL = 32,         // cancel flag observed
    DEV_ERR_BOUNDS = 64,         // an index check failed
    DEV_ERR_UNION = 128          // a component union ran out of attempts
};

// counters written by device code, read back for dcm_get_stats
struct DevStats {
    unsigned long long guard_rechecks;
    unsigned long long pairs;
    int kmeans_iters;            // largest over the systems
    int cfsm_iters;              // passes of the last CFSM run
    double c_liquid;             // system 0
    double c_vapor;
    int class_count[DCM_MAX_CLASSES];
    unsigned int barrier[8];     // [0..1] grid barrier, [2] force queue, [3] CFSM result buffer,
                                 // [4] first CFSM pass of the cluster tail, [5] list-force queue,
                                 // [6] particles queued for the double-float refinement,
                                 // [7] particles the list kernels refined in place
    unsigned long long list_builds;
    unsigned long long list_entries;
    unsigned long long cc_flipped;   // voxels the small-component removal changed (last detection)
};

// Verlet-list control words (device): see dcm_list.cu
// Verlet-list control words: rebuild decision, lists valid, the two maxima
// of the check, its block counter, a per-particle capacity overflow seen by
// the last fill, the capacity density scale (float bits), the largest skin
// share of the build (float bits), the fill gate
enum { LF_REBUILD = 0, LF_OK = 1, LF_PARTNER = 2, LF_EXCESS = 3, LF_DONE = 4, LF_OVERFLOW = 5,
       LF_SCALE = 6, LF_SHMAX = 7, LF_FILL = 8, LF_WORDS = 9 };
// LF_PARTNER and LF_EXCESS hold order-preserving int images of floats; this
// is the image of -3.39e38 (every byte 0x80, so a memset writes it too)
constexpr int LF_EXCESS_RESET = (int)0x80808080u;

constexpr int MAX_SYSTEMS = 1024;

// geometry and parameters passed by value to kernels
struct Geom {
    int n;
    double L[3], halfL[3];
    int nc[3];                   // link cells per axis
    double inv_c[3];             // nc / L  (cell index = floor(x * inv_c))
    double cedge[3];             // L / nc
    float cf[3], inv_cf[3];      // FP32 cell edges (cf: a multiple of qpos) and inverses
    float cfl[3];                // cedge - cf in FP32 (the low part of the cell edge)
    float qpos;                  // grid of the FP32 cell-relative positions (a power of two)
    float inv_qpos;              // 1 / qpos (exact)
    float qtop;                  // 2^24 qpos: grid values below it in magnitude are exact in FP32
    int smax[3];                 // largest stencil radius in cells
    int gd[3];                   // voxels per axis
    double inv_h[3];             // gd / L
    double h[3];                 // L / gd
    double r_grid;               // CFSM band: rc_max + max h
    double w_h[3];               // 1 / h^2 per axis (the Godunov weights)
    double e_min;                // 1 / sqrt(sum w): smallest possible Godunov step
    double rc_min, rc_max, alpha, cut_a, cut_b;
    int cut_fn;                  // DCM_CUTOFF_EXP (Eq. 7) or DCM_CUTOFF_LINEAR (Fig. 12)
    double cut_slope;            // linear: (rc_max - rc_min) / rc_max
    int K;
    double thr[DCM_MAX_CLASSES]; // class thresholds on d (descending)
    double dt, hdtm;             // dt, dt/(2m)
    double eps, sigma;
    double skin;                 // Verlet-list skin (0: direct cell walk)
    int64_t corner_off;          // this system's cell corner coordinates in Batch::corner
    float halfLf[3];             // FP32 half edges
    float skin_time, skin_floor; // velocity-adaptive skin shares (skin_time 0: skin/2 each)
    int cc_min;                  // Section 4.2: components below this many voxels change phase (0: off)
    double ms_nu;                // Eq. 13: perimeter weight (number-density units)
    float ms_nuf;                // ... rounded to FP32 once (the iteration's precision)
    int ms_seg;                  // Eq. 13 segmentation after K-means (DCM_SEG_MUMFORD_SHAH)
    double ms_inv_scale;         // Eq. 13: 1 / (2^(3 smooth_order) V): smoothed counts -> number density
    unsigned long long div_gd[2];  // ceil(2^64 / gd[a]), a = 0, 1: exact 32-bit division by gd[a]
    unsigned long long div_nc[2];  // ceil(2^64 / nc[a]), a = 0, 1: exact 32-bit division by nc[a]
                                   // as the high word of a 64-bit product (Granlund-Montgomery)
    double eps24, eps48, eps2, sig2;     // LJ force/energy constants
    float eps24f, eps48f, eps2f, sig2f;
    float eps24l, eps48l, sig2l;         // low parts: eps48 - eps48f, ... (close pairs)
    float rclose2;               // mixed: pairs with FP32 r^2 below this take the double-float path
    float redo_f2;               // mixed: a particle whose |F|^2 is below this is redone in double-float
    // this system's slices of the concatenated arrays
    int64_t p0, c0, v0;
    int64_t ncell, nvox;
};

// the system table every kernel receives
struct Batch {
    const Geom *sys;             // device table [M]
    const int64_t *p_off;        // [M+1] particle offsets
    const int64_t *c_off;        // [M+1] cell offsets
    const int64_t *v_off;        // [M+1] voxel offsets
    const uint16_t *psys;        // [N] system of each particle (null when M == 1)
    const uint16_t *vsys;        // [NV] system of each voxel (null when M == 1)
    const double *corner;        // cell corner coordinate c * L/n per axis and system
    int M;
    int K;                       // cutoff classes (same for all systems)
    int64_t N, NC, NV;           // totals
};

// system of particle i / voxel v: a table lookup (M == 1: system 0)
__device__ __forceinline__ int sys_p(const Batch &b, int64_t i) { return b.M == 1 ? 0 : (int)b.psys[i]; }
__device__ __forceinline__ int sys_v(const Batch &b, int64_t v) { return b.M == 1 ? 0 : (int)b.vsys[v]; }

// system owning element idx of a concatenated array (largest s with off[s] <= idx)
__device__ __forceinline__ int sys_of(const int64_t *off, int M, int64_t idx)
{
    int lo = 0, hi = M - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&off[mid]) <= idx)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

}  // namespace dcm

struct dcm_handle {
    int M;                       // systems in this handle
    dcm_box box;                 // system 0 (single-system convenience)
    int64_t n;                   // total particles
    dcm_params p;                // system 0's parameters (shared fields:
                                 // precision, detect_every, n_classes,
                                 // smooth_order, iteration caps)
    dcm_tuning tune;
    dcm::Geom g;                 // system 0's geometry
    dcm::Geom *geo_host;         // [M]
    dcm_params *par_host;        // [M]
    int64_t *off_host;           // [3*(M+1)]: p_off, c_off, v_off
    dcm::Geom *geo_dev;
    int64_t *off_dev;
    dcm::Batch b;
    cudaStream_t stream;
    bool own_stream;
    dcm_alloc_fn alloc;          // the caller's allocator (null: cudaMallocAsync on the stream)
    dcm_release_fn release;
    void *alloc_ctx;
    int device;
    int num_sms;
    int64_t ncell, nvox;
    int64_t bytes;
    double *corner, *corner_host;   // cell corner coordinates (device, host copy)

    // state
    double *x, *v, *f;
    double *tmp3n;               // AoS <-> SoA staging, 3N doubles
    double *d, *rc;
    uint8_t *cls;
    // link cells
    int32_t *cell_of, *slot, *cell_count, *cell_start, *sorted_id, *scan_tmp;
    float4 *sp4;
    float4 *spl4;                // MIXED: low parts of the cell-relative positions
    int32_t *refq;               // MIXED: sorted slots queued for the double-float refinement
    double4_32a *spd;
    float4 *rq;                  // MIXED: per sorted slot r_c^2, guard band, culling radius
    int32_t *inv;                // sorted slot of each particle (id order), MIXED
    uint16_t *psys, *vsys;       // system of each particle / voxel (M > 1)
    int4 *pk;                    // MIXED: per sorted slot particle id, cell y, cell z
    int32_t *class_list;         // sorted slots grouped by class
    int32_t *class_count_dev;    // [K] counts, [K..2K) cursors
    // grid
    int32_t *B;
    uint32_t *sm1, *sm2;
    double *Bs;
    uint8_t *S;
    double *D0, *D1;
    int32_t *stamp;
    int32_t *flist;              // 4 * nvox
    int32_t *fcount;             // 4 counters
    int32_t *cc;                 // small components: parent and count of each phase, local sizes
                                 // (5 * nvox), a uniform flag per tile
    int64_t *cc_tiles;           // [M+1] offsets of the systems' 8^3 tiles (device)
    float *msbuf;                // Eq. 13 segmentation (FP32): u, u-bar x 2, r, duals x 2 x 3 planes (10 * nvox)
    unsigned long long *msacc;   // ... per system: phase sums and voxel counts (4 * M)
    double *msc;                 // ... per system: the round's densities (2 * M)
    int *msflag;                 // ... per system: segmenting, changed (2 * M)
    int64_t cc_ntiles, cc_ntiles0;   // tiles of all systems / of system 0
    bool cc_on;                  // some system removes small components
    // Verlet lists (skin > 0), indexed by sorted slot of the last build
    int32_t *nl;                 // entries: j | (dy+8) << 24 | (dz+8) << 28
    int64_t nl_cap;
    int32_t *nl_cnt, *nl_start, *nl_tiles;
    double *x_ref;               // positions at the build (id order)
    float *rl_ref;               // own list radius of each particle at the build (id order)
    float *sh_ref;               // skin share of each particle at the build (id order)
    float *sh;                   // skin share per sorted slot (the fill's partners)
    float4 *u_ref;               // warp lists: cell-relative FP32 position at the build (id order)
    float *disp;                 // warp lists: |displacement| since the build, this step (id order)
    bool cut_detected;           // cutoffs come from detection (lists anticipate d moves)
    bool list_warp;              // lists built and walked by the warp kernels (set per capture)
    bool step_detect;            // the step being enqueued re-detects the interface
    float list_scale0;           // initial capacity density of those lists
    float list_margin;           // interface-distance margin of the list radius (sigma)
    int *lflags;                 // LF_* words
    // per particle diagnostics / energies
    int32_t *npair;
    double *pe, *vir;
    double *red_part, *red_out;
    unsigned long long *kacc;    // K-means accumulators: M x (max, min, total, 3 x (count, sum))
    double *kstate;              // K-means per-system centres / previous counts: M x 4
    int *err;
    dcm::DevStats *stats;
    double *dfinal;              // which D buffer holds the result

    // host-side status
    bool have_state, have_cut, forces_valid, cells_valid;
    bool keep_lists;             // the next eager force evaluation lets the reuse test decide
    int64_t step;
    int class_count_host[DCM_MAX_CLASSES];

    // CUDA graphs of one step (without / with detection)
    cudaGraphExec_t g_plain, g_detect;
    bool graphs_ready;
    int coop_blocks;             // co-resident blocks for the persistent kernels
    // conditional branches of a captured step: k_list_check sets `cond` to
    // the rebuild decision, graph IF nodes on it hold the rebuild-only work
    cudaStream_t side;                  // records the branch bodies
    cudaGraphConditionalHandle cond;    // the rebuild decision of the graph being captured
    bool branching;                     // enqueue_step is recording a graph with branches
    bool fold_check;                    // the step's drift / cutoff kernel runs the reuse test
    bool in_step;                       // enqueue_step: the drift zeroes the force queues
    int br_kernels[2];                  // kernels in bodies taken on rebuild / reuse
    // kernel nodes of one captured step: [plain, detect] x [rebuild, reuse]
    int kernels_plain, kernels_detect, kernels_plain_reuse, kernels_detect_reuse;
    // phase timing: events[0..DCM_NUM_PHASES] bracket the phases
    bool timing;
    cudaEvent_t ev[DCM_NUM_PHASES + 1];
    bool last_detect;
};

namespace dcm {

int fail(int code, const char *fmt, ...);
int fail_cuda(cudaError_t e, const char *what, const char *file, int line);

// launchers (each enqueues on h->stream; return DCM_OK or an error code)
int launch_kick_drift(dcm_handle *h);
int launch_kick(dcm_handle *h);
int launch_bin(dcm_handle *h);                      // full cell sort + classes
int launch_bin_gated(dcm_handle *h, const int *gate, const int *class_gate);  // sort, gather, classes
int launch_sort_gather(dcm_handle *h, const int *gate);    // cell sort + gather
int launch_classes(dcm_handle *h, const int *class_gate);  // class lists
void list_mode(dcm_handle *h);          // sets list_warp from precision, tuning and lists
struct ListTest;
ListTest list_test(dcm_handle *h, bool partner, bool excess, bool decide);
void launch_iota(dcm_handle *h, int32_t *p, int64_t n);
void launch_sys_tables(dcm_handle *h);
int launch_scan(dcm_handle *h, const int32_t *in, int32_t *out, int32_t *tiles, int64_t m,
                int32_t total, const int *gate);     // exclusive scan (total < 0: out[m] = sum)
int launch_list_step(dcm_handle *h, bool force_rebuild);  // decide, [rebin], lists
int launch_list_walk(dcm_handle *h, bool fill, const int *gate, float delta);
int launch_forces(dcm_handle *h, bool energy);   // list mode when skin > 0 and the lists are ok
// warp Verlet-list forces: part 0 the rebuild step's direct walk + fill,
// part 1 the list force, 2 both (each kernel returns at once when it is not
// its step)
int launch_list_forces(dcm_handle *h, bool energy, int part);
int launch_detect(dcm_handle *h);
int launch_ms_detect(dcm_handle *h);     // Eq. 13 from the K-means labels (DCM_SEG_MUMFORD_SHAH)
// Section 4.2 on labels S of the systems in b (thr >= 0 overrides every
// system's min_component_voxels); tiles: their 8^3 tiles
int launch_components(dcm_handle *h, const Batch &b, uint8_t *S, int thr, int64_t tiles);
int launch_reduce_energy(dcm_handle *h, int k);
int launch_reduce_pairs(dcm_handle *h);
int launch_classify_rc(dcm_handle *h);   // classes from supplied rc

// A branch of a captured step on the Verlet-list rebuild decision (a CUDA
// graph IF node on h->cond).  Between branch_open and branch_close the work
// enqueued on h->stream is recorded into body 0, taken on a step that
// rebuilds the lists, and after branch_else into body 1, taken on a step that
// reuses them.  Outside a capture, or without the warp list kernels, the
// three calls do nothing and the kernels' own gates decide.
struct Branch {
    bool active;
    int nbody, cur;
    cudaGraph_t body[2];
    cudaStream_t main;
};
int branch_open(dcm_handle *h, Branch &b, int nbody);     // an IF node on h->cond
int branch_else(dcm_handle *h, Branch &b);
int branch_close(dcm_handle *h, Branch &b);

// device scratch from the handle's allocator, in its stream order
int dev_alloc(dcm_handle *h, void **p, size_t bytes);
void dev_free(dcm_handle *h, void *p, size_t bytes);

// lower-level helpers
int coop_grid_size(dcm_handle *h, const void *kernel, int block, size_t smem);
int prepare_kernels(dcm_handle *h);      // per-handle kernel attributes
int prepare_force_kernels();             // force-kernel attributes
int launch_barrier_timeout_check(dcm_handle *h);

}  // namespace dcm
