// dcm_force.cu -- the DCM force sum, Algorithm 3.2:
//     F_i = sum_{j != i, |r_ij| < r_c[i]} F_LJ(r_ij)
// over a full neighbourhood with no Newton-3 (the thesis, Section 3.2: the
// interaction is asymmetric, so each particle sums its own force only).
//
// GPU design (not the thesis's LAMMPS/Verlet-list design):
//  * Particles are sorted by link cell (cells of edge ~r_c,min/2, the
//    "improved bins" of Fig. 13b).  For particle i the stencil is walked row
//    by row: a row is a run of cells along x at fixed (y, z) cell offset and
//    is contiguous in the sorted arrays.  Rows whose y/z box distance
//    exceeds r_c[i] are skipped and each row is trimmed in x to the chord of
//    the cutoff sphere, so the candidates approach the sphere volume.
//  * DCM_FP64 (the lanes walk, k_force): G lanes (1..32, per cutoff class)
//    share one particle and stride through the row, so loads of the sorted
//    double stream are coalesced; a shuffle tree combines the G partial
//    sums.  Absolute FP64 positions, minimum image and r^2 evaluated exactly
//    as the FP64 definition; FP64 forces and accumulation.
//  * Work is handed out warp by warp from a device queue ordered from the
//    largest-cutoff class down (the GPU analogue of the thesis's
//    schedule(dynamic,20), Algorithm 5.1): interfacial particles, whose
//    cutoff makes them 8-13x more expensive, start first and the cheap bulk
//    fills in behind them.
//  * DCM_MIXED (the warp kernels: direct walk k_force_warp, Verlet-list
//    force k_force_list_warp): positions are stored relative to their cell
//    corner in FP32 on a power-of-two grid, with their FP32 remainders
//    beside them.  Pair distances and forces are FP32 for pairs beyond
//    1.5 sigma; closer pairs, whose forces are large and cancel in the sum,
//    are evaluated in double-float arithmetic from the exact displacement.
//    Lane partials are summed exactly in fixed point.  Pairs whose FP32 r^2
//    is within a relative 2^-18 of r_c^2 are re-decided in FP64 with the
//    exact FP64 rule, so the set of interacting pairs is the same as in FP64.
// Bound: FP32 pipe (mixed) or FP64 pipe (FP64); algorithmic work per
// in-cutoff pair = 8 flops for the distance test + 16 for the force.
#include "dcm_device.cuh"

namespace dcm {

constexpr int FORCE_THREADS = 256;

// the cell and LJ constants of a single-system launch (kernel parameters)
struct ListConst {
    float cf[3], cfl[3], ncx, halfnc, inv_ncx;
    float sig2f, eps48f, eps24f, eps2f;
    float sig2l, eps48l, eps24l, rclose2, redo_f2, qtop;
};

struct ForceArgs {
    Batch b;
    const int32_t *class_buf;     // [0..K) counts, [K..2K) offsets
    int list_g[DCM_MAX_CLASSES];  // list force, per-class schedule: lanes per particle of class q
    const int32_t *class_list;    // sorted slots grouped by class
    int lanes[DCM_MAX_CLASSES];   // lanes per particle per class
    const float4 *sp4;
    const float4 *spl4;           // MIXED: remainders of the cell-relative positions
    int32_t *refq;                // MIXED: sorted slots queued for the double-float refinement
    unsigned int *refq_n;         // ... and their number
    unsigned int *refined_n;      // particles the list kernels refined in place
    const double4_32a *spd;
    const float4 *rq;             // MIXED: r_c^2, guard band, culling radius per slot
    const int4 *pk;               // MIXED: id, cell y, cell z per slot
    const int32_t *cell_start;
    const int32_t *sorted_id;
    const int32_t *cell_of;
    const double *x;              // id-order SoA (FP64 re-decisions)
    const double *rc;
    double *f;
    int32_t *npair;
    double *pe, *vir;
    unsigned int *queue;          // work counter
    unsigned long long *guard_count;
    unsigned long long *list_entries;
    int *list_flags;              // LF_* words (Verlet lists)
    // Verlet lists (skin > 0): used while *list_ok
    const int *list_ok;
    const int32_t *nl_start;
    const int32_t *nl;
    // list build (k_list_walk)
    int32_t *nl_cnt, *nl_w;
    float *rl_ref;                // own list radius of each particle at the build (id order)
    float *sh_ref;                // skin share of each particle at the build (id order)
    const float *sh;              // skin share per sorted slot (warp fill)
    ListConst lc;                 // one system: its cell and LJ constants
    Geom g0;                      // one system: its geometry (kernel parameter space)
    const double *d;
    float list_delta;
    const int *gate;
};

// exact FP64 decision |r_ij| < r_c[i] (the definition's arithmetic)
__device__ __forceinline__ bool fp64_inside(const ForceArgs &a, const Geom &g, int i, int j,
                                            double rci2)
{
    size_t n = (size_t)a.b.N;
    double dx = min_image(DSUB(a.x[i], a.x[j]), g.L[0], g.halfL[0]);
    double dy = min_image(DSUB(a.x[n + i], a.x[n + j]), g.L[1], g.halfL[1]);
    double dz = min_image(DSUB(a.x[2 * n + i], a.x[2 * n + j]), g.L[2], g.halfL[2]);
    return r2_rn(dx, dy, dz) < rci2;
}

// per-lane FP64 sums of one particle (the lanes walk of the FP64 path)
template <bool ENERGY>
struct Acc64 {
    double fx = 0.0, fy = 0.0, fz = 0.0, pe = 0.0;
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
};

// one FP64 pair (the definition's arithmetic: minimum image, r^2, the
// strict test against r_c[i]^2)
template <bool ENERGY>
__device__ __forceinline__ void pair64(const Geom &g, double4_32a pi, double4_32a pj, double rci2,
                                       bool self, Acc64<ENERGY> &acc, int &np)
{
    double dx = min_image(DSUB(pi.x, pj.x), g.L[0], g.halfL[0]);
    double dy = min_image(DSUB(pi.y, pj.y), g.L[1], g.halfL[1]);
    double dz = min_image(DSUB(pi.z, pj.z), g.L[2], g.halfL[2]);
    double r2 = r2_rn(dx, dy, dz);
    if (r2 < rci2 && !self) {
        double r2inv = 1.0 / r2;
        double sr2 = g.sig2 * r2inv;
        double sr6 = sr2 * sr2 * sr2;
        double fr = r2inv * sr6 * (g.eps48 * sr6 - g.eps24);
        acc.fx += fr * dx;
        acc.fy += fr * dy;
        acc.fz += fr * dz;
        ++np;
        if constexpr (ENERGY) {
            acc.pe += g.eps2 * sr6 * (sr6 - 1.0);
            double fx = fr * dx, fy = fr * dy, fz = fr * dz;
            acc.v[0] += 0.5 * dx * fx;
            acc.v[1] += 0.5 * dy * fy;
            acc.v[2] += 0.5 * dz * fz;
            acc.v[3] += 0.5 * dx * fy;
            acc.v[4] += 0.5 * dx * fz;
            acc.v[5] += 0.5 * dy * fz;
        }
    }
}

// box distance along one axis from a point at u in [0, c) of its own cell
// to the cell at offset d
__device__ __forceinline__ float box_gap(int d, float u, float c)
{
    float gap = d > 0 ? (float)d * c - u : (d < 0 ? u - (float)(d + 1) * c : 0.f);
    return gap > 0.f ? gap : 0.f;
}

template <bool ENERGY>
__device__ __forceinline__ void reduce_and_store(const ForceArgs &a, Acc64<ENERGY> &acc, int i,
                                                 int lane, int G, unsigned gmask, int np)
{
    // combine the G lanes of this particle
    double fx = acc.fx, fy = acc.fy, fz = acc.fz, pe = 0.0, vir[6] = {0, 0, 0, 0, 0, 0};
    if constexpr (ENERGY) {
        pe = acc.pe;
        for (int q = 0; q < 6; ++q) vir[q] = acc.v[q];
    }
    for (int off = G >> 1; off > 0; off >>= 1) {
        fx += __shfl_xor_sync(gmask, fx, off);
        fy += __shfl_xor_sync(gmask, fy, off);
        fz += __shfl_xor_sync(gmask, fz, off);
        np += __shfl_xor_sync(gmask, np, off);
        if constexpr (ENERGY) {
            pe += __shfl_xor_sync(gmask, pe, off);
            for (int q = 0; q < 6; ++q) vir[q] += __shfl_xor_sync(gmask, vir[q], off);
        }
    }
    if (lane == 0) {
        size_t n = (size_t)a.b.N;
        a.f[i] = fx;
        a.f[n + i] = fy;
        a.f[2 * n + i] = fz;
        a.npair[i] = np;
        if constexpr (ENERGY) {
            a.pe[i] = pe;
            for (int q = 0; q < 6; ++q) a.vir[q * n + i] = vir[q];
        }
    }
}

// FP64 lanes walk of particle k (sorted slot): G lanes stride through each
// stencil row; rows beyond r_c[i] are skipped and each row is trimmed in x
// to the chord of the cutoff sphere (FP32 geometry on the cell-relative
// positions, conservative by the culling margin)
template <bool ENERGY>
__device__ __forceinline__ void particle_force(const ForceArgs &a, int k, int lane, int G, unsigned gmask, int &ng)
{
    const Geom &g = a.b.sys[sys_p(a.b, k)];
    int i = a.sorted_id[k];
    float4 ui = a.sp4[k];
    int c = a.cell_of[i] - (int)g.c0;
    int cx = (int)ui.w;
    int cy = (c / g.nc[0]) % g.nc[1];
    int cz = c / (g.nc[0] * g.nc[1]);
    double rci = a.rc[i];
    double rci2 = DMUL(rci, rci);
    // conservative culling radius (covers the FP32 geometry error)
    float rcull = fmaf((float)rci, 1.00002f, 1e-4f);
    float rcull2 = rcull * rcull;
    int sx = min(g.smax[0], (int)ceilf(rcull * g.inv_cf[0]));
    int sy = min(g.smax[1], (int)ceilf(rcull * g.inv_cf[1]));
    int sz = min(g.smax[2], (int)ceilf(rcull * g.inv_cf[2]));
    const double4_32a pi = a.spd[k];
    Acc64<ENERGY> acc;
    int np = 0;
    auto segment = [&](int j0, int j1) {
        for (int j = j0 + lane; j < j1; j += G) pair64<ENERGY>(g, pi, a.spd[j], rci2, j == k, acc, np);
    };
    for (int dz = -sz; dz <= sz; ++dz) {
        float gz = box_gap(dz, ui.z, g.cf[2]);
        float remz = fmaf(-gz, gz, rcull2);
        if (remz < 0.f) continue;
        int czz = cz + dz;
        czz += czz < 0 ? g.nc[2] : (czz >= g.nc[2] ? -g.nc[2] : 0);
        for (int dy = -sy; dy <= sy; ++dy) {
            float gy = box_gap(dy, ui.y, g.cf[1]);
            float w2 = fmaf(-gy, gy, remz);
            if (w2 < 0.f) continue;
            int cyy = cy + dy;
            cyy += cyy < 0 ? g.nc[1] : (cyy >= g.nc[1] ? -g.nc[1] : 0);
            float w = sqrtf(w2);
            int xlo = max(-sx, (int)floorf((ui.x - w) * g.inv_cf[0]));
            int xhi = min(sx, (int)floorf((ui.x + w) * g.inv_cf[0]));
            int row = (int)g.c0 + g.nc[0] * (cyy + g.nc[1] * czz);
            int lo = cx + xlo, hi = cx + xhi;
            if (lo < 0) {
                // cells at the top end seen through the x = 0 face
                segment(a.cell_start[row + lo + g.nc[0]], a.cell_start[row + g.nc[0]]);
                lo = 0;
            }
            if (hi >= g.nc[0]) {
                segment(a.cell_start[row], a.cell_start[row + hi - g.nc[0] + 1]);
                hi = g.nc[0] - 1;
            }
            if (lo <= hi) segment(a.cell_start[row + lo], a.cell_start[row + hi + 1]);
        }
    }
    reduce_and_store<ENERGY>(a, acc, i, lane, G, gmask, np);
}

// Algorithm 3.2 over particle k's Verlet list (entries: sorted slot j,
// cell row offsets dy, dz) in FP64: the same pair rule, so the interacting
// pairs are those of the direct walk
template <bool ENERGY>
__device__ __forceinline__ void particle_force_list(const ForceArgs &a, int k, int lane, int G,
                                                    unsigned gmask, int &ng)
{
    const Geom &g = a.b.sys[sys_p(a.b, k)];
    int i = a.sorted_id[k];
    double rci = a.rc[i];
    double rci2 = DMUL(rci, rci);
    const double4_32a pi = a.spd[k];
    Acc64<ENERGY> acc;
    int np = 0;
    const int e0 = a.nl_start[k], e1 = a.nl_start[k + 1];
    int p = e0 + lane;
    for (; p + G < e1; p += 2 * G) {
        int ea = a.nl[p], eb = a.nl[p + G];
        pair64<ENERGY>(g, pi, a.spd[ea & 0xffffff], rci2, false, acc, np);
        pair64<ENERGY>(g, pi, a.spd[eb & 0xffffff], rci2, false, acc, np);
    }
    for (; p < e1; p += G) pair64<ENERGY>(g, pi, a.spd[a.nl[p] & 0xffffff], rci2, false, acc, np);
    reduce_and_store<ENERGY>(a, acc, i, lane, G, gmask, np);
}

// one particle of the list build: the direct row walk with radius
// list_radius; COUNT stores the number of entries, FILL writes them in
// walk order (a ballot over the G lanes keeps the order)
template <bool FILL>
__device__ __forceinline__ void list_particle(const ForceArgs &a, int k, int lane, int G,
                                              unsigned gmask)
{
    const Geom &g = a.b.sys[sys_p(a.b, k)];
    int i = a.sorted_id[k];
    float4 ui = a.sp4[k];
    int c = a.cell_of[i] - (int)g.c0;
    int cx = (int)ui.w;
    int cy = (c / g.nc[0]) % g.nc[1];
    int cz = c / (g.nc[0] * g.nc[1]);
    // uniform skin shares here: the pair radius is the own radius + skin/2
    const float share = 0.5f * (float)g.skin;
    float rl = list_radius(g, a.rc[i], a.d[i], a.list_delta, share) + share;
    float rl2 = rl * rl;
    float rcull = fmaf(rl, 1.00002f, 1e-4f);
    float rcull2 = rcull * rcull;
    int sx = min(g.smax[0], (int)ceilf(rcull * g.inv_cf[0]));
    int sy = min(g.smax[1], (int)ceilf(rcull * g.inv_cf[1]));
    int sz = min(g.smax[2], (int)ceilf(rcull * g.inv_cf[2]));
    const int gbase = (threadIdx.x & 31) & ~(G - 1);
    const unsigned gbits = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
    const unsigned below = (1u << lane) - 1u;
    int n = 0;
    int32_t *out = FILL ? a.nl_w + a.nl_start[k] : nullptr;
    for (int dz = -sz; dz <= sz; ++dz) {
        float gz = box_gap(dz, ui.z, g.cf[2]);
        float remz = fmaf(-gz, gz, rcull2);
        if (remz < 0.f) continue;
        int czz = cz + dz;
        czz += czz < 0 ? g.nc[2] : (czz >= g.nc[2] ? -g.nc[2] : 0);
        float az = fmaf(-(float)dz, g.cf[2], ui.z);
        for (int dy = -sy; dy <= sy; ++dy) {
            float gy = box_gap(dy, ui.y, g.cf[1]);
            float w2 = fmaf(-gy, gy, remz);
            if (w2 < 0.f) continue;
            int cyy = cy + dy;
            cyy += cyy < 0 ? g.nc[1] : (cyy >= g.nc[1] ? -g.nc[1] : 0);
            float ay = fmaf(-(float)dy, g.cf[1], ui.y);
            float w = sqrtf(w2);
            int xlo = max(-sx, (int)floorf((ui.x - w) * g.inv_cf[0]));
            int xhi = min(sx, (int)floorf((ui.x + w) * g.inv_cf[0]));
            int row = (int)g.c0 + g.nc[0] * (cyy + g.nc[1] * czz);
            uint32_t tag = ((uint32_t)(dy + 8) << 24) | ((uint32_t)(dz + 8) << 28);
            int lo = cx + xlo, hi = cx + xhi;
            for (int q = 0; q < 3; ++q) {
                int j0, j1;
                float ax;
                if (q == 0) {            // cells at the top end seen through x = 0
                    if (lo >= 0) continue;
                    j0 = a.cell_start[row + lo + g.nc[0]];
                    j1 = a.cell_start[row + g.nc[0]];
                    ax = (float)(cx + g.nc[0]);
                } else if (q == 1) {     // cells at the bottom end seen through x = L
                    if (hi < g.nc[0]) continue;
                    j0 = a.cell_start[row];
                    j1 = a.cell_start[row + hi - g.nc[0] + 1];
                    ax = (float)(cx - g.nc[0]);
                } else {
                    int l2 = lo < 0 ? 0 : lo, h2 = hi >= g.nc[0] ? g.nc[0] - 1 : hi;
                    if (l2 > h2) continue;
                    j0 = a.cell_start[row + l2];
                    j1 = a.cell_start[row + h2 + 1];
                    ax = (float)cx;
                }
                for (int base = j0; base < j1; base += G) {
                    int j = base + lane;
                    bool hit = false;
                    if (j < j1 && j != k) {
                        float4 uj = a.sp4[j];
                        float ddx = fmaf(ax - uj.w, g.cf[0], ui.x - uj.x);
                        float ddy = ay - uj.y;
                        float ddz = az - uj.z;
                        hit = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz)) < rl2;
                    }
                    if constexpr (FILL) {
                        unsigned m = (__ballot_sync(gmask, hit) >> gbase) & gbits;
                        if (hit) out[n + __popc(m & below)] = (int32_t)((uint32_t)j | tag);
                        n += __popc(m);
                    } else {
                        n += hit ? 1 : 0;
                    }
                }
            }
        }
    }
    if constexpr (!FILL) {
        for (int off = G >> 1; off > 0; off >>= 1) n += __shfl_xor_sync(gmask, n, off);
        if (lane == 0) a.nl_cnt[k] = n;
    } else {
        if (lane == 0) {
            a.rl_ref[i] = rl - share;
            a.sh_ref[i] = share;
        }
    }
}

// the class-ordered work queue shared by the force and list kernels
struct Queue {
    int cnt[DCM_MAX_CLASSES], off[DCM_MAX_CLASSES], items[DCM_MAX_CLASSES + 1];
};

__device__ __forceinline__ void queue_init(const ForceArgs &a, Queue &sq)
{
    const int K = a.b.K;
    if (threadIdx.x == 0) {
        int run = 0;
        // heaviest (largest cutoff) class first
        for (int q = K - 1, t = 0; q >= 0; --q, ++t) {
            sq.cnt[q] = a.class_buf[q];
            sq.off[q] = a.class_buf[K + q];
            int per = 32 / a.lanes[q];
            sq.items[t] = run;
            run += (sq.cnt[q] + per - 1) / per;
        }
        sq.items[K] = run;
    }
}

template <bool FILL>
__global__ void __launch_bounds__(FORCE_THREADS, 3) k_list_walk(ForceArgs a)
{
    __shared__ Queue sq;
    __shared__ int s_run;
    queue_init(a, sq);
    if (threadIdx.x == 0) s_run = *a.gate;
    __syncthreads();
    if (!s_run) return;
    const int K = a.b.K;
    const int total = sq.items[K];
    const int lane32 = threadIdx.x & 31;
    while (true) {
        int item = 0;
        if (lane32 == 0) item = (int)atomicAdd(a.queue, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total) break;
        int t = 0;
        while (t + 1 < K && item >= sq.items[t + 1]) ++t;
        int q = K - 1 - t;
        int G = a.lanes[q];
        int per = 32 / G;
        int local = (item - sq.items[t]) * per + lane32 / G;
        int lane = lane32 & (G - 1);
        unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane32 & ~(G - 1)));
        if (local < sq.cnt[q]) list_particle<FILL>(a, sq.off[q] >= 0 ? a.class_list[sq.off[q] + local] : 0,
                                                    lane, G, gmask);
        __syncwarp();
    }
}

// persistent warps draining the class-ordered work queue (FP64 path)
template <bool ENERGY>
__global__ void __launch_bounds__(FORCE_THREADS, 3) k_force(ForceArgs a)
{
    __shared__ int s_cnt[DCM_MAX_CLASSES], s_off[DCM_MAX_CLASSES], s_items[DCM_MAX_CLASSES + 1];
    const int K = a.b.K;
    if (threadIdx.x == 0) {
        int run = 0;
        // heaviest (largest cutoff) class first
        for (int q = K - 1, t = 0; q >= 0; --q, ++t) {
            s_cnt[q] = a.class_buf[q];
            s_off[q] = a.class_buf[K + q];
            int per = 32 / a.lanes[q];
            s_items[t] = run;
            run += (s_cnt[q] + per - 1) / per;
        }
        s_items[K] = run;
    }
    __shared__ int s_list;
    if (threadIdx.x == 0) s_list = a.list_ok ? *a.list_ok : 0;
    __syncthreads();
    const int total = s_items[K];
    const int lane32 = threadIdx.x & 31;
    const bool use_list = s_list != 0;
    int ng = 0;   // guard-band re-decisions (diagnostic), one atomic per block
    while (true) {
        int item = 0;
        if (lane32 == 0) item = (int)atomicAdd(a.queue, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total) break;
        int t = 0;
        while (t + 1 < K && item >= s_items[t + 1]) ++t;
        int q = K - 1 - t;
        int G = a.lanes[q];
        int per = 32 / G;
        int local = (item - s_items[t]) * per + lane32 / G;
        int lane = lane32 & (G - 1);
        unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane32 & ~(G - 1)));
        if (local < s_cnt[q]) {
            int k = a.class_list[s_off[q] + local];
            if (use_list)
                particle_force_list<ENERGY>(a, k, lane, G, gmask, ng);
            else
                particle_force<ENERGY>(a, k, lane, G, gmask, ng);
        }
        __syncwarp();
    }
    for (int off = 16; off > 0; off >>= 1) ng += __shfl_xor_sync(0xffffffffu, ng, off);
    __shared__ int s_ng;
    if (threadIdx.x == 0) s_ng = 0;
    __syncthreads();
    if (lane32 == 0 && ng) atomicAdd(&s_ng, ng);
    __syncthreads();
    if (threadIdx.x == 0 && s_ng) atomicAdd(a.guard_count, (unsigned long long)s_ng);
}

// ---- warp per particle over a flattened candidate list (mixed precision) ----
// The lanes kernel above gives each particle G lanes that walk its stencil
// rows one after another; rows hold a handful of candidates, so the lanes of
// a warp spend much of their time in different loop phases.  Here one warp
// owns one particle and every step is lane-parallel:
//  1. rows: lane L sets up row L of a pass of 32 stencil rows (box-gap
//     culling and the x chord, as in particle_force); the non-empty rows are
//     compacted into a per-warp table with their offsets in one flattened
//     candidate list (a warp prefix sum of the row lengths);
//  2. candidates: lane L takes list positions base + L; its row is found
//     from a 32-bit mask of the row starts inside the chunk (one warp OR
//     reduction and a popcount), so a chunk may span any number of rows;
//     the pair test and the force are evaluated without branches (the FP64
//     re-decision at the cutoff edge is the only branch, and it is rare);
//  3. close pairs (FP32 r^2 below r_close^2 = (1.5 sigma)^2, about 13 of a
//     liquid particle's ~110 pairs) are not evaluated there: they are
//     appended to a per-warp stash (a ballot keeps the warp converged) and
//     evaluated together at the end of the particle in double-float
//     arithmetic (close_pair): their forces are large (up to a few hundred
//     epsilon/sigma), cancel in the sum, and change fast with r, so their
//     FP32 rounding would dominate the per-particle error;
//  4. the lane partials are summed exactly: each FP32 partial is split
//     into a multiple of 2^-8 and a remainder, both scaled to integers and
//     added with warp integer reductions, so the total is the exact sum of
//     the partials (up to 2^-30 per partial), independent of lane order.
constexpr int FW_THREADS = 128;
constexpr int FW_WARPS = FW_THREADS / 32;
constexpr int FW_ROWS = 128;                 // row table entries per warp
constexpr int FW_GRAB = 4;                   // particles per queue grab
constexpr int FW_LIST_G = 8;                 // lanes per particle of the list kernel
constexpr int FW_LIST_U = 4;                 // list entries in flight per lane
constexpr int FW_WALK_MINB = 8;              // resident blocks per SM of the direct walk (64 registers)
constexpr int FW_WALK_MINB1 = 9;             // ... one system (56 registers, 186 KB of row tables)
constexpr int FW_LIST_MINB = 8;              // resident blocks per SM of the list kernel (64 registers)
constexpr float FW_FIX_LIMIT = 16384.f;      // |partial| bound of the exact sum
constexpr int FW_CLOSE = 64;                 // close-pair stash of a direct-walk warp (one particle)
constexpr int FW_LIST_CLOSE = 64;            // close-pair stash of a list-kernel group (all its lanes)
constexpr float FW_CMAGIC = 3072.f;          // 1.5 * 2^11: (x + m) - m rounds |x| < 2^10 to 2^-12

struct FwTable {
    int4 ri[FW_ROWS];        // list offset P, main start, main length, wrapped start
    float4 rf[FW_ROWS];      // x cell shift (main, wrapped), row y, row z
    int rp[FW_ROWS];         // P again, read conflict-free by the row search
    int rt[FW_ROWS];         // Verlet-list tag of the row: (dy + 8) << 24 | (dz + 8) << 28
};

// fixed-point image of an FP32 value with |p| < FW_FIX_LIMIT: p = hp * 2^-8
// + lp * 2^-30 up to 2^-31 (rem is exact, and lp its rounding to 2^-30)
__device__ __forceinline__ void fixed_split(float p, int &hp, int &lp)
{
    // nearest integers by the 1.5 * 2^23 shift (exact for |x| <= 2^22, and
    // |p| < FW_FIX_LIMIT = 2^14 keeps p * 256 there): no conversion pipe
    const float M = 12582912.f;
    const float t = fmaf(p, 256.f, M);
    hp = __float_as_int(t) - 0x4B400000;
    const float rem = fmaf(__fsub_rn(t, M), -0.00390625f, p);   // exact
    lp = __float_as_int(fmaf(rem, 1073741824.f, M)) - 0x4B400000;   // rem * 2^30, |.| <= 2^21
}

// Exact warp sum of three FP32 partials per lane whose magnitudes are below
// FW_FIX_LIMIT, as the fixed-point integer V = sum * 2^30 (|V| < 2^52).
// Integer pipes only: on this GPU one FP64 warp instruction costs as much
// issue time as dozens of FP32 ones, and this runs once per particle, not
// once per pair.
__device__ __forceinline__ long long warp_fixed_sum(float p, float q, float r)
{
    int h0, l0, h1, l1, h2, l2;
    fixed_split(p, h0, l0);
    fixed_split(q, h1, l1);
    fixed_split(r, h2, l2);
    long long H = __reduce_add_sync(0xffffffffu, h0 + h1 + h2);
    long long Lo = __reduce_add_sync(0xffffffffu, l0 + l1 + l2);
    return H * 4194304ll + Lo;
}

// V * 2^-30 as a double, built from its bits (exact: |V| < 2^53)
__device__ __forceinline__ double fixed_to_double(long long V)
{
    if (V == 0) return 0.0;
    unsigned long long sign = (unsigned long long)V & 0x8000000000000000ull;
    unsigned long long m = (unsigned long long)(V < 0 ? -V : V);
    int e = 63 - __clzll(m);                                 // leading bit, <= 52
    unsigned long long mant = (m << (52 - e)) & 0x000FFFFFFFFFFFFFull;
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)(e - 30 + 1023) << 52) | mant));
}

__device__ __forceinline__ double warp_tree_sum(float p, float q, float r)
{
    double d = ((double)p + (double)q) + (double)r;
    for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
    return d;
}

// ---- close pairs in double-float arithmetic --------------------------------
// A value is carried as hi + lo (two FP32 numbers): products take their
// exact rounding error from an FMA, sums from TwoSum, and the cross terms
// are kept to first order.  One pair's force scalar g = F/r then carries
// about 2^-44 relative error instead of FP32's ~2^-21.  The displacement
// d = dh + dl is exact: dh from the FP32 grid positions and cell shift (no
// rounding, see cell_rel_position), dl from their FP32 remainders and the
// low part of the cell edge.
//
// c: the system's constants (a Geom or the launch's ListConst): sig2f/l,
// eps48f/l, eps24f/l.  Returns g = (gh, gl) and the FP32 (sigma/r)^6.
template <class C>
__device__ __forceinline__ void close_force_scalar(const C &c, float dxh, float dyh, float dzh,
                                                   float dxl, float dyl, float dzl, float &gh,
                                                   float &gl, float &s6)
{
    // q = |d|^2
    const float p1 = __fmul_rn(dxh, dxh), e1 = fmaf(dxh, dxh, -p1);
    const float p2 = __fmul_rn(dyh, dyh), e2 = fmaf(dyh, dyh, -p2);
    const float p3 = __fmul_rn(dzh, dzh), e3 = fmaf(dzh, dzh, -p3);
    float s12, es, qh, eq;
    two_sum(p1, p2, s12, es);
    two_sum(s12, p3, qh, eq);
    const float cr = fmaf(dzh, dzl, fmaf(dyh, dyl, __fmul_rn(dxh, dxl)));
    const float ql =
        fmaf(2.f, cr, __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), __fadd_rn(e3, es)), eq));
    // w = 1/q: approximate reciprocal, then its residual (q and the low part)
    const float wh = rcp_approx(qh);
    const float rho = fmaf(-ql, wh, fmaf(-qh, wh, 1.f));
    const float wl = __fmul_rn(wh, rho);
    // s = sigma^2 w
    const float sh = __fmul_rn(c.sig2f, wh);
    const float sl = fmaf(c.sig2f, wl, fmaf(c.sig2l, wh, fmaf(c.sig2f, wh, -sh)));
    // s^2, then s6 = (sigma/r)^6
    const float s2h = __fmul_rn(sh, sh);
    const float s2l = fmaf(__fmul_rn(2.f, sh), sl, fmaf(sh, sh, -s2h));
    const float s6h = __fmul_rn(s2h, sh);
    const float s6l = fmaf(s2h, sl, fmaf(s2l, sh, fmaf(s2h, sh, -s6h)));
    // u = 48 eps s6 - 24 eps
    const float mh = __fmul_rn(c.eps48f, s6h);
    const float ml = fmaf(c.eps48f, s6l, fmaf(c.eps48l, s6h, fmaf(c.eps48f, s6h, -mh)));
    float uh, ue;
    two_sum(mh, -c.eps24f, uh, ue);
    const float ul = __fsub_rn(__fadd_rn(ue, ml), c.eps24l);
    // v = s6 u, g = w v
    const float vh = __fmul_rn(s6h, uh);
    const float vl = fmaf(s6h, ul, fmaf(s6l, uh, fmaf(s6h, uh, -vh)));
    gh = __fmul_rn(wh, vh);
    gl = fmaf(wh, vl, fmaf(wl, vh, fmaf(wh, vh, -gh)));
    s6 = s6h;
}

// lane partials of one particle: pair force, pair count, PE, virial
template <bool ENERGY>
struct WarpAcc {
    float fx = 0.f, fy = 0.f, fz = 0.f, pe = 0.f;
    float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f, v4 = 0.f, v5 = 0.f;
    // close pairs: hi parts rounded to multiples of 2^-12 (their FP32 sums
    // are exact while below 2^11 in magnitude), and the small remainders
    float cx = 0.f, cy = 0.f, cz = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
    int np = 0;

    // one candidate (dx, dy, dz) = r_i - r_j with in = "inside r_c[i]";
    // C: the system's LJ constants (a Geom, or the launch's ListConst)
    template <class C>
    __device__ __forceinline__ void pair(const C &g, float dx, float dy, float dz, float r2,
                                         bool in)
    {
        float r2inv = rcp_approx(r2);
        float sr2 = g.sig2f * r2inv;
        float sr6 = sr2 * sr2 * sr2;
        float fr = r2inv * sr6 * fmaf(g.eps48f, sr6, -g.eps24f);
        fr = in ? fr : 0.f;
        fx = fmaf(fr, dx, fx);
        fy = fmaf(fr, dy, fy);
        fz = fmaf(fr, dz, fz);
        np += in ? 1 : 0;
        if constexpr (ENERGY) {
            pe = in ? fmaf(g.eps2f * sr6, sr6 - 1.f, pe) : pe;
            float gx = fr * dx, gy = fr * dy, gz = fr * dz;
            v0 = fmaf(0.5f * dx, gx, v0);
            v1 = fmaf(0.5f * dy, gy, v1);
            v2 = fmaf(0.5f * dz, gz, v2);
            v3 = fmaf(0.5f * dx, gy, v3);
            v4 = fmaf(0.5f * dx, gz, v4);
            v5 = fmaf(0.5f * dy, gz, v5);
        }
    }

    // one close pair from its exact displacement dh + dl: the force g d in
    // double-float, its hi part rounded to 2^-12 into the exact sums and
    // the rest into the remainders
    template <class C>
    __device__ __forceinline__ void close(const C &g, float dxh, float dyh, float dzh, float dxl,
                                          float dyl, float dzl)
    {
        float gh, gl, s6;
        close_force_scalar(g, dxh, dyh, dzh, dxl, dyl, dzl, gh, gl, s6);
        add_close(gh, gl, dxh, dxl, cx, lx);
        add_close(gh, gl, dyh, dyl, cy, ly);
        add_close(gh, gl, dzh, dzl, cz, lz);
        ++np;
        if constexpr (ENERGY) {
            pe = fmaf(g.eps2f * s6, s6 - 1.f, pe);
            float gx = gh * dxh, gy = gh * dyh, gz = gh * dzh;
            v0 = fmaf(0.5f * dxh, gx, v0);
            v1 = fmaf(0.5f * dyh, gy, v1);
            v2 = fmaf(0.5f * dzh, gz, v2);
            v3 = fmaf(0.5f * dxh, gy, v3);
            v4 = fmaf(0.5f * dxh, gz, v4);
            v5 = fmaf(0.5f * dyh, gz, v5);
        }
    }

    static __device__ __forceinline__ void add_close(float gh, float gl, float dh, float dl,
                                                     float &c, float &l)
    {
        const float Fh = __fmul_rn(gh, dh);
        const float Fl = fmaf(gh, dl, fmaf(gl, dh, fmaf(gh, dh, -Fh)));
        const float q = __fsub_rn(__fadd_rn(Fh, FW_CMAGIC), FW_CMAGIC);
        c = __fadd_rn(c, q);
        l = __fadd_rn(l, __fadd_rn(__fsub_rn(Fh, q), Fl));
    }

    __device__ __forceinline__ bool small() const
    {
        bool s = fabsf(fx) < FW_FIX_LIMIT && fabsf(fy) < FW_FIX_LIMIT && fabsf(fz) < FW_FIX_LIMIT &&
                 fabsf(cx) < FW_FIX_LIMIT && fabsf(cy) < FW_FIX_LIMIT && fabsf(cz) < FW_FIX_LIMIT &&
                 fabsf(lx) < FW_FIX_LIMIT && fabsf(ly) < FW_FIX_LIMIT && fabsf(lz) < FW_FIX_LIMIT;
        if constexpr (ENERGY)
            s = s && fabsf(pe) < FW_FIX_LIMIT && fabsf(v0) < FW_FIX_LIMIT &&
                fabsf(v1) < FW_FIX_LIMIT && fabsf(v2) < FW_FIX_LIMIT && fabsf(v3) < FW_FIX_LIMIT &&
                fabsf(v4) < FW_FIX_LIMIT && fabsf(v5) < FW_FIX_LIMIT;
        return s;
    }

    // sum the lane partials and store particle i's results; lane q writes
    // value q.  Returns |F|^2 of the stored force in every lane.
    __device__ __forceinline__ float store(const ForceArgs &a, int i, int lane)
    {
        const size_t n = (size_t)a.b.N;
        const int npt = __reduce_add_sync(0xffffffffu, np);
        if (lane == 3) a.npair[i] = npt;
        float fc = 0.f;
        if (__all_sync(0xffffffffu, small())) {
            long long V = 0, t;
            t = warp_fixed_sum(fx, cx, lx); V = lane == 0 ? t : V;
            t = warp_fixed_sum(fy, cy, ly); V = lane == 1 ? t : V;
            t = warp_fixed_sum(fz, cz, lz); V = lane == 2 ? t : V;
            if constexpr (ENERGY) {
                t = warp_fixed_sum(pe, 0.f, 0.f); V = lane == 4 ? t : V;
                t = warp_fixed_sum(v0, 0.f, 0.f); V = lane == 5 ? t : V;
                t = warp_fixed_sum(v1, 0.f, 0.f); V = lane == 6 ? t : V;
                t = warp_fixed_sum(v2, 0.f, 0.f); V = lane == 7 ? t : V;
                t = warp_fixed_sum(v3, 0.f, 0.f); V = lane == 8 ? t : V;
                t = warp_fixed_sum(v4, 0.f, 0.f); V = lane == 9 ? t : V;
                t = warp_fixed_sum(v5, 0.f, 0.f); V = lane == 10 ? t : V;
            }
            const double out = fixed_to_double(V);
            if (lane < 3) {
                a.f[lane * n + i] = out;
                fc = (float)out;
            }
            if constexpr (ENERGY) {
                if (lane == 4) a.pe[i] = out;
                if (lane >= 5 && lane < 11) a.vir[(lane - 5) * n + i] = out;
            }
        } else {
            // a partial beyond the fixed-point range (or not finite): FP64 tree
            double Fx = warp_tree_sum(fx, cx, lx), Fy = warp_tree_sum(fy, cy, ly),
                   Fz = warp_tree_sum(fz, cz, lz);
            if (lane < 3) a.f[lane * n + i] = lane == 0 ? Fx : (lane == 1 ? Fy : Fz);
            fc = lane == 0 ? (float)Fx : (lane == 1 ? (float)Fy : (lane == 2 ? (float)Fz : 0.f));
            if constexpr (ENERGY) {
                double s7[7] = {warp_tree_sum(pe, 0.f, 0.f), warp_tree_sum(v0, 0.f, 0.f),
                                warp_tree_sum(v1, 0.f, 0.f), warp_tree_sum(v2, 0.f, 0.f),
                                warp_tree_sum(v3, 0.f, 0.f), warp_tree_sum(v4, 0.f, 0.f),
                                warp_tree_sum(v5, 0.f, 0.f)};
                if (lane == 4) a.pe[i] = s7[0];
#pragma unroll
                for (int e = 0; e < 6; ++e)
                    if (lane == 5 + e) a.vir[e * n + i] = s7[1 + e];
            }
        }
        const float f2 = fc * fc;
        return __shfl_sync(0xffffffffu, f2, 0) + __shfl_sync(0xffffffffu, f2, 1) +
               __shfl_sync(0xffffffffu, f2, 2);
    }
};

// the exact displacement r_i - r_j of a close pair from both particles' FP32
// grid positions u and remainders ul: the cell x offset (wrapped like the
// list entries: every true offset is below half the cells along x), the
// y/z cell row offsets dyc, dzc of j's row
template <class C>
__device__ __forceinline__ void close_disp(const C &c, float ncx, float halfnc, float4 ui,
                                           float4 uli, float4 uj, float4 ulj, float dyc,
                                           float dzc, float &dxh, float &dyh, float &dzh,
                                           float &dxl, float &dyl, float &dzl)
{
    float dcx = ui.w - uj.w;
    dcx -= dcx > halfnc ? ncx : 0.f;
    dcx += dcx < -halfnc ? ncx : 0.f;
    // the coordinate differences on the grid: exact below qtop; a rare
    // larger one (two particles drifted apart out of their cells) keeps
    // what its rounding drops by TwoSum
    float ax = __fsub_rn(ui.x, uj.x), ay = __fsub_rn(ui.y, uj.y), az = __fsub_rn(ui.z, uj.z);
    float ex = 0.f, ey = 0.f, ez = 0.f;
    if (fabsf(ax) >= c.qtop) two_sum(ui.x, -uj.x, ax, ex);
    if (fabsf(ay) >= c.qtop) two_sum(ui.y, -uj.y, ay, ey);
    if (fabsf(az) >= c.qtop) two_sum(ui.z, -uj.z, az, ez);
    // plus the cell shift: exact, the result is a short multiple of the grid
    dxh = fmaf(dcx, c.cf[0], ax);
    dyh = fmaf(-dyc, c.cf[1], ay);
    dzh = fmaf(-dzc, c.cf[2], az);
    dxl = __fadd_rn(fmaf(dcx, c.cfl[0], __fsub_rn(uli.x, ulj.x)), ex);
    dyl = __fadd_rn(fmaf(-dyc, c.cfl[1], __fsub_rn(uli.y, ulj.y)), ey);
    dzl = __fadd_rn(fmaf(-dzc, c.cfl[2], __fsub_rn(uli.z, ulj.z)), ez);
}

// The cell x offset of a list pair folded into (-n/2, n/2] with one
// rounding: dcx / n rounded to an integer by the 1.5 * 2^23 shift, then that
// multiple of n taken off (exact: small integers).  Every listed pair has
// |offset| <= s_max with 2 s_max + 1 <= n, so the quotient stays clear of
// 1/2 and the result is the same as comparing against n/2 twice.
__device__ __forceinline__ float wrap_cells(float dcx, float ncx, float inv_ncx)
{
    const float k = __fsub_rn(fmaf(dcx, inv_ncx, 12582912.f), 12582912.f);
    return fmaf(-k, ncx, dcx);
}

__device__ __forceinline__ float entry_dy(int e) { return (float)(((e >> 24) & 15) - 8); }
__device__ __forceinline__ float entry_dz(int e) { return (float)((int)((unsigned)e >> 28) - 8); }

// Direct walk of particle k (sorted slot).  FILL (a Verlet-list rebuild):
// the walk also covers the list radius R_k of the gather kernel and appends
// every neighbour within R_k to k's list, in walk order, up to the capacity
// the gather kernel gave it; the forces still use r_c[i] only.  stash: the
// warp's FW_CLOSE close-pair slots; an entry is (j - k) in 24 bits with
// the row's cell offsets on top (the list-entry tag).  A particle with more
// than FW_CLOSE close pairs (far denser than a liquid) evaluates the rest
// in FP32.
template <bool ENERGY, bool FILL, bool SINGLE, bool FF = false>
__device__ __forceinline__ void particle_force_warp(const ForceArgs &a, FwTable &tb, int *stash,
                                                    int k, int lane, int &ng, bool fill_on,
                                                    long long &entries)
{
    static_assert(!(FF && FILL), "the refinement pass does not fill lists");
    const Geom &g = SINGLE ? a.g0 : a.b.sys[sys_p(a.b, k)];
    const float4 ui = a.sp4[k];
    float4 uli0 = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (FF) uli0 = a.spl4[k];
    const float4 q4 = a.rq[k];
    const int4 pk = a.pk[k];
    const int i = pk.x, cy = pk.y, cz = pk.z;
    const int cx = (int)ui.w;
    const float rc2f = q4.x, rc2lo = q4.y, rc2hi = q4.z;
    const float rcl2 = fminf(g.rclose2, rc2lo);
    float rl = 0.f, rcull = q4.w;
    int32_t *out = nullptr;
    int cap = 0, cnt = 0;
    if constexpr (FILL) {
        if (fill_on) {
            // pair (i, j) listed while closer than i's own radius + j's share
            rl = __int_as_float(pk.w);
            const float shmax = __int_as_float(a.list_flags[LF_SHMAX]);
            rcull = fmaxf(rcull, fmaf(rl + shmax, 1.00002f, 1e-4f));
            out = a.nl_w + a.nl_start[k];
            cap = a.nl_cnt[k];
        }
    }
    const float rcull2 = rcull * rcull;
    const int sx = min(g.smax[0], (int)ceilf(rcull * g.inv_cf[0]));
    const int sy = min(g.smax[1], (int)ceilf(rcull * g.inv_cf[1]));
    const int sz = min(g.smax[2], (int)ceilf(rcull * g.inv_cf[2]));
    const int ny_ = 2 * sy + 1;
    const int nrows = ny_ * (2 * sz + 1);
    const float inv_ny = rcp_approx((float)ny_);
    const int nc0 = g.nc[0];
    const float cf0 = g.cf[0];
    const unsigned lane_le = 0xffffffffu >> (31 - lane);
    WarpAcc<ENERGY> acc;
    int ntab = 0, T = 0, ncs = 0;
    for (int r0 = 0; r0 < nrows; r0 += 32) {
        // ---- 1. one stencil row per lane
        const int r = r0 + lane;
        int len = 0, j0a = 0, len1 = 0, j0b = 0, tag = 0;
        float fa = 0.f, fb = 0.f, ay = 0.f, az = 0.f;
        if (r < nrows) {
            int dzi = (int)(((float)r + 0.5f) * inv_ny);    // r / ny_ (exact for these sizes)
            int dz = dzi - sz, dy = r - dzi * ny_ - sy;
            float gz = box_gap(dz, ui.z, g.cf[2]);
            float remz = fmaf(-gz, gz, rcull2);
            float gy = box_gap(dy, ui.y, g.cf[1]);
            float w2 = fmaf(-gy, gy, remz);
            if (remz >= 0.f && w2 >= 0.f) {
                int czz = cz + dz;
                czz += czz < 0 ? g.nc[2] : (czz >= g.nc[2] ? -g.nc[2] : 0);
                int cyy = cy + dy;
                cyy += cyy < 0 ? g.nc[1] : (cyy >= g.nc[1] ? -g.nc[1] : 0);
                // explicit fused forms: the same bits in every instantiation
                az = fmaf(-(float)dz, g.cf[2], ui.z);
                ay = fmaf(-(float)dy, g.cf[1], ui.y);
                float w = sqrtf(w2);
                int xlo = max(-sx, (int)floorf((ui.x - w) * g.inv_cf[0]));
                int xhi = min(sx, (int)floorf((ui.x + w) * g.inv_cf[0]));
                int row = (int)g.c0 + nc0 * (cyy + g.nc[1] * czz);
                int lo = cx + xlo, hi = cx + xhi;
                int len2 = 0;
                if (lo < 0) {
                    // cells at the top end seen through the x = 0 face
                    j0b = a.cell_start[row + lo + nc0];
                    len2 = a.cell_start[row + nc0] - j0b;
                    fb = (float)(cx + nc0);
                    lo = 0;
                } else if (hi >= nc0) {
                    j0b = a.cell_start[row];
                    len2 = a.cell_start[row + hi - nc0 + 1] - j0b;
                    fb = (float)(cx - nc0);
                    hi = nc0 - 1;
                }
                if (lo <= hi) {
                    j0a = a.cell_start[row + lo];
                    len1 = a.cell_start[row + hi + 1] - j0a;
                }
                fa = (float)cx;
                len = len1 + len2;
                tag = (int)(((uint32_t)(dy + 8) << 24) | ((uint32_t)(dz + 8) << 28));
            }
        }
        // compact the non-empty rows into the table
        int incl = len;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        const unsigned ne = __ballot_sync(0xffffffffu, len > 0);
        if (len > 0) {
            int e = ntab + __popc(ne & (lane_le >> 1));
            int P = T + incl - len;
            tb.ri[e] = make_int4(P, j0a, len1, j0b);
            tb.rf[e] = make_float4(fa, fb, ay, az);
            tb.rp[e] = P;
            tb.rt[e] = tag;
        }
        ntab += __popc(ne);
        T += __shfl_sync(0xffffffffu, incl, 31);
        if (ntab <= FW_ROWS - 32 && r0 + 32 < nrows) continue;
        __syncwarp();
        // ---- 2. the flattened candidates, 32 per chunk
        int S = 0;   // rows that start before the chunk
        for (int base = 0; base < T; base += 32) {
            int q = S + lane;
            unsigned d = (unsigned)((q < ntab ? tb.rp[q] : 0x7fffffff) - base);
            unsigned M = __reduce_or_sync(0xffffffffu, d < 32u ? 1u << d : 0u);
            int rowi = S + __popc(M & lane_le) - 1;
            S += __popc(M);
            int p = base + lane;
            bool hit = false;
            int j = 0;
            float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 3.0e38f;
            if (p < T) {
                int4 ri = tb.ri[rowi];
                float4 rf = tb.rf[rowi];
                int t = p - ri.x;
                bool wr = t >= ri.z;
                j = wr ? ri.w + (t - ri.z) : ri.y + t;
                float ax = wr ? rf.y : rf.x;
                float4 uj = a.sp4[j];
                dx = fmaf(ax - uj.w, cf0, ui.x - uj.x);
                dy = rf.z - uj.y;
                dz = rf.w - uj.z;
                r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if constexpr (FILL) {
                    if (fill_on) {
                        const float rp = rl + a.sh[j];
                        hit = r2 < rp * rp && j != k;
                    }
                }
            }
            // the fill walks out to the list radius: a chunk of candidates
            // all beyond the cutoff adds nothing (exact zeros) and skips the
            // force arithmetic
            if (!FILL || __any_sync(0xffffffffu, r2 < rc2hi)) {
                bool in = false, cl = false;
                if (p < T) {
                    in = r2 < rc2f && j != k;
                    if (r2 >= rc2lo && r2 < rc2hi && j != k) {
                        double rci = a.rc[i];
                        in = fp64_inside(a, g, i, a.sorted_id[j], DMUL(rci, rci));
                        if (!FF) ++ng;
                    }
                    // close pairs go to the stash (the slot offset j - k
                    // must fit its 24 bits)
                    cl = r2 < rcl2 && j != k && (unsigned)(j - k + (1 << 23)) < (1u << 24);
                }
                if constexpr (FF) {
                    // refinement: every pair of the particle in double-float
                    if (in) {
                        const int e = tb.rt[rowi];
                        float dxh, dyh, dzh, dxl, dyl, dzl;
                        close_disp(g, (float)nc0, 0.5f * (float)nc0, ui, uli0, a.sp4[j],
                                   a.spl4[j], entry_dy(e), entry_dz(e), dxh, dyh, dzh, dxl, dyl,
                                   dzl);
                        acc.close(g, dxh, dyh, dzh, dxl, dyl, dzl);
                    }
                } else {
                    // (most chunks hold no close pair: one vote skips the
                    // stash bookkeeping for them)
                    const unsigned cm = __ballot_sync(0xffffffffu, cl);
                    if (cm) {
                        const int at = ncs + __popc(cm & (lane_le >> 1));
                        cl = cl && at < FW_CLOSE;
                        if (cl) stash[at] = ((j - k) & 0xffffff) | tb.rt[rowi];
                        ncs = min(ncs + __popc(cm), FW_CLOSE);
                    }
                    if (p < T) acc.pair(g, dx, dy, dz, r2, in && !cl);
                }
            }
            if constexpr (FILL) {
                const unsigned hm = __ballot_sync(0xffffffffu, hit);
                if (hit) {
                    int at = cnt + __popc(hm & (lane_le >> 1));
                    if (at < cap) out[at] = (int32_t)((uint32_t)j | (uint32_t)tb.rt[rowi]);
                }
                cnt += __popc(hm);
            }
        }
        __syncwarp();
        ntab = 0;
        T = 0;
    }
    // ---- 3. the close pairs, one per lane, in double-float
    if (ncs > 0) {
        const float4 uli = a.spl4[k];
        const float ncx = (float)nc0, halfnc = 0.5f * (float)nc0;
        for (int t = lane; t < ncs; t += 32) {
            const int e = stash[t];
            const int j = k + ((int)((unsigned)e << 8) >> 8);
            float dxh, dyh, dzh, dxl, dyl, dzl;
            close_disp(g, ncx, halfnc, ui, uli, a.sp4[j], a.spl4[j], entry_dy(e), entry_dz(e),
                       dxh, dyh, dzh, dxl, dyl, dzl);
            acc.close(g, dxh, dyh, dzh, dxl, dyl, dzl);
        }
        __syncwarp();
    }
    if constexpr (FILL) {
        if (fill_on && lane == 0) {
            a.nl_cnt[k] = min(cnt, cap);
            a.rl_ref[i] = rl;
            a.sh_ref[i] = a.sh[k];
            if (cnt > cap) atomicOr(a.list_flags + LF_OVERFLOW, 1);
            entries += min(cnt, cap);
        }
    }
    const float f2 = acc.store(a, i, lane);
    if constexpr (!FF) {
        // a net force small against the FP32 error of the pairs beyond
        // r_close: queued for k_force_refine (all its pairs in double-float)
        if (f2 < g.redo_f2 && lane == 0) a.refq[atomicAdd(a.refq_n, 1u)] = k;
    }
}

// exact sum over the G lanes of one group (G a power of two <= 32) of three
// FP32 partials per lane: the same split into a multiple of 2^-8 and a
// remainder as warp_fixed_sum, added by an integer butterfly inside the group
template <int G>
__device__ __forceinline__ long long group_fixed_sum(float p, float q, float r)
{
    int h0, l0, h1, l1, h2, l2;
    fixed_split(p, h0, l0);
    fixed_split(q, h1, l1);
    fixed_split(r, h2, l2);
    int hp = h0 + h1 + h2, lp = l0 + l1 + l2;
#pragma unroll
    for (int off = G >> 1; off > 0; off >>= 1) {
        hp += __shfl_xor_sync(0xffffffffu, hp, off);
        lp += __shfl_xor_sync(0xffffffffu, lp, off);
    }
    return (long long)hp * 4194304ll + lp;
}

template <int G>
__device__ __forceinline__ double group_tree_sum(float p, float q, float r)
{
    double d = ((double)p + (double)q) + (double)r;
#pragma unroll
    for (int off = G >> 1; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
    return d;
}

// Sum one group's lane partials (every lane of the warp calls this: the
// sums shuffle across the whole warp) and, when write, store particle i's
// results, lane q of the group writing value q.  Returns |F|^2 of the
// particle in every lane of the group.
template <bool ENERGY, int G>
__device__ __forceinline__ float group_store(const ForceArgs &a, const WarpAcc<ENERGY> &acc,
                                             bool write, int i, int gl)
{
    const size_t n = (size_t)a.b.N;
    const int wl = threadIdx.x & 31, gb = wl & ~(G - 1);
    int npt = acc.np;
#pragma unroll
    for (int off = G >> 1; off > 0; off >>= 1) npt += __shfl_xor_sync(0xffffffffu, npt, off);
    float fc = 0.f;
    if (__all_sync(0xffffffffu, acc.small())) {
        long long V = 0, t;
        t = group_fixed_sum<G>(acc.fx, acc.cx, acc.lx); V = gl == 0 ? t : V;
        t = group_fixed_sum<G>(acc.fy, acc.cy, acc.ly); V = gl == 1 ? t : V;
        t = group_fixed_sum<G>(acc.fz, acc.cz, acc.lz); V = gl == 2 ? t : V;
        if constexpr (ENERGY) {
            t = group_fixed_sum<G>(acc.pe, 0.f, 0.f); V = gl == 4 ? t : V;
            t = group_fixed_sum<G>(acc.v0, 0.f, 0.f); V = gl == 5 ? t : V;
            t = group_fixed_sum<G>(acc.v1, 0.f, 0.f); V = gl == 6 ? t : V;
            t = group_fixed_sum<G>(acc.v2, 0.f, 0.f); V = gl == 7 ? t : V;
            t = group_fixed_sum<G>(acc.v3, 0.f, 0.f); V = gl == 8 ? t : V;
            t = group_fixed_sum<G>(acc.v4, 0.f, 0.f); V = gl == 9 ? t : V;
            t = group_fixed_sum<G>(acc.v5, 0.f, 0.f); V = gl == 10 ? t : V;
        }
        const double out = fixed_to_double(V);
        if (gl < 3) fc = (float)out;
        if (write) {
            if (gl < 3) a.f[gl * n + i] = out;
            if (gl == 3) a.npair[i] = npt;
            if constexpr (ENERGY) {
                if (gl == 4) a.pe[i] = out;
                if (gl >= 5 && gl < 11) a.vir[(gl - 5) * n + i] = out;
            }
        }
    } else {
        double F[3] = {group_tree_sum<G>(acc.fx, acc.cx, acc.lx),
                       group_tree_sum<G>(acc.fy, acc.cy, acc.ly),
                       group_tree_sum<G>(acc.fz, acc.cz, acc.lz)};
        double s7[7] = {0, 0, 0, 0, 0, 0, 0};
        if constexpr (ENERGY) {
            s7[0] = group_tree_sum<G>(acc.pe, 0.f, 0.f);
            s7[1] = group_tree_sum<G>(acc.v0, 0.f, 0.f);
            s7[2] = group_tree_sum<G>(acc.v1, 0.f, 0.f);
            s7[3] = group_tree_sum<G>(acc.v2, 0.f, 0.f);
            s7[4] = group_tree_sum<G>(acc.v3, 0.f, 0.f);
            s7[5] = group_tree_sum<G>(acc.v4, 0.f, 0.f);
            s7[6] = group_tree_sum<G>(acc.v5, 0.f, 0.f);
        }
        if (gl < 3) fc = (float)F[gl];
        if (write && gl == 0) {
            for (int c = 0; c < 3; ++c) a.f[c * n + i] = F[c];
            a.npair[i] = npt;
            if constexpr (ENERGY) {
                a.pe[i] = s7[0];
                for (int c = 0; c < 6; ++c) a.vir[c * n + i] = s7[1 + c];
            }
        }
    }
    const float f2 = fc * fc;
    return __shfl_sync(0xffffffffu, f2, gb) + __shfl_sync(0xffffffffu, f2, gb + 1) +
           __shfl_sync(0xffffffffu, f2, gb + 2);
}

// Particle k again over its Verlet list, the whole warp on it, its results
// stored again: the same pair decisions as the list kernel (FP32 r^2 from
// the grid positions, FP64 re-decision in the guard band), the in-cutoff
// pairs within 2.5 sigma in double-float and the rest in FP32.  Beyond
// 2.5 sigma a pair force is below 0.04 epsilon/sigma and its slope below
// 0.11 epsilon/sigma^2 (falling as r^-8), so the rounding of the FP32 grid
// positions (~1e-7 sigma) moves it by ~1e-8, a hundredth of the smallest
// per-particle bar.  The near pairs are gathered in 64 stash slots of the warp
// (slot t at st[(t >> 5) * stride + (t & 31)]) and evaluated 32 at a time,
// so the double-float work runs on full warps however near and far entries
// interleave in the list.
constexpr float REFINE_NEAR2 = 6.25f;         // (2.5 sigma)^2 in units of sigma^2

template <bool ENERGY, bool SINGLE>
__device__ __forceinline__ void refine_list(const ForceArgs &a, int k, int lane, int *st,
                                            int stride)
{
    const unsigned full = 0xffffffffu;
    const Geom &g = a.b.sys[SINGLE ? 0 : sys_p(a.b, k)];
    const float ncx = (float)g.nc[0], halfnc = 0.5f * (float)g.nc[0], inv_ncx = 1.f / ncx;
    const float4 ui = a.sp4[k], uli = a.spl4[k], q4 = a.rq[k];
    const int i = a.pk[k].x;
    const float rc2f = q4.x, rc2lo = q4.y, rc2hi = q4.z;
    const float near2 = REFINE_NEAR2 * g.sig2f;
    const int32_t *list = a.nl + a.nl_start[k];
    const int cnt = a.nl_cnt[k];
    const unsigned lane_lt = (1u << lane) - 1u;
    WarpAcc<ENERGY> acc;
    auto slot = [&](int t) -> int & { return st[(t >> 5) * stride + (t & 31)]; };
    auto near_pair = [&](int e) {
        const int j = e & 0xffffff;
        float dxh, dyh, dzh, dxl, dyl, dzl;
        close_disp(g, ncx, halfnc, ui, uli, a.sp4[j], a.spl4[j], entry_dy(e), entry_dz(e), dxh, dyh,
                   dzh, dxl, dyl, dzl);
        acc.close(g, dxh, dyh, dzh, dxl, dyl, dzl);
    };
    int ns = 0;                                   // stash fill (the same in every lane)
    for (int p0 = 0; p0 < cnt; p0 += 32) {
        const int p = p0 + lane;
        bool nr = false;
        int e = 0;
        if (p < cnt) {
            e = list[p];
            const int j = e & 0xffffff;
            const float4 uj = a.sp4[j];
            const float dcx = wrap_cells(ui.w - uj.w, ncx, inv_ncx);
            const float dx = fmaf(dcx, g.cf[0], ui.x - uj.x);
            const float dy = fmaf(-entry_dy(e), g.cf[1], ui.y - uj.y);
            const float dz = fmaf(-entry_dz(e), g.cf[2], ui.z - uj.z);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            bool in = r2 < rc2f;
            if (r2 >= rc2lo && r2 < rc2hi) {
                double rci = a.rc[i];
                in = fp64_inside(a, g, i, a.sorted_id[j], DMUL(rci, rci));
            }
            nr = in && r2 < near2;
            if (in && !nr) acc.pair(g, dx, dy, dz, r2, true);
        }
        const unsigned m = __ballot_sync(full, nr);
        if (nr) slot(ns + __popc(m & lane_lt)) = e;
        ns += __popc(m);
        if (ns >= 32) {
            __syncwarp();
            near_pair(slot(lane));
            __syncwarp();
            if (lane < ns - 32) slot(lane) = slot(32 + lane);
            ns -= 32;
            __syncwarp();
        }
    }
    __syncwarp();
    if (lane < ns) near_pair(slot(lane));
    __syncwarp();
    acc.store(a, i, lane);
}

// close-pair slots of one list-kernel lane (slot-major over the block's
// threads); a lane that meets more close pairs evaluates the rest in FP32
template <int G>
constexpr int list_close_slots() { return FW_LIST_CLOSE / G > 4 ? FW_LIST_CLOSE / G : 4; }

// Particle k over its Verlet list, G lanes (one group) per particle, 32/G
// particles per warp: the list is flat, so a group needs no row structure
// and the per-particle work (loads, the exact sum, the stores) is shared by
// 32/G particles per warp instruction.  Entries: j | (dy + 8) << 24 |
// (dz + 8) << 28; the cell x offset comes from the cell x indices stored
// with the positions (every true offset is below half the cells along x).
// Same pair rule and FP64 re-decision as the direct walk.  Close pairs are
// set aside in the lane's stash slots (stash[s * FW_THREADS + thread]) and
// evaluated in double-float after the list, spread over the group's lanes.
// k < 0: an idle group (past the end of the queue).  SINGLE (one system):
// the cell and LJ constants come from the launch parameters (no registers
// held for them, which lets 9 blocks of 128 threads share an SM).
template <bool ENERGY, int G, bool SINGLE>
__device__ __forceinline__ void particle_force_list_group(const ForceArgs &a, int *stash, int k,
                                                          int gl, int &ng)
{
    constexpr int CSL = list_close_slots<G>();
    WarpAcc<ENERGY> acc;
    int i = 0, ncl = 0;
    const Geom &g = a.b.sys[SINGLE ? 0 : (k >= 0 ? sys_p(a.b, k) : 0)];
    const float ncx = SINGLE ? a.lc.ncx : (float)g.nc[0];
    const float halfnc = SINGLE ? a.lc.halfnc : 0.5f * (float)g.nc[0];
    const float inv_ncx = SINGLE ? a.lc.inv_ncx : 1.f / (float)g.nc[0];
    float4 ui = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k >= 0) {
        ui = a.sp4[k];
        const float4 q4 = a.rq[k];
        i = a.pk[k].x;
        const float rc2f = q4.x, rc2lo = q4.y, rc2hi = q4.z;
        const float rcl2 = fminf(SINGLE ? a.lc.rclose2 : g.rclose2, rc2lo);
        const float cf0 = SINGLE ? a.lc.cf[0] : g.cf[0];
        const float cf1 = SINGLE ? a.lc.cf[1] : g.cf[1];
        const float cf2 = SINGLE ? a.lc.cf[2] : g.cf[2];
        const int32_t *list = a.nl + a.nl_start[k];
        const int cnt = a.nl_cnt[k];
        auto one = [&](int e, float4 uj) {
            int j = e & 0xffffff;
            float dyc = entry_dy(e);
            float dzc = entry_dz(e);
            const float dcx = wrap_cells(ui.w - uj.w, ncx, inv_ncx);
            // coordinate differences first: exact for a close pair
            float dx = fmaf(dcx, cf0, ui.x - uj.x);
            float dy = fmaf(-dyc, cf1, ui.y - uj.y);
            float dz = fmaf(-dzc, cf2, ui.z - uj.z);
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            bool in = r2 < rc2f;
            if (r2 >= rc2lo && r2 < rc2hi) {
                double rci = a.rc[i];
                in = fp64_inside(a, g, i, a.sorted_id[j], DMUL(rci, rci));
                ++ng;
            }
            const bool cl = r2 < rcl2 && ncl < CSL;
            if (cl) {
                stash[ncl * FW_THREADS + threadIdx.x] = e;
                ++ncl;
            }
            if constexpr (SINGLE)
                acc.pair(a.lc, dx, dy, dz, r2, in && !cl);
            else
                acc.pair(g, dx, dy, dz, r2, in && !cl);
        };
        int p = gl;
        // FW_LIST_U entries of the lane in flight per iteration: all entry
        // loads, then all position loads, then the arithmetic
        for (; p + (FW_LIST_U - 1) * G < cnt; p += FW_LIST_U * G) {
            int e[FW_LIST_U];
            float4 u[FW_LIST_U];
#pragma unroll
            for (int q = 0; q < FW_LIST_U; ++q) e[q] = __ldcs(list + p + q * G);
#pragma unroll
            for (int q = 0; q < FW_LIST_U; ++q) u[q] = a.sp4[e[q] & 0xffffff];
#pragma unroll
            for (int q = 0; q < FW_LIST_U; ++q) one(e[q], u[q]);
        }
        for (; p < cnt; p += G) {
            int e0 = __ldcs(list + p);
            one(e0, a.sp4[e0 & 0xffffff]);
        }
    }
    // ---- the group's close pairs, spread over its lanes: item t of the
    // group's concatenated slots lives in the slots of the last lane whose
    // exclusive offset is <= t (a binary search over the G offsets)
    {
        const int wl = threadIdx.x & 31, gb = wl & ~(G - 1);
        int incl = ncl;
#pragma unroll
        for (int off = 1; off < G; off <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, off, G);
            if (gl >= off) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, G - 1, G);
        const int excl = incl - ncl;
        float4 uli = make_float4(0.f, 0.f, 0.f, 0.f);
        if (total > 0) uli = a.spl4[k];
        for (int base = 0; __any_sync(0xffffffffu, base < total); base += G) {
            const int t = base + gl;
            int o = 0;
#pragma unroll
            for (int st = G >> 1; st > 0; st >>= 1) {
                const int ex = __shfl_sync(0xffffffffu, excl, gb + o + st);
                o = ex <= t ? o + st : o;
            }
            const int exo = __shfl_sync(0xffffffffu, excl, gb + o);
            if (t < total) {
                const int e = stash[(t - exo) * FW_THREADS + (threadIdx.x & ~31) + gb + o];
                const int j = e & 0xffffff;
                float dxh, dyh, dzh, dxl, dyl, dzl;
                if constexpr (SINGLE) {
                    close_disp(a.lc, ncx, halfnc, ui, uli, a.sp4[j], a.spl4[j], entry_dy(e),
                               entry_dz(e), dxh, dyh, dzh, dxl, dyl, dzl);
                    acc.close(a.lc, dxh, dyh, dzh, dxl, dyl, dzl);
                } else {
                    close_disp(g, ncx, halfnc, ui, uli, a.sp4[j], a.spl4[j], entry_dy(e),
                               entry_dz(e), dxh, dyh, dzh, dxl, dyl, dzl);
                    acc.close(g, dxh, dyh, dzh, dxl, dyl, dzl);
                }
            }
        }
    }
    // ---- sums over the group; lane q of the group writes value q
    float f2 = group_store<ENERGY, G>(a, acc, k >= 0, i, gl);
    // a net force small against the FP32 error of the pairs beyond r_close:
    // evaluated again at once, all its pairs in double-float, by the whole
    // warp (one such group after another; ~2 % of a slab's particles), which
    // keeps the latency-bound refinement inside this issue-bound kernel
    const bool redo = k >= 0 && f2 < (SINGLE ? a.lc.redo_f2 : g.redo_f2);
    unsigned m = __ballot_sync(0xffffffffu, redo && gl == 0);
    if (m) {
        const int lane = threadIdx.x & 31;
        if (lane == 0) atomicAdd(a.refined_n, (unsigned)__popc(m));
        do {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            refine_list<ENERGY, SINGLE>(a, __shfl_sync(0xffffffffu, k, src), lane,
                                        stash + (threadIdx.x & ~31), FW_THREADS);
        } while (m);
    }
}

// The double-float refinement of the particles the direct walks queued
// (net force below 0.5 epsilon/sigma, about 2-4 % of a slab's particles,
// mostly vapor; the list kernels refine theirs in place): a warp per
// particle.  On a rebuild step whose fill completed, over the fresh lists;
// otherwise (no lists) by the direct walk.  Runs after the force kernels of
// the step, so the queue is complete.
template <bool ENERGY, bool SINGLE>
__global__ void __launch_bounds__(FW_THREADS) k_force_refine(const __grid_constant__ ForceArgs a)
{
    __shared__ FwTable s_tab[FW_WARPS];
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * FW_WARPS + (threadIdx.x >> 5);
    const int nw = gridDim.x * FW_WARPS;
    const int total = (int)*(volatile unsigned int *)a.refq_n;
    // the lists are complete on a step that keeps them, and on a rebuild
    // step once the fill ran and no particle overflowed its capacity
    const bool lists = a.nl != nullptr &&
                       (a.list_flags[LF_REBUILD] == 0 ||
                        (a.list_flags[LF_FILL] != 0 && a.list_flags[LF_OVERFLOW] == 0));
    int ng = 0;
    long long entries = 0;
    for (int t = w; t < total; t += nw) {
        const int k = a.refq[t];
        if (lists)
            refine_list<ENERGY, SINGLE>(a, k, lane, s_tab[threadIdx.x >> 5].rt, 32);
        else
            particle_force_warp<ENERGY, false, SINGLE, true>(a, s_tab[threadIdx.x >> 5], nullptr,
                                                             k, lane, ng, false, entries);
    }
}

// the class-ordered queue (heaviest class first), FW_GRAB particles per grab
struct FwQueue {
    int cnt[DCM_MAX_CLASSES], off[DCM_MAX_CLASSES], items[DCM_MAX_CLASSES + 1];

    __device__ __forceinline__ void init(const ForceArgs &a)
    {
        const int K = a.b.K;
        if (threadIdx.x == 0) {
            int run = 0;
            for (int q = K - 1, t = 0; q >= 0; --q, ++t) {
                cnt[q] = a.class_buf[q];
                off[q] = a.class_buf[K + q];
                items[t] = run;
                run += cnt[q];
            }
            items[K] = run;
        }
    }

    template <typename F>
    __device__ __forceinline__ void drain(const ForceArgs &a, int lane, F &&fn)
    {
        const int K = a.b.K;
        const int total = items[K];
        while (true) {
            int item0 = 0;
            if (lane == 0) item0 = (int)atomicAdd(a.queue, (unsigned)FW_GRAB);
            item0 = __shfl_sync(0xffffffffu, item0, 0);
            if (item0 >= total) break;
            const int item1 = min(item0 + FW_GRAB, total);
            int t = 0;
            for (int item = item0; item < item1; ++item) {
                while (t + 1 < K && item >= items[t + 1]) ++t;
                int q = K - 1 - t;
                fn(a.class_list[off[q] + (item - items[t])]);
            }
        }
    }
};

// guard re-decisions and list entries of the block: one atomic each
__device__ __forceinline__ void block_counts(const ForceArgs &a, int ng, long long entries)
{
    __shared__ int s_ng;
    __shared__ unsigned long long s_ent;
    const int lane = threadIdx.x & 31;
    for (int off = 16; off > 0; off >>= 1) {
        ng += __shfl_xor_sync(0xffffffffu, ng, off);
        entries += __shfl_xor_sync(0xffffffffu, entries, off);
    }
    if (threadIdx.x == 0) {
        s_ng = 0;
        s_ent = 0ull;
    }
    __syncthreads();
    if (lane == 0 && ng) atomicAdd(&s_ng, ng);
    if (lane == 0 && entries) atomicAdd(&s_ent, (unsigned long long)entries);
    __syncthreads();
    if (threadIdx.x == 0 && s_ng) atomicAdd(a.guard_count, (unsigned long long)s_ng);
    if (threadIdx.x == 0 && s_ent) atomicAdd(a.list_entries, s_ent);
}

// direct walk; FILL: runs only on a Verlet-list rebuild step and fills the
// lists when the fill gate is open
template <bool ENERGY, bool FILL, bool SINGLE>
__global__ void __launch_bounds__(FW_THREADS, SINGLE ? FW_WALK_MINB1 : FW_WALK_MINB)
    k_force_warp(const __grid_constant__ ForceArgs a)
{
    __shared__ FwTable s_tab[FW_WARPS];
    __shared__ int s_close[FW_WARPS][FW_CLOSE];
    __shared__ FwQueue sq;
    __shared__ int s_run, s_fill;
    sq.init(a);
    if (threadIdx.x == 0) {
        s_run = FILL ? a.list_flags[LF_REBUILD] : 1;
        s_fill = FILL ? a.list_flags[LF_FILL] : 0;
    }
    __syncthreads();
    if (!s_run) return;
    const int lane = threadIdx.x & 31;
    const bool fill_on = s_fill != 0;
    FwTable &tb = s_tab[threadIdx.x >> 5];
    int ng = 0;
    long long entries = 0;
    sq.drain(a, lane, [&](int k) {
        particle_force_warp<ENERGY, FILL, SINGLE>(a, tb, s_close[threadIdx.x >> 5], k, lane, ng,
                                                  fill_on, entries);
    });
    block_counts(a, ng, entries);
}

// Verlet-list forces; runs only on a step that keeps its lists.  A warp
// takes 32/G consecutive sorted slots per grab, one per lane group: in cell
// order the warps resident on an SM work on nearby particles and share
// their neighbours' positions in L1 (a class-ordered queue, heaviest
// particles first, was 3.5 % slower: the lists' lengths are already known
// to be within a few times of each other and the queue balances them)
template <bool ENERGY, int G, bool SINGLE>
__global__ void __launch_bounds__(FW_THREADS, FW_LIST_MINB) k_force_list_warp(ForceArgs a)
{
    __shared__ int s_run;
    __shared__ int s_close[list_close_slots<G>() * FW_THREADS];
    if (threadIdx.x == 0) s_run = a.list_flags[LF_REBUILD] == 0;
    __syncthreads();
    if (!s_run) return;
    constexpr int PER = 32 / G;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, gl = lane & (G - 1);
    const int total = (int)a.b.N;
    int ng = 0;
    while (true) {
        int item0 = 0;
        if (lane == 0) item0 = (int)atomicAdd(a.queue, (unsigned)PER);
        item0 = __shfl_sync(0xffffffffu, item0, 0);
        if (item0 >= total) break;
        const int k = item0 + grp < total ? item0 + grp : -1;
        particle_force_list_group<ENERGY, G, SINGLE>(a, s_close, k, gl, ng);
    }
    block_counts(a, ng, 0);
}

// The same Verlet-list forces class by class, heaviest class first, with
// the lanes per particle of each cutoff class (a.list_g[q]): the per-class
// schedule of Section 5.1 applied to the list force.  A work unit is one
// warp's grab of 32/G consecutive entries of class q's slot list (the class
// lists of the last list build, in cell order within a class).  Which group
// and lanes a particle gets does not depend on the other particles of its
// warp: its result is that of its own list and G alone.
template <bool ENERGY, bool SINGLE>
__global__ void __launch_bounds__(FW_THREADS, FW_LIST_MINB) k_force_list_cls(ForceArgs a)
{
    __shared__ int s_run, s_total;
    __shared__ int s_close[list_close_slots<4>() * FW_THREADS];   // the most slots (G = 4)
    __shared__ int s_off[DCM_MAX_CLASSES], s_cnt[DCM_MAX_CLASSES], s_g[DCM_MAX_CLASSES];
    __shared__ int s_items[DCM_MAX_CLASSES + 1];
    const int K = a.b.K;
    if (threadIdx.x == 0) {
        s_run = a.list_flags[LF_REBUILD] == 0;
        int run = 0;
        for (int t = 0; t < K; ++t) {            // unit order: class K-1 first
            const int q = K - 1 - t;
            const int G = a.list_g[q];
            s_cnt[t] = a.class_buf[q];
            s_off[t] = a.class_buf[K + q];
            s_g[t] = G;
            s_items[t] = run;
            run += (s_cnt[t] + 32 / G - 1) / (32 / G);
        }
        s_items[K] = run;
        s_total = run;
    }
    __syncthreads();
    if (!s_run) return;
    const int lane = threadIdx.x & 31;
    const int total = s_total;
    int ng = 0;
    while (true) {
        int u = 0;
        if (lane == 0) u = (int)atomicAdd(a.queue, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= total) break;
        int t = 0;
        while (t + 1 < K && u >= s_items[t + 1]) ++t;
        const int G = s_g[t];
        const int grp = lane / G;
        const int local = (u - s_items[t]) * (32 / G) + grp;
        const int k = local < s_cnt[t] ? a.class_list[s_off[t] + local] : -1;
        // (a warp-uniform branch: every lane of the warp has the same G)
        if (G == 4)
            particle_force_list_group<ENERGY, 4, SINGLE>(a, s_close, k, lane & 3, ng);
        else if (G == 8)
            particle_force_list_group<ENERGY, 8, SINGLE>(a, s_close, k, lane & 7, ng);
        else if (G == 16)
            particle_force_list_group<ENERGY, 16, SINGLE>(a, s_close, k, lane & 15, ng);
        else
            particle_force_list_group<ENERGY, 32, SINGLE>(a, s_close, k, lane, ng);
    }
    block_counts(a, ng, 0);
}

static void fill_args(dcm_handle *h, ForceArgs &a);

int launch_list_walk(dcm_handle *h, bool fill, const int *gate, float delta)
{
    ForceArgs a;
    fill_args(h, a);
    a.gate = gate;
    a.list_delta = delta;
    cudaMemsetAsync(a.queue, 0, sizeof(unsigned int), h->stream);
    int block = h->tune.block >= 64 && h->tune.block <= FORCE_THREADS ? h->tune.block : FORCE_THREADS;
    int grid = h->num_sms * (2048 / block);
    if (fill)
        k_list_walk<true><<<grid, block, 0, h->stream>>>(a);
    else
        k_list_walk<false><<<grid, block, 0, h->stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "list walk launch");
}

// the direct walk's persistent grid: its resident blocks
template <bool ENERGY, bool FILL>
static void launch_walk(dcm_handle *h, const ForceArgs &a)
{
    if (h->b.M == 1)
        k_force_warp<ENERGY, FILL, true>
            <<<h->num_sms * FW_WALK_MINB1, FW_THREADS, 0, h->stream>>>(a);
    else
        k_force_warp<ENERGY, FILL, false>
            <<<h->num_sms * FW_WALK_MINB, FW_THREADS, 0, h->stream>>>(a);
}

// the refinement of the queued particles (after the step's force kernels)
template <bool ENERGY>
static void launch_refine(dcm_handle *h, const ForceArgs &a)
{
    const int grid = h->num_sms * 4;
    if (h->b.M == 1)
        k_force_refine<ENERGY, true><<<grid, FW_THREADS, 0, h->stream>>>(a);
    else
        k_force_refine<ENERGY, false><<<grid, FW_THREADS, 0, h->stream>>>(a);
}

// ten single-system walk blocks per SM need the largest shared-memory carveout
int prepare_force_kernels()
{
    const void *fns[] = {(const void *)k_force_warp<false, false, true>,
                         (const void *)k_force_warp<true, false, true>,
                         (const void *)k_force_warp<false, true, true>,
                         (const void *)k_force_warp<true, true, true>};
    for (const void *f : fns) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return fail_cuda(e, "walk carveout", __FILE__, __LINE__);
    }
    // the list force's close-pair slots take shared memory; ask for the
    // smallest carveout that holds them, which leaves the rest of the unified
    // L1 to the neighbour positions it gathers
    const void *lf[] = {(const void *)k_force_list_warp<false, 8, true>,
                        (const void *)k_force_list_warp<false, 8, false>,
                        (const void *)k_force_list_warp<false, 4, true>,
                        (const void *)k_force_list_warp<false, 4, false>,
                        (const void *)k_force_list_warp<false, 16, false>,
                        (const void *)k_force_list_warp<false, 32, false>};
    for (const void *f : lf) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 16);
        if (e != cudaSuccess) return fail_cuda(e, "list carveout", __FILE__, __LINE__);
    }
    return DCM_OK;
}

// rebuild step (part 0): direct walk + list fill; other steps (part 1): the
// lists.  Eagerly (part 2) both are launched and each returns at once unless
// it is its step; a captured step puts them in the two bodies of its graph
// IF node on the rebuild decision.
int launch_list_forces(dcm_handle *h, bool energy, int part)
{
    ForceArgs a;
    fill_args(h, a);
    // inside a captured step the drift has zeroed the queues
    if (!h->in_step) cudaMemsetAsync(a.refq_n, 0, 2 * sizeof(unsigned int), h->stream);
    if (part != 1) {
        if (!h->in_step) cudaMemsetAsync(a.queue, 0, sizeof(unsigned int), h->stream);
        if (energy)
            launch_walk<true, true>(h, a);
        else
            launch_walk<false, true>(h, a);
    }
    if (part != 0) {
        a.queue = &h->stats->barrier[5];
        if (!h->in_step) cudaMemsetAsync(a.queue, 0, sizeof(unsigned int), h->stream);
        const int G = h->tune.list_lanes > 0 ? h->tune.list_lanes : FW_LIST_G;
        const int gl = h->num_sms * FW_LIST_MINB;   // persistent: the resident blocks
        const bool one = h->b.M == 1;
        if (h->tune.list_lanes_class[0] != 0) {
            // per-class lanes (validated by dcm_set_tuning)
            if (energy) {
                if (one) k_force_list_cls<true, true><<<gl, FW_THREADS, 0, h->stream>>>(a);
                else k_force_list_cls<true, false><<<gl, FW_THREADS, 0, h->stream>>>(a);
            } else {
                if (one) k_force_list_cls<false, true><<<gl, FW_THREADS, 0, h->stream>>>(a);
                else k_force_list_cls<false, false><<<gl, FW_THREADS, 0, h->stream>>>(a);
            }
        } else if (energy) {
            k_force_list_warp<true, 8, false><<<gl, FW_THREADS, 0, h->stream>>>(a);   // energy steps are rare
        } else if (G == 4) {
            if (one) k_force_list_warp<false, 4, true><<<gl, FW_THREADS, 0, h->stream>>>(a);
            else k_force_list_warp<false, 4, false><<<gl, FW_THREADS, 0, h->stream>>>(a);
        } else if (G == 16) {
            k_force_list_warp<false, 16, false><<<gl, FW_THREADS, 0, h->stream>>>(a);
        } else if (G == 32) {
            k_force_list_warp<false, 32, false><<<gl, FW_THREADS, 0, h->stream>>>(a);
        } else {
            if (one) k_force_list_warp<false, 8, true><<<gl, FW_THREADS, 0, h->stream>>>(a);
            else k_force_list_warp<false, 8, false><<<gl, FW_THREADS, 0, h->stream>>>(a);
        }
    }
    // the list kernels refine in place; the walk of a rebuild step queues
    if (part != 1) {
        if (energy)
            launch_refine<true>(h, a);
        else
            launch_refine<false>(h, a);
    }
    return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "force launch");
}

int launch_forces(dcm_handle *h, bool energy)
{
    ForceArgs a;
    fill_args(h, a);
    const bool list_warp = h->nl && h->list_warp;
    const bool fp64 = h->p.precision == DCM_FP64;
    if (list_warp) return launch_list_forces(h, energy, 2);
    // (the lanes list walks use the queue before the forces of their step;
    // a captured step's drift zeroes the warp walk's queue)
    if (fp64 || !h->in_step) cudaMemsetAsync(a.queue, 0, sizeof(unsigned int), h->stream);
    if (!fp64) {
        // DCM_MIXED: the warp walk, then the refinement of what it queued
        // (and no particle refined in place by a list kernel this time)
        if (!h->in_step) cudaMemsetAsync(a.refq_n, 0, 2 * sizeof(unsigned int), h->stream);
        if (energy) {
            launch_walk<true, false>(h, a);
            launch_refine<true>(h, a);
        } else {
            launch_walk<false, false>(h, a);
            launch_refine<false>(h, a);
        }
        return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "force launch");
    }
    int block = h->tune.block >= 64 && h->tune.block <= FORCE_THREADS ? h->tune.block : FORCE_THREADS;
    int grid = h->num_sms * (2048 / block);
    if (energy)
        k_force<true><<<grid, block, 0, h->stream>>>(a);
    else
        k_force<false><<<grid, block, 0, h->stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "force launch");
}

static void fill_args(dcm_handle *h, ForceArgs &a)
{
    a.b = h->b;
    a.class_buf = h->class_count_dev;
    for (int q = 0; q < DCM_MAX_CLASSES; ++q) {
        const int G = h->tune.list_lanes_class[q];
        a.list_g[q] = G == 4 || G == 16 || G == 32 ? G : 8;
    }
    a.class_list = h->class_list;
    for (int q = 0; q < DCM_MAX_CLASSES; ++q) {
        int G = h->tune.lanes[q];
        a.lanes[q] = (G >= 1 && G <= 32 && (G & (G - 1)) == 0) ? G : 1;
    }
    a.sp4 = h->sp4;
    a.spl4 = h->spl4;
    a.refq = h->refq;
    a.refq_n = &h->stats->barrier[6];
    a.refined_n = &h->stats->barrier[7];
    a.spd = h->spd;
    a.rq = h->rq;
    a.pk = h->pk;
    a.cell_start = h->cell_start;
    a.sorted_id = h->sorted_id;
    a.cell_of = h->cell_of;
    a.x = h->x;
    a.rc = h->rc;
    a.f = h->f;
    a.npair = h->npair;
    a.pe = h->pe;
    a.vir = h->vir;
    a.queue = &h->stats->barrier[2];
    a.guard_count = &h->stats->guard_rechecks;
    a.list_entries = &h->stats->list_entries;
    a.list_flags = h->lflags;
    a.list_ok = h->nl ? h->lflags + LF_OK : nullptr;
    a.nl_start = h->nl_start;
    a.nl = h->nl;
    a.nl_cnt = h->nl_cnt;
    a.nl_w = h->nl;
    a.rl_ref = h->rl_ref;
    a.sh_ref = h->sh_ref;
    a.sh = h->sh;
    a.g0 = h->geo_host[0];
    {
        const Geom &g0 = h->geo_host[0];
        for (int q = 0; q < 3; ++q) {
            a.lc.cf[q] = g0.cf[q];
            a.lc.cfl[q] = g0.cfl[q];
        }
        a.lc.ncx = (float)g0.nc[0];
        a.lc.halfnc = 0.5f * (float)g0.nc[0];
        a.lc.inv_ncx = 1.f / (float)g0.nc[0];
        a.lc.sig2f = g0.sig2f;
        a.lc.eps48f = g0.eps48f;
        a.lc.eps24f = g0.eps24f;
        a.lc.eps2f = g0.eps2f;
        a.lc.sig2l = g0.sig2l;
        a.lc.eps48l = g0.eps48l;
        a.lc.eps24l = g0.eps24l;
        a.lc.rclose2 = g0.rclose2;
        a.lc.redo_f2 = g0.redo_f2;
        a.lc.qtop = g0.qtop;
    }
    a.d = h->d;
    a.list_delta = 0.f;
    a.gate = nullptr;
}

}  // namespace dcm
