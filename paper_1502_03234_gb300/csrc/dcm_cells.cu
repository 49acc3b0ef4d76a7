// dcm_cells.cu -- link-cell binning (Section 2.2.1, bins per Section 3.2):
// an integer counting sort of the particles by cell, bit-exact with the
// definition (cell index = min(n-1, floor(x * n/L)), ascending particle id
// inside a cell), followed by the gather of the sorted FP32/FP64 positions
// the force kernels stream, and per-class lists of sorted slots.
//
// HBM bound: ~40 B/particle (positions read, cell/slot/id written twice) plus
// 16-32 B/particle for the sorted position streams.
#include "dcm_device.cuh"

namespace dcm {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;                       // per thread
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// cell of every particle + its arrival slot within the cell (atomic order;
// the order inside a cell is fixed afterwards by k_cell_sort)
// (cells of all systems are concatenated: cell_of holds the global index)
// gate: nullptr = always run; otherwise the kernel does nothing while *gate
// is 0 (a step that keeps its Verlet lists keeps its cell sort too)
__device__ __forceinline__ bool gated_off(const int *gate) { return gate && *gate == 0; }

__global__ void k_cell_count(Batch b, const double *__restrict__ x, int32_t *cell_of,
                             int32_t *slot, int32_t *count, const int *gate)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.N || gated_off(gate)) return;
    const Geom &g = b.sys[sys_p(b, i)];
    int cx = bin_of(x[i], g.inv_c[0], g.nc[0]);
    int cy = bin_of(x[(size_t)b.N + i], g.inv_c[1], g.nc[1]);
    int cz = bin_of(x[2 * (size_t)b.N + i], g.inv_c[2], g.nc[2]);
    int c = (int)g.c0 + cx + g.nc[0] * (cy + g.nc[1] * cz);
    cell_of[i] = c;
    slot[i] = atomicAdd(&count[c], 1);
}

// exclusive scan, pass 1: scan each tile, record the tile total
__global__ void k_scan_tiles(const int32_t *__restrict__ in, int32_t *out, int32_t *tile_sum,
                             int64_t m, const int *gate)
{
    __shared__ int32_t s[SCAN_THREADS];
    if (gated_off(gate)) return;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int32_t run = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        int64_t k = base + q;
        v[q] = k < m ? in[k] : 0;
        run += v[q];
    }
    s[threadIdx.x] = run;
    __syncthreads();
    // Hillis-Steele inclusive scan of the per-thread totals
    for (int off = 1; off < SCAN_THREADS; off <<= 1) {
        int32_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    int32_t excl = threadIdx.x ? s[threadIdx.x - 1] : 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        int64_t k = base + q;
        if (k < m) out[k] = excl;
        excl += v[q];
    }
    if (threadIdx.x == SCAN_THREADS - 1) tile_sum[blockIdx.x] = s[SCAN_THREADS - 1];
}

// exclusive scan, pass 2: add the sum of all earlier tiles
// total >= 0: out[m] = total; total < 0: out[m] = the sum of all inputs
__global__ void k_scan_add(int32_t *out, const int32_t *__restrict__ tile_sum, int64_t m,
                           int32_t total, int ntiles, const int *gate)
{
    __shared__ int32_t s[SCAN_THREADS];
    if (gated_off(gate)) return;
    int32_t acc = 0;
    for (int t = threadIdx.x; t < (int)blockIdx.x; t += SCAN_THREADS) acc += tile_sum[t];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = SCAN_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    int32_t off = s[0];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int q = threadIdx.x; q < SCAN_TILE; q += SCAN_THREADS) {
        int64_t k = base + q;
        if (k < m) out[k] += off;
    }
    if (blockIdx.x == ntiles - 1 && threadIdx.x == 0)
        out[m] = total >= 0 ? total : off + tile_sum[blockIdx.x];
}

__global__ void k_cell_scatter(int n, const int32_t *__restrict__ cell_of,
                               const int32_t *__restrict__ slot,
                               const int32_t *__restrict__ start, int32_t *sorted_id,
                               const int *gate)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || gated_off(gate)) return;
    sorted_id[start[cell_of[i]] + slot[i]] = i;
}

// ascending particle id inside each cell (cells hold a handful of particles)
__global__ void k_cell_sort(int64_t ncell, const int32_t *__restrict__ start, int32_t *sorted_id,
                            const int *gate)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell || gated_off(gate)) return;
    int lo = start[c], hi = start[c + 1];
    for (int a = lo + 1; a < hi; ++a) {
        int key = sorted_id[a];
        int b = a - 1;
        while (b >= lo && sorted_id[b] > key) {
            sorted_id[b + 1] = sorted_id[b];
            --b;
        }
        sorted_id[b + 1] = key;
    }
}

// sorted position streams: sp4 = (x - cell corner in FP32, cell x index),
// spl4 = its FP32 remainder (mixed path), spd = absolute FP64 position (FP64
// path only)
__global__ void k_gather(Batch b, const double *__restrict__ x, const double *__restrict__ v,
                         const double *__restrict__ f,
                         const int32_t *__restrict__ sorted_id,
                         const int32_t *__restrict__ cell_of, float4 *sp4, float4 *spl4,
                         double4_32a *spd,
                         const double *__restrict__ rc, float4 *rq, int4 *pk, float *sh,
                         const double *__restrict__ dist, int *lf, float delta, int32_t *capk,
                         int32_t *inv, const int *gate, int32_t *cell_count)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gated_off(gate)) return;
    // the cell counts have served the scan: zero them for the next sort
    for (int64_t c = k; c < b.NC; c += (int64_t)gridDim.x * blockDim.x) cell_count[c] = 0;
    if (k >= b.N) return;
    // sorted slots keep the systems' particle ranges
    const Geom &g = b.sys[sys_p(b, k)];
    int i = sorted_id[k];
    int c = cell_of[i] - (int)g.c0;
    double px = x[i], py = x[(size_t)b.N + i], pz = x[2 * (size_t)b.N + i];
    float4 lo;
    sp4[k] = cell_rel_position(b, g, px, py, pz, c, lo);
    if (spl4) spl4[k] = lo;
    if (spd) spd[k] = make_double4_32a(px, py, pz, 0.0);
    if (inv) inv[i] = (int32_t)k;
    if (rq) {
        // the force walk's per-particle constants, once per particle here
        // instead of once per warp there
        double r = rc[i];
        rq[k] = rc_constants(r);
        int cy = (c / g.nc[0]) % g.nc[1];
        int cz = c / (g.nc[0] * g.nc[1]);
        int w = 0;
        if (capk && lf[LF_REBUILD]) {
            // a Verlet-list build follows: the skin share (from the
            // particle's speed and force) and own list radius of this
            // particle, and its entry capacity, (4/3) pi R^3 for R = own
            // radius + the largest share at the density bound scale (1.0
            // sigma^-3 unless a list overflowed before) + 8, rounded up to
            // 8 entries so that every list starts on a 32-byte sector (the
            // force kernel's 8-lane loads then touch one sector each) and
            // capped so that the int32 offset scan cannot wrap
            const size_t N = (size_t)b.N;
            const float vx = (float)v[i], vy = (float)v[N + i], vz = (float)v[2 * N + i];
            const float fx = (float)f[i], fy = (float)f[N + i], fz = (float)f[2 * N + i];
            const float share = skin_share(g, sqrtf(fmaf(vx, vx, fmaf(vy, vy, vz * vz))),
                                           sqrtf(fmaf(fx, fx, fmaf(fy, fy, fz * fz))));
            const float rl = list_radius(g, r, dist[i], delta, share);
            const float R = rl + 0.5f * (float)g.skin;
            float scale = __int_as_float(lf[LF_SCALE]);
            const float capmax = (float)((int32_t)((0x7fffffffLL - 1024) / b.N) & ~7);
            capk[k] = (int32_t)fminf(ceilf(scale * 4.18879020f * R * R * R) + 15.0f, capmax) & ~7;
            w = __float_as_int(rl);
            sh[k] = share;
            // non-negative floats order like their bit patterns; one
            // atomic per warp
            const unsigned act = __activemask();
            const unsigned mx = __reduce_max_sync(act, (unsigned)__float_as_int(share));
            if ((threadIdx.x & 31) == __ffs(act) - 1) atomicMax(&lf[LF_SHMAX], (int)mx);
        }
        pk[k] = make_int4(i, cy, cz, w);
    }
}

__global__ void k_class_zero(int32_t *buf, const int *gate)
{
    if (gated_off(gate)) return;
    if (threadIdx.x < 3 * DCM_MAX_CLASSES) buf[threadIdx.x] = 0;
}

// per-class lists of sorted slots (warp-aggregated appends keep neighbouring
// slots together); counts[0..K) must be prefix offsets, cursors[0..K) zero
__global__ void k_class_lists(int n, int K, const int32_t *__restrict__ sorted_id,
                              const uint8_t *__restrict__ cls, const int32_t *__restrict__ offs,
                              int32_t *cursor, int32_t *list, const int *gate)
{
    if (gated_off(gate)) return;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int lane = threadIdx.x & 31;
    int c = k < n ? (int)cls[sorted_id[k]] : -1;
    unsigned lt = (1u << lane) - 1u;
    for (int q = 0; q < K; ++q) {
        unsigned m = __ballot_sync(0xffffffffu, c == q);
        if (!m) continue;
        int leader = __ffs(m) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&cursor[q], __popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (c == q) list[offs[q] + base + __popc(m & lt)] = k;
    }
}

__global__ void k_class_count(int n, int K, const uint8_t *__restrict__ cls, int32_t *count,
                              const int *gate)
{
    if (gated_off(gate)) return;
    __shared__ int32_t s[DCM_MAX_CLASSES];
    if (threadIdx.x < DCM_MAX_CLASSES) s[threadIdx.x] = 0;
    __syncthreads();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&s[cls[i]], 1);
    __syncthreads();
    if (threadIdx.x < K && s[threadIdx.x]) atomicAdd(&count[threadIdx.x], s[threadIdx.x]);
}

// counts [0..K) -> exclusive offsets [K..2K), cursors [2K..3K) zeroed
__global__ void k_class_offsets(int K, int32_t *buf, const int *gate)
{
    if (gated_off(gate)) return;
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int run = 0;
    for (int q = 0; q < K; ++q) {
        buf[K + q] = run;
        run += buf[q];
        buf[2 * K + q] = 0;
    }
}

static inline int nblk(int64_t n, int b) { return (int)((n + b - 1) / b); }

int launch_scan(dcm_handle *h, const int32_t *in, int32_t *out, int32_t *tiles, int64_t m,
                int32_t total, const int *gate)
{
    int ntiles = nblk(m, SCAN_TILE);
    k_scan_tiles<<<ntiles, SCAN_THREADS, 0, h->stream>>>(in, out, tiles, m, gate);
    k_scan_add<<<ntiles, SCAN_THREADS, 0, h->stream>>>(out, tiles, m, total, ntiles, gate);
    return DCM_OK;
}

// cell sort (skipped while *gate == 0), then the gather of the sorted
// streams from the current positions and the per-class lists.  With the
// warp Verlet-list kernels the drift and the cutoff kernel keep the sorted
// positions and cutoff constants current between builds, so the gather
// runs only with the sort, and so do the class lists (launch_classes;
// class_gate null: always), which only order the force kernels' work.
int launch_sort_gather(dcm_handle *h, const int *gate)
{
    cudaStream_t s = h->stream;
    int n = (int)h->n;
    // cell_count is zero here: zeroed at creation and again by the gather
    // once the scan has used it
    k_cell_count<<<nblk(n, 256), 256, 0, s>>>(h->b, h->x, h->cell_of, h->slot, h->cell_count, gate);
    launch_scan(h, h->cell_count, h->cell_start, h->scan_tmp, h->ncell, n, gate);
    k_cell_scatter<<<nblk(n, 256), 256, 0, s>>>(n, h->cell_of, h->slot, h->cell_start,
                                                h->sorted_id, gate);
    k_cell_sort<<<nblk(h->ncell, 256), 256, 0, s>>>(h->ncell, h->cell_start, h->sorted_id, gate);
    const bool wl = h->nl && h->list_warp;
    k_gather<<<nblk(n, 256), 256, 0, s>>>(h->b, h->x, h->v, h->f, h->sorted_id, h->cell_of, h->sp4,
                                          h->spl4,
                                          h->p.precision == DCM_FP64 ? h->spd : nullptr, h->rc,
                                          h->rq, h->pk, h->sh, h->d, h->lflags,
                                          h->cut_detected ? h->list_margin : 0.0f, wl ? h->nl_cnt : nullptr,
                                          h->inv, wl ? gate : nullptr, h->cell_count);
    return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "binning launch");
}

// class lists of sorted slots for the force work queue
int launch_classes(dcm_handle *h, const int *class_gate)
{
    cudaStream_t s = h->stream;
    int n = (int)h->n;
    int K = h->b.K;
    k_class_zero<<<1, 32, 0, s>>>(h->class_count_dev, class_gate);
    k_class_count<<<nblk(n, 256), 256, 0, s>>>(n, K, h->cls, h->class_count_dev, class_gate);
    k_class_offsets<<<1, 32, 0, s>>>(K, h->class_count_dev, class_gate);
    k_class_lists<<<nblk(n, 256), 256, 0, s>>>(n, K, h->sorted_id, h->cls,
                                               h->class_count_dev + K,
                                               h->class_count_dev + 2 * K, h->class_list,
                                               class_gate);
    return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "class launch");
}

int launch_bin_gated(dcm_handle *h, const int *gate, const int *class_gate)
{
    int r = launch_sort_gather(h, gate);
    return r ? r : launch_classes(h, class_gate);
}

int launch_bin(dcm_handle *h) { return launch_bin_gated(h, nullptr, nullptr); }

}  // namespace dcm
