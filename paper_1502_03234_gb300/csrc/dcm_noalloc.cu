// dcm_noalloc.cu -- link-cell counting sort that allocates no device memory.
//
// Some callers cannot allocate device memory at the time they need a cell
// list: a host application that hands all device memory to its own pool and
// forbids out-of-band cudaMalloc, a serving loop whose latency budget cannot
// absorb cudaMalloc/cudaFree (they synchronise the device and stall every
// stream), or code that must not allocate while other work is in flight.
// dcm_cell_sort_noalloc gives them the same cell list as the handle-based
// path with caller-owned inputs and outputs and the scratch space in a fixed
// file-scope device array.
//
// The array is a `static __device__` object: every GPU that loads this
// library holds it (DCM_NOALLOC_SCRATCH_BYTES) until the process exits.  In
// host code its name is only a host-side stand-in, so its device address is
// looked up with cudaGetSymbolAddress once per device, with that device
// current, on the first call made on that device.
#include <mutex>

#include "dcm_device.cuh"

namespace dcm {
namespace noalloc {

constexpr int64_t MAX_PARTICLES = DCM_NOALLOC_MAX_PARTICLES;
constexpr int64_t MAX_CELLS = DCM_NOALLOC_MAX_CELLS;
constexpr int THREADS = 256;
constexpr int ITEMS = 8;
constexpr int TILE = THREADS * ITEMS;
constexpr int64_t MAX_TILES = (MAX_CELLS + TILE - 1) / TILE;

// scratch layout: per-cell counts | per-particle arrival slots | tile sums
constexpr int64_t WORDS = MAX_CELLS + MAX_PARTICLES + MAX_TILES;
static_assert(WORDS * 4 == DCM_NOALLOC_SCRATCH_BYTES, "scratch size must match dcm.h");
static __device__ __align__(256) int32_t g_scratch[WORDS];

constexpr int MAX_DEVICES = 64;
static int32_t *g_ptr[MAX_DEVICES];
static std::mutex g_mu;

// device address of the scratch array on the current device (looked up once)
static int scratch_on_current_device(int32_t **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice", __FILE__, __LINE__);
    if (dev < 0 || dev >= MAX_DEVICES) return fail(DCM_ERR_ARG, "device ordinal %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress(scratch)", __FILE__, __LINE__);
        g_ptr[dev] = (int32_t *)p;
    }
    *out = g_ptr[dev];
    return DCM_OK;
}

struct Args {
    const double *x;     // AoS [n][3]
    int64_t n;
    int nc[3];
    double inv_c[3];
    int64_t ncell;
    int32_t *count, *slot, *tiles;
    int32_t *cell_start, *sorted_id;
};

__global__ void k_zero(int32_t *p, int64_t m)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 0;
}

__global__ void k_count(Args a)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    int cx = bin_of(a.x[3 * i + 0], a.inv_c[0], a.nc[0]);
    int cy = bin_of(a.x[3 * i + 1], a.inv_c[1], a.nc[1]);
    int cz = bin_of(a.x[3 * i + 2], a.inv_c[2], a.nc[2]);
    int c = cx + a.nc[0] * (cy + a.nc[1] * cz);
    a.slot[i] = atomicAdd(&a.count[c], 1);
}

__global__ void k_scan_tiles(Args a)
{
    __shared__ int32_t s[THREADS];
    int64_t base = (int64_t)blockIdx.x * TILE + (int64_t)threadIdx.x * ITEMS;
    int32_t v[ITEMS];
    int32_t run = 0;
#pragma unroll
    for (int q = 0; q < ITEMS; ++q) {
        v[q] = base + q < a.ncell ? a.count[base + q] : 0;
        run += v[q];
    }
    s[threadIdx.x] = run;
    __syncthreads();
    for (int off = 1; off < THREADS; off <<= 1) {
        int32_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    int32_t excl = threadIdx.x ? s[threadIdx.x - 1] : 0;
#pragma unroll
    for (int q = 0; q < ITEMS; ++q) {
        if (base + q < a.ncell) a.cell_start[base + q] = excl;
        excl += v[q];
    }
    if (threadIdx.x == THREADS - 1) a.tiles[blockIdx.x] = s[THREADS - 1];
}

__global__ void k_scan_add(Args a)
{
    __shared__ int32_t s[THREADS];
    int32_t acc = 0;
    for (int t = threadIdx.x; t < (int)blockIdx.x; t += THREADS) acc += a.tiles[t];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    int64_t base = (int64_t)blockIdx.x * TILE;
    for (int q = threadIdx.x; q < TILE; q += THREADS)
        if (base + q < a.ncell) a.cell_start[base + q] += s[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) a.cell_start[a.ncell] = (int32_t)a.n;
}

__global__ void k_scatter(Args a)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    int cx = bin_of(a.x[3 * i + 0], a.inv_c[0], a.nc[0]);
    int cy = bin_of(a.x[3 * i + 1], a.inv_c[1], a.nc[1]);
    int cz = bin_of(a.x[3 * i + 2], a.inv_c[2], a.nc[2]);
    int c = cx + a.nc[0] * (cy + a.nc[1] * cz);
    a.sorted_id[a.cell_start[c] + a.slot[i]] = (int32_t)i;
}

__global__ void k_sort_cells(Args a)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.ncell) return;
    int lo = a.cell_start[c], hi = a.cell_start[c + 1];
    for (int q = lo + 1; q < hi; ++q) {
        int key = a.sorted_id[q];
        int b = q - 1;
        while (b >= lo && a.sorted_id[b] > key) {
            a.sorted_id[b + 1] = a.sorted_id[b];
            --b;
        }
        a.sorted_id[b + 1] = key;
    }
}

}  // namespace noalloc
}  // namespace dcm

using namespace dcm;

extern "C" int dcm_cell_sort_noalloc(const double *x, int64_t n, const dcm_box *box,
                                     const int32_t nc[3], int32_t *cell_start,
                                     int32_t *sorted_id, void *stream)
{
    namespace na = dcm::noalloc;
    if (!x || !box || !nc || !cell_start || !sorted_id)
        return fail(DCM_ERR_ARG, "null argument");
    if (n < 1 || n > na::MAX_PARTICLES)
        return fail(DCM_ERR_ARG, "n = %lld outside 1..%lld (DCM_NOALLOC_MAX_PARTICLES)",
                    (long long)n, (long long)na::MAX_PARTICLES);
    double L[3] = {box->lx, box->ly, box->lz};
    int64_t ncell = 1;
    na::Args a;
    for (int d = 0; d < 3; ++d) {
        if (!(L[d] > 0) || nc[d] < 1) return fail(DCM_ERR_ARG, "box edges and cell counts must be positive");
        // each factor and each partial product stays within the limit, so
        // the product never wraps (three int32 counts can exceed int64)
        if ((int64_t)nc[d] > na::MAX_CELLS || ncell * (int64_t)nc[d] > na::MAX_CELLS)
            return fail(DCM_ERR_ARG, "cells %d x %d x %d exceed DCM_NOALLOC_MAX_CELLS = %lld",
                        nc[0], nc[1], nc[2], (long long)na::MAX_CELLS);
        a.nc[d] = nc[d];
        a.inv_c[d] = (double)nc[d] / L[d];
        ncell *= nc[d];
    }
    int32_t *scratch = nullptr;
    int rc = na::scratch_on_current_device(&scratch);
    if (rc) return rc;
    a.x = x;
    a.n = n;
    a.ncell = ncell;
    a.count = scratch;
    a.slot = scratch + na::MAX_CELLS;
    a.tiles = scratch + na::MAX_CELLS + na::MAX_PARTICLES;
    a.cell_start = cell_start;
    a.sorted_id = sorted_id;
    cudaStream_t s = (cudaStream_t)stream;
    int nb = (int)((n + na::THREADS - 1) / na::THREADS);
    int ntiles = (int)((ncell + na::TILE - 1) / na::TILE);
    int cb = (int)((ncell + na::THREADS - 1) / na::THREADS);
    // the array keeps the previous call's contents: the counts start at zero
    na::k_zero<<<cb < 1024 ? cb : 1024, na::THREADS, 0, s>>>(a.count, ncell);
    na::k_count<<<nb, na::THREADS, 0, s>>>(a);
    na::k_scan_tiles<<<ntiles, na::THREADS, 0, s>>>(a);
    na::k_scan_add<<<ntiles, na::THREADS, 0, s>>>(a);
    na::k_scatter<<<nb, na::THREADS, 0, s>>>(a);
    na::k_sort_cells<<<cb, na::THREADS, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(e, "dcm_cell_sort_noalloc launch", __FILE__, __LINE__);
    return DCM_OK;
}
