// dcm_detect.cu -- interface detection (Section 4, Fig. 14) and the per-
// particle cutoff (Algorithm 3.1, Eq. 7-8).
//
//   density   Eq. 9: B_ijk = particles in voxel (integer atomics)
//   smoothing three periodic 1D passes with binomial weights C(order, k).
//             The values are exact integers; passes 1-2 run in uint32 and
//             pass 3 in uint64 -> FP64, which gives exactly the numbers an
//             FP64 evaluation gives (all < 2^53) at integer-pipe cost.
//   K-means   Eq. 14, K = 2, Lloyd iterations from (max, min) in one
//             cooperative kernel; sums are exact integers, so the
//             threshold (c_l + c_v)/2 and the labels (Eq. 11-12) are
//             bit-identical to the definition.  Liquid sets of successive
//             iterations are threshold sets, hence nested: equal counts
//             mean an unchanged assignment (the stopping rule).
//   CFSM      Algorithm 4.3 as a Jacobi fixed point over a frontier: each
//             pass recomputes only the voxels whose neighbours changed in
//             the previous pass, writes the other buffer, and stops when
//             nothing changes (eps = 0) or at iter_max; voxels whose
//             solution exceeds r_grid = r_c,max + h are never updated.  The
//             result is independent of thread scheduling.
//   cutoff    trilinear interpolation from the lower-left-front voxel
//             centre (Algorithm 3.1), then Eq. 7-8 and the class.
// Bound: HBM/L2 (the grid holds ~3.7 voxels per particle at 1 sigma voxels).
#include <cooperative_groups.h>

#include "dcm_device.cuh"

namespace dcm {

constexpr int DET_THREADS = 256;

__global__ void k_density(Geom g, const double *__restrict__ x, int32_t *B)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    int gx = bin_of(x[i], g.inv_h[0], g.gd[0]);
    int gy = bin_of(x[(size_t)g.n + i], g.inv_h[1], g.gd[1]);
    int gz = bin_of(x[2 * (size_t)g.n + i], g.inv_h[2], g.gd[2]);
    atomicAdd(&B[gx + g.gd[0] * (gy + g.gd[1] * gz)], 1);
}

struct SmoothW {
    uint32_t w[17];
    int order;
    uint32_t bmax;      // largest voxel count for which pass 2 cannot overflow
};

// one periodic 1D pass along AXIS (0 = x, 1 = y, 2 = z)
template <int AXIS, typename TIN, typename TOUT>
__global__ void k_smooth(const TIN *__restrict__ in, TOUT *out, int nx, int ny, int nz, SmoothW w,
                         int *err)
{
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nv = (int64_t)nx * ny * nz;
    if (v >= nv) return;
    int x = (int)(v % nx);
    int y = (int)((v / nx) % ny);
    int z = (int)(v / ((int64_t)nx * ny));
    int n = AXIS == 0 ? nx : (AXIS == 1 ? ny : nz);
    int c = AXIS == 0 ? x : (AXIS == 1 ? y : z);
    int64_t stride = AXIS == 0 ? 1 : (AXIS == 1 ? (int64_t)nx : (int64_t)nx * ny);
    int64_t base = v - (int64_t)c * stride;
    int half = w.order / 2;
    if constexpr (AXIS == 0) {
        if ((uint32_t)in[v] > w.bmax) atomicOr(err, DEV_ERR_DENSITY);
    }
    if constexpr (sizeof(TOUT) == 8) {
        unsigned long long s = 0;
        for (int k = 0; k <= w.order; ++k) {
            int q = ((c + k - half) % n + n) % n;
            s += (unsigned long long)w.w[k] * (unsigned long long)in[base + (int64_t)q * stride];
        }
        out[v] = (TOUT)s;
    } else {
        uint32_t s = 0;
        for (int k = 0; k <= w.order; ++k) {
            int q = ((c + k - half) % n + n) % n;
            s += w.w[k] * (uint32_t)in[base + (int64_t)q * stride];
        }
        out[v] = (TOUT)s;
    }
}

// ---- K-means (Eq. 14, K = 2) -------------------------------------------------
// acc words: [0] max, [1] min, [2] total, then 3 rotating (count, sum) pairs
__global__ void k_kmeans_init(unsigned long long *acc)
{
    acc[0] = 0ull;
    acc[1] = ~0ull;
    acc[2] = 0ull;
    for (int q = 3; q < 9; ++q) acc[q] = 0ull;
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v,
                                                            unsigned long long *sh)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
    return t;   // valid in thread 0
}

__global__ void __launch_bounds__(DET_THREADS)
    k_kmeans(const double *__restrict__ Bs, int64_t nv, uint8_t *S, int max_iter,
             unsigned long long *acc, unsigned int *bar, int *err, DevStats *st)
{
    __shared__ unsigned long long sh[DET_THREADS / 32];
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nth = (int64_t)gridDim.x * blockDim.x;
    // extremes and the total (exact integers)
    unsigned long long mx = 0, mn = ~0ull, tot = 0;
    for (int64_t v = tid; v < nv; v += nth) {
        unsigned long long b = (unsigned long long)Bs[v];
        mx = b > mx ? b : mx;
        mn = b < mn ? b : mn;
        tot += b;
    }
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, off);
        mx = o > mx ? o : mx;
        o = __shfl_xor_sync(0xffffffffu, mn, off);
        mn = o < mn ? o : mn;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&acc[0], mx);
        atomicMin(&acc[1], mn);
    }
    unsigned long long t = block_sum_u64(tot, sh);
    if (threadIdx.x == 0) atomicAdd(&acc[2], t);
    if (!grid_barrier(bar, err)) return;
    // values other blocks produced are read through L2 (ld.global.cg): the
    // per-SM L1 caches are not coherent across a grid barrier
    double cl = (double)__ldcg(&acc[0]), cv = (double)__ldcg(&acc[1]);
    unsigned long long total = __ldcg(&acc[2]);
    long long prev = -1;
    double thr = DMUL(DADD(cl, cv), 0.5);
    int it = 0;
    for (; it < max_iter;) {
        thr = DMUL(DADD(cl, cv), 0.5);
        unsigned long long *cur = acc + 3 + 2 * (it % 3);
        unsigned long long cnt = 0, sum = 0;
        for (int64_t v = tid; v < nv; v += nth) {
            double b = Bs[v];
            if (b >= thr) {
                cnt++;
                sum += (unsigned long long)b;
            }
        }
        unsigned long long bc = block_sum_u64(cnt, sh);
        unsigned long long bs = block_sum_u64(sum, sh);
        if (threadIdx.x == 0) {
            atomicAdd(&cur[0], bc);
            atomicAdd(&cur[1], bs);
            if (blockIdx.x == 0) {   // clear the pair used two passes ahead
                unsigned long long *nxt = acc + 3 + 2 * ((it + 1) % 3);
                nxt[0] = 0ull;
                nxt[1] = 0ull;
            }
        }
        if (!grid_barrier(bar, err)) return;
        long long nl = (long long)__ldcg(&cur[0]);
        unsigned long long sl = __ldcg(&cur[1]);
        ++it;
        if (nl == prev) break;   // same threshold set as the previous pass
        long long nvap = nv - nl;
        if (nl > 0) cl = (double)sl / (double)nl;
        if (nvap > 0) cv = (double)(total - sl) / (double)nvap;
        prev = nl;
    }
    for (int64_t v = tid; v < nv; v += nth) S[v] = Bs[v] >= thr ? 0 : 1;
    if (tid == 0) {
        st->kmeans_iters = it;
        st->c_liquid = cl;
        st->c_vapor = cv;
    }
}

// ---- CFSM (Algorithm 4.3) ------------------------------------------------------
__device__ __forceinline__ int64_t vox(int x, int y, int z, int nx, int ny)
{
    return x + (int64_t)nx * (y + (int64_t)ny * z);
}

// D0 = D1 = 0 on vapor, +inf on liquid; frontier 0 = liquid voxels with a
// vapor face neighbour (the "interfacial boxes")
__global__ void k_cfsm_init(int nx, int ny, int nz, const uint8_t *__restrict__ S, double *D0,
                            double *D1, int32_t *stamp, int32_t *list0, int32_t *fcount)
{
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nv = (int64_t)nx * ny * nz;
    if (v >= nv) return;
    bool vap = S[v] == 1;
    double d = vap ? 0.0 : __longlong_as_double(0x7ff0000000000000ll);
    D0[v] = d;
    D1[v] = d;
    int st = -1;
    if (!vap) {
        int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((int64_t)nx * ny));
        int xm = x ? x - 1 : nx - 1, xp = x + 1 < nx ? x + 1 : 0;
        int ym = y ? y - 1 : ny - 1, yp = y + 1 < ny ? y + 1 : 0;
        int zm = z ? z - 1 : nz - 1, zp = z + 1 < nz ? z + 1 : 0;
        if (S[vox(xm, y, z, nx, ny)] | S[vox(xp, y, z, nx, ny)] | S[vox(x, ym, z, nx, ny)] |
            S[vox(x, yp, z, nx, ny)] | S[vox(x, y, zm, nx, ny)] | S[vox(x, y, zp, nx, ny)]) {
            list0[atomicAdd(&fcount[0], 1)] = (int32_t)v;
            st = 0;
        }
    }
    stamp[v] = st;
}

struct CfsmArgs {
    int nx, ny, nz;
    double h0, h1, h2;
    double r_grid;
    int iter_max;
    int64_t cap;              // capacity of one frontier list
    const uint8_t *S;
    double *D0, *D1;
    int32_t *stamp;
    int32_t *lists;           // 4 * cap
    int32_t *fcount;          // 4 counters
    int *result;              // which buffer holds the result
    unsigned int *bar;
    int *err;
    DevStats *st;
};

__global__ void __launch_bounds__(DET_THREADS) k_cfsm(CfsmArgs a)
{
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    int k = 0;
    bool converged = false;
    for (; k < a.iter_max; ++k) {
        const double *X = (k & 1) ? a.D1 : a.D0;
        double *Y = (k & 1) ? a.D0 : a.D1;
        int32_t *F = a.lists + (int64_t)(k & 3) * a.cap;
        int32_t *Fn = a.lists + (int64_t)((k + 1) & 3) * a.cap;
        int nf = ((volatile int32_t *)a.fcount)[k & 3];
        if (nf == 0) {
            converged = true;
            break;
        }
        if (tid == 0) a.fcount[(k + 2) & 3] = 0;   // list two passes ahead
        for (int64_t q = tid; q < nf; q += nth) {
            int v = __ldcg(&F[q]);
            int x = v % nx, y = (v / nx) % ny, z = v / (nx * ny);
            int xm = x ? x - 1 : nx - 1, xp = x + 1 < nx ? x + 1 : 0;
            int ym = y ? y - 1 : ny - 1, yp = y + 1 < ny ? y + 1 : 0;
            int zm = z ? z - 1 : nz - 1, zp = z + 1 < nz ? z + 1 : 0;
            int64_t nb[6] = {vox(xm, y, z, nx, ny), vox(xp, y, z, nx, ny),
                             vox(x, ym, z, nx, ny), vox(x, yp, z, nx, ny),
                             vox(x, y, zm, nx, ny), vox(x, y, zp, nx, ny)};
            // D and the lists were written by other blocks in the previous
            // pass: read them through L2 (ld.global.cg), not a stale L1
            double old = __ldcg(&X[v]);
            double ax = fmin(__ldcg(&X[nb[0]]), __ldcg(&X[nb[1]]));
            double ay = fmin(__ldcg(&X[nb[2]]), __ldcg(&X[nb[3]]));
            double az = fmin(__ldcg(&X[nb[4]]), __ldcg(&X[nb[5]]));
            double dbar = godunov(ax, ay, az, a.h0, a.h1, a.h2);
            bool changed = dbar < old && dbar <= a.r_grid;
            Y[v] = changed ? dbar : old;
            if (changed) {
                // the voxel itself (so Y catches up next pass) and its liquid
                // face neighbours are recomputed in the next pass
                if (atomicExch(&a.stamp[v], k + 1) != k + 1) Fn[atomicAdd(&a.fcount[(k + 1) & 3], 1)] = v;
                for (int e = 0; e < 6; ++e) {
                    int64_t u = nb[e];
                    if (a.S[u] == 1) continue;
                    if (atomicExch(&a.stamp[u], k + 1) != k + 1)
                        Fn[atomicAdd(&a.fcount[(k + 1) & 3], 1)] = (int32_t)u;
                }
            }
        }
        if (!grid_barrier(a.bar, a.err)) return;
    }
    if (tid == 0) {
        // after pass k-1 the current values are in the buffer it wrote
        *a.result = (k & 1) ? 1 : 0;
        a.st->cfsm_iters = k;
        if (!converged) atomicOr(a.err, DEV_ERR_CFSM_CAP);
    }
}

// ---- Algorithm 3.1 + Eq. 7-8 ----------------------------------------------------
__global__ void k_cutoff(Geom g, const double *__restrict__ x, const double *__restrict__ D0,
                         const double *__restrict__ D1, const int *__restrict__ result, double *d,
                         double *rc, uint8_t *cls)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const double *D = *result ? D1 : D0;
    int i0[3], i1[3];
    double t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double gg = DSUB(DMUL(x[(size_t)a * g.n + i], g.inv_h[a]), 0.5);
        double fl = floor(gg);
        t[a] = DSUB(gg, fl);
        int lo = (int)fl;
        int n = g.gd[a];
        lo = lo < 0 ? lo + n : (lo >= n ? lo - n : lo);
        int hi = lo + 1 < n ? lo + 1 : 0;
        i0[a] = lo;
        i1[a] = hi;
    }
    const int nx = g.gd[0], ny = g.gd[1];
    auto Dv = [&](int X, int Y, int Z) {
        double v = D[X + (int64_t)nx * (Y + (int64_t)ny * Z)];
        return v < g.r_grid ? v : g.r_grid;   // voxels CFSM never reached
    };
    double c00 = lerp_rn(Dv(i0[0], i0[1], i0[2]), Dv(i1[0], i0[1], i0[2]), t[0]);
    double c10 = lerp_rn(Dv(i0[0], i1[1], i0[2]), Dv(i1[0], i1[1], i0[2]), t[0]);
    double c01 = lerp_rn(Dv(i0[0], i0[1], i1[2]), Dv(i1[0], i0[1], i1[2]), t[0]);
    double c11 = lerp_rn(Dv(i0[0], i1[1], i1[2]), Dv(i1[0], i1[1], i1[2]), t[0]);
    double c0 = lerp_rn(c00, c10, t[1]);
    double c1 = lerp_rn(c01, c11, t[1]);
    double di = lerp_rn(c0, c1, t[2]);
    double r;
    if (di <= 0.0)
        r = g.rc_max;
    else if (di >= g.rc_max)
        r = g.rc_min;
    else
        r = DADD(DMUL(g.cut_a, exp2(DMUL(g.alpha, DSUB(g.rc_max, di)))), g.cut_b);
    int c = 0;
    if (di < g.rc_max) {
        c = 1;
        for (int k = 0; k < g.K - 2; ++k) c += di < g.thr[k] ? 1 : 0;
    }
    d[i] = di;
    rc[i] = r;
    cls[i] = (uint8_t)c;
}

// classes for cutoffs supplied directly (scheduling only)
__global__ void k_classify_rc(Geom g, const double *__restrict__ rc, uint8_t *cls)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    double r = rc[i];
    int c = 0;
    if (r > g.rc_min) {
        c = 1;
        for (int k = 1; k <= g.K - 2; ++k) {
            double edge = g.rc_min + (g.rc_max - g.rc_min) * (double)k / (double)(g.K - 1);
            c += r > edge ? 1 : 0;
        }
    }
    cls[i] = (uint8_t)c;
}

static inline int nblk(int64_t n, int b) { return (int)((n + b - 1) / b); }

int launch_classify_rc(dcm_handle *h)
{
    k_classify_rc<<<nblk(h->n, 256), 256, 0, h->stream>>>(h->g, h->rc, h->cls);
    return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "classify launch");
}

static int coop_launch(dcm_handle *h, const void *fn, int grid, void **args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(DET_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
    if (e != cudaSuccess) return fail_cuda(e, "cooperative launch", __FILE__, __LINE__);
    return DCM_OK;
}

int coop_grid_size(dcm_handle *h, const void *kernel, int block, size_t smem)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    per_sm = per_sm > 2 ? 2 : per_sm;
    return h->num_sms * per_sm;
}

int launch_detect(dcm_handle *h)
{
    h->kernels += h->p.smooth_order > 0 ? 9 : 7;
    cudaStream_t s = h->stream;
    const Geom &g = h->g;
    int n = (int)h->n;
    int64_t nv = h->nvox;
    // Eq. 9
    cudaMemsetAsync(h->B, 0, sizeof(int32_t) * nv, s);
    k_density<<<nblk(n, 256), 256, 0, s>>>(g, h->x, h->B);
    // smoothing
    int order = h->p.smooth_order;
    if (order > 0) {
        SmoothW w;
        w.order = order;
        for (int k = 0; k <= 16; ++k) w.w[k] = 0;
        w.w[0] = 1;
        for (int r = 1; r <= order; ++r)
            for (int k = r; k >= 1; --k) w.w[k] += w.w[k - 1];
        uint64_t pass = 1ull << order;   // sum of the weights
        w.bmax = (uint32_t)((0xffffffffull / (pass * pass)) < 0xffffffffull
                                ? 0xffffffffull / (pass * pass)
                                : 0xffffffffull);
        int vb = nblk(nv, DET_THREADS);
        k_smooth<0, int32_t, uint32_t><<<vb, DET_THREADS, 0, s>>>(h->B, h->sm1, g.gd[0], g.gd[1],
                                                                 g.gd[2], w, h->err);
        k_smooth<1, uint32_t, uint32_t><<<vb, DET_THREADS, 0, s>>>(h->sm1, h->sm2, g.gd[0],
                                                                  g.gd[1], g.gd[2], w, h->err);
        k_smooth<2, uint32_t, double><<<vb, DET_THREADS, 0, s>>>(h->sm2, h->Bs, g.gd[0], g.gd[1],
                                                                g.gd[2], w, h->err);
    } else {
        SmoothW w;
        w.order = 0;
        w.w[0] = 1;
        w.bmax = 0xffffffffu;
        k_smooth<0, int32_t, double><<<nblk(nv, DET_THREADS), DET_THREADS, 0, s>>>(
            h->B, h->Bs, g.gd[0], g.gd[1], g.gd[2], w, h->err);
    }
    // K-means labels
    k_kmeans_init<<<1, 1, 0, s>>>(h->kacc);
    cudaMemsetAsync(h->stats->barrier, 0, 2 * sizeof(unsigned int), s);
    {
        const double *Bs = h->Bs;
        int64_t nvv = nv;
        uint8_t *S = h->S;
        int mi = h->p.kmeans_max_iter > 0 ? h->p.kmeans_max_iter : 100;
        unsigned long long *acc = h->kacc;
        unsigned int *bar = h->stats->barrier;
        int *err = h->err;
        DevStats *st = h->stats;
        void *args[] = {(void *)&Bs, (void *)&nvv, (void *)&S, (void *)&mi,
                        (void *)&acc, (void *)&bar, (void *)&err, (void *)&st};
        int grid = coop_grid_size(h, (const void *)k_kmeans, DET_THREADS, 0);
        int64_t need = (nv + DET_THREADS - 1) / DET_THREADS;
        if (grid > need) grid = (int)(need > 0 ? need : 1);
        int rc = coop_launch(h, (const void *)k_kmeans, grid, args);
        if (rc) return rc;
    }
    // CFSM
    cudaMemsetAsync(h->fcount, 0, 4 * sizeof(int32_t), s);
    k_cfsm_init<<<nblk(nv, DET_THREADS), DET_THREADS, 0, s>>>(g.gd[0], g.gd[1], g.gd[2], h->S,
                                                              h->D0, h->D1, h->stamp, h->flist,
                                                              h->fcount);
    cudaMemsetAsync(h->stats->barrier, 0, 2 * sizeof(unsigned int), s);
    {
        CfsmArgs a;
        a.nx = g.gd[0];
        a.ny = g.gd[1];
        a.nz = g.gd[2];
        a.h0 = g.h[0];
        a.h1 = g.h[1];
        a.h2 = g.h[2];
        a.r_grid = g.r_grid;
        int dmax = g.gd[0] > g.gd[1] ? g.gd[0] : g.gd[1];
        dmax = dmax > g.gd[2] ? dmax : g.gd[2];
        a.iter_max = h->p.cfsm_iter_max > 0 ? h->p.cfsm_iter_max : 4 * dmax;
        a.cap = nv;
        a.S = h->S;
        a.D0 = h->D0;
        a.D1 = h->D1;
        a.stamp = h->stamp;
        a.lists = h->flist;
        a.fcount = h->fcount;
        a.result = (int *)&h->stats->barrier[3];
        a.bar = h->stats->barrier;
        a.err = h->err;
        a.st = h->stats;
        void *args[] = {(void *)&a};
        int grid = coop_grid_size(h, (const void *)k_cfsm, DET_THREADS, 0);
        int rc = coop_launch(h, (const void *)k_cfsm, grid, args);
        if (rc) return rc;
    }
    // Algorithm 3.1 + Eq. 7
    k_cutoff<<<nblk(n, 256), 256, 0, s>>>(g, h->x, h->D0, h->D1, (const int *)&h->stats->barrier[3],
                                          h->d, h->rc, h->cls);
    return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "detect launch");
}

}  // namespace dcm
