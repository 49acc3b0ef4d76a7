// dcm_detect.cu -- interface detection (Section 4, Fig. 14) and the per-
// particle cutoff (Algorithm 3.1, Eq. 7-8).
//
//   density   Eq. 9: B_ijk = particles in voxel (integer atomics)
//   smoothing three periodic 1D passes with binomial weights C(order, k).
//             The values are exact integers; passes 1-2 run in uint32 and
//             pass 3 in uint64 -> FP64, which gives exactly the numbers an
//             FP64 evaluation gives (all < 2^53) at integer-pipe cost.
//   K-means   Eq. 14, K = 2, Lloyd iterations from (max, min) in one
//             cooperative kernel, every system with its own centres and
//             stopping point; sums are exact integers, so the
//             threshold (c_l + c_v)/2 and the labels (Eq. 11-12) are
//             bit-identical to the definition.  Liquid sets of successive
//             iterations are threshold sets, hence nested: equal counts
//             mean an unchanged assignment (the stopping rule).
//   small components (Section 4.2, optional): dcm_components.cu
//   CFSM      Algorithm 4.3 as a Jacobi fixed point over a frontier: each
//             pass recomputes only the voxels whose neighbours changed in
//             the previous pass, writes the other buffer, and stops when
//             nothing changes (an update must lower a value by more than 16
//             ulps, so eps ~ 1e-15 relative) or at iter_max; voxels whose
//             solution exceeds r_grid = r_c,max + h are never updated.  The
//             result is independent of thread scheduling.
//   cutoff    trilinear interpolation from the lower-left-front voxel
//             centre (Algorithm 3.1), then Eq. 7-8 and the class.
// Bound: HBM/L2 (the grid holds ~3.7 voxels per particle at 1 sigma voxels).
#include <cooperative_groups.h>

#include <type_traits>

#include "dcm_device.cuh"

namespace dcm {

constexpr int DET_THREADS = 256;
constexpr int CFSM_THREADS = 512;           // the grid-wide passes: one block per SM, of
                                            // 256 threads for one system, 512 for several
constexpr int CFSM_TAIL_CTAS = 8;           // one portable cluster
constexpr int CFSM_TAIL_THREADS = 512;

__global__ void k_density(Batch b, const double *__restrict__ x, int32_t *B)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.N) return;
    const Geom &g = b.sys[sys_p(b, i)];
    int gx = bin_of(x[i], g.inv_h[0], g.gd[0]);
    int gy = bin_of(x[(size_t)b.N + i], g.inv_h[1], g.gd[1]);
    int gz = bin_of(x[2 * (size_t)b.N + i], g.inv_h[2], g.gd[2]);
    atomicAdd(&B[g.v0 + gx + g.gd[0] * (gy + (int64_t)g.gd[1] * gz)], 1);
}

struct SmoothW {
    uint32_t w[17];
    int order;
    uint32_t bmax;      // largest voxel count for which pass 2 cannot overflow
};

// one periodic 1D pass along AXIS (0 = x, 1 = y, 2 = z) of every system
template <int AXIS, typename TIN, typename TOUT>
__global__ void k_smooth(Batch b, const TIN *__restrict__ in, TOUT *out, SmoothW w, int *err)
{
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= b.NV) return;
    const Geom &g = b.sys[sys_v(b, v)];
    const int nx = g.gd[0], ny = g.gd[1], nz = g.gd[2];
    const int lv = (int)(v - g.v0);              // 32-bit index math
    const int x = lv % nx, yz = lv / nx;
    const int y = yz % ny, z = yz / ny;
    const int n = AXIS == 0 ? nx : (AXIS == 1 ? ny : nz);
    const int c = AXIS == 0 ? x : (AXIS == 1 ? y : z);
    const int stride = AXIS == 0 ? 1 : (AXIS == 1 ? nx : nx * ny);
    const TIN *line = in + (v - (int64_t)c * stride);
    const int half = w.order / 2;
    if constexpr (AXIS == 0) {
        if ((uint32_t)in[v] > w.bmax) atomicOr(err, DEV_ERR_DENSITY);
    }
    // periodic tap index: one conditional wrap while the kernel fits in the
    // line, a full modulo only for lines shorter than the kernel
    auto tap = [&](int k) {
        int q = c + k - half;
        if (n > w.order) {
            q += q < 0 ? n : 0;
            q -= q >= n ? n : 0;
        } else {
            q = ((q % n) + n) % n;
        }
        return line[q * stride];
    };
    if constexpr (sizeof(TOUT) == 8) {
        unsigned long long s = 0;
        for (int k = 0; k <= w.order; ++k) s += (unsigned long long)w.w[k] * (unsigned long long)tap(k);
        out[v] = (TOUT)s;
    } else {
        uint32_t s = 0;
        for (int k = 0; k <= w.order; ++k) s += w.w[k] * (uint32_t)tap(k);
        out[v] = (TOUT)s;
    }
}

// the default order 8 (weights C(8,k)) with the taps unrolled at compile
// time: interior voxels index their line directly, only the 8 voxels nearest
// the periodic seam wrap
template <int AXIS, typename TIN, typename TOUT>
__global__ void __launch_bounds__(256) k_smooth8(Batch b, const TIN *__restrict__ in, TOUT *out,
                                                 uint32_t bmax, int *err)
{
    constexpr uint32_t W[9] = {1, 8, 28, 56, 70, 56, 28, 8, 1};
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= b.NV) return;
    const Geom &g = b.sys[sys_v(b, v)];
    const int nx = g.gd[0], ny = g.gd[1], nz = g.gd[2];
    const int lv = (int)(v - g.v0);
    int c, n, stride;
    // exact divisions by nx, ny (Geom::div_gd)
    const int yz = (int)__umul64hi((unsigned)lv, g.div_gd[0]);
    if constexpr (AXIS == 0) {
        c = lv - yz * nx;
        n = nx;
        stride = 1;
    } else if constexpr (AXIS == 1) {
        c = yz - (int)__umul64hi((unsigned)yz, g.div_gd[1]) * ny;
        n = ny;
        stride = nx;
    } else {
        c = (int)__umul64hi((unsigned)yz, g.div_gd[1]);
        n = nz;
        stride = nx * ny;
    }
    const TIN *line = in + (v - (int64_t)c * stride);
    if constexpr (AXIS == 0) {
        if ((uint32_t)in[v] > bmax) atomicOr(err, DEV_ERR_DENSITY);
    }
    using ACC = typename std::conditional<sizeof(TOUT) == 8, unsigned long long, uint32_t>::type;
    ACC sum = 0;
    if (c >= 4 && c + 4 < n) {
        const TIN *p = line + (int64_t)(c - 4) * stride;
#pragma unroll
        for (int k = 0; k < 9; ++k) sum += (ACC)W[k] * (ACC)(uint32_t)p[(int64_t)k * stride];
    } else if (n > 8) {
        // near the seam: one conditional wrap (the kernel fits in the line)
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            int q = c + k - 4;
            q += q < 0 ? n : 0;
            q -= q >= n ? n : 0;
            sum += (ACC)W[k] * (ACC)(uint32_t)line[(int64_t)q * stride];
        }
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            int q = c + k - 4;
            q = ((q % n) + n) % n;
            sum += (ACC)W[k] * (ACC)(uint32_t)line[(int64_t)q * stride];
        }
    }
    out[v] = (TOUT)sum;
}

// ---- K-means (Eq. 14, K = 2), all systems in one cooperative kernel ------------
// global accumulators per system s, each spread over SPREAD slots (a block
// adds into slot blockIdx % SPREAD, readers sum the slots) so that hundreds
// of blocks do not serialise on one address: [max | min | total] then three
// rotating (count | sum) pairs
constexpr int SPREAD = 16;
constexpr int KACC = 9 * SPREAD;

// the detection's initial state in one launch: the density grid (Eq. 9
// accumulates into it), the CFSM stamps, the K-means accumulators, the
// grid-barrier words and the CFSM frontier counters
__global__ void k_detect_init(int64_t nv, int32_t *B, int32_t *stamp, int M,
                              unsigned long long *acc, unsigned int *bar, int32_t *fcount)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = t; v < nv; v += nth) {
        B[v] = 0;
        stamp[v] = -1;                           // no CFSM pass has claimed the voxel
    }
    for (int64_t q = t; q < (int64_t)M * KACC; q += nth) {
        int w = (int)(q % KACC) / SPREAD;
        acc[q] = w == 1 ? ~0ull : 0ull;
    }
    if (t < 2) bar[t] = 0u;
    if (t < 4) fcount[t] = 0;
}

__device__ __forceinline__ unsigned long long spread_sum(const unsigned long long *p)
{
    unsigned long long t = 0;
#pragma unroll
    for (int q = 0; q < SPREAD; ++q) t += __ldcg(&p[q]);
    return t;
}

struct KmeansArgs {
    Batch b;
    const double *Bs;
    uint8_t *S;
    int max_iter;
    unsigned long long *acc;
    unsigned long long *part;     // per-block partials (single-system kernel)
    unsigned int *bar;
    int *err;
    DevStats *st;
};

// warp-level reduction of a per-lane value when every lane holds the same
// system (the common case); otherwise each lane adds its own value
template <int OP>
__device__ __forceinline__ void warp_flush(int cur, unsigned long long v, unsigned long long *slot)
{
    const unsigned full = 0xffffffffu;
    int c0 = __shfl_sync(full, cur, 0);
    if (__all_sync(full, cur == c0)) {
        for (int off = 16; off > 0; off >>= 1) {
            unsigned long long o = __shfl_xor_sync(full, v, off);
            v = OP == 0 ? v + o : (OP == 1 ? (o > v ? o : v) : (o < v ? o : v));
        }
        if ((threadIdx.x & 31) == 0 && cur >= 0) {
            if (OP == 0) atomicAdd(&slot[c0], v);
            else if (OP == 1) atomicMax(&slot[c0], v);
            else atomicMin(&slot[c0], v);
        }
    } else if (cur >= 0) {
        if (OP == 0) atomicAdd(&slot[cur], v);
        else if (OP == 1) atomicMax(&slot[cur], v);
        else atomicMin(&slot[cur], v);
    }
}

// The smoothed densities are exact integers below 2^53 held as doubles.  The
// voxel loops never touch the FP64 pipe (one FP64 warp instruction costs
// dozens of issue slots here): a non-negative double compares like its bit
// pattern, and its integer value comes from the bits by a shift.
__device__ __forceinline__ unsigned long long exact_u64(double d)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(d);
    if (b == 0ull) return 0ull;
    int e = (int)(b >> 52) - 1023;                       // 0 <= e <= 52
    unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    return m >> (52 - e);
}

// The systems met by the voxel range [lo, hi): calls fn(s, a0, a1) for each
// segment [a0, a1) of system s, in order (every thread of the block calls
// it; the segments are the same for all of them)
template <typename F>
__device__ __forceinline__ void for_segments(const Batch &b, int64_t lo, int64_t hi, F &&fn)
{
    if (lo >= hi) return;
    for (int s = b.M == 1 ? 0 : sys_of(b.v_off, b.M, lo); s < b.M; ++s) {
        const int64_t a0 = lo > b.v_off[s] ? lo : b.v_off[s];
        const int64_t a1 = hi < b.v_off[s + 1] ? hi : b.v_off[s + 1];
        if (a0 >= hi) break;
        if (a0 < a1) fn(s, a0, a1);
    }
}

constexpr int KM_U = 4;      // voxel loads in flight per thread in the K-means passes
constexpr int KM_THREADS = 512;   // the multi-system K-means: one block of 512 per SM

// per-block shared state: centres, previous liquid count, threshold and the
// done flag of every system (every block derives the same values from the
// same global sums, so no broadcast is needed)
__global__ void __launch_bounds__(KM_THREADS) k_kmeans(KmeansArgs a)
{
    extern __shared__ unsigned char smem[];
    const int M = a.b.M;
    double *s_cl = (double *)smem;
    double *s_cv = s_cl + M;
    double *s_thr = s_cv + M;
    long long *s_prev = (long long *)(s_thr + M);
    unsigned long long *s_c0 = (unsigned long long *)(s_prev + M);   // block partials
    unsigned long long *s_c1 = s_c0 + M;
    unsigned long long *s_c2 = s_c1 + M;
    int *s_done = (int *)(s_c2 + M);
    __shared__ int s_left;
    const int64_t NV = a.b.NV;
    int64_t chunk = (NV + gridDim.x - 1) / gridDim.x;
    int64_t lo = (int64_t)blockIdx.x * chunk, hi = lo + chunk < NV ? lo + chunk : NV;

    // phase A: extremes and totals (exact integers), segment by segment of
    // the block's range, KM_U independent loads in flight per thread
    for (int s = threadIdx.x; s < M; s += blockDim.x) {
        s_c0[s] = 0ull;
        s_c1[s] = ~0ull;
        s_c2[s] = 0ull;
    }
    __syncthreads();
    for_segments(a.b, lo, hi, [&](int sg, int64_t a0, int64_t a1) {
        unsigned long long mx = 0, mn = ~0ull, tot = 0;
        for (int64_t v = a0 + threadIdx.x; v < a1; v += (int64_t)KM_U * blockDim.x) {
            double d[KM_U];
#pragma unroll
            for (int q = 0; q < KM_U; ++q) {
                const int64_t w = v + (int64_t)q * blockDim.x;
                d[q] = w < a1 ? __ldg(&a.Bs[w]) : -1.0;
            }
#pragma unroll
            for (int q = 0; q < KM_U; ++q) {
                if (__double_as_longlong(d[q]) < 0) continue;   // (past the segment)
                const unsigned long long bv = exact_u64(d[q]);
                mx = bv > mx ? bv : mx;
                mn = bv < mn ? bv : mn;
                tot += bv;
            }
        }
        warp_flush<1>(sg, mx, s_c0);
        warp_flush<2>(sg, mn, s_c1);
        warp_flush<0>(sg, tot, s_c2);
    });
    __syncthreads();
    const int slot = blockIdx.x % SPREAD;
    for (int s = threadIdx.x; s < M; s += blockDim.x) {
        if (s_c1[s] == ~0ull) continue;   // no voxel of s in this block
        unsigned long long *g = a.acc + (int64_t)KACC * s;
        atomicMax(&g[0 * SPREAD + slot], s_c0[s]);
        atomicMin(&g[1 * SPREAD + slot], s_c1[s]);
        atomicAdd(&g[2 * SPREAD + slot], s_c2[s]);
    }
    if (!grid_barrier(a.bar, a.err)) return;
    // values other blocks produced are read through L2 (ld.global.cg): the
    // per-SM L1 caches are not coherent across a grid barrier
    for (int s = threadIdx.x; s < M; s += blockDim.x) {
        const unsigned long long *g = a.acc + (int64_t)KACC * s;
        unsigned long long mx = 0, mn = ~0ull;
        for (int q = 0; q < SPREAD; ++q) {
            unsigned long long u = __ldcg(&g[q]), l = __ldcg(&g[SPREAD + q]);
            mx = u > mx ? u : mx;
            mn = l < mn ? l : mn;
        }
        s_cl[s] = (double)mx;
        s_cv[s] = (double)mn;
        s_prev[s] = -1;
        s_done[s] = 0;
        s_thr[s] = DMUL(DADD(s_cl[s], s_cv[s]), 0.5);
    }
    __syncthreads();
    int it = 0;
    while (it < a.max_iter) {
        for (int s = threadIdx.x; s < M; s += blockDim.x) {
            s_c0[s] = 0ull;
            s_c1[s] = 0ull;
        }
        __syncthreads();
        for_segments(a.b, lo, hi, [&](int sg, int64_t a0, int64_t a1) {
            if (s_done[sg]) return;
            const long long thr = __double_as_longlong(s_thr[sg]);
            unsigned long long cnt = 0, sum = 0;
            for (int64_t v = a0 + threadIdx.x; v < a1; v += (int64_t)KM_U * blockDim.x) {
                double d[KM_U];
#pragma unroll
                for (int q = 0; q < KM_U; ++q) {
                    const int64_t w = v + (int64_t)q * blockDim.x;
                    d[q] = w < a1 ? __ldg(&a.Bs[w]) : -1.0;
                }
#pragma unroll
                for (int q = 0; q < KM_U; ++q) {
                    if (__double_as_longlong(d[q]) >= thr) {   // (-1.0: negative bits, never)
                        cnt++;
                        sum += exact_u64(d[q]);
                    }
                }
            }
            warp_flush<0>(sg, cnt, s_c0);
            warp_flush<0>(sg, sum, s_c1);
        });
        __syncthreads();
        for (int s = threadIdx.x; s < M; s += blockDim.x) {
            unsigned long long *g = a.acc + (int64_t)KACC * s + (3 + 2 * (it % 3)) * SPREAD;
            if (s_c0[s]) {
                atomicAdd(&g[slot], s_c0[s]);
                atomicAdd(&g[SPREAD + slot], s_c1[s]);
            }
            if (blockIdx.x == 0) {   // clear the pair of the next pass
                unsigned long long *nx = a.acc + (int64_t)KACC * s + (3 + 2 * ((it + 1) % 3)) * SPREAD;
                for (int q = 0; q < 2 * SPREAD; ++q) nx[q] = 0ull;
            }
        }
        if (!grid_barrier(a.bar, a.err)) return;
        ++it;
        if (threadIdx.x == 0) s_left = 0;
        __syncthreads();
        for (int s = threadIdx.x; s < M; s += blockDim.x) {
            if (s_done[s]) continue;
            const unsigned long long *g = a.acc + (int64_t)KACC * s + (3 + 2 * ((it - 1) % 3)) * SPREAD;
            long long nl = (long long)spread_sum(g);
            unsigned long long sl = spread_sum(g + SPREAD);
            if (nl == s_prev[s]) {   // same threshold set as the previous pass
                s_done[s] = 1;
                continue;
            }
            const Geom &geo = a.b.sys[s];
            long long nvap = geo.nvox - nl;
            unsigned long long total = spread_sum(a.acc + (int64_t)KACC * s + 2 * SPREAD);
            if (nl > 0) s_cl[s] = (double)sl / (double)nl;
            if (nvap > 0) s_cv[s] = (double)(total - sl) / (double)nvap;
            s_prev[s] = nl;
            s_thr[s] = DMUL(DADD(s_cl[s], s_cv[s]), 0.5);
            atomicAdd(&s_left, 1);
        }
        __syncthreads();
        if (s_left == 0) break;
    }
    for_segments(a.b, lo, hi, [&](int sg, int64_t a0, int64_t a1) {
        const long long thr = __double_as_longlong(s_thr[sg]);
        for (int64_t v = a0 + threadIdx.x; v < a1; v += blockDim.x)
            a.S[v] = __double_as_longlong(__ldg(&a.Bs[v])) >= thr ? 0 : 1;
    });
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.st->kmeans_iters = it;
        a.st->c_liquid = s_cl[0];
        a.st->c_vapor = s_cv[0];
    }
}

// The same K-means for one system, with each thread's voxels held in
// registers across the passes: the values never change during the
// iteration, so a pass is a compare-and-add over registers, a block
// reduction and the grid barrier (the multi-system kernel above re-reads the
// field every pass).  A voxel is liquid when its value reaches the
// threshold; for the exact integers held here that is u >= ceil(thr), the
// same decision as the double comparison.
constexpr int KM1_THREADS = 1024;
constexpr int KM1_CACHE = 8;

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// per-block partials of the single-system K-means: [0, 4G) the extremes and
// total of phase A (max, min, total, -), then two parities of (count, sum)
// per block for the Lloyd passes (G <= KM1_MAX_BLOCKS blocks)
constexpr int KM1_MAX_BLOCKS = 1024;
constexpr int KM1_PART = 8 * KM1_MAX_BLOCKS;

__global__ void __launch_bounds__(KM1_THREADS) k_kmeans1(KmeansArgs a)
{
    constexpr int NW = KM1_THREADS / 32;
    __shared__ unsigned long long s_w[3][NW];
    __shared__ double s_cl, s_cv, s_thr;
    __shared__ unsigned long long s_thru, s_total;
    __shared__ long long s_prev;
    __shared__ int s_done, s_ok;
    const int64_t NV = a.b.NV;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int G = gridDim.x;
    unsigned long long *partA = a.part, *partL = a.part + 4 * KM1_MAX_BLOCKS;
    unsigned long long u[KM1_CACHE];
    // phase A: extremes and total (exact integers); the first KM1_CACHE
    // voxels of the thread stay in registers
    unsigned long long mx = 0, mn = ~0ull, tot = 0;
#pragma unroll
    for (int c = 0; c < KM1_CACHE; ++c) {
        const int64_t v = t + (int64_t)c * nth;
        u[c] = v < NV ? exact_u64(a.Bs[v]) : ~0ull;     // ~0: no voxel
        if (v < NV) {
            mx = u[c] > mx ? u[c] : mx;
            mn = u[c] < mn ? u[c] : mn;
            tot += u[c];
        }
    }
    for (int64_t v = t + (int64_t)KM1_CACHE * nth; v < NV; v += nth) {
        const unsigned long long x = exact_u64(a.Bs[v]);
        mx = x > mx ? x : mx;
        mn = x < mn ? x : mn;
        tot += x;
    }
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, off);
        mx = o > mx ? o : mx;
        o = __shfl_xor_sync(0xffffffffu, mn, off);
        mn = o < mn ? o : mn;
    }
    tot = warp_sum_u64(tot);
    if (lane == 0) {
        s_w[0][w] = mx;
        s_w[1][w] = mn;
        s_w[2][w] = tot;
    }
    __syncthreads();
    // one warp: the block's partial out, the grid barrier, every block's
    // partial back in (plain stores ordered by the barrier's release, reads
    // through L2), the centres of the first pass
    if (w == 0) {
        mx = lane < NW ? s_w[0][lane] : 0ull;
        mn = lane < NW ? s_w[1][lane] : ~0ull;
        tot = lane < NW ? s_w[2][lane] : 0ull;
        for (int off = 16; off > 0; off >>= 1) {
            unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, off);
            mx = o > mx ? o : mx;
            o = __shfl_xor_sync(0xffffffffu, mn, off);
            mn = o < mn ? o : mn;
        }
        tot = warp_sum_u64(tot);
        int ok = 1;
        if (lane == 0) {
            partA[4 * blockIdx.x] = mx;
            partA[4 * blockIdx.x + 1] = mn;
            partA[4 * blockIdx.x + 2] = tot;
            ok = grid_arrive_wait(a.bar, a.err) ? 1 : 0;
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        __syncwarp();
        if (ok) {
            mx = 0ull;
            mn = ~0ull;
            tot = 0ull;
            for (int q = lane; q < G; q += 32) {
                const unsigned long long x = __ldcg(&partA[4 * q]), y = __ldcg(&partA[4 * q + 1]);
                mx = x > mx ? x : mx;
                mn = y < mn ? y : mn;
                tot += __ldcg(&partA[4 * q + 2]);
            }
            for (int off = 16; off > 0; off >>= 1) {
                unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, off);
                mx = o > mx ? o : mx;
                o = __shfl_xor_sync(0xffffffffu, mn, off);
                mn = o < mn ? o : mn;
            }
            tot = warp_sum_u64(tot);
            if (lane == 0) {
                s_cl = (double)mx;
                s_cv = (double)mn;
                s_total = tot;
                s_prev = -1;
                s_done = 0;
                s_thr = DMUL(DADD(s_cl, s_cv), 0.5);
                s_thru = (unsigned long long)ceil(s_thr);
            }
        }
        if (lane == 0) s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
    int it = 0;
    while (it < a.max_iter) {
        const unsigned long long thr = s_thru;
        unsigned long long cnt = 0, sum = 0;
#pragma unroll
        for (int c = 0; c < KM1_CACHE; ++c) {
            const bool in = u[c] != ~0ull && u[c] >= thr;
            cnt += in ? 1ull : 0ull;
            sum += in ? u[c] : 0ull;
        }
        for (int64_t v = t + (int64_t)KM1_CACHE * nth; v < NV; v += nth) {
            const unsigned long long x = exact_u64(a.Bs[v]);
            cnt += x >= thr ? 1ull : 0ull;
            sum += x >= thr ? x : 0ull;
        }
        cnt = warp_sum_u64(cnt);
        sum = warp_sum_u64(sum);
        if (lane == 0) {
            s_w[0][w] = cnt;
            s_w[1][w] = sum;
        }
        __syncthreads();
        if (w == 0) {
            unsigned long long *P = partL + (it & 1) * 2 * KM1_MAX_BLOCKS;
            cnt = lane < NW ? s_w[0][lane] : 0ull;
            sum = lane < NW ? s_w[1][lane] : 0ull;
            cnt = warp_sum_u64(cnt);
            sum = warp_sum_u64(sum);
            int ok = 1;
            if (lane == 0) {
                P[2 * blockIdx.x] = cnt;
                P[2 * blockIdx.x + 1] = sum;
                ok = grid_arrive_wait(a.bar, a.err) ? 1 : 0;
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            __syncwarp();
            if (ok) {
                cnt = 0ull;
                sum = 0ull;
                for (int q = lane; q < G; q += 32) {
                    cnt += __ldcg(&P[2 * q]);
                    sum += __ldcg(&P[2 * q + 1]);
                }
                cnt = warp_sum_u64(cnt);
                sum = warp_sum_u64(sum);
                if (lane == 0) {
                    const long long nl = (long long)cnt;
                    if (nl == s_prev) {      // same threshold set as the previous pass
                        s_done = 1;
                    } else {
                        const long long nvap = NV - nl;
                        if (nl > 0) s_cl = (double)sum / (double)nl;
                        if (nvap > 0) s_cv = (double)(s_total - sum) / (double)nvap;
                        s_prev = nl;
                        s_thr = DMUL(DADD(s_cl, s_cv), 0.5);
                        s_thru = (unsigned long long)ceil(s_thr);
                    }
                }
            }
            if (lane == 0) s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return;
        ++it;
        if (s_done) break;
    }
    const unsigned long long thr = s_thru;
#pragma unroll
    for (int c = 0; c < KM1_CACHE; ++c) {
        const int64_t v = t + (int64_t)c * nth;
        if (v < NV) a.S[v] = u[c] >= thr ? 0 : 1;
    }
    for (int64_t v = t + (int64_t)KM1_CACHE * nth; v < NV; v += nth)
        a.S[v] = exact_u64(a.Bs[v]) >= thr ? 0 : 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.st->kmeans_iters = it;
        a.st->c_liquid = s_cl;
        a.st->c_vapor = s_cv;
    }
}

// ---- CFSM (Algorithm 4.3) ------------------------------------------------------
__device__ __forceinline__ int64_t vox(int x, int y, int z, int nx, int ny)
{
    return x + (int64_t)nx * (y + (int64_t)ny * z);
}

// one voxel's Jacobi update (Algorithm 4.3): the Godunov solve from its face
// neighbours' values a{x,y,z} (Eq. 16-19); true when it lowers the voxel's
// value within the band r_grid.  Any solution is at least min(a) +
// 1/sqrt(sum w): when that cannot beat the current value the solve is
// skipped (a lower bound with a relative margin, so no update is lost).
__device__ __forceinline__ bool cfsm_solve(const Geom &g, double old, double ax, double ay,
                                           double az, double &dbar)
{
    double amin = dmin_nonneg(ax, dmin_nonneg(ay, az));
    dbar = old;
    if (isinf(amin) ||
        __double_as_longlong(old) <= __double_as_longlong(amin + 0.999999 * g.e_min))
        return false;
    dbar = godunov_w(ax, ay, az, g.h[0], g.h[1], g.h[2], g.w_h[0], g.w_h[1], g.w_h[2]);
    // non-negative doubles: compare the bit patterns.  An update must lower
    // the value by more than 16 units in the last place: the root of the
    // local solve carries ~1e-14 relative error, and without the margin two
    // neighbours can trade last-bit decreases for many passes (the values
    // stay within ~1e-13 of the exact fixed point)
    return __double_as_longlong(dbar) + 16 < __double_as_longlong(old) &&
           __double_as_longlong(dbar) <= __double_as_longlong(g.r_grid);
}

// a changed voxel v: itself (so the other buffer catches up next pass) and
// its liquid face neighbours go to pass k+1's frontier, each once (stamp
// k+1; the seven exchanges are independent of each other); returns how many
// this thread claimed into push
__device__ __forceinline__ int cfsm_claim(int v, const int nb[6], const bool liq[7], int k,
                                          int32_t *stamp, int32_t push[7])
{
    const int cand[7] = {v, nb[0], nb[1], nb[2], nb[3], nb[4], nb[5]};
    int prev[7];
#pragma unroll
    for (int e = 0; e < 7; ++e) prev[e] = liq[e] ? atomicExch(&stamp[cand[e]], k + 1) : k + 1;
    int n = 0;
#pragma unroll
    for (int e = 0; e < 7; ++e)
        if (prev[e] != k + 1) push[n++] = cand[e];
    return n;
}

// the lanes' claims appended to the next frontier, one atomic per warp
// (every lane of the warp calls it)
__device__ __forceinline__ void cfsm_append(const int32_t push[7], int npush, int32_t *count,
                                            int32_t *Fn, int lane)
{
    int incl = npush;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total) {
        int base = 0;
        if (lane == 31) base = atomicAdd(count, total);
        base = __shfl_sync(0xffffffffu, base, 31) + incl - npush;
        for (int e = 0; e < npush; ++e) Fn[base + e] = push[e];
    }
}

// the initial values, D = 0 on vapor and +inf on liquid (buffer D0), and the
// first pass of the iteration done in place: it reads only those values, so
// the liquid voxels with a vapor face neighbour (the "interfacial boxes")
// solve here (into D1) and claim the next frontier (list 1) as any pass
// would.  The stamps are -1 (k_detect_init).
__global__ void k_cfsm_init(Batch b, const uint8_t *__restrict__ S, double *D0, double *D1,
                            int32_t *stamp, int32_t *list1, int32_t *fcount, unsigned int *bar)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = (int)(threadIdx.x & 31);
    if (v < 2) bar[v] = 0u;                  // the K-means kernel is done with them
    int32_t push[7];
    int npush = 0;
    if (v < b.NV) {
        const double inf = __longlong_as_double(0x7ff0000000000000ll);
        const bool vap = S[v] == 1;
        const double d0 = vap ? 0.0 : inf;
        D0[v] = d0;
        double d1 = d0;
        if (!vap) {
            const Geom &g = b.sys[sys_v(b, v)];
            const int nx = g.gd[0], ny = g.gd[1], nz = g.gd[2];
            const int v0 = (int)g.v0;
            int lv = (int)(v - v0);
            // exact divisions by nx, ny (Geom::div_gd)
            int yz = (int)__umul64hi((unsigned)lv, g.div_gd[0]);
            int z = (int)__umul64hi((unsigned)yz, g.div_gd[1]);
            int x = lv - yz * nx, y = yz - z * ny;
            int xm = x ? x - 1 : nx - 1, xp = x + 1 < nx ? x + 1 : 0;
            int ym = y ? y - 1 : ny - 1, yp = y + 1 < ny ? y + 1 : 0;
            int zm = z ? z - 1 : nz - 1, zp = z + 1 < nz ? z + 1 : 0;
            const int nb[6] = {v0 + xm + nx * yz, v0 + xp + nx * yz,
                               v0 + x + nx * (ym + ny * z), v0 + x + nx * (yp + ny * z),
                               v0 + x + nx * (y + ny * zm), v0 + x + nx * (y + ny * zp)};
            bool liq[7];
            liq[0] = true;
#pragma unroll
            for (int e = 1; e < 7; ++e) liq[e] = S[nb[e - 1]] == 0;
            if (!(liq[1] && liq[2] && liq[3] && liq[4] && liq[5] && liq[6])) {
                // pass 0 on an interfacial box: the face values are 0 (vapor)
                // or +inf (liquid), as in D0
                const double ax = dmin_nonneg(liq[1] ? inf : 0.0, liq[2] ? inf : 0.0);
                const double ay = dmin_nonneg(liq[3] ? inf : 0.0, liq[4] ? inf : 0.0);
                const double az = dmin_nonneg(liq[5] ? inf : 0.0, liq[6] ? inf : 0.0);
                double dbar;
                if (cfsm_solve(g, d0, ax, ay, az, dbar)) {
                    d1 = dbar;
                    npush = cfsm_claim((int)v, nb, liq, 0, stamp, push);
                }
            }
        }
        D1[v] = d1;
    }
    cfsm_append(push, npush, &fcount[1], list1, lane);
}

struct CfsmArgs {
    Batch b;
    int iter_max;
    int64_t cap;              // capacity of one frontier list
    const uint8_t *S;
    double *D0, *D1;
    int32_t *stamp;
    int32_t *lists;           // 4 * cap
    int32_t *fcount;          // 4 counters
    int *result;              // which buffer holds the result
    int *kpass;               // first pass of the tail kernel
    int nf_switch;            // frontier size below which the tail kernel runs
    unsigned int *bar;
    int *err;
    DevStats *st;
};

// one pass k of the frontier iteration: items q = pos, pos + nth, ... of
// frontier list k & 3 (nf items), pushes into list (k + 1) & 3.  With pos =
// threadIdx.x * blocks + block consecutive items go to different blocks, so
// a small frontier spreads over every SM (its FP64 solves would otherwise
// crowd the SMs of the first few blocks)
// the list entry this thread takes first in pass k, loaded before the
// frontier size is known (the two reads overlap; beyond the size it is unused)
__device__ __forceinline__ int32_t cfsm_first(const CfsmArgs &a, int k, int64_t pos)
{
    return pos < a.cap ? __ldcg(&a.lists[(int64_t)(k & 3) * a.cap + pos]) : 0;
}

__device__ __forceinline__ void cfsm_pass(const CfsmArgs &a, int k, int nf, int64_t pos, int64_t nth,
                                          int32_t first)
{
    const double *X = (k & 1) ? a.D1 : a.D0;
    double *Y = (k & 1) ? a.D0 : a.D1;
    int32_t *F = a.lists + (int64_t)(k & 3) * a.cap;
    int32_t *Fn = a.lists + (int64_t)((k + 1) & 3) * a.cap;
    if (pos == 0) a.fcount[(k + 2) & 3] = 0;   // list two passes ahead
    const int lane = (int)(threadIdx.x & 31);
    for (int64_t q0 = 0; __any_sync(0xffffffffu, q0 + pos < nf); q0 += nth) {
        const int64_t q = q0 + pos;
        int32_t push[7];
        int npush = 0;
        if (q < nf) {
            int v = q0 == 0 ? first : __ldcg(&F[q]);
            const Geom &g = a.b.sys[sys_v(a.b, v)];
            const int nx = g.gd[0], ny = g.gd[1], nz = g.gd[2];
            const int v0 = (int)g.v0;
            int lv = v - v0;                         // 32-bit index math
            int yz = (int)__umul64hi((unsigned)lv, g.div_gd[0]);     // lv / nx
            int z = (int)__umul64hi((unsigned)yz, g.div_gd[1]);      // yz / ny
            int x = lv - yz * nx, y = yz - z * ny;
            int xm = x ? x - 1 : nx - 1, xp = x + 1 < nx ? x + 1 : 0;
            int ym = y ? y - 1 : ny - 1, yp = y + 1 < ny ? y + 1 : 0;
            int zm = z ? z - 1 : nz - 1, zp = z + 1 < nz ? z + 1 : 0;
            int nb[6] = {v0 + xm + nx * yz, v0 + xp + nx * yz,
                         v0 + x + nx * (ym + ny * z), v0 + x + nx * (yp + ny * z),
                         v0 + x + nx * (y + ny * zm), v0 + x + nx * (y + ny * zp)};
            // D and the lists were written by other blocks in the previous
            // pass: read them through L2 (ld.global.cg), not a stale L1
            double old = __ldcg(&X[v]);
            double ax = dmin_nonneg(__ldcg(&X[nb[0]]), __ldcg(&X[nb[1]]));
            double ay = dmin_nonneg(__ldcg(&X[nb[2]]), __ldcg(&X[nb[3]]));
            double az = dmin_nonneg(__ldcg(&X[nb[4]]), __ldcg(&X[nb[5]]));
            // the labels of the face neighbours, loaded with the distances
            // (read-only in this kernel) so the push below waits on nothing
            bool liq[7];
            liq[0] = true;
#pragma unroll
            for (int e = 1; e < 7; ++e) liq[e] = __ldg(&a.S[nb[e - 1]]) == 0;
            double dbar;
            const bool changed = cfsm_solve(g, old, ax, ay, az, dbar);
            Y[v] = changed ? dbar : old;
            if (changed) npush = cfsm_claim(v, nb, liq, k, a.stamp, push);
        }
        cfsm_append(push, npush, &a.fcount[(k + 1) & 3], Fn, lane);
    }
}

// the passes over large frontiers, all SMs, a grid barrier between passes;
// once the frontier falls below nf_switch the tail kernel takes over (its
// passes are short latency chains that a grid barrier would dominate)
__global__ void __launch_bounds__(CFSM_THREADS) k_cfsm(CfsmArgs a)
{
    // items of a frontier smaller than the grid go round-robin over the
    // blocks (pos_c); a larger one in contiguous runs per block (pos_l),
    // whose list reads coalesce and whose neighbours share L1.  Both first
    // entries are loaded before the frontier size is known.
    const int64_t pos_c = (int64_t)threadIdx.x * gridDim.x + blockIdx.x;
    const int64_t pos_l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    int k = 1;                                   // pass 0 ran in k_cfsm_init
    for (; k < a.iter_max; ++k) {
        const int32_t first_c = cfsm_first(a, k, pos_c), first_l = cfsm_first(a, k, pos_l);
        const int nf = ((volatile int32_t *)a.fcount)[k & 3];
        if (nf < a.nf_switch) break;             // (also nf == 0: converged)
        const bool rr = nf <= nth;
        cfsm_pass(a, k, nf, rr ? pos_c : pos_l, nth, rr ? first_c : first_l);
        if (!grid_barrier(a.bar, a.err)) return;
    }
    if (pos_l == 0) *a.kpass = k;
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// the remaining passes in one thread-block cluster: the hardware cluster
// barrier replaces the grid barrier; ends the iteration (result, statistics,
// the not-converged flag)
__global__ void __launch_bounds__(CFSM_TAIL_THREADS) k_cfsm_tail(CfsmArgs a)
{
    const int64_t pos = (int64_t)threadIdx.x * CFSM_TAIL_CTAS + cluster_rank();
    const int64_t nth = (int64_t)CFSM_TAIL_CTAS * blockDim.x;
    int k = __ldcg(a.kpass);
    bool converged = false;
    for (; k < a.iter_max; ++k) {
        const int32_t first = cfsm_first(a, k, pos);
        const int nf = ((volatile int32_t *)a.fcount)[k & 3];
        if (nf == 0) {
            converged = true;
            break;
        }
        cfsm_pass(a, k, nf, pos, nth, first);
        cluster_sync_all();
    }
    if (pos == 0) {
        // after pass k-1 the current values are in the buffer it wrote
        *a.result = (k & 1) ? 1 : 0;
        a.st->cfsm_iters = k;
        if (!converged) atomicOr(a.err, DEV_ERR_CFSM_CAP);
    }
}

// ---- Algorithm 3.1 + Eq. 7-8 ----------------------------------------------------
// Algorithm 3.1 (trilinear lookup of the distance grid) and Eq. 7 for
// particle i.  rq given (warp Verlet-list kernels): the new cutoff's force
// constants go straight to the particle's sorted slot inv[i].  With a reuse
// test, the particle's headroom term for the new cutoff.
__device__ __forceinline__ void cutoff_one(Batch b, int64_t i, const double *__restrict__ x,
                                           const double *__restrict__ D0,
                                           const double *__restrict__ D1,
                                           const int *__restrict__ result, double *d, double *rc,
                                           uint8_t *cls, float4 *rq, const int32_t *__restrict__ inv,
                                           const ListTest &lt, float &mq)
{
    const Geom &g = b.sys[sys_p(b, i)];
    const double *D = (*result ? D1 : D0) + g.v0;
    int i0[3], i1[3];
    double t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double gg = DSUB(DMUL(x[(size_t)a * b.N + i], g.inv_h[a]), 0.5);
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
    const double rg = g.r_grid;
    const long long rgb = __double_as_longlong(rg);
    // distances are >= 0 (or +inf), so min(v, r_grid) is an integer
    // comparison of the bit patterns (no FP64 compare on the slow pipe)
    auto Dv = [&](int X, int Y, int Z) {
        double v = D[X + (int64_t)nx * (Y + (int64_t)ny * Z)];
        return __double_as_longlong(v) < rgb ? v : rg;   // voxels CFSM never reached
    };
    double v000 = Dv(i0[0], i0[1], i0[2]), v100 = Dv(i1[0], i0[1], i0[2]);
    double v010 = Dv(i0[0], i1[1], i0[2]), v110 = Dv(i1[0], i1[1], i0[2]);
    double v001 = Dv(i0[0], i0[1], i1[2]), v101 = Dv(i1[0], i0[1], i1[2]);
    double v011 = Dv(i0[0], i1[1], i1[2]), v111 = Dv(i1[0], i1[1], i1[2]);
    long long b0 = __double_as_longlong(v000);
    bool flat = b0 == __double_as_longlong(v100) && b0 == __double_as_longlong(v010) &&
                b0 == __double_as_longlong(v110) && b0 == __double_as_longlong(v001) &&
                b0 == __double_as_longlong(v101) && b0 == __double_as_longlong(v011) &&
                b0 == __double_as_longlong(v111);
    double di;
    if (flat) {
        di = v000;   // a + t (a - a) == a exactly: the lerps reproduce it
    } else {
        double c00 = lerp_rn(v000, v100, t[0]);
        double c10 = lerp_rn(v010, v110, t[0]);
        double c01 = lerp_rn(v001, v101, t[0]);
        double c11 = lerp_rn(v011, v111, t[0]);
        double c0 = lerp_rn(c00, c10, t[1]);
        double c1 = lerp_rn(c01, c11, t[1]);
        di = lerp_rn(c0, c1, t[2]);
    }
    // d >= 0 here (a convex combination of non-negative distances), so the
    // comparisons below are exact integer comparisons of the bit patterns
    const long long db = __double_as_longlong(di);
    const long long rmaxb = __double_as_longlong(g.rc_max);
    double r;
    if (db <= 0)
        r = g.rc_max;
    else if (db >= rmaxb)
        r = g.rc_min;
    else if (g.cut_fn == DCM_CUTOFF_LINEAR)
        r = DSUB(g.rc_max, DMUL(g.cut_slope, di));                  // Fig. 12
    else
        r = DADD(DMUL(g.cut_a, exp2(DMUL(g.alpha, DSUB(g.rc_max, di)))), g.cut_b);   // Eq. 7
    int c = 0;
    if (db < rmaxb) {
        c = 1;
        for (int k = 0; k < b.K - 2; ++k)
            c += db < __double_as_longlong(g.thr[k]) ? 1 : 0;   // thresholds are >= 0
    }
    d[i] = di;
    rc[i] = r;
    cls[i] = (uint8_t)c;
    if (rq) rq[inv[i]] = rc_constants(r);
    if (lt.lf) {
        // the displacement the drift found this step (warp lists), or in FP64
        const size_t N = (size_t)b.N;
        const float disp = lt.disp ? lt.disp[i] : list_disp(lt, g, N, i, x[i], x[N + i], x[2 * N + i]);
        float unused = -3.0e38f;
        list_terms(lt, i, disp, r, unused, mq);
    }
}

__global__ void k_cutoff(Batch b, const double *__restrict__ x, const double *__restrict__ D0,
                         const double *__restrict__ D1, const int *__restrict__ result, double *d,
                         double *rc, uint8_t *cls, float4 *rq, const int32_t *__restrict__ inv,
                         ListTest lt)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float mp = -3.0e38f, mq = -3.0e38f;
    if (i < b.N) cutoff_one(b, i, x, D0, D1, result, d, rc, cls, rq, inv, lt, mq);
    // the headroom term for the new cutoffs and the decision
    if (lt.lf) list_test_block(lt, mp, mq);
}

// classes for cutoffs supplied directly (scheduling only)
__global__ void k_classify_rc(Batch b, const double *__restrict__ rc, uint8_t *cls)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.N) return;
    const Geom &g = b.sys[sys_p(b, i)];
    double r = rc[i];
    int c = 0;
    if (r > g.rc_min) {
        c = 1;
        for (int k = 1; k <= b.K - 2; ++k) {
            double edge = g.rc_min + (g.rc_max - g.rc_min) * (double)k / (double)(b.K - 1);
            c += r > edge ? 1 : 0;
        }
    }
    cls[i] = (uint8_t)c;
}

static inline int nblk(int64_t n, int b) { return (int)((n + b - 1) / b); }

int launch_classify_rc(dcm_handle *h)
{
    k_classify_rc<<<nblk(h->n, 256), 256, 0, h->stream>>>(h->b, h->rc, h->cls);
    return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "classify launch");
}

static int coop_launch(dcm_handle *h, const void *fn, int grid, size_t smem, void **args,
                       int block = DET_THREADS)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
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

// Failure-detection check of the bounded grid barrier: block 1 leaves
// without arriving, so block 0 waits for an arrival that never comes; the
// bounded poll gives up, sets DEV_ERR_BARRIER and the kernel returns.
__global__ void k_barrier_timeout_check(unsigned int *bar, int *err)
{
    if (blockIdx.x == 1) return;
    grid_barrier(bar, err);
}

int launch_barrier_timeout_check(dcm_handle *h)
{
    cudaMemsetAsync(h->stats->barrier, 0, 2 * sizeof(unsigned int), h->stream);
    unsigned int *bar = h->stats->barrier;
    int *err = h->err;
    void *args[] = {(void *)&bar, (void *)&err};
    return coop_launch(h, (const void *)k_barrier_timeout_check, 2, 0, args);
}

static size_t kmeans_smem(int M) { return (size_t)M * (4 * 8 + 3 * 8 + 4); }

int prepare_kernels(dcm_handle *h)
{
    int r = prepare_force_kernels();
    if (r) return r;
    size_t smem = kmeans_smem(h->M);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute((const void *)k_kmeans,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return fail_cuda(e, "k_kmeans shared memory", __FILE__, __LINE__);
    }
    return DCM_OK;
}

int launch_detect(dcm_handle *h)
{
    cudaStream_t s = h->stream;
    const Batch &b = h->b;
    int64_t nv = b.NV;
    // Eq. 9
    k_detect_init<<<h->num_sms * 4, 256, 0, s>>>(nv, h->B, h->stamp, b.M, h->kacc,
                                                 h->stats->barrier, h->fcount);
    k_density<<<nblk(b.N, 256), 256, 0, s>>>(b, h->x, h->B);
    // smoothing
    int order = h->p.smooth_order;
    int vb = nblk(nv, DET_THREADS);
    if (order > 0) {
        SmoothW w;
        w.order = order;
        for (int k = 0; k <= 16; ++k) w.w[k] = 0;
        w.w[0] = 1;
        for (int r = 1; r <= order; ++r)
            for (int k = r; k >= 1; --k) w.w[k] += w.w[k - 1];
        uint64_t pass = 1ull << order;   // sum of the weights
        w.bmax = (uint32_t)(0xffffffffull / (pass * pass));
        if (order == 8) {
            k_smooth8<0, int32_t, uint32_t><<<vb, DET_THREADS, 0, s>>>(b, h->B, h->sm1, w.bmax, h->err);
            k_smooth8<1, uint32_t, uint32_t><<<vb, DET_THREADS, 0, s>>>(b, h->sm1, h->sm2, w.bmax, h->err);
            k_smooth8<2, uint32_t, double><<<vb, DET_THREADS, 0, s>>>(b, h->sm2, h->Bs, w.bmax, h->err);
        } else {
            k_smooth<0, int32_t, uint32_t><<<vb, DET_THREADS, 0, s>>>(b, h->B, h->sm1, w, h->err);
            k_smooth<1, uint32_t, uint32_t><<<vb, DET_THREADS, 0, s>>>(b, h->sm1, h->sm2, w, h->err);
            k_smooth<2, uint32_t, double><<<vb, DET_THREADS, 0, s>>>(b, h->sm2, h->Bs, w, h->err);
        }
    } else {
        SmoothW w;
        w.order = 0;
        w.w[0] = 1;
        w.bmax = 0xffffffffu;
        k_smooth<0, int32_t, double><<<vb, DET_THREADS, 0, s>>>(b, h->B, h->Bs, w, h->err);
    }
    // K-means labels (accumulators and barrier words zeroed by k_detect_init)
    {
        KmeansArgs a;
        a.b = b;
        a.Bs = h->Bs;
        a.S = h->S;
        a.max_iter = h->p.kmeans_max_iter > 0 ? h->p.kmeans_max_iter : 100;
        a.acc = h->kacc;
        a.part = h->kacc + 9 * 16 * (int64_t)b.M;   // after the multi-system accumulators
        a.bar = h->stats->barrier;
        a.err = h->err;
        a.st = h->stats;
        void *args[] = {(void *)&a};
        int rc;
        // one block per SM where the registers hold every voxel: each pass
        // ends in a grid barrier, whose cost grows with the arrivals
        if (b.M == 1) {
            int grid = coop_grid_size(h, (const void *)k_kmeans1, KM1_THREADS, 0);
            if ((int64_t)h->num_sms * KM1_THREADS * KM1_CACHE >= nv) grid = h->num_sms;
            if (grid > KM1_MAX_BLOCKS) grid = KM1_MAX_BLOCKS;
            int64_t need = (nv + KM1_THREADS - 1) / KM1_THREADS;
            if (grid > need) grid = (int)(need > 0 ? need : 1);
            rc = coop_launch(h, (const void *)k_kmeans1, grid, 0, args, KM1_THREADS);
        } else {
            size_t smem = kmeans_smem(b.M);
            int grid = coop_grid_size(h, (const void *)k_kmeans, KM_THREADS, smem);
            if (grid > h->num_sms) grid = h->num_sms;
            int64_t need = (nv + KM_THREADS - 1) / KM_THREADS;
            if (grid > need) grid = (int)(need > 0 ? need : 1);
            rc = coop_launch(h, (const void *)k_kmeans, grid, smem, args, KM_THREADS);
        }
        if (rc) return rc;
    }
    // Eq. 13 from the K-means labels
    if (h->p.segmentation == DCM_SEG_MUMFORD_SHAH) {
        int rc = launch_ms_detect(h);
        if (rc) return rc;
    }
    // Section 4.2: small components of either phase change phase
    if (h->cc_on) {
        int rc = launch_components(h, b, h->S, -1, h->cc_ntiles);
        if (rc) return rc;
    }
    // CFSM (frontier counters zeroed by k_detect_init, barrier words by k_cfsm_init)
    k_cfsm_init<<<vb, DET_THREADS, 0, s>>>(b, h->S, h->D0, h->D1, h->stamp, h->flist + nv,
                                           h->fcount, h->stats->barrier);
    {
        CfsmArgs a;
        a.b = b;
        int dmax = 1;
        for (int q = 0; q < b.M; ++q)
            for (int ax = 0; ax < 3; ++ax) dmax = h->geo_host[q].gd[ax] > dmax ? h->geo_host[q].gd[ax] : dmax;
        a.iter_max = h->p.cfsm_iter_max > 0 ? h->p.cfsm_iter_max : 4 * dmax;
        a.cap = nv;
        a.S = h->S;
        a.D0 = h->D0;
        a.D1 = h->D1;
        a.stamp = h->stamp;
        a.lists = h->flist;
        a.fcount = h->fcount;
        a.result = (int *)&h->stats->barrier[3];
        a.kpass = (int *)&h->stats->barrier[4];
        a.nf_switch = 256;          // measured: 262k, 2M and ensemble detection all best here
        a.bar = h->stats->barrier;
        a.err = h->err;
        a.st = h->stats;
        void *args[] = {(void *)&a};
        // one block per SM: a pass is a short latency chain over a small
        // frontier, and the grid barrier costs less with half the arrivals
        // (measured: 0.302 against 0.359 ms per detection at 262k atoms)
        int grid = h->num_sms;
        int rc = coop_launch(h, (const void *)k_cfsm, grid, 0, args,
                             b.M == 1 ? CFSM_THREADS / 2 : CFSM_THREADS);
        if (rc) return rc;
        // the small frontiers of the last passes: one cluster of 8 SMs
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(CFSM_TAIL_CTAS);
        cfg.blockDim = dim3(CFSM_TAIL_THREADS);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CFSM_TAIL_CTAS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelExC(&cfg, (const void *)k_cfsm_tail, args);
        if (e != cudaSuccess) return fail_cuda(e, "cfsm tail launch", __FILE__, __LINE__);
    }
    // Algorithm 3.1 + Eq. 7
    const bool wl = h->nl && h->list_warp;
    ListTest lt = list_test(h, false, true, true);     // the drift added the other term
    if (!h->fold_check) lt.lf = nullptr;
    k_cutoff<<<nblk(b.N, 256), 256, 0, s>>>(b, h->x, h->D0, h->D1,
                                            (const int *)&h->stats->barrier[3], h->d, h->rc, h->cls,
                                            wl ? h->rq : nullptr, h->inv, lt);
    return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "detect launch");
}

}  // namespace dcm
