// dcm_device.cuh -- device helpers shared by the libdcm kernels.
//
// Every FP64 expression whose result decides an integer (a bin index, a
// pair inside/outside the cutoff, a class) or must reproduce a defined
// value (the Godunov solve, the trilinear lookup) is written with explicit
// round-to-nearest intrinsics so that the compiler cannot contract it into
// an FMA.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dcm_internal.cuh"

namespace dcm {

#define DADD(a, b) __dadd_rn((a), (b))
#define DSUB(a, b) __dsub_rn((a), (b))
#define DMUL(a, b) __dmul_rn((a), (b))

// bin of coordinate x on n bins of a periodic edge: min(n-1, floor(x*inv))
__device__ __forceinline__ int bin_of(double x, double inv, int n)
{
    int k = (int)floor(DMUL(x, inv));
    k = k > n - 1 ? n - 1 : k;
    return k < 0 ? 0 : k;
}

// minimum image of a coordinate difference (same rule on every code path)
__device__ __forceinline__ double min_image(double dx, double L, double halfL)
{
    if (dx > halfL) return DSUB(dx, L);
    if (dx < -halfL) return DADD(dx, L);
    return dx;
}

// wrap into [0, L) for a move smaller than L
__device__ __forceinline__ double wrap_coord(double x, double L)
{
    if (x < 0.0) x = DADD(x, L);
    if (x >= L) x = DSUB(x, L);
    return x;
}

// The same wrap with the comparisons done on the IEEE bit patterns (for
// L > 0 and non-NaN x, x < 0 is the sign bit and, for x >= 0, x >= L is an
// integer comparison of the patterns): GB300 runs FP64 compares on its
// FP64 pipe at 1/64 of the FP32 rate.  Returns false when x is still out of
// [0, L) afterwards (a move of more than one edge).
__device__ __forceinline__ bool wrap_coord_bits(double &x, double L)
{
    const long long Lb = __double_as_longlong(L);
    long long b = __double_as_longlong(x);
    if (b < 0) {                              // sign bit: x < 0 (or -0)
        x = DADD(x, L);
        b = __double_as_longlong(x);
    } else if (b >= Lb) {
        x = DSUB(x, L);
        b = __double_as_longlong(x);
    }
    if (b == (long long)0x8000000000000000ll) {   // -0 -> +0
        x = 0.0;
        b = 0;
    }
    return b >= 0 && b < Lb;
}

// r^2 = dx*dx + dy*dy + dz*dz, left to right, no FMA
__device__ __forceinline__ double r2_rn(double dx, double dy, double dz)
{
    return DADD(DADD(DMUL(dx, dx), DMUL(dy, dy)), DMUL(dz, dz));
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// add a float into a (hi, lo) double-float accumulator
__device__ __forceinline__ void ff_add(float &hi, float &lo, float a)
{
    float s, e;
    two_sum(hi, a, s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
}

// ---- bounded grid barrier for cooperative (co-resident) launches --------
// words[0] counts arrivals and is never reset inside a launch: the k-th
// barrier of the launch is complete when the count reaches k * (blocks),
// and a block learns k from the value its own arrival returned.  One atomic
// per block and polling with acquire loads; no reset or generation word, so
// the last block to arrive does no extra round trips.  words[0] must be zero
// at launch.  Gives up after a bounded number of polls, sets
// DEV_ERR_BARRIER and returns false.
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// arrival with release semantics at GPU scope: after the block's bar.sync it
// publishes every write of the block (release is cumulative), so no separate
// fence is needed; the acquire loads of the poll order what follows
__device__ __forceinline__ unsigned int atom_add_release_u32(unsigned int *p, unsigned int v)
{
    unsigned int old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// the arrival and the wait of grid_barrier for one thread, the caller
// synchronising its block around it (a block whose other threads have
// nothing to do across the barrier); true when every block arrived
__device__ __forceinline__ bool grid_arrive_wait(unsigned int *words, int *err)
{
    const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
    const unsigned int arrived = atom_add_release_u32(words, 1u);
    const unsigned int target = (arrived / nb + 1u) * nb;
    long long polls = 0;
    while ((int)(ld_acquire_u32(words) - target) < 0) {
        ++polls;
        if ((polls & 255) == 0) {
            if (polls > (1ll << 21)) {
                atomicOr(err, DEV_ERR_BARRIER);
                return false;
            }
            if (*(volatile int *)err & DEV_ERR_BARRIER) return false;
        }
        if (polls > 4096) __nanosleep(128);
    }
    return true;
}

__device__ __forceinline__ bool grid_barrier(unsigned int *words, int *err)
{
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
        const unsigned int arrived = atom_add_release_u32(words, 1u);
        const unsigned int target = (arrived / nb + 1u) * nb;
        int ok = 1;
        // tight polling first (a healthy barrier completes in a few
        // microseconds), then back off; the error word is read only every
        // 256 polls.  The limit bounds the wait to well under a second.
        long long polls = 0;
        while ((int)(ld_acquire_u32(words) - target) < 0) {
            ++polls;
            if ((polls & 255) == 0) {
                if (polls > (1ll << 21)) {
                    atomicOr(err, DEV_ERR_BARRIER);
                    ok = 0;
                    break;
                }
                if (*(volatile int *)err & DEV_ERR_BARRIER) {
                    ok = 0;
                    break;
                }
            }
            if (polls > 4096) __nanosleep(128);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---- Godunov upwind local solve (Eq. 16-19, per-axis spacing) -----------
// The oracle's sequence of cases (one, two, three upwind axes) and
// expressions, with two changes for this GPU, whose FP64 pipe runs at 1/64
// of FP32: the comparisons of the non-negative (or +inf) values use their
// bit patterns (integer pipe), and the quadratic's root (B + sqrt(disc)) / A
// takes FP32 seeds for the square root and 1/A, each refined by one FP64
// Newton step (relative error ~1e-14 instead of the correctly rounded
// 1e-16; the distances agree with the oracle to ~1e-13 absolute).  The
// weights w_k = 1/h_k^2 come precomputed (the same IEEE quotients).
__device__ __forceinline__ bool dle_nonneg(double a, double b)
{
    return __double_as_longlong(a) <= __double_as_longlong(b);
}

__device__ __forceinline__ double godunov_root(double A, double B, double disc)
{
    double s = 0.0;
    if (__double_as_longlong(disc) > 0) {
        const float sf = sqrtf(__double2float_rn(disc));
        if (sf > 1e-18f) {
            const double s0 = (double)sf;
            const double t = fma(-s0, s0, disc);                  // disc - s0^2
            s = fma(t, (double)(0.5f * __frcp_rn(sf)), s0);        // s0 + t / (2 s0)
        } else {
            s = __dsqrt_rn(disc);                                 // (below FP32's range)
        }
    }
    const double num = DADD(B, s);
    const double r = (double)__frcp_rn(__double2float_rn(A));     // A = sum of w: FP32-safe
    const double q0 = DMUL(num, r);
    return fma(fma(-q0, A, num), r, q0);                          // q0 + (num - q0 A) / A
}

__device__ __forceinline__ double godunov_w(double a0, double a1, double a2, double h0, double h1,
                                            double h2, double w1, double w2, double w3)
{
    // stable sort of (a, h, w) by a
    if (!dle_nonneg(a0, a1)) {
        double t = a0; a0 = a1; a1 = t; t = h0; h0 = h1; h1 = t; t = w1; w1 = w2; w2 = t;
    }
    if (!dle_nonneg(a1, a2)) {
        double t = a1; a1 = a2; a2 = t; t = h1; h1 = h2; h2 = t; t = w2; w2 = w3; w3 = t;
        if (!dle_nonneg(a0, a1)) {
            t = a0; a0 = a1; a1 = t; t = h0; h0 = h1; h1 = t; t = w1; w1 = w2; w2 = t;
        }
    }
    if (__double_as_longlong(a0) == 0x7ff0000000000000ll) return a0;    // +inf
    double d2 = DSUB(a1, a0);
    double d3 = DSUB(a2, a0);
    double e = h0;
    if (dle_nonneg(e, d2)) return DADD(a0, e);
    double wd2 = DMUL(w2, d2);
    double A = DADD(w1, w2);
    double B = wd2;
    double C = DSUB(DMUL(wd2, d2), 1.0);
    double disc = DSUB(DMUL(B, B), DMUL(A, C));
    e = godunov_root(A, B, disc);
    if (dle_nonneg(e, d3)) return DADD(a0, e);
    double wd3 = DMUL(w3, d3);
    A = DADD(DADD(w1, w2), w3);
    B = DADD(wd2, wd3);
    C = DSUB(DADD(DMUL(wd2, d2), DMUL(wd3, d3)), 1.0);
    disc = DSUB(DMUL(B, B), DMUL(A, C));
    e = godunov_root(A, B, disc);
    return DADD(a0, e);
}

__device__ __forceinline__ double godunov(double a0, double a1, double a2, double h0, double h1,
                                          double h2)
{
    return godunov_w(a0, a1, a2, h0, h1, h2, __ddiv_rn(1.0, DMUL(h0, h0)),
                     __ddiv_rn(1.0, DMUL(h1, h1)), __ddiv_rn(1.0, DMUL(h2, h2)));
}

// min of two non-negative doubles (or +inf) by their bit patterns
__device__ __forceinline__ double dmin_nonneg(double a, double b)
{
    return __double_as_longlong(a) < __double_as_longlong(b) ? a : b;
}

__device__ __forceinline__ double lerp_rn(double a, double b, double t)
{
    return DADD(a, DMUL(t, DSUB(b, a)));
}

// Own Verlet-list radius of particle i: the cutoff it would get if its
// interface distance dropped by delta (so small moves of the detected
// interface do not force a rebuild), never below its current cutoff, plus
// its skin share; a pair (i, j) is listed while closer than this plus j's
// share.  The margin (1e-5 relative + 1e-4) covers the FP32 distances of
// the build; the reuse check takes it off again.
__device__ __forceinline__ float list_radius(const Geom &g, double rci, double di, float delta,
                                             float share)
{
    float r = (float)rci;
    if (delta > 0.f && g.rc_max > g.rc_min) {
        float dd = fmaxf((float)di - delta, 0.f);
        float rmax = (float)g.rc_max, rmin = (float)g.rc_min;
        float ra = dd <= 0.f ? rmax
                 : (dd >= rmax ? rmin
                    : (g.cut_fn == DCM_CUTOFF_LINEAR
                           ? fmaf(-(float)g.cut_slope, dd, rmax)
                           : fmaf((float)g.cut_a, exp2f((float)g.alpha * (rmax - dd)), (float)g.cut_b)));
        r = fmaxf(r, ra);
    }
    return fmaf(r, 1.00001f, 1e-4f) + share;
}

// an own list radius without the build margin (for the reuse check)
__device__ __forceinline__ float list_radius_unpadded(float rl, float share)
{
    return fmaf(rl - share - 1e-4f, 0.99999f, share);
}

// skin share of a particle with speed |v| under force |F|: skin/2, or with
// adaptive skins the distance it would cover in skin_time at constant
// acceleration, tau |v| + tau^2 |F| / (2 m), clamped to [skin_floor, skin/2]
__device__ __forceinline__ float skin_share(const Geom &g, float speed, float force)
{
    const float half = 0.5f * (float)g.skin;
    if (g.skin_time <= 0.f) return half;
    const float tau = g.skin_time;
    const float inv_m = (float)(2.0 * g.hdtm / g.dt);      // hdtm = dt / (2 m)
    const float reach = tau * fmaf(0.5f * tau * inv_m, force, speed);
    return fminf(fmaxf(reach, g.skin_floor), half);
}

// The FP32 grid value and remainder of a cell-relative coordinate u: hi is u
// rounded (to nearest, ties to even) to a multiple of the grid step 2^gexp,
// or to 24 significant bits where those are coarser (|u| >= 2^(gexp + 24),
// a particle that drifted beyond the bound the grid was sized for); lo is
// the rest u - hi rounded to FP32.  Computed from the bits of u with integer
// instructions: on this GPU a double/float conversion issues at the FP64
// rate, 1/64 of FP32, and this runs for three coordinates of every particle
// every step.  |u| below 2^-70 gives hi = lo = 0.
__device__ __forceinline__ void grid_split(double u, int gexp, float &hi, float &lo)
{
    const long long b = __double_as_longlong(u);
    const int E = (int)((b >> 52) & 0x7ff) - 1075;        // u = +-M 2^E, M < 2^53
    if (E < -1075 + 1023 - 70) {
        hi = 0.f;
        lo = 0.f;
        return;
    }
    const long long M = (b & 0xFFFFFFFFFFFFFll) | (1ll << 52);
    int s = gexp - E;                                      // bits of M below the step
    s = s < 29 ? 29 : s;
    long long N = 0, r = M;
    if (s < 54) {
        N = M >> s;
        const long long rem = M - (N << s), half = 1ll << (s - 1);
        N += (rem > half || (rem == half && (N & 1))) ? 1 : 0;
        r = M - (N << s);                                  // |r| <= 2^(s-1)
    }
    // N <= 2^24 and |r| < 2^53: both convert exactly or correctly rounded;
    // the scales are powers of two inside the normal FP32 range
    const float h = __int2float_rn((int)N) * __int_as_float((s + E + 127) << 23);
    const float l = __ll2float_rn(r) * __int_as_float((E + 127) << 23);
    hi = b < 0 ? -h : h;
    lo = b < 0 ? -l : l;
}

// FP32 position of a particle relative to the corner of its link cell
// (cell index c_local within its system) and that cell's x index; a particle
// that wrapped through the box since its cell was assigned (between
// Verlet-list builds) is folded back next to that cell.  Shared by the
// gather kernel and the drift, which must produce the same bits.  The
// corner coordinates c * L/n come from a table (the same rounded products
// as computing them here), and the cell coordinates from exact magic-number
// divisions, which keeps this to one FP64 subtraction per axis: the FP64
// pipe runs at 1/64 of the FP32 rate.
// The FP32 coordinate is a multiple of the system's grid qpos (a power of
// two chosen so that coordinates and close-pair distances have at most 24
// significant bits), and lo receives the FP32 remainder u - hi: a close
// pair's cell shift is then exact in FP32, and hi + lo carries the FP64
// position to about 2^-47 for the double-float close-pair forces.
__device__ __forceinline__ float4 cell_rel_position(const Batch &b, const Geom &g, double px,
                                                   double py, double pz, int c_local, float4 &lo)
{
    const int yz = (int)__umul64hi((unsigned)c_local, g.div_nc[0]);      // c / nc0
    const int cx = c_local - yz * g.nc[0];
    const int cz = (int)__umul64hi((unsigned)yz, g.div_nc[1]);           // yz / nc1
    const int cy = yz - cz * g.nc[1];
    const double *corner = b.corner + g.corner_off;
    const double p[3] = {px, py, pz};
    const int c[3] = {cx, g.nc[0] + cy, g.nc[0] + g.nc[1] + cz};
    const int gexp = ((__float_as_int(g.qpos) >> 23) & 0xff) - 127;
    float uf[3], ul[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double u = DSUB(p[a], corner[c[a]]);
        // wrapped through the box: |u| above half the box (integer compare
        // of the magnitudes' bits; the FP32 half box widened exactly)
        const unsigned hb = (unsigned)__float_as_int(g.halfLf[a]);
        const long long half_bits = ((long long)((hb >> 23) + 896) << 52) |
                                    ((long long)(hb & 0x7fffff) << 29);
        const long long ub = __double_as_longlong(u);
        if ((ub & 0x7FFFFFFFFFFFFFFFll) > half_bits) u = ub < 0 ? DADD(u, g.L[a]) : DSUB(u, g.L[a]);
        grid_split(u, gexp, uf[a], ul[a]);
    }
    lo = make_float4(ul[0], ul[1], ul[2], 0.f);
    return make_float4(uf[0], uf[1], uf[2], (float)cx);
}

// the force walks' per-particle cutoff constants: FP32 r_c^2, its 2^-18
// guard band below and above, and the conservative culling radius
__device__ __forceinline__ float4 rc_constants(double r)
{
    float rc2f = (float)DMUL(r, r);
    return make_float4(rc2f, rc2f * (1.f - 3.814697265625e-06f), rc2f * (1.f + 3.814697265625e-06f),
                       fmaf((float)r, 1.00002f, 1e-4f));
}

// ---- the Verlet-list reuse test (condition: dcm_list.cu) ----------------
// Any kernel that visits every particle once can carry it: the drift on a
// step without detection, the cutoff kernel (new cutoffs) and the drift
// together on a step with one, the stand-alone check otherwise.
struct ListTest {
    int *lf;                           // null: no test in this kernel
    const double *x_ref;
    const float *rl_ref, *sh_ref;
    const float4 *u_ref;               // warp lists: FP32 cell-relative positions at the build
    float *disp;                       // warp lists: this step's |displacement| per particle
    int excess;                        // the headroom term here (needs the cutoffs)
    int partner;                       // the displacement-share term here
    int decide;                        // this kernel's last block decides
    int force;                         // decide "rebuild" whatever the terms
    int set_cond;                      // also set the step graph's branch condition
    cudaGraphConditionalHandle cond;
};

// order-preserving int image of a float (for atomicMax over signed values);
// the image is its own inverse
__device__ __forceinline__ int ordered_int(float f)
{
    int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}

// |displacement| of particle i since the build; a coordinate wrapped through
// the box shows up as a jump of about one edge and is folded back (moves are
// far below half an edge)
__device__ __forceinline__ float list_disp(const ListTest &t, const Geom &g, size_t N, int64_t i,
                                           double x, double y, double z)
{
    float dx = (float)(x - t.x_ref[i]);
    float dy = (float)(y - t.x_ref[N + i]);
    float dz = (float)(z - t.x_ref[2 * N + i]);
    // (an approximate reciprocal suffices: rint only decides between 0 and
    // +-1 edges, and a move near half an edge cannot happen)
    const float Lx = (float)g.L[0], Ly = (float)g.L[1], Lz = (float)g.L[2];
    dx -= Lx * rintf(dx * rcp_approx(Lx));
    dy -= Ly * rintf(dy * rcp_approx(Ly));
    dz -= Lz * rintf(dz * rcp_approx(Lz));
    return sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
}

// the same from the FP32 cell-relative positions now and at the build: the
// cell of a particle is fixed between builds, so the difference is the
// displacement (FP32 only)
__device__ __forceinline__ float list_disp32(float4 u, float4 u0)
{
    const float dx = u.x - u0.x, dy = u.y - u0.y, dz = u.z - u0.z;
    return sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
}

// particle i's two terms: partner |d_i| - s_i, headroom |d_i| - (R_i - r_c[i])
__device__ __forceinline__ void list_terms(const ListTest &t, int64_t i, float disp, double rci,
                                           float &mp, float &mq)
{
    const float s = t.sh_ref[i];
    if (t.partner) mp = fmaxf(mp, disp - s);
    if (t.excess) mq = fmaxf(mq, disp - (list_radius_unpadded(t.rl_ref[i], s) - (float)rci));
}

// the decision from the two maxima (one thread, after every block added its own)
__device__ __forceinline__ void list_decide(const ListTest &t)
{
    int *lf = t.lf;
    // reset both maxima to the image of -3.4e38 for the next step
    float partner = __int_as_float(ordered_int(__int_as_float(atomicExch(&lf[LF_PARTNER], LF_EXCESS_RESET))));
    float excess = __int_as_float(ordered_int(__int_as_float(atomicExch(&lf[LF_EXCESS], LF_EXCESS_RESET))));
    int ok = atomicAdd(&lf[LF_OK], 0);
    if (atomicExch(&lf[LF_OVERFLOW], 0)) {
        // a particle had more neighbours than its capacity at the last
        // fill: its list is incomplete, rebuild with 25 % more room
        ok = 0;
        lf[LF_OK] = 0;
        lf[LF_SCALE] = __float_as_int(__int_as_float(lf[LF_SCALE]) * 1.25f);
    }
    int rebuild = t.force || !ok || (partner + excess >= 0.f);
    lf[LF_REBUILD] = rebuild;
    if (rebuild) lf[LF_SHMAX] = 0;          // the gather of the build takes the max
    lf[LF_DONE] = 0;
    if (t.set_cond) cudaGraphSetConditional(t.cond, (unsigned)rebuild);
}

// the block's maxima into the control words and, in the last block of a
// deciding kernel, the decision; every thread of the block calls it, and
// t.lf and t.decide are the same for all of them
__device__ __forceinline__ void list_test_block(const ListTest &t, float mp, float mq)
{
    // warp maxima, then the block's in shared memory: one atomic per word
    // and block (the kernels that carry the test launch a block per 256
    // particles; per-warp atomics on two words serialised in L2)
    for (int off = 16; off > 0; off >>= 1) {
        mp = fmaxf(mp, __shfl_xor_sync(0xffffffffu, mp, off));
        mq = fmaxf(mq, __shfl_xor_sync(0xffffffffu, mq, off));
    }
    __shared__ float s_mp[32], s_mq[32];
    __shared__ int s_last;
    const int warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_mp[warp] = mp;
        s_mq[warp] = mq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nwarps; ++w) {
            mp = fmaxf(mp, s_mp[w]);
            mq = fmaxf(mq, s_mq[w]);
        }
        if (t.partner) atomicMax(&t.lf[LF_PARTNER], ordered_int(mp));
        if (t.excess) atomicMax(&t.lf[LF_EXCESS], ordered_int(mq));
        if (t.decide) {
            __threadfence();
            s_last = atomicAdd(&t.lf[LF_DONE], 1) == (int)(gridDim.x * gridDim.y * gridDim.z) - 1;
            if (s_last) {
                __threadfence();
                list_decide(t);
            }
        }
    }
}

}  // namespace dcm
