// dcm_ms.cu -- two-phase piecewise-constant Mumford-Shah segmentation (Eq. 13)
// on a voxel image: the convex relaxation of Chan, Esedoglu and Nikolova,
//     min over u in [0,1] of  sum_v u_v r_v + nu sum_faces |u_a - u_b|,
//     r_v = (rho_v - c_l)^2 - (rho_v - c_v)^2   (u = 1: liquid),
// solved by the first-order primal-dual iteration of Chambolle and Pock with
// one dual variable per grid face (|p| <= nu), step sizes tau = sigma =
// 0.99/sqrt(12) (convergence needs tau sigma |grad|^2 < 1, and |grad|^2 = 12
// for periodic forward differences in 3D), u from 1/2, a fixed number of
// iterations; liquid (s = 0) where u > 1/2.  The perimeter counts the
// periodic faces between liquid and vapor voxels, for which thresholded
// relaxed minimisers are exact minimisers of Eq. 13.
//
// Two uses:
//  * dcm_ms_segment: the densities fixed, on a caller's image;
//  * the segmentation step of the interface detection (DCM_SEG_MUMFORD_SHAH):
//    on the smoothed number density rho = Bs * inv_scale, from the K-means
//    labels, rounds of exact phase means (integer sums of Bs) and
//    segmentation (one round by default: the thesis's flow, K-means
//    densities then Eq. 13; more alternate) until the labels repeat or
//    ms_outer rounds, for every
//    system of the handle at once (a system whose labels repeated, or with
//    an empty phase, stops; its later rounds are no-ops).
//
// One iteration is one kernel: each voxel updates the duals of its three
// upper faces and recomputes, with the same expression, the new duals of
// its three lower faces (which the voxel below also writes), then its
// primal value, reading the previous iteration's u-bar and duals and
// writing the next ones (two buffers of each, alternating).  The thesis
// fixes no precision for the segmentation and the labels are a threshold
// decision, so the iteration runs in FP32 (the data term is formed in FP64
// and rounded once), with round-to-nearest intrinsics in the oracle's
// operation order and no reduction: the result does not depend on the
// thread layout and equals the oracle's two-pass single-precision iteration
// bit for bit.  (In FP64 the ~40 FP64 operations per voxel made each
// iteration FP64-pipe bound, 1/64 of the FP32 rate on this GPU.)  Bound:
// L2 (the iteration's ~40 B per voxel stay resident), then launch latency.
// Duals are stored as three planes (x, y, z faces) for coalesced access.
#include "dcm_device.cuh"

namespace dcm {

constexpr int MS_THREADS = 256;

static inline int ms_blocks(int64_t n) { return (int)((n + MS_THREADS - 1) / MS_THREADS); }

// the step sizes (host: the same expression as the oracle's)
static double ms_tau() { return 0.99 / sqrt(12.0); }

// the iteration's buffers: u, u-bar (two), duals (two x 3 planes), r
struct MsBufs {
    float *u, *ub[2], *p[2], *r;
    int64_t ps;        // plane stride of the duals
};

// one system's voxel grid and the voxel's coordinates in it
struct MsCell {
    int nx, ny, nz;
    int64_t v0;                    // first voxel of the system
    unsigned long long mx, my;     // exact division by nx, ny (Geom::div_gd)
};

__device__ __forceinline__ MsCell ms_cell(const Batch &b, int64_t v, int &sys)
{
    sys = sys_v(b, v);
    const Geom &g = b.sys[sys];
    MsCell c;
    c.nx = g.gd[0];
    c.ny = g.gd[1];
    c.nz = g.gd[2];
    c.v0 = g.v0;
    c.mx = g.div_gd[0];
    c.my = g.div_gd[1];
    return c;
}

// The duals of one axis at voxel v: the face above v (stored) and, with the
// same expression, the face below v (the lower voxel's upper face);
// returns their contribution to grad^T p at v.  live: the axis has more
// than one voxel (otherwise its faces carry no dual).
__device__ __forceinline__ float ms_axis(const float *__restrict__ pa, float *__restrict__ po,
                                         const float *__restrict__ ubi, int64_t v, float ubv,
                                         int upo, int dno, bool live, float sigma, float nu)
{
    // dual ascent on the face above v, projected on |p| <= nu
    float q = live ? __fadd_rn(pa[v], __fmul_rn(sigma, __fsub_rn(ubi[v + upo], ubv))) : 0.0f;
    if (q > nu) q = nu;
    if (q < -nu) q = -nu;
    po[v] = q;
    float qd = live ? __fadd_rn(pa[v + dno], __fmul_rn(sigma, __fsub_rn(ubv, ubi[v + dno]))) : 0.0f;
    if (qd > nu) qd = nu;
    if (qd < -nu) qd = -nu;
    // inflow from the lower face minus outflow
    return __fsub_rn(qd, q);
}

// One Chambolle-Pock iteration at voxel v (global index), system grid c:
// reads u-bar and the duals of buffer k (the previous iteration), writes
// those of buffer k ^ 1 and u.  Voxel coordinates and neighbour offsets in
// 32 bits (a system's grid holds fewer than 2^31 voxels).
__device__ __forceinline__ void ms_iter_voxel(const MsCell &c, int64_t v, const MsBufs &m, int k,
                                              float tau, float sigma, float nu)
{
    const unsigned nx = (unsigned)c.nx, ny = (unsigned)c.ny, nz = (unsigned)c.nz;
    const unsigned lv = (unsigned)(v - c.v0);
    const unsigned t = (unsigned)__umul64hi(lv, c.mx);          // lv / nx
    const unsigned z = (unsigned)__umul64hi(t, c.my);           // t / ny
    const unsigned x = lv - t * nx, y = t - z * ny;
    const int sxy = (int)(nx * ny), sv = (int)(nz * (unsigned)sxy);
    // (selects, not m.ub[k]: a run-time index into the parameter struct
    // would copy it to local memory)
    const float *__restrict__ ubi = k ? m.ub[1] : m.ub[0];
    float *ubo = k ? m.ub[0] : m.ub[1];
    const float *pi = k ? m.p[1] : m.p[0];
    float *po = k ? m.p[0] : m.p[1];
    const float ubv = ubi[v];
    // grad^T p at v, axes in order x, y, z (periodic neighbours)
    float gtp = 0.0f;
    gtp = __fadd_rn(gtp, ms_axis(pi, po, ubi, v, ubv, x + 1 < nx ? 1 : 1 - (int)nx,
                                 x > 0 ? -1 : (int)nx - 1, nx > 1, sigma, nu));
    gtp = __fadd_rn(gtp, ms_axis(pi + m.ps, po + m.ps, ubi, v, ubv,
                                 y + 1 < ny ? (int)nx : (int)nx - sxy,
                                 y > 0 ? -(int)nx : sxy - (int)nx, ny > 1, sigma, nu));
    gtp = __fadd_rn(gtp, ms_axis(pi + 2 * m.ps, po + 2 * m.ps, ubi, v, ubv,
                                 z + 1 < nz ? sxy : sxy - sv, z > 0 ? -sxy : sv - sxy, nz > 1,
                                 sigma, nu));
    // primal descent u -= tau (grad^T p + r), clipped to [0, 1], and the
    // extrapolation u-bar = 2 u_new - u_old
    const float uo = m.u[v];
    float un = __fsub_rn(uo, __fmul_rn(tau, __fadd_rn(gtp, m.r[v])));
    if (un < 0.0f) un = 0.0f;
    if (un > 1.0f) un = 1.0f;
    ubo[v] = __fsub_rn(__fmul_rn(2.0f, un), uo);
    m.u[v] = un;
}

// the relaxation's start at voxel v: data term (FP64, rounded once), u and
// u-bar at 1/2, duals at 0
__device__ __forceinline__ void ms_start_voxel(const MsBufs &m, int64_t v, double rho, double c_l,
                                               double c_v)
{
    const double a = DSUB(rho, c_l), b = DSUB(rho, c_v);
    m.r[v] = __double2float_rn(DSUB(DMUL(a, a), DMUL(b, b)));
    m.u[v] = 0.5f;
    m.ub[0][v] = 0.5f;
    m.p[0][v] = 0.0f;
    m.p[0][m.ps + v] = 0.0f;
    m.p[0][2 * m.ps + v] = 0.0f;
}

// ---- dcm_ms_segment: one image, densities fixed -----------------------------
__global__ void k_ms_init(int64_t nv, const double *__restrict__ rho, double c_l, double c_v,
                          MsBufs m)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    ms_start_voxel(m, v, rho[v], c_l, c_v);
}

__global__ void k_ms_iter(MsCell c, int64_t nv, MsBufs m, int k, float tau, float sigma, float nu)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    ms_iter_voxel(c, v, m, k, tau, sigma, nu);
}

// labels (liquid where u > 1/2) and u in double for the caller
__global__ void k_ms_labels(int64_t nv, const float *__restrict__ u, uint8_t *S, double *u_out)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    S[v] = u[v] > 0.5f ? 0 : 1;
    u_out[v] = (double)u[v];
}

// ---- the detection's segmentation step, every system of the handle --------
// per system: [0] liquid sum of Bs, [1] liquid voxels, [2] vapor sum, [3]
// vapor voxels (exact: Bs holds integers below 2^53); c[2s], c[2s + 1] the
// round's densities; flag[2s] the system is still segmenting, flag[2s + 1]
// this round changed a label
struct MsSys {
    unsigned long long *acc;
    double *c;
    int *flag;
};

// the phase sums of labels S for the systems still segmenting: warp sums,
// then one atomic per counter and block when the whole block lies in one
// system (per warp otherwise), so a large grid does not serialise on the
// four counters of its system
__global__ void __launch_bounds__(MS_THREADS) k_ms_sums(Batch b, const double *__restrict__ Bs,
                                                       const uint8_t *__restrict__ S, MsSys ms)
{
    constexpr int W = MS_THREADS / 32;
    __shared__ unsigned long long s_acc[W][4];
    __shared__ int s_sys[W];
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int sys = -1;
    unsigned long long q[4] = {0ull, 0ull, 0ull, 0ull};
    if (v < b.NV) {
        sys = sys_v(b, v);
        if (ms.flag[2 * sys]) {
            const unsigned long long val = (unsigned long long)Bs[v];
            const bool liq = S[v] == 0;
            q[0] = liq ? val : 0ull;
            q[1] = liq ? 1ull : 0ull;
            q[2] = liq ? 0ull : val;
            q[3] = liq ? 0ull : 1ull;
        }
    }
    // (lanes past the end take the first lane's system: they add zeros)
    const int s0 = __shfl_sync(full, sys, 0);
    if (sys < 0) sys = s0;
    const bool uniform = __all_sync(full, sys == s0);
    if (uniform) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            for (int off = 16; off > 0; off >>= 1) q[c] += __shfl_xor_sync(full, q[c], off);
        if (lane == 0) {
            for (int c = 0; c < 4; ++c) s_acc[w][c] = q[c];
            s_sys[w] = s0;
        }
    } else {
        if (lane == 0) s_sys[w] = -1;
        if (sys >= 0 && (q[1] | q[3])) {
            unsigned long long *a = ms.acc + 4 * sys;
            for (int c = 0; c < 4; ++c)
                if (q[c]) atomicAdd(a + c, q[c]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // warps of one system add up first
        for (int i = 0; i < W; ++i) {
            if (s_sys[i] < 0) continue;
            unsigned long long t[4] = {s_acc[i][0], s_acc[i][1], s_acc[i][2], s_acc[i][3]};
            for (int j = i + 1; j < W; ++j)
                if (s_sys[j] == s_sys[i]) {
                    for (int c = 0; c < 4; ++c) t[c] += s_acc[j][c];
                    s_sys[j] = -1;
                }
            unsigned long long *a = ms.acc + 4 * s_sys[i];
            for (int c = 0; c < 4; ++c)
                if (t[c]) atomicAdd(a + c, t[c]);
        }
    }
}

// every system segments from its K-means labels; accumulators at zero
__global__ void k_ms_start(Batch b, MsSys ms)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.M) return;
    ms.flag[2 * s] = 1;
    ms.flag[2 * s + 1] = 0;
    unsigned long long *a = ms.acc + 4 * s;
    a[0] = a[1] = a[2] = a[3] = 0ull;
}

// a round's start, one thread per system: the densities from the sums (the
// oracle's (sum / count) * inv_scale), the sums cleared for the next round;
// a system with an empty phase stops
__global__ void k_ms_begin(Batch b, MsSys ms)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.M) return;
    unsigned long long *a = ms.acc + 4 * s;
    if (a[1] == 0 || a[3] == 0) ms.flag[2 * s] = 0;
    if (ms.flag[2 * s]) {
        const double inv = b.sys[s].ms_inv_scale;
        ms.c[2 * s] = DMUL(__ddiv_rn((double)a[0], (double)a[1]), inv);
        ms.c[2 * s + 1] = DMUL(__ddiv_rn((double)a[2], (double)a[3]), inv);
    }
    ms.flag[2 * s + 1] = 0;
    a[0] = a[1] = a[2] = a[3] = 0ull;
}

// the relaxation's start for the systems still segmenting
__global__ void k_ms_prep(Batch b, const double *__restrict__ Bs, MsSys ms, MsBufs m)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= b.NV) return;
    const int s = sys_v(b, v);
    if (!ms.flag[2 * s]) return;
    ms_start_voxel(m, v, DMUL(Bs[v], b.sys[s].ms_inv_scale), ms.c[2 * s], ms.c[2 * s + 1]);
}

__global__ void k_ms_iter_sys(Batch b, MsSys ms, MsBufs m, int k, float tau, float sigma)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= b.NV) return;
    int s;
    const MsCell c = ms_cell(b, v, s);
    if (!ms.flag[2 * s]) return;
    ms_iter_voxel(c, v, m, k, tau, sigma, b.sys[s].ms_nuf);
}

// the round's labels and whether any changed
__global__ void k_ms_end(Batch b, MsSys ms, const float *u, uint8_t *S)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= b.NV) return;
    const int s = sys_v(b, v);
    if (!ms.flag[2 * s]) return;
    const uint8_t nl = u[v] > 0.5f ? 0 : 1;
    if (nl != S[v]) {
        S[v] = nl;
        if (!*(volatile int *)&ms.flag[2 * s + 1]) atomicOr(&ms.flag[2 * s + 1], 1);
    }
}

// a system whose labels repeated stops
__global__ void k_ms_check(Batch b, MsSys ms)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.M) return;
    if (!ms.flag[2 * s + 1]) ms.flag[2 * s] = 0;
}

static MsBufs ms_bufs(float *base, int64_t nv)
{
    MsBufs m;
    m.u = base;
    m.ub[0] = base + nv;
    m.ub[1] = base + 2 * nv;
    m.r = base + 3 * nv;
    m.p[0] = base + 4 * nv;
    m.p[1] = base + 7 * nv;
    m.ps = nv;
    return m;
}

int launch_ms_detect(dcm_handle *h)
{
    const Batch &b = h->b;
    cudaStream_t s = h->stream;
    const int64_t nv = b.NV;
    MsBufs m = ms_bufs(h->msbuf, nv);
    MsSys ms;
    ms.acc = h->msacc;
    ms.c = h->msc;
    ms.flag = h->msflag;
    const float tau = (float)ms_tau();
    const int iters = h->p.ms_iters > 0 ? h->p.ms_iters : 50;
    const int outer = h->p.ms_outer > 0 ? h->p.ms_outer : 1;
    const int vb = ms_blocks(nv), sb = (b.M + 127) / 128;
    // the sums of the K-means labels (every system starts segmenting; the
    // accumulators are left at zero by each round's begin)
    k_ms_start<<<sb, 128, 0, s>>>(b, ms);
    k_ms_sums<<<vb, MS_THREADS, 0, s>>>(b, h->Bs, h->S, ms);
    for (int round = 0; round < outer; ++round) {
        k_ms_begin<<<sb, 128, 0, s>>>(b, ms);
        k_ms_prep<<<vb, MS_THREADS, 0, s>>>(b, h->Bs, ms, m);
        for (int it = 0; it < iters; ++it)
            k_ms_iter_sys<<<vb, MS_THREADS, 0, s>>>(b, ms, m, it & 1, tau, tau);
        // (the last iteration wrote u; u-bar and the duals are not read)
        k_ms_end<<<vb, MS_THREADS, 0, s>>>(b, ms, m.u, h->S);
        k_ms_check<<<sb, 128, 0, s>>>(b, ms);
        if (round + 1 < outer) k_ms_sums<<<vb, MS_THREADS, 0, s>>>(b, h->Bs, h->S, ms);
    }
    return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "segmentation launch");
}

}  // namespace dcm

using namespace dcm;

extern "C" int dcm_ms_segment(dcm_handle *h, const double *rho, double c_l, double c_v, double nu,
                              int32_t iters, uint8_t *labels, double *u_out, int mem)
{
    if (!h || !rho || !labels) return fail(DCM_ERR_ARG, "null handle, image or labels");
    if (!(nu >= 0.0) || iters < 0) return fail(DCM_ERR_ARG, "need nu >= 0 and iters >= 0");
    if (mem != DCM_HOST && mem != DCM_DEVICE) return fail(DCM_ERR_ARG, "mem must be DCM_HOST or DCM_DEVICE");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    DCM_CHECK_CUDA(cudaStreamIsCapturing(h->stream, &cap));
    if (cap != cudaStreamCaptureStatusNone) return fail(DCM_ERR_STATE, "not callable during stream capture");
    MsCell c;
    c.nx = h->g.gd[0];
    c.ny = h->g.gd[1];
    c.nz = h->g.gd[2];
    c.v0 = 0;
    c.mx = h->g.div_gd[0];
    c.my = h->g.div_gd[1];
    const int64_t nvi = (int64_t)c.nx * c.ny * c.nz;
    const size_t nv = (size_t)nvi;
    // 10 floats per voxel for the iteration, then the image (double)
    const size_t bytes = sizeof(float) * 10 * nv + sizeof(double) * nv;
    void *vbuf = nullptr, *vS = nullptr;
    int rc = dev_alloc(h, &vbuf, bytes);
    if (rc == DCM_OK) rc = dev_alloc(h, &vS, nv);
    if (rc != DCM_OK) {
        if (vbuf) dev_free(h, vbuf, bytes);
        if (vS) dev_free(h, vS, nv);
        cudaStreamSynchronize(h->stream);
        return rc;
    }
    float *buf = (float *)vbuf;
    uint8_t *S = (uint8_t *)vS;
    cudaError_t e = cudaSuccess;
    MsBufs m = ms_bufs(buf, nvi);
    double *rh = (double *)(buf + 10 * nv);    // the image; after the start, u as double
    cudaStream_t s = h->stream;
    const cudaMemcpyKind in = mem == DCM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind out = mem == DCM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (e == cudaSuccess) e = cudaMemcpyAsync(rh, rho, sizeof(double) * nv, in, s);
    const int grid = ms_blocks(nvi);
    const float tau = (float)ms_tau();
    if (e == cudaSuccess) {
        k_ms_init<<<grid, MS_THREADS, 0, s>>>(nvi, rh, c_l, c_v, m);
        for (int it = 0; it < iters; ++it)
            k_ms_iter<<<grid, MS_THREADS, 0, s>>>(c, nvi, m, it & 1, tau, tau, (float)nu);
        k_ms_labels<<<grid, MS_THREADS, 0, s>>>(nvi, m.u, S, rh);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(labels, S, nv, out, s);
    if (e == cudaSuccess && u_out) e = cudaMemcpyAsync(u_out, rh, sizeof(double) * nv, out, s);
    dev_free(h, buf, bytes);
    dev_free(h, S, nv);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return fail_cuda(e, "segmentation", __FILE__, __LINE__);
    return DCM_OK;
}
