// dcm_ms.cu -- two-phase piecewise-constant Mumford-Shah segmentation (Eq. 13)
// with the densities fixed, on a voxel image: the convex relaxation of Chan,
// Esedoglu and Nikolova,
//     min over u in [0,1] of  sum_v u_v r_v + nu sum_faces |u_a - u_b|,
//     r_v = (rho_v - c_l)^2 - (rho_v - c_v)^2   (u = 1: liquid),
// solved by the first-order primal-dual iteration of Chambolle and Pock with
// one dual variable per grid face (|p| <= nu), tau = 1/4, sigma = 1/3, u from
// 1/2, a fixed number of iterations; liquid (s = 0) where u > 1/2.  The
// perimeter counts the periodic faces between liquid and vapor voxels, for
// which thresholded relaxed minimisers are exact minimisers of Eq. 13.
//
// Each iteration is two element-wise passes (the faces, then the voxels), in
// FP64 with round-to-nearest intrinsics in a fixed order and no reduction, so
// the result does not depend on the thread layout.  Bound: HBM (per voxel and
// iteration ~100 B: u-bar and the 3 face values read and written, u, r).
#include "dcm_device.cuh"

namespace dcm {

constexpr int MS_THREADS = 256;

struct MsGrid {
    int nx, ny, nz;
    int64_t nv;
};

__device__ __forceinline__ void ms_coords(const MsGrid &g, int64_t v, int &x, int &y, int &z)
{
    const int64_t t = v / g.nx;
    x = (int)(v - t * g.nx);
    y = (int)(t % g.ny);
    z = (int)(t / g.ny);
}

__global__ void k_ms_init(MsGrid g, const double *__restrict__ rho, double c_l, double c_v,
                          double *u, double *ub, double *r, double *p)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.nv) return;
    const double a = DSUB(rho[v], c_l), b = DSUB(rho[v], c_v);
    r[v] = DSUB(DMUL(a, a), DMUL(b, b));
    u[v] = 0.5;
    ub[v] = 0.5;
    p[3 * v] = 0.0;
    p[3 * v + 1] = 0.0;
    p[3 * v + 2] = 0.0;
}

// dual ascent on the three upper faces of each voxel, projected on |p| <= nu
__global__ void k_ms_dual(MsGrid g, const double *__restrict__ ub, double *p, double sigma,
                          double nu)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.nv) return;
    int x, y, z;
    ms_coords(g, v, x, y, z);
    const int n[3] = {g.nx, g.ny, g.nz};
    const int64_t up[3] = {v + (x + 1 < g.nx ? 1 : -(int64_t)(g.nx - 1)),
                           v + (y + 1 < g.ny ? (int64_t)g.nx : -(int64_t)(g.ny - 1) * g.nx),
                           v + (z + 1 < g.nz ? (int64_t)g.nx * g.ny
                                             : -(int64_t)(g.nz - 1) * g.nx * g.ny)};
    const double ubv = ub[v];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double q = n[a] > 1 ? DADD(p[3 * v + a], DMUL(sigma, DSUB(ub[up[a]], ubv))) : 0.0;
        if (q > nu) q = nu;
        if (q < -nu) q = -nu;
        p[3 * v + a] = q;
    }
}

// primal descent u -= tau (grad^T p + r), clipped to [0, 1], and the
// extrapolation u-bar = 2 u_new - u_old
__global__ void k_ms_primal(MsGrid g, const double *__restrict__ p, const double *__restrict__ r,
                            double *u, double *ub, double tau)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.nv) return;
    int x, y, z;
    ms_coords(g, v, x, y, z);
    const int64_t dn[3] = {v + (x > 0 ? -1 : (int64_t)(g.nx - 1)),
                           v + (y > 0 ? -(int64_t)g.nx : (int64_t)(g.ny - 1) * g.nx),
                           v + (z > 0 ? -(int64_t)g.nx * g.ny : (int64_t)(g.nz - 1) * g.nx * g.ny)};
    double gtp = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) gtp = DADD(gtp, DSUB(p[3 * dn[a] + a], p[3 * v + a]));
    const double uo = u[v];
    double un = DSUB(uo, DMUL(tau, DADD(gtp, r[v])));
    if (un < 0.0) un = 0.0;
    if (un > 1.0) un = 1.0;
    ub[v] = DSUB(DMUL(2.0, un), uo);
    u[v] = un;
}

__global__ void k_ms_labels(MsGrid g, const double *__restrict__ u, uint8_t *S)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.nv) return;
    S[v] = u[v] > 0.5 ? 0 : 1;
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
    MsGrid g;
    g.nx = h->g.gd[0];
    g.ny = h->g.gd[1];
    g.nz = h->g.gd[2];
    g.nv = (int64_t)g.nx * g.ny * g.nz;
    const size_t nv = (size_t)g.nv;
    double *buf = nullptr;
    uint8_t *S = nullptr;
    cudaError_t e = cudaMalloc((void **)&buf, sizeof(double) * 7 * nv);
    if (e == cudaSuccess) e = cudaMalloc((void **)&S, nv);
    if (e != cudaSuccess) {
        cudaFree(buf);
        cudaFree(S);
        return fail(DCM_ERR_OOM, "segmentation buffers");
    }
    double *u = buf, *ub = buf + nv, *r = buf + 2 * nv, *rh = buf + 3 * nv, *p = buf + 4 * nv;
    cudaStream_t s = h->stream;
    const cudaMemcpyKind in = mem == DCM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind out = mem == DCM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    e = cudaMemcpyAsync(rh, rho, sizeof(double) * nv, in, s);
    const unsigned grid = (unsigned)((g.nv + MS_THREADS - 1) / MS_THREADS);
    const double tau = 0.25, sigma = 1.0 / 3.0;
    if (e == cudaSuccess) {
        k_ms_init<<<grid, MS_THREADS, 0, s>>>(g, rh, c_l, c_v, u, ub, r, p);
        for (int it = 0; it < iters; ++it) {
            k_ms_dual<<<grid, MS_THREADS, 0, s>>>(g, ub, p, sigma, nu);
            k_ms_primal<<<grid, MS_THREADS, 0, s>>>(g, p, r, u, ub, tau);
        }
        k_ms_labels<<<grid, MS_THREADS, 0, s>>>(g, u, S);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(labels, S, nv, out, s);
    if (e == cudaSuccess && u_out) e = cudaMemcpyAsync(u_out, u, sizeof(double) * nv, out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(buf);
    cudaFree(S);
    if (e != cudaSuccess) return fail_cuda(e, "segmentation", __FILE__, __LINE__);
    return DCM_OK;
}
