// dcm_integrate.cu -- velocity Verlet (Eq. 1-2) and deterministic FP64
// reductions for energy, virial and pair counts.
//
// HBM bound: a kick-drift reads x, v, f (72 B/particle) and writes x, v
// (48 B); a kick reads v, f and writes v (48 + 24 B).
#include "dcm_device.cuh"

namespace dcm {

// v += dt/(2m) F;  x += dt v;  wrap into the box  (first half of a step).
// GB300 issues FP64 at 1/64 of the FP32 rate, so the update uses two fused
// multiply-adds per component and integer tests of the exponent bits.
// With sp4 given (warp Verlet-list kernels) the drift also refreshes the
// particle's FP32 cell-relative position and its remainder (spl4) at its
// sorted slot inv[i], in the cell of the last sort, so no gather pass is
// needed between list builds.
__global__ void k_kick_drift(Batch b, double *__restrict__ x, double *__restrict__ v,
                             const double *__restrict__ f, int *err, float4 *sp4, float4 *spl4,
                             const int32_t *__restrict__ inv, const int32_t *__restrict__ cell_of,
                             const double *__restrict__ rc, ListTest t, unsigned int *queues)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // the step's force work queues and refinement queue (a captured step
    // has no memset nodes)
    if (queues && i == 0) {
        queues[0] = 0u;
        queues[3] = 0u;
        queues[4] = 0u;
        queues[5] = 0u;
    }
    float mp = -3.0e38f, mq = -3.0e38f;
    if (i < b.N) {
        const Geom &g = b.sys[sys_p(b, i)];
        int bad = 0;
        double xn[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            size_t o = (size_t)a * b.N + i;
            double vi = fma(g.hdtm, f[o], v[o]);
            double xi = fma(g.dt, vi, x[o]);
            // non-finite: exponent bits all ones
            if (((__double_as_longlong(xi) >> 52) & 0x7ff) == 0x7ff ||
                ((__double_as_longlong(vi) >> 52) & 0x7ff) == 0x7ff)
                bad |= DEV_ERR_NONFINITE;
            if (!wrap_coord_bits(xi, g.L[a])) {   // moved more than one box edge
                bad |= DEV_ERR_JUMP;
                xi = 0.0;
            }
            v[o] = vi;
            x[o] = xi;
            xn[a] = xi;
        }
        if (bad) atomicOr(err, bad);
        float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
        if (sp4) {
            float4 lo;
            u = cell_rel_position(b, g, xn[0], xn[1], xn[2], cell_of[i] - (int)g.c0, lo);
            const int k = inv[i];
            sp4[k] = u;
            spl4[k] = lo;
        }
        if (t.lf) {
            // warp lists: the displacement from the FP32 cell-relative
            // positions (kept for the cutoff kernel's term); else in FP64
            float d;
            if (t.u_ref) {
                d = list_disp32(u, t.u_ref[i]);
                t.disp[i] = d;
            } else {
                d = list_disp(t, g, (size_t)b.N, i, xn[0], xn[1], xn[2]);
            }
            list_terms(t, i, d, t.excess ? rc[i] : 0.0, mp, mq);
        }
    }
    if (t.lf) list_test_block(t, mp, mq);
}

__global__ void k_iota(int32_t *p, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (int32_t)i;
}

// v += dt/(2m) F  (second half of a step)
__global__ void k_kick(Batch b, double *__restrict__ v, const double *__restrict__ f)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.N) return;
    const double hdtm = b.sys[sys_p(b, i)].hdtm;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        size_t o = (size_t)a * b.N + i;
        v[o] = fma(hdtm, f[o], v[o]);
    }
}

// ---- deterministic reductions -------------------------------------------
// Fixed partition (RED_BLOCKS contiguous chunks) and a fixed tree order in
// each block, so the result does not depend on scheduling.
constexpr int RED_BLOCKS = 256;
constexpr int RED_THREADS = 256;
constexpr int RED_VALUES = 8;   // pe, sum v^2, w_xx w_yy w_zz w_xy w_xz w_yz

// partial sums over the particles [p0, p0 + n) of one system
__global__ void k_reduce_energy_part(int64_t p0, int n, int64_t N, const double *__restrict__ pe,
                                     const double *__restrict__ vir,
                                     const double *__restrict__ v, double *part)
{
    __shared__ double s[RED_VALUES][RED_THREADS];
    int chunk = (n + RED_BLOCKS - 1) / RED_BLOCKS;
    int lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    pe += p0;
    vir += p0;
    v += p0;
    double acc[RED_VALUES];
#pragma unroll
    for (int q = 0; q < RED_VALUES; ++q) acc[q] = 0.0;
    for (int i = lo + threadIdx.x; i < hi; i += RED_THREADS) {
        acc[0] += pe[i];
        double vx = v[i], vy = v[(size_t)N + i], vz = v[2 * (size_t)N + i];
        acc[1] += vx * vx + vy * vy + vz * vz;
#pragma unroll
        for (int q = 0; q < 6; ++q) acc[2 + q] += vir[(size_t)q * N + i];
    }
#pragma unroll
    for (int q = 0; q < RED_VALUES; ++q) s[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < RED_VALUES; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < RED_VALUES) part[blockIdx.x * RED_VALUES + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void k_reduce_final(const double *part, int nvals, double *out)
{
    __shared__ double s[RED_BLOCKS];
    for (int q = 0; q < nvals; ++q) {
        s[threadIdx.x] = part[threadIdx.x * nvals + q];
        __syncthreads();
        for (int w = RED_BLOCKS / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[q] = s[0];
        __syncthreads();
    }
}

__global__ void k_reduce_pairs(int64_t n, const int32_t *__restrict__ npair,
                               unsigned long long *out)
{
    __shared__ unsigned long long s[RED_THREADS];
    unsigned long long acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc += (unsigned long long)npair[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, s[0]);   // integer: order-free
}

static inline int nblk(int64_t n, int b) { return (int)((n + b - 1) / b); }

int launch_kick_drift(dcm_handle *h)
{
    const bool wl = h->nl && h->list_warp;
    // a captured step with lists runs the reuse test here: all of it on a
    // step without detection, the displacement-share term on one with (the
    // cutoff kernel adds the headroom term for the new cutoffs and decides)
    ListTest t = list_test(h, true, !h->step_detect, !h->step_detect);
    if (!h->fold_check) t.lf = nullptr;
    k_kick_drift<<<nblk(h->n, 256), 256, 0, h->stream>>>(h->b, h->x, h->v, h->f, h->err,
                                                         wl ? h->sp4 : nullptr, h->spl4, h->inv,
                                                         h->cell_of,
                                                         h->rc, t,
                                                         h->in_step ? &h->stats->barrier[2] : nullptr);
    return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "kick_drift launch");
}

__global__ void k_sys_table(const int64_t *__restrict__ off, int M, int64_t n, uint16_t *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint16_t)sys_of(off, M, i);
}

// the system of every particle and voxel, once at creation
void launch_sys_tables(dcm_handle *h)
{
    const int M = h->M;
    k_sys_table<<<nblk(h->n, 256), 256, 0, h->stream>>>(h->off_dev, M, h->n, h->psys);
    k_sys_table<<<nblk(h->nvox, 256), 256, 0, h->stream>>>(h->off_dev + 2 * (M + 1), M, h->nvox,
                                                            h->vsys);
}

void launch_iota(dcm_handle *h, int32_t *p, int64_t n)
{
    k_iota<<<nblk(n, 256), 256, 0, h->stream>>>(p, n);
}

int launch_kick(dcm_handle *h)
{
    k_kick<<<nblk(h->n, 256), 256, 0, h->stream>>>(h->b, h->v, h->f);
    return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "kick launch");
}

// energy and virial of system k into red_out[8*k .. 8*k+8)
int launch_reduce_energy(dcm_handle *h, int k)
{
    const Geom &g = h->geo_host[k];
    k_reduce_energy_part<<<RED_BLOCKS, RED_THREADS, 0, h->stream>>>(g.p0, g.n, h->n, h->pe, h->vir,
                                                                  h->v, h->red_part);
    k_reduce_final<<<1, RED_BLOCKS, 0, h->stream>>>(h->red_part, RED_VALUES, h->red_out + 8 * k);
    return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "reduce launch");
}

int launch_reduce_pairs(dcm_handle *h)
{
    cudaMemsetAsync(&h->stats->pairs, 0, sizeof(unsigned long long), h->stream);
    k_reduce_pairs<<<RED_BLOCKS, RED_THREADS, 0, h->stream>>>(h->n, h->npair,
                                                             &h->stats->pairs);
    return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "reduce launch");
}

}  // namespace dcm
