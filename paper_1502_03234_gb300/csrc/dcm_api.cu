// dcm_api.cu -- the C ABI of libdcm (see include/dcm.h): handle life cycle,
// geometry, device allocation, state transfer, the CUDA-graph step loop and
// the diagnostic read-backs.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dcm_device.cuh"

// NVTX range around an entry point (for a host-side timeline in Nsight
// Systems; a no-op when no tool is attached)
namespace {
struct Trace {
    explicit Trace(const char *name) { nvtxRangePushA(name); }
    ~Trace() { nvtxRangePop(); }
    Trace(const Trace &) = delete;
    Trace &operator=(const Trace &) = delete;
};
}  // namespace

static thread_local char g_errmsg[512] = "";

namespace dcm {

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_errmsg, sizeof(g_errmsg), fmt, ap);
    va_end(ap);
    return code;
}

int fail_cuda(cudaError_t e, const char *what, const char *file, int line)
{
    (void)cudaGetLastError();
    int code = (e == cudaErrorMemoryAllocation) ? DCM_ERR_OOM : DCM_ERR_CUDA;
    return fail(code, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

// AoS [n][3] -> SoA slice [3][N] at particles p0 .. p0+n, wrapping positions
// into their system's box
__global__ void k_aos_to_soa(Batch b, int64_t p0, int64_t n, const double *__restrict__ in,
                             double *out, int wrap)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Geom &g = b.sys[sys_p(b, p0 + i)];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double v = in[3 * i + a];
        if (wrap) {
            double L = g.L[a];
            if (v < 0.0 || v >= L) v = DSUB(v, DMUL(L, floor(__ddiv_rn(v, L))));
            v = wrap_coord(v, L);
            if (!(v >= 0.0 && v < L)) v = 0.0;
        }
        out[(size_t)a * b.N + p0 + i] = v;
    }
}

__global__ void k_soa_to_aos(int64_t N, int64_t p0, int64_t n, const double *__restrict__ in,
                             double *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int a = 0; a < 3; ++a) out[3 * i + a] = in[(size_t)a * N + p0 + i];
}

static inline int nblk(int64_t n, int b) { return (int)((n + b - 1) / b); }

}  // namespace dcm

using namespace dcm;

// ---------------------------------------------------------------------------
extern "C" void dcm_default_params(dcm_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->rc_min = 3.0;
    p->rc_max = 6.0;
    p->alpha = -0.5;
    p->dt = 0.005;
    p->mass = 1.0;
    p->eps = 1.0;
    p->sigma = 1.0;
    p->voxel = 1.0;
    p->smooth_order = 8;
    p->detect_every = 2;
    p->kmeans_max_iter = 100;
    p->cfsm_iter_max = 0;
    p->list_density = 1.0f;
    p->list_margin = 1.0f;
    p->cfsm_eps = 0.0;
    p->precision = DCM_FP64;
    p->n_classes = 4;
    p->cell_min = 0.0;
    p->segmentation = DCM_SEG_KMEANS;
    p->ms_iters = 50;
    p->ms_outer = 1;
    p->ms_nu = 0.005;
}

extern "C" const char *dcm_last_error(void) { return g_errmsg; }
extern "C" int dcm_version(void) { return DCM_ABI_VERSION; }

static int check_params(const dcm_box *box, int64_t n, const dcm_params *p)
{
    if (!box || !p) return fail(DCM_ERR_ARG, "null box or params");
    if (n < 1 || n > (int64_t)0x7fffffff / 4) return fail(DCM_ERR_ARG, "n out of range: %lld", (long long)n);
    if (!(box->lx > 0 && box->ly > 0 && box->lz > 0)) return fail(DCM_ERR_ARG, "box edges must be > 0");
    if (!(p->rc_min > 0 && p->rc_max >= p->rc_min)) return fail(DCM_ERR_ARG, "need 0 < rc_min <= rc_max");
    if (!(p->alpha < 0)) return fail(DCM_ERR_ARG, "alpha must be negative (Eq. 7)");
    if (!(p->dt > 0 && p->mass > 0 && p->eps > 0 && p->sigma > 0))
        return fail(DCM_ERR_ARG, "dt, mass, eps, sigma must be > 0");
    if (!(p->voxel > 0)) return fail(DCM_ERR_ARG, "voxel must be > 0");
    if (p->smooth_order < 0 || p->smooth_order > 12 || (p->smooth_order & 1))
        return fail(DCM_ERR_ARG, "smooth_order must be even, 0..12");
    if (p->precision != DCM_FP64 && p->precision != DCM_MIXED)
        return fail(DCM_ERR_ARG, "precision must be DCM_FP64 or DCM_MIXED");
    if (p->n_classes < 2 || p->n_classes > DCM_MAX_CLASSES)
        return fail(DCM_ERR_ARG, "n_classes must be 2..%d", DCM_MAX_CLASSES);
    if (p->detect_every < 0) return fail(DCM_ERR_ARG, "detect_every must be >= 0");
    if (!(p->skin >= 0) || p->skin > 2.0) return fail(DCM_ERR_ARG, "skin must be in [0, 2] sigma");
    // (the shares only matter with lists)
    if (!(p->skin_time >= 0.f) || !(p->skin_floor >= 0.f) ||
        (p->skin > 0 && p->skin_time > 0.f && p->skin_floor > 0.5 * p->skin))
        return fail(DCM_ERR_ARG, "skin_time, skin_floor must be >= 0, skin_floor <= skin/2");
    if (p->min_component_voxels < 0) return fail(DCM_ERR_ARG, "min_component_voxels must be >= 0");
    if (p->segmentation != DCM_SEG_KMEANS && p->segmentation != DCM_SEG_MUMFORD_SHAH)
        return fail(DCM_ERR_ARG, "segmentation must be DCM_SEG_KMEANS or DCM_SEG_MUMFORD_SHAH");
    if (!(p->ms_nu >= 0) || p->ms_iters > 100000 || p->ms_outer > 1000)
        return fail(DCM_ERR_ARG, "need ms_nu >= 0, ms_iters <= 100000, ms_outer <= 1000");
    if (p->cutoff_fn != DCM_CUTOFF_EXP && p->cutoff_fn != DCM_CUTOFF_LINEAR)
        return fail(DCM_ERR_ARG, "cutoff_fn must be DCM_CUTOFF_EXP or DCM_CUTOFF_LINEAR");
    return DCM_OK;
}

// geometry of the system (same definitions as the FP64 reference: bins of
// edge L/n with index min(n-1, floor(x * n/L)), Eq. 7-8 constants)
static int setup_geometry(const dcm_box *box, int64_t n, const dcm_params *p, Geom &g)
{
    memset(&g, 0, sizeof(g));
    g.n = (int)n;
    double L[3] = {box->lx, box->ly, box->lz};
    double target = p->cell_min > 0 ? p->cell_min : 0.5 * p->rc_min;
    double reach = p->rc_max + (p->skin > 0 ? p->skin : 0.0);   // Verlet lists reach r_c + skin
    double rcull = reach * 1.00002 + 1e-4;
    bool ok = false;
    for (int tries = 0; tries < 64 && target >= 0.25; ++tries, target *= 0.9) {
        ok = true;
        for (int a = 0; a < 3; ++a) {
            int nc = (int)floor(L[a] / target);
            nc = nc < 1 ? 1 : nc;
            double inv = (double)nc / L[a];
            int s = (int)ceil(rcull * inv);
            if (2 * s + 1 > nc) ok = false;
            g.nc[a] = nc;
            g.inv_c[a] = inv;
            g.cedge[a] = L[a] / nc;
            g.smax[a] = s;
        }
        if (ok) break;
    }
    if (!ok)
        return fail(DCM_ERR_BOX_TOO_SMALL,
                    "box too small for rc_max=%g: each edge must exceed 2*rc_max plus a few link cells",
                    p->rc_max);
    for (int a = 0; a < 3; ++a) {
        g.L[a] = L[a];
        g.halfL[a] = 0.5 * L[a];
        g.halfLf[a] = (float)g.halfL[a];
        g.inv_cf[a] = (float)g.inv_c[a];
        int gd = (int)floor(L[a] / p->voxel);
        g.gd[a] = gd < 3 ? 3 : gd;
        g.inv_h[a] = (double)g.gd[a] / L[a];
        g.h[a] = L[a] / g.gd[a];
    }
    double hmax = fmax(g.h[0], fmax(g.h[1], g.h[2]));
    g.r_grid = p->rc_max + hmax;
    // the same expression as the oracle's: voxel volume from the three
    // quotients L / n, scaled by the smoothing mass 2^(3 order)
    {
        const double V = (L[0] / g.gd[0]) * (L[1] / g.gd[1]) * (L[2] / g.gd[2]);
        g.ms_inv_scale = 1.0 / ldexp(V, 3 * (p->smooth_order > 0 ? p->smooth_order : 0));
    }
    // q = floor(n / d) = high word of n * ceil(2^64 / d) for every 32-bit n
    // (the product's error n (ceil(2^64/d) - 2^64/d) / 2^64 stays below 1/d)
    for (int a = 0; a < 2; ++a) g.div_gd[a] = ~0ull / (unsigned long long)g.gd[a] + 1ull;
    for (int a = 0; a < 3; ++a) g.w_h[a] = 1.0 / (g.h[a] * g.h[a]);
    g.e_min = 1.0 / sqrt(g.w_h[0] + g.w_h[1] + g.w_h[2]);
    g.rc_min = p->rc_min;
    g.rc_max = p->rc_max;
    g.alpha = p->alpha;
    g.K = p->n_classes;
    g.cut_fn = p->cutoff_fn;
    g.cut_slope = 0.0;
    if (p->rc_max > p->rc_min && p->cutoff_fn == DCM_CUTOFF_LINEAR) {
        // Fig. 12's line; the class edges invert it
        g.cut_a = 0.0;
        g.cut_b = p->rc_min;
        g.cut_slope = (p->rc_max - p->rc_min) / p->rc_max;
        for (int k = 1; k <= g.K - 2; ++k) {
            double r = p->rc_min + (p->rc_max - p->rc_min) * (double)k / (double)(g.K - 1);
            g.thr[k - 1] = (p->rc_max - r) * p->rc_max / (p->rc_max - p->rc_min);
        }
    } else if (p->rc_max > p->rc_min) {
        g.cut_fn = DCM_CUTOFF_EXP;
        g.cut_a = (p->rc_max - p->rc_min) / (pow(2.0, p->alpha * p->rc_max) - 1.0);
        g.cut_b = p->rc_min - g.cut_a;
        for (int k = 1; k <= g.K - 2; ++k) {
            double r = p->rc_min + (p->rc_max - p->rc_min) * (double)k / (double)(g.K - 1);
            g.thr[k - 1] = p->rc_max - log2((r - g.cut_b) / g.cut_a) / p->alpha;
        }
    } else {
        g.cut_fn = DCM_CUTOFF_EXP;
        g.cut_a = 0.0;
        g.cut_b = p->rc_min;
        for (int k = 1; k <= g.K - 2; ++k) g.thr[k - 1] = 0.0;
    }
    g.dt = p->dt;
    g.hdtm = 0.5 * p->dt / p->mass;
    g.eps = p->eps;
    g.sigma = p->sigma;
    g.skin = p->skin > 0 ? p->skin : 0.0;
    g.skin_time = p->skin_time;
    g.skin_floor = p->skin_floor;
    g.cc_min = p->min_component_voxels;
    g.ms_nu = p->ms_nu;
    g.ms_nuf = (float)p->ms_nu;
    g.ms_seg = p->segmentation == DCM_SEG_MUMFORD_SHAH ? 1 : 0;
    g.eps24 = 24.0 * p->eps;
    g.eps48 = 48.0 * p->eps;
    g.eps2 = 2.0 * p->eps;
    g.sig2 = p->sigma * p->sigma;
    g.eps24f = (float)g.eps24;
    g.eps48f = (float)g.eps48;
    g.eps2f = (float)g.eps2;
    g.sig2f = (float)g.sig2;
    g.eps24l = (float)(g.eps24 - (double)g.eps24f);
    g.eps48l = (float)(g.eps48 - (double)g.eps48f);
    g.sig2l = (float)(g.sig2 - (double)g.sig2f);
    // Mixed precision: pairs closer than 1.5 sigma, whose forces are large
    // and change fast with r, take the double-float path.  The FP32
    // cell-relative positions live on a grid qpos = 2^(e - 24) with 2^e above
    // every coordinate (a cell edge plus the drift allowed between list
    // builds) and every close-pair distance, so these have at most 24
    // significant bits: a close pair's cell shift is then exact in FP32, and
    // the rounding of its coordinate difference is recovered by TwoSum.
    const double rclose = 1.5 * p->sigma;
    g.rclose2 = (float)(rclose * rclose);
    // The FP32 error left by the pairs beyond r_close is at most a few 1e-6
    // epsilon/sigma at liquid density; a particle whose net force is below
    // 0.5 epsilon/sigma (where the tolerance 1e-6 + 1e-5 |F| falls under
    // 6e-6) has all its pairs evaluated again in double-float.
    const double fredo = 0.5 * p->eps / p->sigma;
    g.redo_f2 = (float)(fredo * fredo);
    double cmax = fmax(g.cedge[0], fmax(g.cedge[1], g.cedge[2]));
    double bound = fmax(cmax + 0.5 * g.skin, rclose);
    int e = (int)ceil(log2(bound));
    g.qpos = (float)ldexp(1.0, e - 24);
    g.inv_qpos = (float)ldexp(1.0, 24 - e);
    g.qtop = (float)ldexp(1.0, e);
    for (int a = 0; a < 3; ++a) {
        double cq = nearbyint(g.cedge[a] * (double)g.inv_qpos) * (double)g.qpos;
        g.cf[a] = (float)cq;   // exact: below 2^24 grid steps
        g.cfl[a] = (float)(g.cedge[a] - cq);
    }
    g.ncell = (int64_t)g.nc[0] * g.nc[1] * g.nc[2];
    for (int a = 0; a < 2; ++a) g.div_nc[a] = ~0ull / (unsigned long long)g.nc[a] + 1ull;
    g.nvox = (int64_t)g.gd[0] * g.gd[1] * g.gd[2];
    if (g.nvox > INT32_MAX)
        return fail(DCM_ERR_ARG, "voxel grid of %lld voxels: at most 2^31 - 1 per system (raise voxel)",
                    (long long)g.nvox);
    return DCM_OK;
}

// Verlet-list entries reserved for one system: every particle may hold
// the neighbours of a sphere of r_c,max + skin, but no more than three times
// those of r_c,min + skin (bulk particles are the vast majority), at a
// density bound of 1.0, plus the 15 entries of slack and the rounding up to
// 8 that each particle's own capacity adds (without them a box of uniform
// cutoff at liquid density asks for more than this and never keeps a list)
static int64_t list_cap(const Geom &g, int64_t n)
{
    if (g.skin <= 0) return 0;
    const double c43pi = 4.18879020478639;
    double big = c43pi * pow(g.rc_max + g.skin, 3.0);
    double small = 3.0 * c43pi * pow(g.rc_min + g.skin, 3.0);
    return n * ((int64_t)ceil(big < small ? big : small) + 23) + 1024;
}

// the small-component buffers (5 ints per voxel and a flag per tile) and the
// systems' tile offsets, on creation with min_component_voxels or on first use
template <typename T>
static int dalloc(dcm_handle *h, T **ptr, int64_t count);

static int cc_setup(dcm_handle *h)
{
    if (h->cc) return DCM_OK;
    if (h->b.NV > 0x7fffffffLL) return fail(DCM_ERR_ARG, "small-component removal indexes at most 2^31 voxels");
    std::vector<int64_t> off(h->M + 1, 0);
    for (int k = 0; k < h->M; ++k) {
        const Geom &g = h->geo_host[k];
        off[k + 1] = off[k] + (int64_t)((g.gd[0] + 7) / 8) * ((g.gd[1] + 7) / 8) * ((g.gd[2] + 7) / 8);
    }
    int rc;
    if ((rc = dalloc(h, &h->cc, 5 * h->b.NV + off[h->M]))) return rc;
    if ((rc = dalloc(h, &h->cc_tiles, (int64_t)h->M + 1))) return rc;
    DCM_CHECK_CUDA(cudaMemcpyAsync(h->cc_tiles, off.data(), sizeof(int64_t) * (h->M + 1),
                                   cudaMemcpyHostToDevice, h->stream));
    DCM_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    h->cc_ntiles = off[h->M];
    h->cc_ntiles0 = off[1];
    return DCM_OK;
}

static int64_t bytes_for(const Geom &g, int64_t n, int precision)
{
    int64_t ncell = g.ncell;
    int64_t nv = g.nvox;
    int64_t per_p = 3 * 8 * 3 + 8 + 8 + 1 + 4 * 3 + 16 + 4 + 4 + 8 + 48 + 24 + 2;
    per_p += precision == DCM_FP64 ? 36 : 56;   // spd (FP64) or spl4 + refq + rq + pk + inv (MIXED)
    int64_t per_v = 4 + 4 + 4 + 8 + 1 + 8 + 8 + 4 + 16 + 2 + (g.cc_min > 0 ? 20 : 0) +
                    (g.ms_seg ? 40 : 0);
    int64_t ntiles = (ncell + 2047) / 2048 + 1;
    int64_t lists = g.skin > 0 ? 4 * list_cap(g, n) + n * (4 + 4 + 24 + 8 + 8 + 20) : 0;
    return n * per_p + ncell * 8 + 8 + nv * per_v + ntiles * 4 + 4096 + 256 * 8 * 8 +
           8 * 1024 * 8 + lists;
}

extern "C" int64_t dcm_estimate_bytes(const dcm_box *box, int64_t n, const dcm_params *p)
{
    if (check_params(box, n, p)) return -1;
    Geom g;
    if (setup_geometry(box, n, p, g)) return -1;
    return bytes_for(g, n, p->precision);
}

// the allocator new handles take (process-wide; each handle keeps a copy)
static std::mutex g_alloc_mu;
static dcm_alloc_fn g_alloc = nullptr;
static dcm_release_fn g_release = nullptr;
static void *g_alloc_ctx = nullptr;

extern "C" int dcm_set_allocator(dcm_alloc_fn alloc, dcm_release_fn release, void *ctx)
{
    if ((alloc == nullptr) != (release == nullptr))
        return fail(DCM_ERR_ARG, "give both allocator functions or neither");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_release = release;
    g_alloc_ctx = ctx;
    return DCM_OK;
}

static void take_allocator(dcm_handle *h)
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    h->alloc = g_alloc;
    h->release = g_release;
    h->alloc_ctx = g_alloc_ctx;
}

// device buffers in the stream order of the handle's stream
template <typename T>
static int dalloc(dcm_handle *h, T **ptr, int64_t count)
{
    size_t b = sizeof(T) * (size_t)(count > 0 ? count : 1);
    if (h->alloc) {
        *ptr = (T *)h->alloc(b, (void *)h->stream, h->alloc_ctx);
        if (!*ptr) return fail(DCM_ERR_OOM, "the caller's allocator returned no memory (%zu bytes)", b);
    } else {
        cudaError_t e = cudaMallocAsync((void **)ptr, b, h->stream);
        if (e != cudaSuccess) {
            *ptr = nullptr;
            return fail_cuda(e, "cudaMallocAsync", __FILE__, __LINE__);
        }
    }
    h->bytes += (int64_t)b;
    return DCM_OK;
}

static void dfree(dcm_handle *h, void *p)
{
    if (!p) return;
    if (h->release)
        h->release(p, (void *)h->stream, h->alloc_ctx);
    else
        cudaFreeAsync(p, h->stream);
}

namespace dcm {
// scratch of an entry point outside the step (the same allocator)
int dev_alloc(dcm_handle *h, void **p, size_t bytes)
{
    char *q = nullptr;
    int rc = dalloc(h, &q, (int64_t)bytes);
    *p = q;
    return rc;
}
void dev_free(dcm_handle *h, void *p, size_t bytes)
{
    dfree(h, p);
    h->bytes -= (int64_t)(bytes > 0 ? bytes : 1);
}
}  // namespace dcm

extern "C" int dcm_destroy(dcm_handle *h)
{
    if (!h) return DCM_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->g_plain) cudaGraphExecDestroy(h->g_plain);
    if (h->g_detect) cudaGraphExecDestroy(h->g_detect);
    for (int q = 0; q <= DCM_NUM_PHASES; ++q)
        if (h->ev[q]) cudaEventDestroy(h->ev[q]);
    void *ptrs[] = {h->x, h->v, h->f, h->d, h->rc, h->cls, h->cell_of, h->slot, h->cell_count,
                    h->cell_start, h->sorted_id, h->scan_tmp, h->sp4, h->spl4, h->refq, h->spd, h->rq, h->pk, h->inv, h->psys, h->vsys, h->class_list,
                    h->class_count_dev, h->B, h->sm1, h->sm2, h->Bs, h->S, h->D0, h->D1, h->stamp,
                    h->flist, h->fcount, h->kacc, h->npair, h->pe, h->vir, h->red_part, h->red_out,
                    h->err, h->stats, h->tmp3n, h->geo_dev, h->off_dev, h->nl, h->nl_cnt,
                    h->nl_start, h->nl_tiles, h->x_ref, h->rl_ref, h->sh_ref, h->sh, h->u_ref,
                    h->disp, h->corner, h->lflags, h->cc, h->cc_tiles,
                    h->msbuf, h->msacc, h->msc, h->msflag};
    if (h->stream) {
        for (void *q : ptrs) dfree(h, q);
        cudaStreamSynchronize(h->stream);
    }
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    if (h->side) cudaStreamDestroy(h->side);
    delete[] h->geo_host;
    delete[] h->corner_host;
    delete[] h->par_host;
    delete[] h->off_host;
    delete h;
    return DCM_OK;
}

// one creation path for M >= 1 systems; the shared run-time fields
// (precision, detection cadence and caps, classes, smoothing) come from
// system 0's parameters and must agree across systems
static int create_systems(int M, const dcm_box *boxes, const int64_t *ns, const dcm_params *ps,
                          void *stream, dcm_handle **out)
{
    if (!out) return fail(DCM_ERR_ARG, "null out");
    *out = nullptr;
    if (M < 1 || M > MAX_SYSTEMS) return fail(DCM_ERR_ARG, "system count must be 1..%d", MAX_SYSTEMS);
    if (!boxes || !ns || !ps) return fail(DCM_ERR_ARG, "null boxes, sizes or params");
    int64_t ntot = 0;
    for (int k = 0; k < M; ++k) {
        int rc = check_params(&boxes[k], ns[k], &ps[k]);
        if (rc) return rc;
        const dcm_params &a = ps[0], &q = ps[k];
        if (q.precision != a.precision || q.detect_every != a.detect_every ||
            q.n_classes != a.n_classes || q.smooth_order != a.smooth_order ||
            q.segmentation != a.segmentation || q.ms_iters != a.ms_iters ||
            q.ms_outer != a.ms_outer)
            return fail(DCM_ERR_ARG, "system %d: precision, detect_every, n_classes, "
                                     "smooth_order, segmentation, ms_iters and ms_outer must "
                                     "match system 0", k);
        ntot += ns[k];
    }
    if (ntot > (int64_t)0x7fffffff / 4) return fail(DCM_ERR_ARG, "too many particles in total");
    dcm_handle *h = new dcm_handle();
    memset((void *)h, 0, sizeof(*h));
    h->M = M;
    h->box = boxes[0];
    h->n = ntot;
    h->p = ps[0];
    if (h->p.kmeans_max_iter <= 0) h->p.kmeans_max_iter = 100;
    h->geo_host = new Geom[M];
    h->par_host = new dcm_params[M];
    h->off_host = new int64_t[3 * (M + 1)];
    int64_t *po = h->off_host, *co = po + (M + 1), *vo = co + (M + 1);
    po[0] = co[0] = vo[0] = 0;
    for (int k = 0; k < M; ++k) {
        h->par_host[k] = ps[k];
        int rc = setup_geometry(&boxes[k], ns[k], &ps[k], h->geo_host[k]);
        if (rc) {
            dcm_destroy(h);
            return rc;
        }
        Geom &g = h->geo_host[k];
        g.K = ps[0].n_classes;
        g.p0 = po[k];
        g.c0 = co[k];
        g.v0 = vo[k];
        po[k + 1] = po[k] + ns[k];
        co[k + 1] = co[k] + g.ncell;
        vo[k + 1] = vo[k] + g.nvox;
    }
    // cell corner coordinates c * L/n of every axis and system (IEEE
    // products, the same on the host as on the device)
    int64_t ncorner = 0;
    for (int k = 0; k < M; ++k) {
        Geom &g = h->geo_host[k];
        g.corner_off = ncorner;
        ncorner += (int64_t)g.nc[0] + g.nc[1] + g.nc[2];
    }
    h->corner_host = new double[ncorner];
    for (int k = 0; k < M; ++k) {
        const Geom &g = h->geo_host[k];
        double *c = h->corner_host + g.corner_off;
        for (int a = 0, o = 0; a < 3; o += g.nc[a], ++a)
            for (int q = 0; q < g.nc[a]; ++q) c[o + q] = (double)q * g.cedge[a];
    }
    if (co[M] > (int64_t)0x7fffffff - 2 || vo[M] > (int64_t)0x7fffffff / 4) {
        dcm_destroy(h);
        return fail(DCM_ERR_ARG, "too many cells or voxels in total");
    }
    h->g = h->geo_host[0];
    // default launch shape of the FP64 lanes walk: 16 lanes per particle for
    // the lower half of the cutoff classes, 32 for the upper (measured on
    // slabs of 4k-262k atoms: 1.1-8x faster than 1-2 lanes, whose few
    // threads leave small systems latency-bound)
    for (int q = 0; q < DCM_MAX_CLASSES; ++q) h->tune.lanes[q] = 2 * q < h->p.n_classes ? 16 : 32;
    h->tune.block = 128;
    h->tune.walk = DCM_WALK_WARP;
    h->tune.list_lanes = 8;
    cudaGetDevice(&h->device);
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (stream) {
        h->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            dcm_destroy(h);
            return fail_cuda(e, "cudaStreamCreate", __FILE__, __LINE__);
        }
        h->own_stream = true;
    }
    take_allocator(h);
    h->ncell = co[M];
    h->nvox = vo[M];
    int64_t N = ntot, nc = h->ncell, nv = h->nvox;
    int64_t ntiles = (nc + 2047) / 2048 + 1;
    int rc;
#define ALLOC(ptr, cnt)                 \
    if ((rc = dalloc(h, &(ptr), (cnt)))) { \
        dcm_destroy(h);                 \
        return rc;                      \
    }
    ALLOC(h->geo_dev, M);
    ALLOC(h->off_dev, 3 * (M + 1));
    ALLOC(h->corner, ncorner);
    ALLOC(h->x, 3 * N);
    ALLOC(h->v, 3 * N);
    ALLOC(h->f, 3 * N);
    ALLOC(h->tmp3n, 3 * N);
    ALLOC(h->d, N);
    ALLOC(h->rc, N);
    ALLOC(h->cls, N);
    ALLOC(h->cell_of, N);
    ALLOC(h->slot, N);
    ALLOC(h->sorted_id, N);
    ALLOC(h->cell_count, nc);
    ALLOC(h->cell_start, nc + 1);
    ALLOC(h->scan_tmp, ntiles);
    ALLOC(h->sp4, N);
    if (h->p.precision == DCM_FP64) ALLOC(h->spd, N);
    if (M > 1) {
        ALLOC(h->psys, N);
        ALLOC(h->vsys, nv);
    }
    if (h->p.precision != DCM_FP64) {
        ALLOC(h->spl4, N);
        ALLOC(h->refq, N);
        ALLOC(h->rq, N);
        ALLOC(h->pk, N);
        ALLOC(h->inv, N);
    }
    ALLOC(h->class_list, N);
    ALLOC(h->class_count_dev, 3 * DCM_MAX_CLASSES);
    ALLOC(h->B, nv);
    ALLOC(h->sm1, nv);
    ALLOC(h->sm2, nv);
    ALLOC(h->Bs, nv);
    ALLOC(h->S, nv);
    ALLOC(h->D0, nv);
    ALLOC(h->D1, nv);
    ALLOC(h->stamp, nv);
    ALLOC(h->flist, 4 * nv);
    for (int k = 0; k < M; ++k) h->cc_on = h->cc_on || h->geo_host[k].cc_min > 0;
    ALLOC(h->fcount, 4);
    // K-means sums, 16 spread slots each, then the single-system kernel's
    // per-block partials (8 x 1024)
    ALLOC(h->kacc, 9 * 16 * (int64_t)M + 8 * 1024);
    if (h->p.segmentation == DCM_SEG_MUMFORD_SHAH) {
        ALLOC(h->msbuf, 10 * nv);
        ALLOC(h->msacc, 4 * (int64_t)M);
        ALLOC(h->msc, 2 * (int64_t)M);
        ALLOC(h->msflag, 2 * (int64_t)M);
    }
    ALLOC(h->npair, N);
    ALLOC(h->pe, N);
    ALLOC(h->vir, 6 * N);
    ALLOC(h->red_part, 256 * 8);
    ALLOC(h->red_out, 8 * (int64_t)M);
    ALLOC(h->err, 1);
    ALLOC(h->stats, 1);
    bool lists = false;
    int64_t cap = 0;
    for (int k = 0; k < M; ++k) {
        cap += list_cap(h->geo_host[k], ns[k]);
        lists = lists || h->geo_host[k].skin > 0;
    }
    if (lists) {
        for (int k = 0; k < M; ++k)
            if (h->geo_host[k].skin <= 0 || h->geo_host[k].smax[1] > 7 || h->geo_host[k].smax[2] > 7) {
                dcm_destroy(h);
                return fail(DCM_ERR_ARG, "system %d: Verlet lists need skin > 0 in every system "
                                         "and a stencil of at most 7 cells in y and z", k);
            }
        if (N >= (1 << 24)) {
            dcm_destroy(h);
            return fail(DCM_ERR_ARG, "Verlet lists hold at most 2^24 particles per handle");
        }
        if (cap > 0x7fffffffLL) {
            dcm_destroy(h);
            return fail(DCM_ERR_ARG, "Verlet lists need %lld entries, above the 2^31 a handle "
                                     "can index: fewer particles or a smaller skin", (long long)cap);
        }
        h->nl_cap = cap;
        ALLOC(h->nl, cap);
        ALLOC(h->nl_cnt, N);
        ALLOC(h->nl_start, N + 1);
        ALLOC(h->nl_tiles, (N + 2047) / 2048 + 1);
        ALLOC(h->x_ref, 3 * N);
        ALLOC(h->rl_ref, N);
        ALLOC(h->sh_ref, N);
        ALLOC(h->sh, N);
        ALLOC(h->u_ref, N);
        ALLOC(h->disp, N);
        ALLOC(h->lflags, LF_WORDS);
    }
#undef ALLOC
    h->b.sys = h->geo_dev;
    h->b.p_off = h->off_dev;
    h->b.c_off = h->off_dev + (M + 1);
    h->b.v_off = h->off_dev + 2 * (M + 1);
    h->b.psys = h->psys;
    h->b.vsys = h->vsys;
    h->b.corner = h->corner;
    h->b.M = M;
    h->b.K = h->p.n_classes;
    h->b.N = N;
    h->b.NC = nc;
    h->b.NV = nv;
    if (h->cc_on && (rc = cc_setup(h))) {       // small-component buffers (Section 4.2)
        dcm_destroy(h);
        return rc;
    }
    cudaMemcpyAsync(h->geo_dev, h->geo_host, sizeof(Geom) * M, cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(h->corner, h->corner_host, sizeof(double) * ncorner, cudaMemcpyHostToDevice,
                    h->stream);
    cudaMemcpyAsync(h->off_dev, h->off_host, sizeof(int64_t) * 3 * (M + 1), cudaMemcpyHostToDevice,
                    h->stream);
    cudaMemsetAsync(h->err, 0, sizeof(int), h->stream);
    cudaMemsetAsync(h->stats, 0, sizeof(DevStats), h->stream);
    cudaMemsetAsync(h->v, 0, sizeof(double) * 3 * N, h->stream);
    cudaMemsetAsync(h->f, 0, sizeof(double) * 3 * N, h->stream);
    cudaMemsetAsync(h->cls, 0, N, h->stream);
    cudaMemsetAsync(h->cell_count, 0, sizeof(int32_t) * nc, h->stream);
    if (h->inv) launch_iota(h, h->inv, N);       // a valid permutation before the first sort
    if (M > 1) launch_sys_tables(h);
    if (h->nl) {
        cudaMemsetAsync(h->lflags, 0, sizeof(int) * LF_WORDS, h->stream);
        cudaMemsetAsync(h->lflags + LF_EXCESS, 0x80, sizeof(int), h->stream);    // LF_EXCESS_RESET
        cudaMemsetAsync(h->lflags + LF_PARTNER, 0x80, sizeof(int), h->stream);
        // capacity density of the warp list fill (float bits); a host member
        // so the asynchronous copy reads live memory
        h->list_scale0 = h->par_host[0].list_density > 0.f ? h->par_host[0].list_density : 1.0f;
        const float lm = h->par_host[0].list_margin;
        h->list_margin = lm > 0.f ? lm : (lm < 0.f ? 0.f : 1.0f);
        cudaMemcpyAsync(h->lflags + LF_SCALE, &h->list_scale0, sizeof(float), cudaMemcpyHostToDevice,
                        h->stream);
        // every entry a valid slot from the start (entries past a list's
        // count are never read, but stay harmless if they were)
        cudaMemsetAsync(h->nl, 0, sizeof(int32_t) * h->nl_cap, h->stream);
        cudaMemsetAsync(h->x_ref, 0, sizeof(double) * 3 * N, h->stream);
        cudaMemsetAsync(h->rl_ref, 0, sizeof(float) * N, h->stream);
        cudaMemsetAsync(h->sh_ref, 0, sizeof(float) * N, h->stream);
        cudaMemsetAsync(h->sh, 0, sizeof(float) * N, h->stream);
        cudaMemsetAsync(h->u_ref, 0, sizeof(float4) * N, h->stream);
        cudaMemsetAsync(h->disp, 0, sizeof(float) * N, h->stream);
    }
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        dcm_destroy(h);
        return fail_cuda(e, "create sync", __FILE__, __LINE__);
    }
    rc = prepare_kernels(h);
    if (rc) {
        dcm_destroy(h);
        return rc;
    }
    *out = h;
    return DCM_OK;
}

extern "C" int dcm_create(const dcm_box *box, int64_t n, const dcm_params *p, void *stream,
                          dcm_handle **out)
{
    Trace trace("dcm_create");
    if (!box || !p) return fail(DCM_ERR_ARG, "null box or params");
    return create_systems(1, box, &n, p, stream, out);
}

extern "C" int dcm_ensemble_create(int count, const dcm_box *boxes, const int64_t *n,
                                   const dcm_params *params, void *stream, dcm_handle **out)
{
    Trace trace("dcm_ensemble_create");
    return create_systems(count, boxes, n, params, stream, out);
}

extern "C" int dcm_system_count(const dcm_handle *h) { return h ? h->M : 0; }

extern "C" int dcm_system_range(const dcm_handle *h, int k, int64_t *first, int64_t *count)
{
    if (!h || k < 0 || k >= h->M) return fail(DCM_ERR_ARG, "bad handle or system index");
    if (first) *first = h->geo_host[k].p0;
    if (count) *count = h->geo_host[k].n;
    return DCM_OK;
}

static void invalidate_graphs(dcm_handle *h)
{
    if (h->g_plain) cudaGraphExecDestroy(h->g_plain);
    if (h->g_detect) cudaGraphExecDestroy(h->g_detect);
    h->g_plain = h->g_detect = nullptr;
    h->graphs_ready = false;
}

static int set_state_range(dcm_handle *h, int64_t p0, int64_t n, const double *x,
                           const double *v, int mem)
{
    size_t bytes = sizeof(double) * 3 * (size_t)n;
    const double *src[2] = {x, v};
    double *dst[2] = {h->x, h->v};
    for (int q = 0; q < 2; ++q) {
        if (!src[q]) {
            for (int a = 0; a < 3; ++a)
                DCM_CHECK_CUDA(cudaMemsetAsync(dst[q] + (size_t)a * h->n + p0, 0,
                                               sizeof(double) * n, h->stream));
            continue;
        }
        DCM_CHECK_CUDA(cudaMemcpyAsync(h->tmp3n, src[q], bytes,
                                       mem == DCM_DEVICE ? cudaMemcpyDeviceToDevice
                                                         : cudaMemcpyHostToDevice,
                                       h->stream));
        k_aos_to_soa<<<nblk(n, 256), 256, 0, h->stream>>>(h->b, p0, n, h->tmp3n, dst[q], q == 0);
    }
    DCM_CHECK_CUDA(cudaGetLastError());
    if (mem != DCM_DEVICE) DCM_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    h->have_state = true;
    h->have_cut = false;
    h->forces_valid = false;
    h->cells_valid = false;
    return DCM_OK;
}

static int get_state_range(dcm_handle *h, int64_t p0, int64_t n, double *x, double *v, double *f,
                           int mem)
{
    size_t bytes = sizeof(double) * 3 * (size_t)n;
    double *src[3] = {h->x, h->v, h->f};
    double *dst[3] = {x, v, f};
    // (the staging buffer is reused in stream order: one wait at the end)
    for (int q = 0; q < 3; ++q) {
        if (!dst[q]) continue;
        k_soa_to_aos<<<nblk(n, 256), 256, 0, h->stream>>>(h->n, p0, n, src[q], h->tmp3n);
        DCM_CHECK_CUDA(cudaGetLastError());
        DCM_CHECK_CUDA(cudaMemcpyAsync(dst[q], h->tmp3n, bytes,
                                       mem == DCM_DEVICE ? cudaMemcpyDeviceToDevice
                                                         : cudaMemcpyDeviceToHost,
                                       h->stream));
    }
    if (mem != DCM_DEVICE) DCM_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    return DCM_OK;
}

extern "C" int dcm_set_state(dcm_handle *h, const double *x, const double *v, int mem)
{
    Trace trace("dcm_set_state");
    if (!h || !x) return fail(DCM_ERR_ARG, "null handle or positions");
    int r = set_state_range(h, 0, h->n, x, v, mem);
    if (!r) h->step = 0;
    h->keep_lists = false;
    return r;
}

// the FP32 cell-relative positions of every particle from x, in the cell
// of the last sort (what the drift writes in a step): a state update that
// keeps the Verlet lists
__global__ void k_refresh_rel(Batch b, const double *__restrict__ x,
                              const int32_t *__restrict__ cell_of, const int32_t *__restrict__ inv,
                              float4 *sp4, float4 *spl4)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.N) return;
    const Geom &g = b.sys[sys_p(b, i)];
    const size_t N = (size_t)b.N;
    float4 lo;
    const float4 u = cell_rel_position(b, g, x[i], x[N + i], x[2 * N + i], cell_of[i] - (int)g.c0, lo);
    const int32_t k = inv[i];
    sp4[k] = u;
    spl4[k] = lo;
}

extern "C" int dcm_update_state(dcm_handle *h, const double *x, const double *v, int mem)
{
    Trace trace("dcm_update_state");
    if (!h || !x) return fail(DCM_ERR_ARG, "null handle or positions");
    if (h->M != 1) return fail(DCM_ERR_ARG, "dcm_update_state takes single-system handles");
    const bool keep = h->have_state && h->have_cut && h->forces_valid;
    int r = set_state_range(h, 0, h->n, x, v, mem);
    if (r) return r;
    if (!keep) return DCM_OK;                    // (set_state, the step counter kept)
    h->have_cut = true;                          // the last detection's cutoffs stay
    h->keep_lists = h->nl != nullptr;
    if (h->nl && h->list_warp) {
        k_refresh_rel<<<nblk(h->n, 256), 256, 0, h->stream>>>(h->b, h->x, h->cell_of, h->inv,
                                                              h->sp4, h->spl4);
        DCM_CHECK_CUDA(cudaGetLastError());
    }
    return DCM_OK;
}

extern "C" int dcm_ensemble_set_state(dcm_handle *h, int k, const double *x, const double *v,
                                      int mem)
{
    if (!h || !x || k < 0 || k >= h->M) return fail(DCM_ERR_ARG, "bad handle, system or positions");
    return set_state_range(h, h->geo_host[k].p0, h->geo_host[k].n, x, v, mem);
}

extern "C" int dcm_ensemble_get_state(dcm_handle *h, int k, double *x, double *v, double *f,
                                      int mem)
{
    if (!h || k < 0 || k >= h->M) return fail(DCM_ERR_ARG, "bad handle or system");
    return get_state_range(h, h->geo_host[k].p0, h->geo_host[k].n, x, v, f, mem);
}

extern "C" int dcm_set_step(dcm_handle *h, int64_t step)
{
    if (!h || step < 0) return fail(DCM_ERR_ARG, "bad handle or step");
    h->step = step;
    return DCM_OK;
}

extern "C" int dcm_get_state(dcm_handle *h, double *x, double *v, double *f, int mem)
{
    Trace trace("dcm_get_state");
    if (!h) return fail(DCM_ERR_ARG, "null handle");
    return get_state_range(h, 0, h->n, x, v, f, mem);
}

extern "C" int dcm_set_cutoffs(dcm_handle *h, const double *rc, int mem)
{
    if (!h || !rc) return fail(DCM_ERR_ARG, "null handle or cutoffs");
    int64_t N = h->n;
    std::vector<double> tmp;
    if (mem != DCM_DEVICE) {
        for (int k = 0; k < h->M; ++k) {
            const Geom &g = h->geo_host[k];
            for (int64_t i = g.p0; i < g.p0 + g.n; ++i)
                if (!(rc[i] >= g.rc_min && rc[i] <= g.rc_max))
                    return fail(DCM_ERR_ARG, "cutoff %lld = %g outside [rc_min, rc_max]",
                                (long long)i, rc[i]);
        }
    }
    DCM_CHECK_CUDA(cudaMemcpyAsync(h->rc, rc, sizeof(double) * N,
                                   mem == DCM_DEVICE ? cudaMemcpyDeviceToDevice
                                                     : cudaMemcpyHostToDevice,
                                   h->stream));
    int r = launch_classify_rc(h);
    if (r) return r;
    if (mem != DCM_DEVICE) DCM_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    h->have_cut = true;
    h->cut_detected = false;
    h->forces_valid = false;
    invalidate_graphs(h);   // the captured list builds depend on where cutoffs come from
    return DCM_OK;
}

extern "C" int dcm_detect_interface(dcm_handle *h)
{
    Trace trace("dcm_detect_interface");
    if (!h) return fail(DCM_ERR_ARG, "null handle");
    if (!h->have_state) return fail(DCM_ERR_STATE, "no state set");
    if (!h->cut_detected) invalidate_graphs(h);   // list builds anticipate detected cutoffs
    int r = launch_detect(h);
    if (r) return r;
    h->have_cut = true;
    h->cut_detected = true;
    h->forces_valid = false;
    return DCM_OK;
}

static int forces_now(dcm_handle *h, bool energy)
{
    if (!h->have_cut) {
        int r = launch_detect(h);
        if (r) return r;
        h->have_cut = true;
        h->cut_detected = true;
    }
    h->step_detect = true;                       // classes may have changed
    // after dcm_update_state the reuse test decides whether the lists are
    // rebuilt; after anything else they are
    const bool rebuild = !h->keep_lists;
    h->keep_lists = false;
    int r = h->nl ? launch_list_step(h, rebuild) : launch_bin(h);
    if (r) return r;
    r = launch_forces(h, energy);
    if (r) return r;
    h->forces_valid = true;
    return DCM_OK;
}

extern "C" int dcm_compute_forces(dcm_handle *h)
{
    Trace trace("dcm_compute_forces");
    if (!h) return fail(DCM_ERR_ARG, "null handle");
    if (!h->have_state) return fail(DCM_ERR_STATE, "no state set");
    return forces_now(h, false);
}

static void mark(dcm_handle *h, int q, bool capturing)
{
    if (!h->timing) return;
    if (capturing)
        cudaEventRecordWithFlags(h->ev[q], h->stream, cudaEventRecordExternal);
    else
        cudaEventRecord(h->ev[q], h->stream);
}

// ---- conditional branches of a captured step ----------------------------
namespace dcm {

int branch_open(dcm_handle *h, Branch &b, int nbody)
{
    b.active = false;
    if (!h->branching) return DCM_OK;
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edges = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(h->stream, &st, nullptr, &g, &deps, &edges, &ndeps);
    if (e != cudaSuccess) return fail_cuda(e, "capture info", __FILE__, __LINE__);
    if (st != cudaStreamCaptureStatusActive) return fail(DCM_ERR_STATE, "branch outside a capture");
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = h->cond;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = (unsigned)nbody;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, deps, edges, ndeps, &p);
    if (e != cudaSuccess) return fail_cuda(e, "conditional node", __FILE__, __LINE__);
    e = cudaStreamUpdateCaptureDependencies(h->stream, &node, nullptr, 1,
                                            cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return fail_cuda(e, "capture dependencies", __FILE__, __LINE__);
    b.nbody = nbody;
    b.cur = 0;
    b.body[0] = p.conditional.phGraph_out[0];
    b.body[1] = nbody > 1 ? p.conditional.phGraph_out[1] : nullptr;
    e = cudaStreamBeginCaptureToGraph(h->side, b.body[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail_cuda(e, "body capture", __FILE__, __LINE__);
    b.main = h->stream;
    h->stream = h->side;
    b.active = true;
    return DCM_OK;
}

static int count_kernel_nodes(cudaGraph_t g)
{
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return -1;
    std::vector<cudaGraphNode_t> nodes(n);
    if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return -1;
    int k = 0;
    for (cudaGraphNode_t q : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(q, &t) != cudaSuccess) return -1;
        k += t == cudaGraphNodeTypeKernel;
    }
    return k;
}

static int branch_end_body(dcm_handle *h, Branch &b)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->side, &g);
    if (e != cudaSuccess) return fail_cuda(e, "end body capture", __FILE__, __LINE__);
    int k = count_kernel_nodes(b.body[b.cur]);
    if (k < 0) return fail(DCM_ERR_CUDA, "graph node count");
    h->br_kernels[b.cur] += k;
    return DCM_OK;
}

int branch_else(dcm_handle *h, Branch &b)
{
    if (!b.active) return DCM_OK;
    if (b.nbody < 2 || b.cur != 0) return fail(DCM_ERR_STATE, "branch has no else body");
    int r = branch_end_body(h, b);
    if (r) return r;
    b.cur = 1;
    cudaError_t e = cudaStreamBeginCaptureToGraph(h->side, b.body[1], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail_cuda(e, "body capture", __FILE__, __LINE__);
    return DCM_OK;
}

int branch_close(dcm_handle *h, Branch &b)
{
    if (!b.active) return DCM_OK;
    int r = branch_end_body(h, b);
    h->stream = b.main;
    b.active = false;
    return r;
}

}  // namespace dcm

// one velocity-Verlet step; detection after the drift when detect is set
static int enqueue_step(dcm_handle *h, bool detect, bool capturing)
{
    list_mode(h);
    h->step_detect = detect;
    h->fold_check = h->nl != nullptr;        // the reuse test rides on the drift / cutoff kernel
    h->in_step = true;
    mark(h, 0, capturing);
    int r = launch_kick_drift(h);
    mark(h, 1, capturing);
    if (!r && detect) r = launch_detect(h);
    mark(h, 2, capturing);
    if (h->branching) {
        // warp Verlet lists in a captured graph: one IF node on the rebuild
        // decision holds the list build and the force walk of a rebuild step
        // (body 0) and the list force of every other step (body 1).  Events
        // cannot sit in a body, so the binning phase is empty here and the
        // force phase covers both.
        mark(h, 3, capturing);
        Branch br = {};
        if (!r) r = branch_open(h, br, 2);
        if (!r) r = launch_list_step(h, false);
        if (!r) r = launch_list_forces(h, false, 0);
        if (!r) r = branch_else(h, br);
        if (!r) r = launch_list_forces(h, false, 1);
        int r2 = branch_close(h, br);
        if (!r) r = r2;
    } else {
        if (!r) r = h->nl ? launch_list_step(h, false) : launch_bin(h);
        mark(h, 3, capturing);
        if (!r) r = launch_forces(h, false);
    }
    mark(h, 4, capturing);
    if (!r) r = launch_kick(h);
    mark(h, 5, capturing);
    h->fold_check = false;
    h->in_step = false;
    return r;
}

static int capture(dcm_handle *h, bool detect, cudaGraphExec_t *exec)
{
    cudaGraph_t graph = nullptr;
    if (!h->side) {
        cudaError_t e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail_cuda(e, "cudaStreamCreate", __FILE__, __LINE__);
    }
    cudaStream_t main = h->stream;
    cudaError_t e = cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail_cuda(e, "begin capture", __FILE__, __LINE__);
    // the rebuild decision of this graph's list check (default: rebuild);
    // only graphs with branches may hold a handle
    list_mode(h);
    h->branching = h->list_warp && h->tune.step_graph == DCM_GRAPH_BRANCHED;
    if (h->branching) {
        cudaStreamCaptureStatus st;
        cudaGraph_t g = nullptr;
        e = cudaStreamGetCaptureInfo(main, &st, nullptr, &g);
        if (e == cudaSuccess)
            e = cudaGraphConditionalHandleCreate(&h->cond, g, 1, cudaGraphCondAssignDefault);
    }
    int r = e == cudaSuccess ? DCM_OK : fail_cuda(e, "conditional handle", __FILE__, __LINE__);
    h->br_kernels[0] = h->br_kernels[1] = 0;
    if (!r) r = enqueue_step(h, detect, true);
    h->branching = false;
    if (h->stream != main) {                 // an error inside a branch body
        cudaGraph_t body = nullptr;
        (void)cudaStreamEndCapture(h->side, &body);
        h->stream = main;
    }
    e = cudaStreamEndCapture(main, &graph);
    if (r || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        (void)cudaGetLastError();
        return r ? r : fail_cuda(e, "end capture", __FILE__, __LINE__);
    }
    int top = count_kernel_nodes(graph);
    (detect ? h->kernels_detect : h->kernels_plain) = top + h->br_kernels[0];
    (detect ? h->kernels_detect_reuse : h->kernels_plain_reuse) = top + h->br_kernels[1];
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail_cuda(e, "graph instantiate", __FILE__, __LINE__);
    return DCM_OK;
}

extern "C" int dcm_step(dcm_handle *h, int64_t nsteps)
{
    Trace trace("dcm_step");
    if (!h || nsteps < 0) return fail(DCM_ERR_ARG, "bad handle or nsteps");
    if (!h->have_state) return fail(DCM_ERR_STATE, "no state set");
    if (nsteps == 0) return DCM_OK;
    if (!h->forces_valid) {
        int r = forces_now(h, false);
        if (r) return r;
    }
    if (!h->graphs_ready) {
        int r = capture(h, false, &h->g_plain);
        if (!r) r = capture(h, true, &h->g_detect);
        if (r) {
            invalidate_graphs(h);
            return r;
        }
        h->graphs_ready = true;
    }
    for (int64_t s = 0; s < nsteps; ++s) {
        int64_t step = ++h->step;
        bool det = h->p.detect_every > 0 && step % h->p.detect_every == 0;
        DCM_CHECK_CUDA(cudaGraphLaunch(det ? h->g_detect : h->g_plain, h->stream));
        h->last_detect = det;
    }
    return DCM_OK;
}

extern "C" int dcm_set_timing(dcm_handle *h, int on)
{
    if (!h) return fail(DCM_ERR_ARG, "null handle");
    if ((on != 0) == h->timing) return DCM_OK;
    if (on && !h->ev[0])
        for (int q = 0; q <= DCM_NUM_PHASES; ++q) DCM_CHECK_CUDA(cudaEventCreate(&h->ev[q]));
    h->timing = on != 0;
    invalidate_graphs(h);
    return DCM_OK;
}

extern "C" int dcm_get_phase_times(dcm_handle *h, float ms[DCM_NUM_PHASES])
{
    if (!h || !ms) return fail(DCM_ERR_ARG, "null handle or output");
    if (!h->timing || !h->graphs_ready) return fail(DCM_ERR_STATE, "timing off or no step run");
    DCM_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    for (int q = 0; q < DCM_NUM_PHASES; ++q) {
        float t = 0.f;
        DCM_CHECK_CUDA(cudaEventElapsedTime(&t, h->ev[q], h->ev[q + 1]));
        ms[q] = t;
    }
    return DCM_OK;
}

static int energies(dcm_handle *h, std::vector<double> &out)
{
    if (!h->have_state) return fail(DCM_ERR_STATE, "no state set");
    int r = forces_now(h, true);
    if (r) return r;
    for (int k = 0; k < h->M && !r; ++k) r = launch_reduce_energy(h, k);
    if (r) return r;
    out.resize(8 * (size_t)h->M);
    DCM_CHECK_CUDA(cudaMemcpyAsync(out.data(), h->red_out, sizeof(double) * out.size(),
                                   cudaMemcpyDeviceToHost, h->stream));
    DCM_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    return DCM_OK;
}

static void energy_of(const dcm_handle *h, const double *o, int k, double *pe, double *ke,
                      double *w, bool add)
{
    double m = h->par_host[k].mass;
    if (pe) *pe = (add ? *pe : 0.0) + o[0];
    if (ke) *ke = (add ? *ke : 0.0) + 0.5 * m * o[1];
    if (w)
        for (int q = 0; q < 6; ++q) w[q] = (add ? w[q] : 0.0) + o[2 + q];
}

extern "C" int dcm_energy_virial(dcm_handle *h, double *pe, double *ke, double w[6])
{
    Trace trace("dcm_energy_virial");
    if (!h) return fail(DCM_ERR_ARG, "null handle");
    std::vector<double> out;
    int r = energies(h, out);
    if (r) return r;
    for (int k = 0; k < h->M; ++k) energy_of(h, out.data() + 8 * k, k, pe, ke, w, k > 0);
    return DCM_OK;
}

extern "C" int dcm_ensemble_energy_virial(dcm_handle *h, int k, double *pe, double *ke, double w[6])
{
    if (!h || k < 0 || k >= h->M) return fail(DCM_ERR_ARG, "bad handle or system");
    std::vector<double> out;
    int r = energies(h, out);
    if (r) return r;
    energy_of(h, out.data() + 8 * k, k, pe, ke, w, false);
    return DCM_OK;
}

extern "C" int dcm_get_grid(dcm_handle *h, int32_t dims[3], int32_t *counts, double *smoothed,
                            uint8_t *labels, double *dist)
{
    if (!h) return fail(DCM_ERR_ARG, "null handle");
    if (dims)
        for (int a = 0; a < 3; ++a) dims[a] = h->g.gd[a];
    size_t nv = (size_t)h->g.nvox;   // system 0 (voxels of system 0 come first)
    if (counts) DCM_CHECK_CUDA(cudaMemcpyAsync(counts, h->B, 4 * nv, cudaMemcpyDeviceToHost, h->stream));
    if (smoothed)
        DCM_CHECK_CUDA(cudaMemcpyAsync(smoothed, h->Bs, 8 * nv, cudaMemcpyDeviceToHost, h->stream));
    if (labels) DCM_CHECK_CUDA(cudaMemcpyAsync(labels, h->S, nv, cudaMemcpyDeviceToHost, h->stream));
    if (dist) {
        DevStats st;
        DCM_CHECK_CUDA(cudaMemcpyAsync(&st, h->stats, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
        DCM_CHECK_CUDA(cudaStreamSynchronize(h->stream));
        const double *D = st.barrier[3] ? h->D1 : h->D0;
        DCM_CHECK_CUDA(cudaMemcpyAsync(dist, D, 8 * nv, cudaMemcpyDeviceToHost, h->stream));
    }
    DCM_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    if (dist)
        for (size_t q = 0; q < nv; ++q)
            if (dist[q] > h->g.r_grid) dist[q] = h->g.r_grid;   // CFSM cap
    return DCM_OK;
}

extern "C" int dcm_remove_small_components(dcm_handle *h, uint8_t *labels, int32_t min_voxels,
                                           int mem, int64_t *flipped)
{
    if (!h || !labels) return fail(DCM_ERR_ARG, "null handle or labels");
    if (min_voxels < 0) return fail(DCM_ERR_ARG, "min_voxels must be >= 0");
    if (mem != DCM_HOST && mem != DCM_DEVICE) return fail(DCM_ERR_ARG, "mem must be DCM_HOST or DCM_DEVICE");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    DCM_CHECK_CUDA(cudaStreamIsCapturing(h->stream, &cap));
    if (cap != cudaStreamCaptureStatusNone) return fail(DCM_ERR_STATE, "not callable during stream capture");
    const int64_t nv = h->g.nvox;   // system 0 (its voxels come first)
    int rc;
    if ((rc = cc_setup(h))) return rc;
    uint8_t *S = nullptr;
    if ((rc = dalloc(h, &S, nv))) return rc;
    cudaMemcpyKind in = mem == DCM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaMemcpyKind out = mem == DCM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    cudaError_t e = cudaMemcpyAsync(S, labels, (size_t)nv, in, h->stream);
    Batch b0 = h->b;              // system 0 alone
    b0.M = 1;
    b0.NV = nv;
    b0.vsys = nullptr;
    if (e == cudaSuccess) rc = launch_components(h, b0, S, min_voxels, h->cc_ntiles0);
    if (e == cudaSuccess && rc == DCM_OK) e = cudaMemcpyAsync(labels, S, (size_t)nv, out, h->stream);
    DevStats st;
    if (e == cudaSuccess && rc == DCM_OK)
        e = cudaMemcpyAsync(&st, h->stats, sizeof(st), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dfree(h, S);
    h->bytes -= nv > 0 ? nv : 1;
    if (e != cudaSuccess) return fail_cuda(e, "small-component removal", __FILE__, __LINE__);
    if (rc) return rc;
    if (flipped) *flipped = (int64_t)st.cc_flipped;
    return dcm_sync(h);
}

extern "C" int dcm_get_cutoffs(dcm_handle *h, double *d, double *rc, uint8_t *cls)
{
    if (!h) return fail(DCM_ERR_ARG, "null handle");
    size_t N = (size_t)h->n;
    if (d) DCM_CHECK_CUDA(cudaMemcpyAsync(d, h->d, 8 * N, cudaMemcpyDeviceToHost, h->stream));
    if (rc) DCM_CHECK_CUDA(cudaMemcpyAsync(rc, h->rc, 8 * N, cudaMemcpyDeviceToHost, h->stream));
    if (cls) DCM_CHECK_CUDA(cudaMemcpyAsync(cls, h->cls, N, cudaMemcpyDeviceToHost, h->stream));
    DCM_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    return DCM_OK;
}

extern "C" int dcm_get_cells(dcm_handle *h, int32_t nc[3], int32_t *cell_start, int32_t *sorted_id)
{
    if (!h) return fail(DCM_ERR_ARG, "null handle");
    if (nc)
        for (int a = 0; a < 3; ++a) nc[a] = h->g.nc[a];
    // system 0: its cells and sorted slots come first in the concatenation
    if (cell_start)
        DCM_CHECK_CUDA(cudaMemcpyAsync(cell_start, h->cell_start, 4 * (size_t)(h->g.ncell + 1),
                                       cudaMemcpyDeviceToHost, h->stream));
    if (sorted_id)
        DCM_CHECK_CUDA(cudaMemcpyAsync(sorted_id, h->sorted_id, 4 * (size_t)h->g.n,
                                       cudaMemcpyDeviceToHost, h->stream));
    DCM_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    return DCM_OK;
}

extern "C" int dcm_get_pair_counts(dcm_handle *h, int32_t *npair)
{
    if (!h || !npair) return fail(DCM_ERR_ARG, "null handle or output");
    DCM_CHECK_CUDA(cudaMemcpyAsync(npair, h->npair, 4 * (size_t)h->n, cudaMemcpyDeviceToHost,
                                   h->stream));
    DCM_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    return DCM_OK;
}

extern "C" int dcm_get_stats(dcm_handle *h, dcm_stats *s)
{
    if (!h || !s) return fail(DCM_ERR_ARG, "null handle or output");
    int r = launch_reduce_pairs(h);
    if (r) return r;
    DevStats st;
    int32_t cc[3 * DCM_MAX_CLASSES];
    DCM_CHECK_CUDA(cudaMemcpyAsync(&st, h->stats, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    DCM_CHECK_CUDA(cudaMemcpyAsync(cc, h->class_count_dev, sizeof(cc), cudaMemcpyDeviceToHost,
                                   h->stream));
    DCM_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    memset(s, 0, sizeof(*s));
    s->step = h->step;
    s->pairs = (int64_t)st.pairs;
    s->kmeans_iters = st.kmeans_iters;
    s->cfsm_iters = st.cfsm_iters;
    for (int q = 0; q < h->b.K; ++q) s->class_count[q] = cc[q];
    for (int a = 0; a < 3; ++a) {
        s->grid[a] = h->g.gd[a];
        s->cells[a] = h->g.nc[a];
    }
    s->c_liquid = st.c_liquid;
    s->c_vapor = st.c_vapor;
    s->guard_rechecks = (int64_t)st.guard_rechecks;
    s->kernels_plain = h->kernels_plain;
    s->kernels_detect = h->kernels_detect;
    s->kernels_plain_reuse = h->kernels_plain_reuse;
    s->kernels_detect_reuse = h->kernels_detect_reuse;
    s->list_builds = (int64_t)st.list_builds;
    s->list_entries = (int64_t)st.list_entries;
    s->cc_flipped = (int64_t)st.cc_flipped;
    s->refined = (int64_t)st.barrier[6] + (int64_t)st.barrier[7];
    return DCM_OK;
}

extern "C" int dcm_set_tuning(dcm_handle *h, const dcm_tuning *t)
{
    if (!h || !t) return fail(DCM_ERR_ARG, "null handle or tuning");
    for (int q = 0; q < DCM_MAX_CLASSES; ++q) {
        int G = t->lanes[q];
        if (G < 1 || G > 32 || (G & (G - 1))) return fail(DCM_ERR_ARG, "lanes must be 1..32, pow2");
    }
    if (t->block < 64 || t->block > 256 || (t->block & 31))
        return fail(DCM_ERR_ARG, "block must be a multiple of 32 in 64..256");
    if (t->walk != DCM_WALK_WARP && t->walk != DCM_WALK_LANES)
        return fail(DCM_ERR_ARG, "walk must be DCM_WALK_WARP or DCM_WALK_LANES");
    if (t->walk == DCM_WALK_LANES && h->p.precision == DCM_MIXED)
        return fail(DCM_ERR_ARG, "DCM_WALK_LANES is the FP64 walk; DCM_MIXED runs the warp kernels");
    if (t->list_lanes != 0 && t->list_lanes != 4 && t->list_lanes != 8 && t->list_lanes != 16 &&
        t->list_lanes != 32)
        return fail(DCM_ERR_ARG, "list_lanes must be 4, 8, 16 or 32 (0: 8)");
    if (t->step_graph != DCM_GRAPH_BRANCHED && t->step_graph != DCM_GRAPH_FLAT)
        return fail(DCM_ERR_ARG, "step_graph must be DCM_GRAPH_BRANCHED or DCM_GRAPH_FLAT");
    bool per_class = false;
    for (int q = 0; q < DCM_MAX_CLASSES; ++q) per_class = per_class || t->list_lanes_class[q] != 0;
    if (per_class) {
        for (int q = 0; q < h->p.n_classes; ++q) {
            const int G = t->list_lanes_class[q];
            if (G != 4 && G != 8 && G != 16 && G != 32)
                return fail(DCM_ERR_ARG, "list_lanes_class[%d] must be 4, 8, 16 or 32 (or all 0)", q);
        }
        if (h->p.precision != DCM_MIXED)
            return fail(DCM_ERR_ARG, "list_lanes_class applies to the DCM_MIXED list force");
    }
    h->tune = *t;
    invalidate_graphs(h);
    // the two list layouts differ (the warp kernels place each list at its
    // capacity offset and keep its length in nl_cnt, the lanes kernels pack
    // them): the next step rebuilds the lists for the kernels now selected
    if (h->nl) DCM_CHECK_CUDA(cudaMemsetAsync(h->lflags + LF_OK, 0, sizeof(int), h->stream));
    return DCM_OK;
}

extern "C" int dcm_get_tuning(dcm_handle *h, dcm_tuning *t)
{
    if (!h || !t) return fail(DCM_ERR_ARG, "null handle or tuning");
    *t = h->tune;
    return DCM_OK;
}

extern "C" int dcm_sync(dcm_handle *h)
{
    if (!h) return fail(DCM_ERR_ARG, "null handle");
    DCM_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    int err = 0;
    DCM_CHECK_CUDA(cudaMemcpyAsync(&err, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DCM_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    if (!err) return DCM_OK;
    DCM_CHECK_CUDA(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
    DCM_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    if (err & DEV_ERR_CANCEL) return fail(DCM_ERR_CANCELLED, "cancelled");
    if (err & DEV_ERR_CFSM_CAP)
        return fail(DCM_ERR_NOT_CONVERGED, "CFSM reached its iteration cap (device flags 0x%x)", err);
    return fail(DCM_ERR_DEVICE_CHECK, "device check failed (flags 0x%x: 1 non-finite, 2 jump, "
                                      "4 barrier timeout, 16 density, 64 bounds, 128 union)",
                err);
}

extern "C" int64_t dcm_device_bytes(const dcm_handle *h) { return h ? h->bytes : 0; }

extern "C" int dcm_check_bounded_wait(dcm_handle *h)
{
    if (!h) return fail(DCM_ERR_ARG, "null handle");
    int r = launch_barrier_timeout_check(h);
    if (r) return r;
    return dcm_sync(h);
}
