// dcm_list.cu -- Verlet pair lists with a skin for the DCM force (Section
// 2.2.1 and Algorithm 3.3 of the thesis: store every j within r_c[i] + r_s,
// reuse the list while no particle moved r_s/2).
//
// With per-particle cutoffs the reuse condition also covers cutoff growth,
// and each particle carries its own share s_i of the skin: particle i's
// list holds every j closer than R_i + s_j at the build, where R_i is i's
// own list radius (anticipated cutoff + s_i).  A pair inside r_c[i](t) now
// was closer than r_c[i](t) + |d_i| + |d_j| at the build (d the
// displacements since), so every list stays complete while
//     max_i (|d_i| - (R_i - r_c[i](t))) + max_j (|d_j| - s_j) < 0,
// both maxima taken in one pass.  With uniform shares s = skin/2 this is
// the usual rule "no two displacements add up to the skin"; with
// velocity-adaptive shares (s_i growing with the particle's speed at the
// build) slow particles keep short lists and the few fast ones do not
// force early rebuilds.
// The anticipated cutoff in R_i is the one particle i would get if its
// interface distance dropped by a margin (list_margin, 1 sigma by default):
// the detected interface jitters by about a voxel, and Eq. 7 is steep near
// d = r_c,max, so lists sized by the current cutoff alone would be rebuilt
// at nearly every detection.  Every step one kernel measures both maxima
// and decides; the cell sort and the list build that follow run only on a
// rebuild step (graph IF nodes, or their own gates when launched eagerly).
//
// Lists are indexed by the sorted slot k of the build; an entry holds the
// sorted slot j of a neighbour (24 bits) and its row's cell offsets dy, dz
// (4 bits each); the x offset comes from the cell x index stored with j's
// position.  If the entries would not fit the storage reserved at creation,
// that step uses the direct cell walk and the next step rebuilds.
#include "dcm_device.cuh"

namespace dcm {

// order-preserving int image of a float (for atomicMax over signed values)
__device__ __forceinline__ int ordered_int(float f)
{
    int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}

// the two maxima of the reuse condition; the last block to finish turns
// them into the decision
__global__ void k_list_check(Batch b, const double *__restrict__ x, const double *__restrict__ x_ref,
                             const double *__restrict__ rc, const float *__restrict__ rl_ref,
                             const float *__restrict__ sh_ref, int *lf, int force,
                             cudaGraphConditionalHandle cond0, cudaGraphConditionalHandle cond1,
                             int set_cond)
{
    float mp = -3.0e38f, mq = -3.0e38f;
    const size_t N = (size_t)b.N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        float dx = (float)(x[i] - x_ref[i]);
        float dy = (float)(x[N + i] - x_ref[N + i]);
        float dz = (float)(x[2 * N + i] - x_ref[2 * N + i]);
        // a coordinate wrapped through the box shows up as a jump of about
        // one box edge: fold it back (moves are far below half an edge)
        const Geom &g = b.sys[sys_p(b, i)];
        float Lx = (float)g.L[0], Ly = (float)g.L[1], Lz = (float)g.L[2];
        dx -= Lx * rintf(dx / Lx);
        dy -= Ly * rintf(dy / Ly);
        dz -= Lz * rintf(dz / Lz);
        const float d = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        const float s = sh_ref[i];
        mp = fmaxf(mp, d - s);
        mq = fmaxf(mq, d - (list_radius_unpadded(rl_ref[i], s) - (float)rc[i]));
    }
    for (int off = 16; off > 0; off >>= 1) {
        mp = fmaxf(mp, __shfl_xor_sync(0xffffffffu, mp, off));
        mq = fmaxf(mq, __shfl_xor_sync(0xffffffffu, mq, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&lf[LF_PARTNER], ordered_int(mp));
        atomicMax(&lf[LF_EXCESS], ordered_int(mq));
    }
    __syncthreads();
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&lf[LF_DONE], 1) == (int)(gridDim.x * gridDim.y * gridDim.z) - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        // the images are their own inverses; reset both to that of -3.4e38
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
        int rebuild = force || !ok || (partner + excess >= 0.f);
        lf[LF_REBUILD] = rebuild;
        if (rebuild) lf[LF_SHMAX] = 0;          // the gather of the build takes the max
        lf[LF_DONE] = 0;
        if (set_cond) {
            cudaGraphSetConditional(cond0, (unsigned)rebuild);
            cudaGraphSetConditional(cond1, (unsigned)rebuild);
        }
    }
}

// after the count scan: does the list fit?  FILL gate = rebuild && fits
__global__ void k_list_total(int64_t N, const int32_t *__restrict__ start, int64_t cap, int *lf,
                             DevStats *st, int fill_counts)
{
    if (lf[LF_REBUILD] == 0) {
        lf[LF_FILL] = 0;         // no fill on a step that keeps its lists
        return;
    }
    int64_t total = start[N];
    int ok = total <= cap;
    lf[LF_OK] = ok;
    lf[LF_FILL] = ok;            // fill gate
    st->list_builds += 1ull;
    // the warp fill walk adds its entries (start[] sums capacities there)
    st->list_entries = fill_counts ? 0ull : (unsigned long long)total;
}

__global__ void k_list_save(int64_t N, const double *__restrict__ x, double *x_ref, const int *gate)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || *gate == 0) return;
    x_ref[i] = x[i];
    x_ref[N + i] = x[N + i];
    x_ref[2 * N + i] = x[2 * N + i];
}

static inline int nblk(int64_t n, int b) { return (int)((n + b - 1) / b); }

void list_mode(dcm_handle *h)
{
    h->list_warp = h->nl && h->p.precision == DCM_MIXED && h->tune.walk == DCM_WALK_WARP;
}

// decide, [cell sort], gather + classes, then
//  warp kernels (MIXED, warp walk): [capacity scan, total, save]; the list
//      fill happens in the force phase, inside the direct force walk of the
//      rebuild step (launch_forces).  In a captured step the bracketed work
//      sits in a graph IF node on the decision, so a step that reuses its
//      lists launches none of it;
//  lanes kernels: [list count, scan, total, fill, save]
int launch_list_step(dcm_handle *h, bool force_rebuild)
{
    int64_t N = h->n;
    int cgrid = h->num_sms * 2;
    list_mode(h);
    const bool set_cond = h->branching;
    k_list_check<<<cgrid, 256, 0, h->stream>>>(h->b, h->x, h->x_ref, h->rc, h->rl_ref, h->sh_ref,
                                               h->lflags, force_rebuild ? 1 : 0, h->cond[0],
                                               h->cond[1], set_cond ? 1 : 0);
    const int *rebuild = h->lflags + LF_REBUILD;
    const int *fill = h->lflags + LF_FILL;
    if (h->list_warp) {
        Branch br;
        int r = branch_open(h, br, 1, 0);
        if (!r) r = launch_sort_gather(h, rebuild);
        // class lists change with a detection or with the sort
        if (!r && !h->step_detect) r = launch_classes(h, rebuild);
        if (!r) {
            // the gather wrote each particle's capacity into nl_cnt
            cudaStream_t s = h->stream;
            launch_scan(h, h->nl_cnt, h->nl_start, h->nl_tiles, N, -1, rebuild);
            k_list_total<<<1, 1, 0, s>>>(N, h->nl_start, h->nl_cap, h->lflags, h->stats, 1);
            k_list_save<<<nblk(N, 256), 256, 0, s>>>(N, h->x, h->x_ref, fill);
            if (cudaGetLastError() != cudaSuccess) r = fail(DCM_ERR_CUDA, "list launch");
        }
        int r2 = branch_close(h, br);
        if (!r) r = r2;
        if (!r && h->step_detect) r = launch_classes(h, nullptr);
        return r;
    }
    cudaStream_t s = h->stream;
    int r = launch_bin_gated(h, rebuild, nullptr);
    if (r) return r;
    float delta = h->cut_detected ? h->list_margin : 0.0f;
    r = launch_list_walk(h, false, rebuild, delta);
    if (r) return r;
    launch_scan(h, h->nl_cnt, h->nl_start, h->nl_tiles, N, -1, rebuild);
    k_list_total<<<1, 1, 0, s>>>(N, h->nl_start, h->nl_cap, h->lflags, h->stats, 0);
    r = launch_list_walk(h, true, fill, delta);
    if (r) return r;
    k_list_save<<<nblk(N, 256), 256, 0, s>>>(N, h->x, h->x_ref, fill);
    return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "list launch");
}

}  // namespace dcm
