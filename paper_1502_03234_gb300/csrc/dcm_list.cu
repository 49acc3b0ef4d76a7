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

// the stand-alone reuse test (eager list steps and forced rebuilds; a
// captured step folds it into the drift or the cutoff kernel)
__global__ void k_list_check(Batch b, const double *__restrict__ x, const double *__restrict__ rc,
                             ListTest t)
{
    float mp = -3.0e38f, mq = -3.0e38f;
    const size_t N = (size_t)b.N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Geom &g = b.sys[sys_p(b, i)];
        const float d = list_disp(t, g, N, i, x[i], x[N + i], x[2 * N + i]);
        list_terms(t, i, d, rc[i], mp, mq);
    }
    list_test_block(t, mp, mq);
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

// the build's positions: FP64, and with the warp lists the FP32
// cell-relative ones of the fresh sort (id order)
__global__ void k_list_save(int64_t N, const double *__restrict__ x, double *x_ref, const int *gate,
                            const float4 *__restrict__ sp4, const int32_t *__restrict__ inv,
                            float4 *u_ref)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || *gate == 0) return;
    x_ref[i] = x[i];
    x_ref[N + i] = x[N + i];
    x_ref[2 * N + i] = x[2 * N + i];
    if (u_ref) u_ref[i] = sp4[inv[i]];
}

static inline int nblk(int64_t n, int b) { return (int)((n + b - 1) / b); }

ListTest list_test(dcm_handle *h, bool partner, bool excess, bool decide)
{
    ListTest t;
    t.lf = h->lflags;
    t.x_ref = h->x_ref;
    t.rl_ref = h->rl_ref;
    t.sh_ref = h->sh_ref;
    // the warp kernels keep FP32 cell-relative positions current every step
    t.u_ref = h->list_warp ? h->u_ref : nullptr;
    t.disp = h->list_warp ? h->disp : nullptr;
    t.partner = partner ? 1 : 0;
    t.excess = excess ? 1 : 0;
    t.decide = decide ? 1 : 0;
    t.force = 0;
    t.set_cond = h->branching ? 1 : 0;
    t.cond = h->cond;
    return t;
}

void list_mode(dcm_handle *h)
{
    h->list_warp = h->nl && h->p.precision == DCM_MIXED;
}

// decide, [cell sort], gather + classes, then
//  warp kernels (MIXED, warp walk): [capacity scan, total, save]; the list
//      fill happens in the force phase, inside the direct force walk of the
//      rebuild step (launch_list_forces).  In a captured step the bracketed
//      work sits in the rebuild body of the step's graph IF node (see
//      enqueue_step), so a step that reuses its lists launches none of it;
//  lanes kernels: [list count, scan, total, fill, save]
int launch_list_step(dcm_handle *h, bool force_rebuild)
{
    int64_t N = h->n;
    int cgrid = h->num_sms * 2;
    list_mode(h);
    if (force_rebuild || !h->fold_check) {
        ListTest t = list_test(h, true, true, true);
        t.force = force_rebuild ? 1 : 0;
        k_list_check<<<cgrid, 256, 0, h->stream>>>(h->b, h->x, h->rc, t);
    }
    const int *rebuild = h->lflags + LF_REBUILD;
    const int *fill = h->lflags + LF_FILL;
    if (h->list_warp) {
        int r = launch_sort_gather(h, rebuild);
        // the class lists only order the work queue: they are redone with
        // the sort (new slots) and left as they are after a detection that
        // keeps the lists (every slot is still in exactly one list; the
        // order is slightly off until the next build)
        if (!r) r = launch_classes(h, rebuild);
        if (!r) {
            // the gather wrote each particle's capacity into nl_cnt
            cudaStream_t s = h->stream;
            launch_scan(h, h->nl_cnt, h->nl_start, h->nl_tiles, N, -1, rebuild);
            k_list_total<<<1, 1, 0, s>>>(N, h->nl_start, h->nl_cap, h->lflags, h->stats, 1);
            k_list_save<<<nblk(N, 256), 256, 0, s>>>(N, h->x, h->x_ref, fill, h->sp4, h->inv,
                                                     h->u_ref);
            if (cudaGetLastError() != cudaSuccess) r = fail(DCM_ERR_CUDA, "list launch");
        }
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
    k_list_save<<<nblk(N, 256), 256, 0, s>>>(N, h->x, h->x_ref, fill, nullptr, nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? DCM_OK : fail(DCM_ERR_CUDA, "list launch");
}

}  // namespace dcm
