// dcm_components.cu -- removal of small connected components from the
// segmented voxel grid (Section 4.2, Fig. 20-21): after the K-means labels,
// each liquid component of fewer than min_component_voxels voxels becomes
// vapor, then each vapor component of the updated grid with fewer than that
// many voxels becomes liquid.  Components are 6-connected (face neighbours)
// across the periodic faces.
//
// The thesis labels in one row-major pass with an equivalence table
// (Algorithm 4.1) and, across processes, merges boundary labels so that the
// component sizes are lower bounds (Algorithm 5.3).  On one GPU the grid is
// labelled exactly with a two-level union-find over the voxel indices:
//   local    one block per 8x8x8 tile labels the tile's components in
//            shared memory (a tile wholly in the phase is one component;
//            otherwise minimum-label propagation with pointer jumping), points
//            each voxel of the phase at its tile-local root (the component's
//            smallest index) and records the local sizes at those roots;
//   global   the links that cross a tile face join the local roots in global
//            memory (roots linked larger under smaller by compare-and-swap,
//            so parent[v] <= v at all times and every find ends).  Finds
//            start at the local roots, so the slots of the other voxels keep
//            their local roots throughout, and a link whose in-plane
//            predecessor on the face joins the same two roots is left to
//            that one (a uniform face takes one union, not 64);
//   count    each tile-local root adds its local size to its global root's
//            count while that count is below the threshold (only "fewer
//            than the threshold" matters, so a large component stops
//            counting after a few atomics);
//   flip     voxels whose root's count is below the threshold change phase.
// The partition into components is unique, so the labels that come out do
// not depend on thread scheduling.
#include "dcm_device.cuh"

namespace dcm {

constexpr int CC_THREADS = 256;                  // blocks of the per-voxel passes
constexpr int CC_T = 8;                          // tile edge (voxels)
constexpr int CC_TILE = CC_T * CC_T * CC_T;      // voxels per tile = threads of a local block
// compare-and-swap attempts per union; a failed attempt means another union
// linked the root meanwhile, so this bounds a loop that always progresses
constexpr int CC_UNION_TRIES = 1 << 16;

struct CcArgs {
    Batch b;
    uint8_t *S;
    int32_t *parent;     // this phase's forest (voxel indices)
    int32_t *size;       // voxels per global root, counted up to the threshold
    int32_t *lsize;      // voxels per tile-local root (0 elsewhere)
    int32_t *uniform;    // per tile: every voxel of the tile in the phase
    const int64_t *tile_off;   // [M+1] tile offsets of the systems
    int phase;           // 0: liquid components, 1: vapor components
    int thr;             // >= 0: this threshold for every system; < 0: each system's own
    int *err;
    DevStats *st;
};

__device__ __forceinline__ int cc_threshold(const CcArgs &a, const Geom &g)
{
    return a.thr >= 0 ? a.thr : g.cc_min;
}

// root of v; every voxel visited is pointed at its grandparent on the way
// (an ancestor, so parent[v] <= v still holds and concurrent finds agree)
__device__ __forceinline__ int cc_find(int32_t *parent, int v)
{
    while (true) {
        const int p = __ldcg(parent + v);
        if (p == v) return v;
        const int gp = __ldcg(parent + p);
        if (gp == p) return p;
        __stcg(parent + v, gp);
        v = gp;
    }
}

// root of v without writes (after the unions the forest no longer changes)
__device__ __forceinline__ int cc_root(const int32_t *parent, int v)
{
    int p = __ldcg(parent + v);
    while (p != v) {
        v = p;
        p = __ldcg(parent + v);
    }
    return v;
}

__device__ __forceinline__ bool cc_union(int32_t *parent, int a, int b)
{
    for (int t = 0; t < CC_UNION_TRIES; ++t) {
        a = cc_find(parent, a);
        b = cc_find(parent, b);
        if (a == b) return true;
        if (a < b) {
            const int c = a;
            a = b;
            b = c;
        }
        if (atomicCAS(parent + a, a, b) == a) return true;
    }
    return false;
}

// a block's tile and a thread's voxel in it (local index lx + 8 (ly + 8 lz),
// whose order is the order of the voxels' global indices)
struct CcTile {
    const Geom *g;
    int tx, ty, tz, lx, ly, lz, x, y, z;
    int64_t sy, sz, v;
    bool inside;
    int thr;
};

__device__ __forceinline__ CcTile cc_tile(const CcArgs &a)
{
    CcTile c;
    const int s = a.b.M == 1 ? 0 : sys_of(a.tile_off, a.b.M, blockIdx.x);
    c.g = &a.b.sys[s];
    const Geom &g = *c.g;
    const int ntx = (g.gd[0] + CC_T - 1) / CC_T, nty = (g.gd[1] + CC_T - 1) / CC_T;
    const int t = (int)((int64_t)blockIdx.x - a.tile_off[s]);
    c.tx = t % ntx;
    c.ty = (t / ntx) % nty;
    c.tz = t / (ntx * nty);
    const int tid = threadIdx.x;
    c.lx = tid & (CC_T - 1);
    c.ly = (tid / CC_T) & (CC_T - 1);
    c.lz = tid / (CC_T * CC_T);
    c.x = c.tx * CC_T + c.lx;
    c.y = c.ty * CC_T + c.ly;
    c.z = c.tz * CC_T + c.lz;
    c.inside = c.x < g.gd[0] && c.y < g.gd[1] && c.z < g.gd[2];
    c.sy = g.gd[0];
    c.sz = (int64_t)g.gd[0] * g.gd[1];
    c.v = g.v0 + c.x + c.sy * c.y + c.sz * c.z;
    c.thr = cc_threshold(a, g);
    return c;
}

// the tile's components in shared memory: each voxel of the phase points at
// its tile-local root (the component's smallest index), which records the
// component's size; zeroes the tile's count slots
__device__ __forceinline__ void cc_local(const CcArgs &a, const CcTile &c)
{
    __shared__ int lab[CC_TILE];
    __shared__ int cnt[CC_TILE];
    const int tid = threadIdx.x;
    const Geom &g = *c.g;
    const bool in = c.inside && c.thr > 0 && a.S[c.v] == a.phase;
    if (c.inside) {
        a.size[c.v] = 0;
        a.lsize[c.v] = 0;
    }
    cnt[tid] = 0;
    const bool uniform = __syncthreads_and(in || !c.inside);
    if (tid == 0) a.uniform[blockIdx.x] = uniform ? 1 : 0;
    if (uniform) {
        // the tile's voxels all in the phase: one box-shaped component whose
        // smallest index is the tile's first voxel (local 0, always inside)
        lab[tid] = 0;
    } else {
        lab[tid] = in ? tid : CC_TILE;
        // face neighbours inside the tile and in the phase (the periodic wrap
        // stays in the tile only when the tile spans the axis); an absent one
        // is the voxel itself, which leaves the minimum alone
        int nb[6];
        const int xs[2] = {c.x == 0 ? g.gd[0] - 1 : c.x - 1, c.x + 1 == g.gd[0] ? 0 : c.x + 1};
        const int ys[2] = {c.y == 0 ? g.gd[1] - 1 : c.y - 1, c.y + 1 == g.gd[1] ? 0 : c.y + 1};
        const int zs[2] = {c.z == 0 ? g.gd[2] - 1 : c.z - 1, c.z + 1 == g.gd[2] ? 0 : c.z + 1};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            nb[q] = in && xs[q] / CC_T == c.tx && xs[q] != c.x && a.S[c.v + xs[q] - c.x] == a.phase
                        ? tid + xs[q] - c.x : tid;
            nb[2 + q] = in && ys[q] / CC_T == c.ty && ys[q] != c.y &&
                                a.S[c.v + c.sy * (ys[q] - c.y)] == a.phase
                            ? tid + CC_T * (ys[q] - c.y) : tid;
            nb[4 + q] = in && zs[q] / CC_T == c.tz && zs[q] != c.z &&
                                a.S[c.v + c.sz * (zs[q] - c.z)] == a.phase
                            ? tid + CC_T * CC_T * (zs[q] - c.z) : tid;
        }
        __syncthreads();
        // labels only decrease and stay inside the component, so they end at
        // the component's smallest local index; the minimum crosses at least
        // one link per pass, and no component has more than 511 links in a path
        for (int it = 0; it < CC_TILE; ++it) {
            bool changed = false;
            if (in) {
                int l = lab[tid];
                l = min(l, lab[l]);                      // pointer jumping
#pragma unroll
                for (int q = 0; q < 6; ++q) l = min(l, lab[nb[q]]);
                if (l < lab[tid]) {
                    lab[tid] = l;
                    changed = true;
                }
            }
            if (!__syncthreads_or(changed)) break;
        }
    }
    __syncthreads();
    if (in) {
        const int r = lab[tid];
        const int rx = c.tx * CC_T + (r & (CC_T - 1)), ry = c.ty * CC_T + ((r / CC_T) & (CC_T - 1)),
                  rz = c.tz * CC_T + r / (CC_T * CC_T);
        a.parent[c.v] = (int32_t)(g.v0 + rx + c.sy * ry + c.sz * rz);
        atomicAdd(&cnt[r], 1);
    }
    __syncthreads();
    if (in && cnt[tid] > 0) a.lsize[c.v] = cnt[tid];   // tid is a local root
}

// voxels of the phase whose root counted fewer than the threshold change phase
__device__ __forceinline__ void cc_flip(const CcArgs &a, const CcTile &c)
{
    if (!c.inside || c.thr <= 0 || a.S[c.v] != a.phase) return;
    // v -> its local root -> the global root (the count pass pointed every
    // local root at its global root)
    const int r = __ldcg(a.parent + __ldcg(a.parent + c.v));
    if (__ldcg(a.size + r) < c.thr) {
        a.S[c.v] = (uint8_t)(1 - a.phase);
        atomicAdd(&a.st->cc_flipped, 1ull);
    }
}

__global__ void __launch_bounds__(CC_TILE) k_cc_local(CcArgs a)
{
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.phase == 0) a.st->cc_flipped = 0ull;
    cc_local(a, cc_tile(a));
}

// voxel coordinates of v in its system (32-bit: a handle with this pass
// holds fewer than 2^31 voxels)
__device__ __forceinline__ void cc_coords(const Geom &g, int64_t v, int co[3])
{
    const int loc = (int)(v - g.v0);
    const int t = loc / g.gd[0];
    co[0] = loc - t * g.gd[0];
    co[1] = t % g.gd[1];
    co[2] = t / g.gd[1];
}

// the links across tile faces, in global memory, between local roots (one
// thread per voxel in index order: coalesced)
__global__ void k_cc_global(CcArgs a)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.b.NV || a.S[v] != a.phase) return;
    const Geom &g = a.b.sys[sys_v(a.b, v)];
    if (cc_threshold(a, g) <= 0) return;
    int co[3];
    cc_coords(g, v, co);
    const int64_t st[3] = {1, g.gd[0], (int64_t)g.gd[0] * g.gd[1]};
    const int nt[3] = {(g.gd[0] + CC_T - 1) / CC_T, (g.gd[1] + CC_T - 1) / CC_T, 0};
    const int tc[3] = {co[0] / CC_T, co[1] / CC_T, co[2] / CC_T};
    const int64_t t0 = a.b.M == 1 ? 0 : a.tile_off[sys_v(a.b, v)];
    const bool uni = __ldg(a.uniform + t0 + tc[0] + nt[0] * (tc[1] + nt[1] * tc[2])) != 0;
    bool ok = true;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const int cu = co[ax] + 1 == g.gd[ax] ? 0 : co[ax] + 1;
        if (cu / CC_T == tc[ax]) continue;                 // a link inside the tile
        const int64_t u = v + st[ax] * (cu - co[ax]);
        if (uni) {
            // both tiles wholly in the phase: their roots are their first
            // voxels, and the face's in-plane corner joins them for all 64
            int tu[3] = {tc[0], tc[1], tc[2]};
            tu[ax] = cu / CC_T;
            if (__ldg(a.uniform + t0 + tu[0] + nt[0] * (tu[1] + nt[1] * tu[2])) != 0) {
                if (co[(ax + 1) % 3] % CC_T == 0 && co[(ax + 2) % 3] % CC_T == 0)
                    ok = cc_union(a.parent, __ldcg(a.parent + v), __ldcg(a.parent + u)) && ok;
                continue;
            }
        }
        if (a.S[u] != a.phase) continue;
        const int pa = __ldcg(a.parent + v), pb = __ldcg(a.parent + u);
        if (pa == pb) continue;
        // the link one step back along each in-plane axis of the face, if it
        // is on the same face and joins the same two roots, covers this one
        bool covered = false;
#pragma unroll
        for (int d = 1; d <= 2; ++d) {
            const int bx = (ax + d) % 3;
            if (covered || co[bx] % CC_T == 0) continue;
            const int64_t w = v - st[bx], wu = u - st[bx];
            covered = a.S[w] == a.phase && a.S[wu] == a.phase && __ldcg(a.parent + w) == pa &&
                      __ldcg(a.parent + wu) == pb;
        }
        if (!covered) ok = cc_union(a.parent, pa, pb) && ok;
    }
    if (!ok) atomicOr(a.err, DEV_ERR_UNION);
}

// tile-local roots add their sizes to their global roots and point at them
__global__ void k_cc_count(CcArgs a)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.b.NV) return;
    const int ls = a.lsize[v];
    if (ls == 0 || a.S[v] != a.phase) return;
    const int thr = cc_threshold(a, a.b.sys[sys_v(a.b, v)]);
    if (thr <= 0) return;
    const int r = cc_root(a.parent, (int)v);
    if (__ldcg(a.size + r) < thr) atomicAdd(a.size + r, ls);
    __stcg(a.parent + v, r);
}

__global__ void k_cc_flip(CcArgs a)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.b.NV || a.S[v] != a.phase) return;
    const int thr = cc_threshold(a, a.b.sys[sys_v(a.b, v)]);
    if (thr <= 0) return;
    const int r = __ldcg(a.parent + __ldcg(a.parent + v));
    if (__ldcg(a.size + r) < thr) {
        a.S[v] = (uint8_t)(1 - a.phase);
        atomicAdd(&a.st->cc_flipped, 1ull);
    }
}

// the liquid pass's flip, then the vapor pass's tile labelling of the same
// tile (it reads only the tile's own labels)
__global__ void __launch_bounds__(CC_TILE) k_cc_flip_local(CcArgs a0, CcArgs a1)
{
    const CcTile c = cc_tile(a0);
    cc_flip(a0, c);
    __syncthreads();
    cc_local(a1, c);
}

// Section 4.2 on the labels S of the systems in b (the first systems of the
// handle: their voxels and tiles come first): seven launches, the tile
// passes one block per tile, the others one thread per voxel
int launch_components(dcm_handle *h, const Batch &b, uint8_t *S, int thr, int64_t tiles)
{
    cudaStream_t s = h->stream;
    if (b.NV <= 0 || tiles <= 0) return DCM_OK;
    CcArgs a[2];
    for (int phase = 0; phase <= 1; ++phase) {
        a[phase].b = b;
        a[phase].S = S;
        a[phase].parent = h->cc + (2 * phase) * h->b.NV;
        a[phase].size = h->cc + (2 * phase + 1) * h->b.NV;
        a[phase].lsize = h->cc + 4 * h->b.NV;
        a[phase].uniform = h->cc + 5 * h->b.NV;
        a[phase].tile_off = h->cc_tiles;
        a[phase].phase = phase;
        a[phase].thr = thr;
        a[phase].err = h->err;
        a[phase].st = h->stats;
    }
    const unsigned tgrid = (unsigned)tiles;
    const unsigned vgrid = (unsigned)((b.NV + CC_THREADS - 1) / CC_THREADS);
    k_cc_local<<<tgrid, CC_TILE, 0, s>>>(a[0]);
    k_cc_global<<<vgrid, CC_THREADS, 0, s>>>(a[0]);
    k_cc_count<<<vgrid, CC_THREADS, 0, s>>>(a[0]);
    k_cc_flip_local<<<tgrid, CC_TILE, 0, s>>>(a[0], a[1]);
    k_cc_global<<<vgrid, CC_THREADS, 0, s>>>(a[1]);
    k_cc_count<<<vgrid, CC_THREADS, 0, s>>>(a[1]);
    k_cc_flip<<<vgrid, CC_THREADS, 0, s>>>(a[1]);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DCM_OK : fail_cuda(e, "component launch", __FILE__, __LINE__);
}

}  // namespace dcm
