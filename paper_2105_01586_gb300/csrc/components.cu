// components.cu -- connected components of the unknown-vertex graph and a
// component-ordered numbering of the unknowns (rows of A_UU, Sec. 2.2).
//
// A_UU couples two unknown vertices only through a mesh edge with a nonzero
// stiffness entry.  In meshes made by the spatial optimisation nearly every
// unknown vertex sits among mask vertices, so A_UU splits into many small
// independent blocks: a 4 % mesh of a 2049 x 2049 image has 19,622 unknowns
// in 9,561 blocks, the largest with 224 rows.  When the unknowns are
// numbered component by component, each block is a contiguous range of rows
// whose columns stay inside the range, and the solver treats the blocks as
// independent systems (solve_comp.cu).
//
// The numbering does not depend on thread scheduling: components are
// ordered by their smallest vertex id, the rows of a component by vertex id.
//   1. union-find over the edges (parents start at the smallest unknown
//      neighbour; the larger root is hooked under the smaller one by
//      atomicCAS; finds halve paths), so the final root of a component is
//      its smallest vertex;
//   2. sizes per root, then one scan over the roots gives the first row of
//      each component;
//   3. members are dropped into their component's range in any order, and
//      each range is sorted by vertex id (a warp with shuffles, a block in
//      shared memory, or a block in global memory for long ranges).
// Components are then addressed by their first row (rowcomp holds their
// size there), listed by size class for the solver.
#include <algorithm>
#include <climits>

#include "fem_internal.cuh"

namespace fem {

constexpr int kSortSmem = 4096;   // ranges up to this size are sorted in shared memory
constexpr int kSortThreads = 256;
constexpr int kUniteCap = 1 << 20;

// Root of x.  Parents only point to smaller ids, so the walk ends; path
// halving stores an ancestor, which stays an ancestor as trees merge.
__device__ __forceinline__ int cc_find(int* parent, int x) {
    for (;;) {
        int p = ld_volatile_i32(parent + x);
        if (p == x) return x;
        int gp = ld_volatile_i32(parent + p);
        if (gp == p) return p;
        parent[x] = gp;
        x = gp;
    }
}

// One thread per (vertex, direction) slot: each edge is united once, from
// its larger endpoint.  A thread follows one chain of dependent loads only.
__global__ void k_cc_hook(const unsigned char* __restrict__ mask, const int* __restrict__ nbr,
                          const float* __restrict__ coef, int V, int* parent, int* __restrict__ err) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8LL * V) return;
    int v = (int)(t % V);
    int j = nbr[t];
    if (j < 0 || j >= v || mask[v] || coef[t] == 0.0f || mask[j]) return;
    int a = v, b = j;
    bool done = false;
    for (int it = 0; it < kUniteCap && !done; ++it) {
        a = cc_find(parent, a);
        b = cc_find(parent, b);
        if (a == b) { done = true; break; }
        if (a < b) { int x = a; a = b; b = x; }
        done = atomicCAS(parent + a, a, b) == a;
    }
    if (!done) atomicCAS(err, 0, (int)FEM_E_INVALID);
}

// Final root of every unknown vertex (into a separate array: a path-halving
// find here could overwrite a root just stored by another thread with an
// older ancestor) and the component sizes.  The forest no longer changes, so
// a read-only walk suffices.
__global__ void k_cc_flatten(const unsigned char* __restrict__ mask, int V, const int* __restrict__ parent,
                             int* __restrict__ root, int* __restrict__ size) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V || mask[v]) return;
    int r = v;
    for (int p = parent[r]; p != r; p = parent[r]) r = p;
    root[v] = r;
    atomicAdd(size + r, 1);
}

// Members into their ranges (any order).  Every member writes its slot of
// rowcomp (the size at the component's first row, 0 elsewhere); the root
// lists its component by size class; a one-row component needs no sort, so
// its vertex gets its row here.
__global__ void k_cc_place(const unsigned char* __restrict__ mask, int V, const int* __restrict__ root,
                           const int* __restrict__ size, const int* __restrict__ cstart, int* __restrict__ fill,
                           int* __restrict__ members, int* __restrict__ rowcomp, int* __restrict__ uidx,
                           int* __restrict__ blk_list, int* __restrict__ warp_list, int* __restrict__ cnt, int nU) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V || mask[v]) return;
    int r = root[v], sz = size[r], st = cstart[r];
    int slot = st + atomicAdd(fill + r, 1);
    if (slot >= nU || st + sz > nU) {  // more unknowns than rows: a malformed mesh count
        atomicCAS(cnt + CC_ERR, 0, (int)FEM_E_INVALID);
        return;
    }
    members[slot] = v;
    rowcomp[slot] = slot == st ? sz : 0;
    if (sz == 1) uidx[v] = slot;
    if (r == v) {
        if (sz > kWarpComp) {
            blk_list[atomicAdd(cnt + CC_NBLK, 1)] = st;
            if (sz > kBlockComp) atomicAdd(cnt + CC_NBIG, 1);
        } else if (sz > 1) {
            warp_list[atomicAdd(cnt + CC_NWARP, 1)] = st;
        }
    }
}

// All-ascending bitonic network: for each merge size k, compare i with its
// mirror i ^ (k - 1), then with i ^ s for s = k/4 .. 1; the smaller key goes
// to the smaller index.  Keys past the range act as +infinity, which never
// moves, so a range is sorted in place without padding.
__device__ __forceinline__ void cas_asc(int* a, int lo, int hi, int n) {
    if (hi >= n) return;
    int x = a[lo], y = a[hi];
    if (y < x) { a[lo] = y; a[hi] = x; }
}

__device__ void block_sort_range(int* a, int n) {
    int P = 1;
    while (P < n) P <<= 1;
    for (int k = 2; k <= P; k <<= 1) {
        int h = k >> 1;
        for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
            int blk = i / h, off = i % h;
            cas_asc(a, blk * k + off, blk * k + k - 1 - off, n);
        }
        __syncthreads();
        for (int s = k >> 2; s > 0; s >>= 1) {
            for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
                int lo = (i / s) * 2 * s + i % s;
                cas_asc(a, lo, lo + s, n);
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ int warp_sort_asc(int key) {
    const unsigned FULL = 0xffffffffu;
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
        int j = lane ^ (k - 1);
        int o = __shfl_sync(FULL, key, j);
        key = lane < j ? min(key, o) : max(key, o);
#pragma unroll
        for (int s = k >> 2; s > 0; s >>= 1) {
            int j2 = lane ^ s;
            int o2 = __shfl_sync(FULL, key, j2);
            key = lane < j2 ? min(key, o2) : max(key, o2);
        }
    }
    return key;
}

// Sort every component's range by vertex id and write uidx (vertex -> row):
// blocks take the components above one warp, warps those of 2..32 rows.
__global__ void __launch_bounds__(kSortThreads) k_cc_sort(const int* __restrict__ rowcomp,
                                                           const int* __restrict__ blk_list,
                                                           const int* __restrict__ warp_list,
                                                           const int* __restrict__ cnt, int* __restrict__ members,
                                                           int* __restrict__ uidx) {
    __shared__ int s_keys[kSortSmem];
    if (cnt[CC_ERR] != 0) return;
    const int nblk = cnt[CC_NBLK], nwarp = cnt[CC_NWARP];
    for (int i = blockIdx.x; i < nblk; i += gridDim.x) {
        int s0 = blk_list[i], n = rowcomp[s0];
        int* rng = members + s0;
        if (n <= kSortSmem) {
            for (int k = threadIdx.x; k < n; k += blockDim.x) s_keys[k] = rng[k];
            __syncthreads();
            block_sort_range(s_keys, n);
            for (int k = threadIdx.x; k < n; k += blockDim.x) {
                int v = s_keys[k];
                rng[k] = v;
                uidx[v] = s0 + k;
            }
            __syncthreads();
        } else {
            block_sort_range(rng, n);
            for (int k = threadIdx.x; k < n; k += blockDim.x) uidx[rng[k]] = s0 + k;
            __syncthreads();
        }
    }
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = gw; i < nwarp; i += nw) {
        int s0 = warp_list[i], n = rowcomp[s0];
        int key = lane < n ? members[s0 + lane] : INT_MAX;
        key = warp_sort_asc(key);
        if (lane < n) {
            members[s0 + lane] = key;
            uidx[key] = s0 + lane;
        }
    }
}

fem_status build_components(fem_mesh* m, cudaStream_t s) {
    int V = m->V, nU = m->nU;
    size_t nr = (size_t)(nU > 0 ? nU : 1) + 1;
    FEM_TRY(ensure(m->cc_root, (size_t)V, s));
    FEM_TRY(ensure(m->cc_cstart, (size_t)V + 1, s));
    FEM_TRY(ensure(m->rowcomp, nr, s));
    FEM_TRY(ensure(m->blk_list, nr, s));
    FEM_TRY(ensure(m->warp_list, nr, s));
    FEM_CUDA(cudaMemsetAsync(m->ccount.p, 0, sizeof(int) * CC_COUNTERS, s));
    if (nU == 0) return FEM_OK;
    int vb = (V + 255) / 256;
    int* cnt = m->ccount.p;
    FEM_LAUNCH(F_ASSEMBLY, s, k_cc_hook, (int)((8LL * V + 255) / 256), 256, 0, m->mask.p, m->nbr.p, m->coefA.p, V,
               m->cc_parent.p, cnt + CC_ERR);
    FEM_LAUNCH(F_ASSEMBLY, s, k_cc_flatten, vb, 256, 0, m->mask.p, V, m->cc_parent.p, m->cc_root.p, m->cc_size.p);
    FEM_TRY(scan_component_rows(m, m->mask.p, m->cc_root.p, m->cc_size.p, m->cc_cstart.p, V, s, cnt + CC_NROWS));
    FEM_LAUNCH(F_ASSEMBLY, s, k_cc_place, vb, 256, 0, m->mask.p, V, m->cc_root.p, m->cc_size.p, m->cc_cstart.p,
               m->cc_fill.p, m->urow_vertex.p, m->rowcomp.p, m->uidx.p, m->blk_list.p, m->warp_list.p, cnt, nU);
    // about one component of 2..32 rows per warp (at most half the rows)
    int grid = std::max(1, std::min(m->num_sms * 8, (nU / 2 + 7) / 8));
    FEM_LAUNCH(F_ASSEMBLY, s, k_cc_sort, grid, kSortThreads, 0, m->rowcomp.p, m->blk_list.p, m->warp_list.p, cnt,
               m->urow_vertex.p, m->uidx.p);
    return FEM_OK;
}

}  // namespace fem
