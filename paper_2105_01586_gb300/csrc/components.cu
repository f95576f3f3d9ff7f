// components.cu -- the Laplace system of a mesh in one cooperative kernel:
// P1 stiffness per vertex and lattice direction (Sec. 2.2), the K/U split,
// the connected components of the unknown-vertex graph, a component-ordered
// numbering of the unknowns, and the ELL rows of A_UU.
//
// Every triangle of a newest-vertex-bisection mesh of the pixel square is a
// right isosceles triangle, so its P1 stiffness matrix is the same for all
// sizes: with c at the right angle, K_cc = 1, K_aa = K_bb = 1/2,
// K_ac = K_bc = -1/2, K_ab = 0.  All entries of A are multiples of 1/2 and
// exact in FP32, and their sums do not depend on the order of the additions.
// All edges point in one of 8 lattice directions, so A is stored per vertex
// and direction (nbr / coef, slot-major).
//
// A_UU couples two unknown vertices only through a mesh edge with a nonzero
// stiffness entry.  In meshes made by the spatial optimisation nearly every
// unknown vertex sits among mask vertices, so A_UU splits into many small
// independent blocks: a 4 % mesh of a 2049 x 2049 image has 19,622 unknowns
// in 10,233 blocks, the largest with 216 rows.  When the unknowns are
// numbered component by component, each block is a contiguous range of rows
// whose columns stay inside the range, and the solver treats the blocks as
// independent systems (solve_comp.cu).  The numbering does not depend on
// thread scheduling: components are ordered by their smallest vertex id, the
// rows of a component by vertex id.
//
// The phases, separated by bounded grid barriers (one launch instead of a
// chain of kernels and memsets):
//   0. clear the per-vertex stiffness arrays, the union-find forest (every
//      vertex its own parent) and the counters; count mask vertices per
//      chunk of vertices;
//   1. assemble: per triangle, neighbours and stiffness per direction; mask
//      vertices are numbered by the count of mask vertices before them;
//   2. union-find over the edges of A_UU (a thread per vertex takes the
//      edges to its smaller neighbours; the larger root is hooked under the
//      smaller by atomicCAS; finds halve paths), so the final root of a
//      component is its smallest vertex;
//   3. final roots (a read-only walk) and component sizes;
//   4. sums of the sizes at the roots per chunk of vertices;
//   5. their scan: the first row of each component;
//   6. members dropped into their component's range in any order; sizes at
//      the first rows; components listed by size class;
//   7. every range sorted by vertex id (a warp with shuffles, a block in
//      shared memory, or a block in global memory for long ranges);
//   8. ELL rows of A_UU, and (optionally) the right-hand side and start of a
//      solve on the current vertex values.
// Data written in one phase and read in a later one is read through L2
// (__ldcg): an SM's L1 is not kept coherent with other SMs' writes.
#include <algorithm>
#include <climits>

#include "fem_internal.cuh"
#include "scan.cuh"

namespace fem {

constexpr int kBuildThreads = 256;
static_assert(kBuildThreads == SCAN_BT, "the block scan assumes SCAN_BT threads");
constexpr int kSortSmem = 4096;  // ranges up to this size are sorted in shared memory
constexpr int kUniteCap = 1 << 20;
// Up to this many vertices one block builds the whole system: its phases are
// then separated by block barriers, which cost far less than grid barriers,
// while each thread takes a few more vertices per phase.
constexpr int kBuildOneBlockV = 512;

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

// All-ascending bitonic network: for each merge size k, compare i with its
// mirror i ^ (k - 1), then with i ^ s for s = k/4 .. 1; the smaller key goes
// to the smaller index.  Keys past the range act as +infinity, which never
// moves, so a range is sorted in place without padding.  GLOBAL: the range
// lives in global memory and was written by other blocks (loads through L2).
template <bool GLOBAL>
__device__ __forceinline__ void cas_asc(int* a, int lo, int hi, int n) {
    if (hi >= n) return;
    int x = GLOBAL ? __ldcg(a + lo) : a[lo], y = GLOBAL ? __ldcg(a + hi) : a[hi];
    if (y < x) { a[lo] = y; a[hi] = x; }
}

template <bool GLOBAL>
__device__ void block_sort_range(int* a, int n) {
    int P = 1;
    while (P < n) P <<= 1;
    for (int k = 2; k <= P; k <<= 1) {
        int h = k >> 1;
        for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
            int blk = i / h, off = i % h;
            cas_asc<GLOBAL>(a, blk * k + off, blk * k + k - 1 - off, n);
        }
        __syncthreads();
        for (int s = k >> 2; s > 0; s >>= 1) {
            for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
                int lo = (i / s) * 2 * s + i % s;
                cas_asc<GLOBAL>(a, lo, lo + s, n);
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

// integer sum over the block, the same value in every thread
__device__ __forceinline__ int block_sum_int(int v) {
    __shared__ int s_w[kBuildThreads / 32];
    __shared__ int s_tot;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) s_w[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < kBuildThreads / 32; ++i) t += s_w[i];
        s_tot = t;
    }
    __syncthreads();
    int t = s_tot;
    __syncthreads();
    return t;
}

// Exclusive scan over [0, n) inside the cooperative kernel, in two halves
// that the caller places in consecutive phases (a grid barrier between
// them): block b owns a contiguous chunk; scan_count sums in(i) over the
// chunk into tsum[b]; scan_emit adds the sums of the chunks before b and
// scans the chunk one element per thread per step, calling
// out(i, prefix, in(i)).  in(i) must give the same value in both halves.
__device__ __forceinline__ void scan_chunk(int n, int& lo, int& hi) {
    const int chunk = (n + gridDim.x - 1) / gridDim.x;
    lo = min(n, (int)blockIdx.x * chunk);
    hi = min(n, lo + chunk);
}

template <class In>
__device__ void scan_count(In in, int n, int* tsum) {
    int lo, hi;
    scan_chunk(n, lo, hi);
    int part = 0;
    for (int i = lo + threadIdx.x; i < hi; i += kBuildThreads) part += in(i);
    part = block_sum_int(part);
    if (threadIdx.x == 0) tsum[blockIdx.x] = part;
}

template <class In, class Out>
__device__ void scan_emit(In in, Out out, int n, const int* tsum, int* total) {
    int lo, hi;
    scan_chunk(n, lo, hi);
    const int b = blockIdx.x;
    int pre = 0;
    for (int j = threadIdx.x; j < b; j += kBuildThreads) pre += __ldcg(tsum + j);
    pre = block_sum_int(pre);
    if (total && b == (int)gridDim.x - 1 && threadIdx.x == 0) *total = pre + __ldcg(tsum + b);
    for (int base = lo; base < hi; base += kBuildThreads) {
        const int i = base + threadIdx.x;
        int v[1] = {i < hi ? in(i) : 0};
        const int own = v[0];
        const int seg = block_exclusive_scan<1>(v);
        if (i < hi) out(i, pre + v[0], own);
        pre += seg;
    }
}

struct BuildArgs {
    const int4* tri;
    const int2* vxy;
    const unsigned char* mask;
    int T, V, nU;
    int* nbr;
    float* coef;
    float* diag;
    int* parent;
    int* root;
    int* size;
    int* fill;
    int* cstart;
    int* uidx;
    int* kidx;
    int* kvert;
    int* members;  // urow_vertex: vertex of each row
    int* ulist;    // the unknown vertices in ascending id (phase 1)
    int* rowcomp;
    int* blk_list;
    int* warp_list;
    int* cnt;      // CC_* counters
    int* nU_dev;
    int* ucol;
    float* uval;
    float* udiag;
    int* ucnt;
    float* udinv;
    double* udinv64;
    const double* uv;  // right-hand side and start (optional: b == nullptr)
    double* b;
    double* x;
    int* tsum;  // per-block sums of the scans
    unsigned* bar;
    int* err;
    // ahead of the host (dV != nullptr): V and T are the counts before the
    // refinement round and the refined mesh has V + *dV vertices and
    // T + *dT triangles; nothing is built when the round failed (guard[7]:
    // closure or top-k error, guard[9]: scan error) or when the refined mesh
    // exceeds the capacities Vcap (every per-vertex and per-unknown array)
    // and Tcap (triangles).  nU < 0: the unknown count is the kernel's own.
    const int* dV;
    const int* dT;
    const int* guard;
    int Vcap, Tcap;
    // only the rows of unknown vertices (nbr, coef, diag): all that the
    // Laplace solve reads; the adjoint also reads the mask vertices' rows
    bool unknown_rows;
};

struct UnknownFlagIn {
    const unsigned char* mask;
    __device__ __forceinline__ int operator()(int i) const { return mask[i] ? 0 : 1; }
};

struct IndexMapOut {
    const BuildArgs* A;
    __device__ __forceinline__ void operator()(int i, int u, int unk) const {
        const BuildArgs& a = *A;
        if (!unk) {
            int k = i - u;
            a.kidx[i] = k;
            a.kvert[k] = i;
            a.uidx[i] = -1;
        } else {
            a.kidx[i] = -1;
            a.ulist[u] = i;
        }
    }
};

// over the unknown list: the component size at a root, else 0
struct RootSizeIn {
    const BuildArgs* A;
    __device__ __forceinline__ int operator()(int k) const {
        const BuildArgs& a = *A;
        const int v = __ldcg(a.ulist + k);
        return __ldcg(a.root + v) == v ? __ldcg(a.size + v) : 0;
    }
};

// the first row of the component at root ulist[k]
struct CStartOut {
    const BuildArgs* A;
    __device__ __forceinline__ void operator()(int k, int pre, int) const {
        const BuildArgs& a = *A;
        a.cstart[__ldcg(a.ulist + k)] = pre;
    }
};

// the kernel stops at a failed barrier; the solve then reports the code
__device__ __forceinline__ void build_fail(const BuildArgs& A) {
    if (threadIdx.x == 0) atomicCAS(A.cnt + CC_ERR, 0, (int)FEM_E_TIMEOUT);
}

__global__ void __launch_bounds__(kBuildThreads) k_build_system(BuildArgs A) {
    pdl_wait();
    __shared__ int s_keys[kSortSmem];
    const int tid0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    int V = A.V, T = A.T;
    if (A.dV) {
        // every block reads the same words, so all return or none does
        if (ld_volatile_i32(A.guard + 7) != 0 || ld_volatile_i32(A.guard + 9) != 0) return;
        V += __ldcg(A.dV);
        T += __ldcg(A.dT);
        if (V > A.Vcap || T > A.Tcap) return;
    }
    const long long V8 = 8LL * V;
    // 0. clear; union-find forest of singletons; mask counts per chunk
    if (!A.unknown_rows) {
        for (long long i = tid0; i < V8; i += stride) {
            A.nbr[i] = -1;
            A.coef[i] = 0.0f;
        }
    }
    for (int i = tid0; i < V; i += stride) {
        if (A.unknown_rows) {
            if (A.mask[i]) continue;
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                A.nbr[(size_t)d * V + i] = -1;
                A.coef[(size_t)d * V + i] = 0.0f;
            }
        }
        A.diag[i] = 0.0f;
        A.parent[i] = i;
        A.size[i] = 0;
        A.fill[i] = 0;
    }
    if (tid0 < CC_COUNTERS) A.cnt[tid0] = 0;
    scan_count(UnknownFlagIn{A.mask}, V, A.tsum);
    if (!grid_barrier(A.bar, A.err)) { build_fail(A); return; }
    // 1. assemble: legs (c,a) and (c,b) carry -1/2 each, the hypotenuse is
    //    adjacency only; K_cc = 1, K_aa = K_bb = 1/2 on the diagonal.
    //    Mask vertices are numbered by the count of mask vertices before them.
    //    With unknown_rows a triangle writes only its unknown corners' rows
    //    (and none when all three are mask vertices).
    for (int t = tid0; t < T; t += stride) {
        int4 tr = A.tri[t];
        int a = tr.x, b = tr.y, c = tr.z;
        const bool ra = !A.unknown_rows || !A.mask[a];
        const bool rb = !A.unknown_rows || !A.mask[b];
        const bool rc = !A.unknown_rows || !A.mask[c];
        if (!(ra || rb || rc)) continue;
        int2 pa = A.vxy[a], pb = A.vxy[b], pc = A.vxy[c];
        int d = dir_index(pa.x - pc.x, pa.y - pc.y);
        if (rc) {
            A.nbr[(size_t)d * V + c] = a;
            atomicAdd(A.coef + (size_t)d * V + c, -0.5f);
        }
        d = (d + 4) & 7;
        if (ra) {
            A.nbr[(size_t)d * V + a] = c;
            atomicAdd(A.coef + (size_t)d * V + a, -0.5f);
        }
        d = dir_index(pb.x - pc.x, pb.y - pc.y);
        if (rc) {
            A.nbr[(size_t)d * V + c] = b;
            atomicAdd(A.coef + (size_t)d * V + c, -0.5f);
        }
        d = (d + 4) & 7;
        if (rb) {
            A.nbr[(size_t)d * V + b] = c;
            atomicAdd(A.coef + (size_t)d * V + b, -0.5f);
        }
        d = dir_index(pb.x - pa.x, pb.y - pa.y);
        if (ra) A.nbr[(size_t)d * V + a] = b;
        if (rb) A.nbr[(size_t)((d + 4) & 7) * V + b] = a;
        if (rc) atomicAdd(A.diag + c, 1.0f);
        if (ra) atomicAdd(A.diag + a, 0.5f);
        if (rb) atomicAdd(A.diag + b, 0.5f);
    }
    scan_emit(UnknownFlagIn{A.mask}, IndexMapOut{&A}, V, A.tsum, A.nU_dev);
    if (!grid_barrier(A.bar, A.err)) { build_fail(A); return; }
    const int nU = A.nU >= 0 ? A.nU : __ldcg(A.nU_dev);
    if (nU == 0) return;  // uniform: no unknowns, no components
    // 2. union-find over the edges of A_UU, each from its larger endpoint;
    //    the 8 slots of a vertex are loaded together.  Phases 2-6 run over
    //    the list of unknowns (a few per cent of the vertices), in ascending
    //    vertex id, which keeps the numbering of the vertex-order loops.
    const int nUl = __ldcg(A.nU_dev);
    for (int k = tid0; k < nUl; k += stride) {
        const int v = __ldcg(A.ulist + k);
        int nb[8];
        float cf[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            nb[d] = __ldcg(A.nbr + (size_t)d * V + v);
            cf[d] = __ldcg(A.coef + (size_t)d * V + v);
        }
        bool on[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) on[d] = nb[d] >= 0 && nb[d] < v && cf[d] != 0.0f;
#pragma unroll
        for (int d = 0; d < 8; ++d) on[d] = on[d] && !A.mask[nb[d]];
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            if (!on[d]) continue;
            int a = v, b = nb[d];
            bool done = false;
            for (int it = 0; it < kUniteCap && !done; ++it) {
                a = cc_find(A.parent, a);
                b = cc_find(A.parent, b);
                if (a == b) { done = true; break; }
                if (a < b) { int x = a; a = b; b = x; }
                done = atomicCAS(A.parent + a, a, b) == a;
            }
            if (!done) atomicCAS(A.cnt + CC_ERR, 0, (int)FEM_E_INVALID);
        }
    }
    if (!grid_barrier(A.bar, A.err)) { build_fail(A); return; }
    // 3. final roots (into a separate array: the forest no longer changes)
    //    and component sizes
    for (int k = tid0; k < nUl; k += stride) {
        const int v = __ldcg(A.ulist + k);
        int r = v;
        for (int p = __ldcg(A.parent + r); p != r; p = __ldcg(A.parent + r)) r = p;
        A.root[v] = r;
        atomicAdd(A.size + r, 1);
    }
    if (!grid_barrier(A.bar, A.err)) { build_fail(A); return; }
    // 4.-5. first row of each component: scan of the sizes at the roots
    scan_count(RootSizeIn{&A}, nUl, A.tsum);
    if (!grid_barrier(A.bar, A.err)) { build_fail(A); return; }
    scan_emit(RootSizeIn{&A}, CStartOut{&A}, nUl, A.tsum, A.cnt + CC_NROWS);
    if (!grid_barrier(A.bar, A.err)) { build_fail(A); return; }
    // 6. members into their ranges; a one-row component needs no sort
    for (int k = tid0; k < nUl; k += stride) {
        const int v = __ldcg(A.ulist + k);
        int r = __ldcg(A.root + v), sz = __ldcg(A.size + r), st = __ldcg(A.cstart + r);
        int slot = st + atomicAdd(A.fill + r, 1);
        if (slot >= nU || st + sz > nU) {  // more unknowns than rows: a malformed mesh count
            atomicCAS(A.cnt + CC_ERR, 0, (int)FEM_E_INVALID);
            continue;
        }
        A.members[slot] = v;
        A.rowcomp[slot] = slot == st ? sz : 0;
        if (sz == 1) A.uidx[v] = slot;
        if (r == v) {
            if (sz > kWarpComp) {
                A.blk_list[atomicAdd(A.cnt + CC_NBLK, 1)] = st;
                if (sz > kBlockComp) atomicAdd(A.cnt + CC_NBIG, 1);
            } else if (sz > 1) {
                A.warp_list[atomicAdd(A.cnt + CC_NWARP, 1)] = st;
            }
        }
    }
    if (!grid_barrier(A.bar, A.err)) { build_fail(A); return; }
    // 7. sort every range by vertex id and write uidx (vertex -> row)
    if (__ldcg(A.cnt + CC_ERR) == 0) {
        const int nblk = __ldcg(A.cnt + CC_NBLK), nwarp = __ldcg(A.cnt + CC_NWARP);
        for (int i = blockIdx.x; i < nblk; i += gridDim.x) {
            int s0 = __ldcg(A.blk_list + i), n = __ldcg(A.rowcomp + s0);
            int* rng = A.members + s0;
            if (n <= kSortSmem) {
                for (int k = threadIdx.x; k < n; k += blockDim.x) s_keys[k] = __ldcg(rng + k);
                __syncthreads();
                block_sort_range<false>(s_keys, n);
                for (int k = threadIdx.x; k < n; k += blockDim.x) {
                    int v = s_keys[k];
                    rng[k] = v;
                    A.uidx[v] = s0 + k;
                }
                __syncthreads();
            } else {
                block_sort_range<true>(rng, n);
                for (int k = threadIdx.x; k < n; k += blockDim.x) A.uidx[__ldcg(rng + k)] = s0 + k;
                __syncthreads();
            }
        }
        const int lane = threadIdx.x & 31;
        const int gw = tid0 >> 5, nw = stride >> 5;
        for (int i = gw; i < nwarp; i += nw) {
            int s0 = __ldcg(A.warp_list + i), n = __ldcg(A.rowcomp + s0);
            int key = lane < n ? __ldcg(A.members + s0 + lane) : INT_MAX;
            key = warp_sort_asc(key);
            if (lane < n) {
                A.members[s0 + lane] = key;
                A.uidx[key] = s0 + lane;
            }
        }
    }
    if (!grid_barrier(A.bar, A.err)) { build_fail(A); return; }
    if (__ldcg(A.cnt + CC_ERR) != 0) return;  // rows incomplete: the solve reports the code
    // 8. ELL rows of A_UU (padded with the own row and value 0); with b the
    //    right-hand side b_r = -sum over mask neighbours of A_ij uv_j and the
    //    start x_r = uv of the row's vertex
    for (int r = tid0; r < nU; r += stride) {
        int i = __ldcg(A.members + r);
        int s = 0;
        double bs = 0.0;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            int j = __ldcg(A.nbr + (size_t)d * V + i);
            float c = __ldcg(A.coef + (size_t)d * V + i);
            if (j >= 0 && c != 0.0f) {
                int uj = __ldcg(A.uidx + j);
                if (uj >= 0) {
                    A.ucol[(size_t)s * nU + r] = uj;
                    A.uval[(size_t)s * nU + r] = c;
                    s++;
                } else if (A.b) {
                    bs -= (double)c * A.uv[j];
                }
            }
        }
        A.ucnt[r] = s;
        for (; s < 8; ++s) {
            A.ucol[(size_t)s * nU + r] = r;
            A.uval[(size_t)s * nU + r] = 0.0f;
        }
        float dg = __ldcg(A.diag + i);
        A.udiag[r] = dg;
        A.udinv[r] = 1.0f / dg;
        A.udinv64[r] = 1.0 / (double)dg;
        if (A.b) {
            A.b[r] = bs;
            A.x[r] = A.uv[i];
        }
    }
}

// algorithmic bytes of a build: the mesh read once (16 B per triangle,
// 9 B per vertex), the stencil and index maps written once (76 B per
// vertex, 4 B per mask vertex), the ELL rows with diagonal, inverse
// diagonals, row counts, vertex and component of each row (92 B per
// unknown); with the right-hand side, 8 B per vertex read and 16 B per
// unknown written.  The union-find forest is working state, not counted.
// With the unknown vertices' rows only: the triangles (16 B) and the mask
// (1 B per vertex) read, the index maps written (4 B per vertex, 4 B per
// mask vertex), the stencil rows of the unknowns (68 B) with their ELL
// rows (92 B), and for the right-hand side the values of the at most 8
// neighbours and the own vertex read (72 B) and 16 B written per unknown.
double build_bytes(long long T, long long V, long long nU, bool rhs, bool unknown_rows) {
    if (unknown_rows)
        return 16.0 * T + 5.0 * V + 4.0 * (V - nU) + 160.0 * nU + (rhs ? 88.0 * nU : 0.0);
    return 16.0 * T + 85.0 * V + 4.0 * (V - nU) + 92.0 * nU + (rhs ? 8.0 * V + 16.0 * nU : 0.0);
}

namespace {

// Ensure the system arrays for nv vertices and nu unknowns (nu <= nv) and
// launch k_build_system on the mesh counts V, T (host) or, ahead of the
// host, on the counts of the round in flight (dV, dT, guard; then nU < 0).
fem_status launch_build(fem_mesh* m, cudaStream_t s, int V, int T, int nU, size_t nv, size_t nu, bool rhs,
                        const int* dV, const int* dT, const int* guard, int Vcap, int Tcap, bool unknown_rows) {
    const size_t n = nu > 0 ? nu : 1, nr = n + 1;
    FEM_TRY(ensure(m->nbr, (size_t)8 * nv, s));
    FEM_TRY(ensure(m->coefA, (size_t)8 * nv, s));
    FEM_TRY(ensure(m->diagA, nv, s));
    FEM_TRY(ensure(m->uidx, nv, s));
    FEM_TRY(ensure(m->kidx, nv, s));
    FEM_TRY(ensure(m->urow_vertex, nv, s));
    FEM_TRY(ensure(m->ulist, nv, s));
    FEM_TRY(ensure(m->kvert, nv, s));
    FEM_TRY(ensure(m->cc_parent, nv, s));
    FEM_TRY(ensure(m->cc_root, nv, s));
    FEM_TRY(ensure(m->cc_size, nv, s));
    FEM_TRY(ensure(m->cc_fill, nv, s));
    FEM_TRY(ensure(m->cc_cstart, nv + 1, s));
    FEM_TRY(ensure(m->rowcomp, nr, s));
    FEM_TRY(ensure(m->blk_list, nr, s));
    FEM_TRY(ensure(m->warp_list, nr, s));
    FEM_TRY(ensure(m->ucol, 8 * n, s));
    FEM_TRY(ensure(m->uval32, 8 * n, s));
    FEM_TRY(ensure(m->udiag, n, s));
    FEM_TRY(ensure(m->ucnt, n, s));
    FEM_TRY(ensure(m->dinv32, n, s));
    FEM_TRY(ensure(m->dinv64, n, s));
    if (rhs) {
        FEM_TRY(ensure(m->b64, n, s));
        FEM_TRY(ensure(m->x64, n, s));
    }
    static const int occ = [] {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)k_build_system, kBuildThreads, 0);
        return nb < 1 ? 1 : nb;
    }();
    // one block for small systems; else about one vertex per thread, at most
    // the co-resident blocks
    const int grid = V <= kBuildOneBlockV
                         ? 1
                         : std::max(1, std::min(occ * m->num_sms, (V + kBuildThreads - 1) / kBuildThreads));
    FEM_TRY(ensure(m->scan_pre, (size_t)grid + 1, s));
    BuildArgs A;
    A.tri = m->tri.p;
    A.vxy = m->vxy.p;
    A.mask = m->mask.p;
    A.T = T;
    A.V = V;
    A.nU = nU;
    A.nbr = m->nbr.p;
    A.coef = m->coefA.p;
    A.diag = m->diagA.p;
    A.parent = m->cc_parent.p;
    A.root = m->cc_root.p;
    A.size = m->cc_size.p;
    A.fill = m->cc_fill.p;
    A.cstart = m->cc_cstart.p;
    A.uidx = m->uidx.p;
    A.kidx = m->kidx.p;
    A.kvert = m->kvert.p;
    A.members = m->urow_vertex.p;
    A.ulist = m->ulist.p;
    A.rowcomp = m->rowcomp.p;
    A.blk_list = m->blk_list.p;
    A.warp_list = m->warp_list.p;
    A.cnt = m->ccount.p;
    A.nU_dev = m->dcount.p + 1;
    A.ucol = m->ucol.p;
    A.uval = m->uval32.p;
    A.udiag = m->udiag.p;
    A.ucnt = m->ucnt.p;
    A.udinv = m->dinv32.p;
    A.udinv64 = m->dinv64.p;
    A.uv = m->uv.p;
    A.b = rhs ? m->b64.p : nullptr;
    A.x = rhs ? m->x64.p : nullptr;
    A.tsum = m->scan_pre.p;
    A.bar = m->bar.p;
    A.err = m->dflag.p + 2;
    A.dV = dV;
    A.dT = dT;
    A.guard = guard;
    A.Vcap = Vcap;
    A.Tcap = Tcap;
    A.unknown_rows = unknown_rows;
    // *A.err is zero: cleared at creation, left at zero by every completed
    // launch, and cleared again after a failed one (reset_coop_state)
    void* args[] = {&A};
    return launch_coop(F_ASSEMBLY, (const void*)k_build_system, grid, kBuildThreads, 0, s, args, "k_build_system");
}

}  // namespace

// with_rhs (optional): on input asks for b64/x64 of a solve on the current
// vertex values to be filled with the system; on output true when that
// happened (the system was rebuilt, or built ahead with them by the last
// refinement round), false when the caller must fill them
fem_status build_system_rhs(fem_mesh* m, cudaStream_t s, bool* with_rhs) {
    bool want = with_rhs && *with_rhs;
    if (with_rhs) *with_rhs = false;
    if (m->sys_version == m->mesh_version && (m->sys_full || m->unknown_rows_ok)) {
        if (want && m->rhs_fresh) *with_rhs = true;
        m->rhs_fresh = false;
        return FEM_OK;
    }
    m->rhs_fresh = false;
    const int V = m->V, T = m->T;
    // the mask count is kept on the host by create / import / refinement, so
    // the unknown count needs no read-back
    const int nU = V - m->nK;
    m->nU = nU;
    const bool rhs = want && nU > 0;
    FEM_TRY(launch_build(m, s, V, T, nU, (size_t)V, (size_t)(nU > 0 ? nU : 1), rhs, nullptr, nullptr, nullptr, 0, 0,
                         false));
    note_bytes(F_ASSEMBLY, build_bytes(T, V, nU, rhs));
    if (rhs) *with_rhs = true;
    m->sys_version = m->mesh_version;
    m->sys_full = true;
    return FEM_OK;
}


// The system of the mesh that the refinement round in flight produces,
// launched behind that round's last kernel before the host has read the
// round's counts (mesh of V vertices and T triangles before the round; the
// refined counts are the round's device counters, guard the round's staged
// status words).  The arrays are sized for V + V/4 + 64 vertices; the kernel
// builds nothing when the refined mesh is larger, or when the round failed.
// *Vcap / *Tcap receive the capacities: the caller knows the system is built
// once it has read counts within them.
fem_status build_system_ahead(fem_mesh* m, cudaStream_t s, int V, int T, const int* guard, int* Vcap, int* Tcap) {
    const size_t nv = (size_t)V + V / 4 + 64;
    long long vc = (long long)std::min({nv, m->vxy.n, m->mask.n, m->uv.n, m->uvf.n});
    long long tc = (long long)m->tri.n;
    *Vcap = (int)std::min<long long>(vc, INT_MAX);
    *Tcap = (int)std::min<long long>(tc, INT_MAX);
    return launch_build(m, s, V, T, -1, nv, nv, true, m->dcount.p + 4, m->dcount.p + 5, guard, *Vcap, *Tcap, true);
}

fem_status build_system(fem_mesh* m, cudaStream_t s) { return build_system_rhs(m, s, nullptr); }

}  // namespace fem
