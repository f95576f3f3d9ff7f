// fem_internal.cuh -- internal declarations of the GB300 FEM inpainting library.
//
// Device data layout (all arrays live in HBM, owned by the mesh handle):
//   vxy[V]   int2   vertex pixel positions (x, y)
//   mask[V]  uint8  1 = mask vertex (Dirichlet set K), 0 = unknown vertex (U)
//   tri[T]   int4   (a, b, c, 0): refinement edge (a, b), newest vertex c
//   uv[V]    double vertex values (g at K, Laplace solution at U), kept
//                   between rounds as the warm start
// Per-round scratch is sized by capacity and reused.
#pragma once
#include <atomic>
#include <utility>

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/feminpaint.h"
#include <nvtx3/nvToolsExt.h>

namespace fem {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);

// NVTX range for the lifetime of a scope: API calls, spatial rounds, Laplace
// solves and tonal iterations show up by name in Nsight timelines (a no-op
// unless a tool is attached).
struct Nvtx {
    explicit Nvtx(const char* name) { nvtxRangePushA(name); }
    ~Nvtx() { nvtxRangePop(); }
    Nvtx(const Nvtx&) = delete;
    Nvtx& operator=(const Nvtx&) = delete;
};
fem_status cuda_fail(cudaError_t e, const char* what);

#define FEM_CUDA(call)                                              \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return ::fem::cuda_fail(e_, #call);  \
    } while (0)

#define FEM_TRY(expr)                        \
    do {                                     \
        fem_status s_ = (expr);              \
        if (s_ != FEM_OK) return s_;         \
    } while (0)

// ------------------------------------------------------ launch accounting
// F_SQPASS: the square-tiled FP32 error pass (one kernel, so
// that its roofline can be taken alone); the rest of the error work (plan,
// band, image layout) is F_RASTER
enum Family { F_RASTER = 0, F_CG = 1, F_ASSEMBLY = 2, F_TOPK = 3, F_REFINE = 4, F_TONAL = 5, F_OTHER = 6, F_SQPASS = 7,
              F_COUNT = 8 };
void note_launch_begin(int family, cudaStream_t s);
bool profiling(int family);
// algorithmic bytes moved by work of a family (counted only while profiling)
void note_bytes(int family, double bytes);
// algorithmic bytes of the incremental FP32 passes since the last call,
// counted on the device while F_SQPASS is profiled (raster_sq.cu)
double sq_inc_bytes_take();
void note_launch_end(int family, cudaStream_t s);

// Launch a kernel with accounting; returns FEM_E_CUDA on a launch error.
// Launches use programmatic dependent launch: the kernel may be set up
// while the previous kernel of the stream is still running, and every
// kernel of this library starts with pdl_wait(), which returns once the
// previous grid has completed and its memory is visible.  So the stream
// order of results is kept; only the launch latency is hidden.
bool pdl_enabled();

template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

#define FEM_LAUNCH(family, stream, kernel, grid, block, smem, ...)                                    \
    do {                                                                                              \
        ::fem::note_launch_begin((family), (stream));                                                 \
        cudaError_t e_ = ::fem::launch_pdl(kernel, dim3(grid), dim3(block), (smem), (stream), __VA_ARGS__); \
        ::fem::note_launch_end((family), (stream));                                                   \
        if (e_ != cudaSuccess) return ::fem::cuda_fail(e_, #kernel);                                  \
    } while (0)

// Cooperative launch (all blocks co-resident; used by kernels with grid barriers).
fem_status launch_coop(int family, const void* func, int grid, int block, size_t smem, cudaStream_t s,
                       void** args, const char* name);

// ------------------------------------------------------------ device utils
// First statement of every kernel: waits for the grid launched before it in
// the stream (a no-op for launches without the programmatic attribute).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) {
    return *(const volatile int*)p;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Bounded grid-wide barrier for cooperatively launched kernels, one atomic
// per block: block 0 adds 2^31 - (nb - 1) to bar[0], every other block adds
// 1, so the nb arrivals add exactly 2^31: the top bit of bar[0] flips with
// the last arrival and no earlier (every partial sum stays below 2^31), and
// the low 31 bits return to their value before the barrier.  A block waits
// until the top bit differs from the one its own arrival saw.  A block that
// waits longer than kBarrierLimitNs records FEM_E_TIMEOUT in *err and stops
// waiting; once *err is set every later barrier returns at once, so the
// kernel winds down (the word must then be cleared before the next launch).
// A grid of one block needs only the block barrier, which orders the block's
// global memory accesses; no other block can time out, so *err is not read.
// Returns false when the kernel must stop.
constexpr unsigned long long kBarrierLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err) {
    __syncthreads();
    if (gridDim.x * gridDim.y * gridDim.z == 1) return true;
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
        const bool first = blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
        const unsigned add = first ? 0x80000000u - (nb - 1u) : 1u;
        __threadfence();
        const unsigned old = atomicAdd(bar, add);
        if (((old + add) ^ old) & 0x80000000u) {
            // this arrival completed the barrier
        } else {
            unsigned long long t0 = globaltimer_ns();
            while (!((ld_acquire_u32(bar) ^ old) & 0x80000000u)) {
                if (ld_volatile_i32(err) != 0) { ok = 0; break; }
                if (globaltimer_ns() - t0 > kBarrierLimitNs) {
                    atomicCAS(err, 0, (int)FEM_E_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        if (ld_volatile_i32(err) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The pixel domain of a mesh: side N = 2^L + 1, and the W x H image at its
// top-left whose pixels alone are data (W = H = N for a square image).  A
// triangle owns the pixels of the ownership rule that lie in the image.  It
// can be selected when its refinement edge (a, b) can be bisected (the
// midpoint is a pixel) and its bounding box meets the image.
struct Dom {
    int N, W, H;
};

constexpr int kMaxChannels = 4;  // channels of a colour image in the spatial optimisation

__host__ __device__ __forceinline__ bool dom_eligible(int ax, int ay, int bx, int by, int cx, int cy, const Dom& D) {
    return (((ax + bx) | (ay + by)) & 1) == 0 && min(ax, min(bx, cx)) < D.W && min(ay, min(by, cy)) < D.H;
}

// Direction index (0..7) of a nonzero lattice step whose components are each
// -1, 0 or +1 after taking signs: E, NE(+x,+y), N(+y), NW, W, SW, S, SE.
__host__ __device__ __forceinline__ int dir_index(int dx, int dy) {
    int sx = (dx > 0) - (dx < 0), sy = (dy > 0) - (dy < 0);
    // table over (sx+1)*3 + (sy+1)
    const int tab[9] = {5, 4, 3, 6, -1, 2, 7, 0, 1};
    return tab[(sx + 1) * 3 + (sy + 1)];
}

// ------------------------------------------------------------ device arrays
template <class T>
struct DArr {
    T* p = nullptr;
    size_t n = 0;  // capacity in elements
};

fem_status dalloc_raw(void** p, size_t bytes, cudaStream_t s);
void dfree_raw(void* p, cudaStream_t s);

// Ensure capacity >= need; keep_n leading elements are preserved when growing.
template <class T>
fem_status ensure(DArr<T>& a, size_t need, cudaStream_t s, size_t keep_n = 0) {
    if (need <= a.n && a.p) return FEM_OK;
    size_t cap = a.n ? a.n : 64;
    while (cap < need) cap *= 2;
    void* np = nullptr;
    FEM_TRY(dalloc_raw(&np, cap * sizeof(T), s));
    if (keep_n && a.p) {
        cudaError_t e = cudaMemcpyAsync(np, a.p, keep_n * sizeof(T), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) { dfree_raw(np, s); return cuda_fail(e, "cudaMemcpyAsync(grow)"); }
    }
    if (a.p) dfree_raw(a.p, s);
    a.p = (T*)np;
    a.n = cap;
    return FEM_OK;
}

template <class T>
void release(DArr<T>& a, cudaStream_t s) {
    if (a.p) dfree_raw(a.p, s);
    a.p = nullptr;
    a.n = 0;
}

}  // namespace fem

// ------------------------------------------------------------------ mesh
struct fem_mesh {
    int N = 0;          // domain side (2^L + 1): the mesh lives on [0, N-1]^2
    long long P = 0;    // domain pixels N^2
    int W = 0, H = 0;   // the image, at the domain's top-left (W = H = N: square image)
    long long PI = 0;   // image pixels W H
    int V = 0, T = 0, nK = 0, nU = 0;
    int dev = 0, num_sms = 0;
    cudaStream_t last_stream = nullptr;
    // set by the server for a running request: the spatial rounds and the
    // tonal iterations stop with FEM_E_CANCELLED once it reads nonzero
    const std::atomic<int>* cancel = nullptr;

    // mesh proper
    fem::DArr<int2> vxy;
    fem::DArr<unsigned char> mask;
    fem::DArr<int4> tri;
    fem::DArr<double> uv;
    fem::DArr<int> order;      // triangle ids along the space-filling curve
    fem::DArr<int> order_tmp, ocnt, ooff;
    bool order_is_curve = true;  // the curve of the bisection tree (also after an import)
    fem::DArr<float2> uvf;  // float-float copy of uv, written with it in the spatial loop

    // rasterisation plan (valid for plan_T triangles of plan_version)
    fem::DArr<int> item_cnt, item_off, item_tri;
    // fast keys (FP32 with error bounds, exact band): intervals, histograms, band lists
    fem::DArr<float> keys_lo, keys_hi;
    fem::DArr<unsigned> fast_hist;
    fem::DArr<int> band;
    fem::DArr<double> partial;
    fem::DArr<double> keys;
    fem::DArr<unsigned long long> keyc;  // composite selection keys (eligible flag | key bits)
    long long plan_version = -1, mesh_version = 0;
    int n_items = 0;

    // refinement
    fem::DArr<unsigned> bmM, bmS, wpre;  // edge bitmaps: two buffers each, alternating by round
    int bm_parity = 0;
    bool bm_clean = false;              // the buffer of the next round is known to be clear
    fem::DArr<int> flags, fscan, wcnt;
    fem::DArr<unsigned> topk_hist;

    // Laplace system on U
    long long sys_version = -1;
    bool sys_full = false;          // the built system has every vertex's stiffness row
    bool unknown_rows_ok = false;   // set by the spatial loop: the unknowns' rows suffice
    bool rhs_fresh = false;         // b64/x64 hold the right-hand side and start of the built system
    cudaEvent_t round_ev = nullptr; // end of a refinement round's last kernel
    fem::DArr<int> uidx;            // vertex -> U row or -1
    fem::DArr<int> kidx;            // vertex -> K index or -1
    fem::DArr<int> nbr;             // 8*V neighbour per direction (-1 none)
    fem::DArr<float> coefA;         // 8*V stiffness entry per direction
    fem::DArr<float> diagA;         // V stiffness diagonal
    fem::DArr<int> ucol;            // 8*nU ELL columns (slot-major), padded with own row
    fem::DArr<float> uval32;        // 8*nU ELL values (0 in padding)
    fem::DArr<double> uval64;
    fem::DArr<float> udiag;         // nU diagonal of A_UU (exact)
    fem::DArr<int> ucnt;            // nU used ELL slots per row
    fem::DArr<float> dinv32;        // nU inverse diagonal
    fem::DArr<double> dinv64;
    fem::DArr<int> urow_vertex;     // nU: vertex of each U row (rows numbered by component)
    fem::DArr<int> ulist;           // nU: the unknown vertices in ascending id (system build)
    fem::DArr<int> gcnt;            // new-vertex numbering of large bitmaps: marks per group of words, prefixes
    // components of the unknown-vertex graph (components.cu)
    fem::DArr<int> cc_parent, cc_root, cc_size, cc_fill, cc_cstart;
    fem::DArr<int> rowcomp;     // nU: rows of the component starting at this row, else 0
    fem::DArr<int> blk_list;    // first rows of the components above one warp
    fem::DArr<int> warp_list;   // first rows of the components of 2..32 rows
    fem::DArr<int> ccount;      // CC_* counters
    fem::DArr<unsigned long long> comp_stats;  // component solve totals, zero between launches
    fem::DArr<int> kvert;           // nK: vertex of each K index
    // CG work
    fem::DArr<double> x64, b64, r64, p64, q64, z64;
    fem::DArr<float> r32, p32, q32, z32, d32;
    fem::DArr<float> bvec;              // one-block solve: global fallback vectors
    fem::DArr<int> browptr;
    fem::DArr<unsigned short> bent;
    fem::DArr<unsigned char> bdg2;
    fem::DArr<float2> bxff, bbff;       // float-float iterate and right-hand side
    fem::DArr<unsigned long long> scan_status;  // look-back scan tile status words
    fem::DArr<unsigned long long> scan_ctr;     // look-back scan tile counter
    fem::DArr<int> scan_vals, scan_pre;         // unfused scans of large inputs: values, prefixes
    unsigned long long scan_tiles_issued = 0;
    unsigned scan_epoch = 0;
    fem::DArr<double> red;          // grid-reduction partials
    fem::DArr<unsigned> bar;        // grid barrier words
    fem::DArr<int> dflag;           // device status/flags
    fem::DArr<double> dscal;        // device scalars
    fem::DArr<int> dcount;          // device counters

    // tonal (pixel mass matrix M = P^T P, incidence by sector)
    long long tonal_version = -1;
    fem::DArr<int> inc;             // 8*V triangle per sector (-1 none)
    fem::DArr<double> loc;          // 6*T local pixel-mass or 3*T scatter sums
    fem::DArr<double> Moff;         // 8*V pixel-mass off-diagonal per direction
    fem::DArr<double> Mdiag;        // V
    fem::DArr<double> tv, ty, tz, tg, tr, tp, tw, tc;  // tonal work vectors
    fem::DArr<double> tyr;             // tonal: y = P^T (f - B g), the residual recursion

    // square-tiled error pass (raster_sq.cu): the image as squares, the node
    // tables of the plan, per-node partial sums, the band's squares
    fem::DArr<float> fsq, fedge;       // Q*Q squares of s rows of s + 1 floats; the image's last row (N)
    fem::DArr<float> fpad;             // a W x H input image padded to the domain with its edge values
    // channels 1..3 of a colour image in the spatial optimisation (channel 0
    // uses uv, uvf, fsq, fedge, fpad), and the keys of one channel
    fem::DArr<double> uvc[3];
    fem::DArr<float2> uvfc[3];
    fem::DArr<float> fsqc[3], fedgec[3], fpadc[3];
    fem::DArr<double> keys_acc;
    fem::DArr<float> wimg, wfimg;      // IRLS weights w and w f of the L1 data term (domain layout)
    fem::DArr<int> sq_nodeof, sq_off;  // per curve position: node (fine) or -1; first bounding-box square
    fem::DArr<int> sq_pos;             // per triangle: its curve position
    fem::DArr<int> sq_bcoarse;         // curve positions of the band's coarse triangles
    fem::DArr<int> sq_cov, sq_slot;    // per node: covering triangle's curve position or -1; partial slot
    fem::DArr<int2> sq_seg;            // per node: curve segment of its triangles
    fem::DArr<float4> sq_part;         // partial sums (hi, lo, pixel count)
    fem::DArr<int> sq_coarse, sq_list; // curve positions of the coarse triangles; listed squares
    fem::DArr<int4> sq_long;           // long coarse triangles (curve position, first piece, pieces, slots)
    fem::DArr<int2> sq_piece;          // pieces of the long ones (triangle, index)
    fem::DArr<float4> sq_psum;         // their sums
    fem::DArr<int> sq_pdone;           // finished pieces per long triangle
    fem::DArr<int> sq_ctr;             // [0] coarse bounding-box squares, [1] coarse triangles
    fem::DArr<int4> sq_rec;            // 2 int4 per curve position: fine-triangle records of the FP32 pass
    fem::DArr<unsigned char> sq_mark, bsel;  // squares with a band triangle; band flag per triangle
    long long sq_plan_version = -1;
    // Incremental FP32 pass (spatial rounds after a call's first): the vertex
    // values the kept intervals were formed with, the triangles rewritten by
    // the last bisection, and the counts at that pass.
    fem::DArr<double> uvk;
    fem::DArr<float2> uvfk;
    fem::DArr<unsigned char> vchg, tchg, tdirty, sq_dmark;  // per vertex, triangle, triangle, square
    fem::DArr<unsigned char> hcnt;     // per triangle: its interval is counted in the histograms
    fem::DArr<int> sq_dlist;           // squares of the incremental pass
    int inc_V = 0, inc_T = 0;
    bool inc_ok = false;               // keys_lo/hi and uvk/uvfk belong to the current mesh
    fem::DArr<double> lossk, lossred;  // tonal loss: per-triangle squared errors, block partial sums

    // host staging (pinned)
    void* host_stage = nullptr;
    void* host_stage_dev = nullptr;  // the same memory as seen by kernels (mapped), or null
    bool round_ctr_clear = true;     // dcount[6..63] known to be zero (refinement rounds)

    fem_stats stats{};
};

namespace fem {
// A cancelled request stops between spatial rounds and tonal iterations.
inline Dom dom_of(const fem_mesh* m) { return Dom{m->N, m->W, m->H}; }

// The image the kernels read, indexed over the domain (pixel (x, y) at
// y N + x): f itself for a square image, else a copy of the W x H image f
// padded to N x N with the values of its nearest pixels (fem_mesh::fpad).
// Pixels outside the image are only ever read as the values of mask
// vertices there, never as data.
fem_status domain_image(fem_mesh* m, const float* f, cudaStream_t s, const float** out);

inline fem_status check_cancel(const fem_mesh* m) {
    if (m->cancel && m->cancel->load(std::memory_order_relaxed) != 0) {
        set_error("request cancelled");
        return FEM_E_CANCELLED;
    }
    return FEM_OK;
}

// component sizes: up to kWarpComp rows a warp solves the component, up to
// kBlockComp a block; a larger component sends the whole system to the
// grid-wide solver
constexpr int kWarpComp = 32;
constexpr int kBlockComp = 1024;
// counters of the component search (fem_mesh::ccount)
enum CcCounter { CC_NWARP = 0, CC_NROWS = 1, CC_NBLK = 2, CC_NBIG = 3, CC_ERR = 4, CC_WORK = 5, CC_DONE = 6,
                 CC_COUNTERS = 16 };
fem_status solve_components(fem_mesh* m, const double* b, double* x, bool use_fp64, double tol, int maxit,
                            bool deferred, bool scatter, int* clear_word, cudaStream_t s);

// helpers implemented in the .cu files
fem_status exclusive_scan_i32(const int* in, int* out, int n, cudaStream_t s, int* total_dev);
// the system of the current mesh, with every vertex's stiffness row (the
// tonal step's adjoint and pixel-mass products read the mask vertices'
// rows); inside the spatial loop (m->unknown_rows_ok) a system built ahead
// with the unknown vertices' rows only, all that a Laplace solve reads, is
// kept
fem_status build_system(fem_mesh* m, cudaStream_t s);
// with_rhs (optional): on input asks for b64/x64 of a solve on the current
// vertex values; on output true when the build filled them
fem_status build_system_rhs(fem_mesh* m, cudaStream_t s, bool* with_rhs);
// the system of the mesh the refinement round in flight produces, launched
// before the host reads the round's counts, with the unknown vertices' rows
// only (components.cu)
fem_status build_system_ahead(fem_mesh* m, cudaStream_t s, int V, int T, const int* guard, int* Vcap, int* Tcap);
// algorithmic bytes of one system build (unknown_rows: of the unknown
// vertices' stiffness rows only)
double build_bytes(long long T, long long V, long long nU, bool rhs, bool unknown_rows = false);
fem_status solve_laplace(fem_mesh* m, bool use_fp64, double tol, int maxit, cudaStream_t s,
                         int* iters_out, double* relres_out, bool deferred = false);
// scatter: the solution also goes to m->uv / m->uvf at the rows' vertices
fem_status run_solve(fem_mesh* m, const double* b, double* x, bool use_fp64, double tol, int maxit, cudaStream_t s,
                     int* iters_out, double* relres_out, bool deferred = false, bool scatter = false);
fem_status solve_totals_reset(fem_mesh* m, cudaStream_t s);
fem_status solve_totals_read(fem_mesh* m, cudaStream_t s);
fem_status set_uv_from_g(fem_mesh* m, const float* g_dev, cudaStream_t s);
fem_status set_uv_from_f(fem_mesh* m, const float* f_dev, cudaStream_t s);
fem_status raster_plan(fem_mesh* m, cudaStream_t s);
// exact keys of every triangle (square-tiled pass, raster_sq.cu); the image
// must have been laid out in squares by sq_image for the call
fem_status raster_errors(fem_mesh* m, const double* uv, const float2* uvf, double* err, cudaStream_t s,
                         unsigned long long* keyc_out = nullptr);
fem_status raster_image(fem_mesh* m, const double* uv, float* u, int* owner, cudaStream_t s);
fem_status raster_keys_fast(fem_mesh* m, const double* uv, const float2* uvf, double frac, long long vcap,
                            cudaStream_t s, bool incremental = false);
// the image f as squares for the square-tiled pass (once per call that reads f)
fem_status sq_image(fem_mesh* m, const float* f, cudaStream_t s);
fem_status raster_local(fem_mesh* m, int mode, const float* r, cudaStream_t s);
fem_status raster_weights(fem_mesh* m, const double* uv, const float* f, float eps, float* w_dom, float* wf_dom,
                          cudaStream_t s);
fem_status refine_round(fem_mesh* m, const float* f, double frac, long long vstar, cudaStream_t s,
                        double* margin_out, int* k_out, bool band = false);
// fast keys: histogram bins (top 16 bits of a non-negative float) and the
// counters after the two histograms in fem_mesh::fast_hist
constexpr int kFastBins = 32768;
// ints into fem_mesh::host_stage where a refinement round leaves its counters
constexpr int kRoundStageInts = 1024;
enum FastCounter { FC_IN = 0, FC_BAND = 1, FC_BAND_SQUARES = 2, FC_BAND_COARSE = 3 };
fem_status sync_counts(fem_mesh* m, cudaStream_t s);
fem_status ensure_mesh_capacity(fem_mesh* m, int needV, int needT, cudaStream_t s);
void reset_coop_state(fem_mesh* m, cudaStream_t s);
int sm_count();

// caller-provided scratch for the allocation-free error pass
struct RasterScratch {
    int* item_cnt;   // T
    int* item_off;   // T + 1
    int* item_tri;   // item_cap
    double* partial; // item_cap
    int item_cap;
    int* counters;   // [0] item count, [1] overflow flag; zeroed by the caller
    int* scan_tmp;
    int scan_tmp_n;
    int grid;
};
int scan_tmp_ints(int n);
fem_status exclusive_scan_i32_scratch(const int* in, int* out, int n, cudaStream_t s, int* total_dev, int* tmp,
                                      int tmp_n);
fem_status raster_errors_scratch(const int4* tri, const int2* vxy, int T, int N, const double* uv, const float* f,
                                 double* err_out, cudaStream_t s, const RasterScratch& w);
}  // namespace fem
