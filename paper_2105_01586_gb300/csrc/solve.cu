// solve.cu -- the Laplace solve on the unknown vertices (Sec. 2.2):
// A_UU x_U = -A_UK g_K by Jacobi-preconditioned CG.  The system itself
// (stiffness, K/U split, ELL rows of A_UU) is built in components.cu.
//
// The solve is one cooperative kernel with bounded grid barriers:
//   FP32_IR: repeat { r = b - A x in FP64; stop if ||r|| <= tol ||b||;
//                     solve A d = r/||r|| by FP32 PCG to relative 1e-5;
//                     x += ||r|| d (FP64) }
//   FP64:    PCG in FP64 from the warm start until ||r|| <= tol ||b||, then
//            the residual is recomputed from scratch to confirm.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fem_internal.cuh"
#include "ff.cuh"
#include "scan.cuh"

namespace fem {

constexpr int kSolveThreads = 256;
constexpr int kSingleThreads = 1024;
constexpr int kSingleMaxRows = 8192;   // systems up to this size run in one block
constexpr double kInnerEta = 1e-5;
constexpr int kInnerCap = 4000;        // FP32 iterations per refinement step

// b_r = -sum over mask neighbours j of A_ij uv_j;  x_r = uv of the row's vertex
__global__ void k_rhs_and_start(int nU, int V, const int* __restrict__ urow_vertex, const int* __restrict__ nbr,
                                const float* __restrict__ coef, const unsigned char* __restrict__ mask,
                                const double* __restrict__ uv, double* __restrict__ b, double* __restrict__ x) {
    pdl_wait();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nU) return;
    int i = urow_vertex[r];
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        int j = nbr[d * V + i];
        float c = coef[d * V + i];
        if (j >= 0 && c != 0.0f && mask[j]) s -= (double)c * uv[j];
    }
    b[r] = s;
    x[r] = uv[i];
}

// x -> vertex values; nothing when the system build failed (gate: the
// component counters), since the row order is then incomplete
__global__ void k_scatter_solution(int nU, int V, const int* __restrict__ urow_vertex, const double* __restrict__ x,
                                   double* __restrict__ uv, float2* __restrict__ uvf, const int* __restrict__ gate) {
    pdl_wait();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nU || gate[CC_ERR] != 0) return;
    int i = urow_vertex[r];
    if (i < 0 || i >= V) return;
    double v = x[r];
    uv[i] = v;
    ff q = ff_from_double(v);
    uvf[i] = make_float2(q.hi, q.lo);
}

// ------------------------------------------------------------ device solve
struct SolveArgs {
    int n;
    const int* col;       // 8*n ELL columns, slot-major
    const float* val;     // 8*n ELL values (exact)
    const int* cnt;       // n entries used per row
    const float* diag;    // n diagonal (exact)
    const float* dinv;    // n 1/diag (FP32)
    const double* dinv64; // n 1/diag (FP64)
    const double* b;
    double* x;
    double* r64;
    double* p64;
    double* q64;
    double* z64;
    float* r32;
    float* p32;
    float* q32;
    float* z32;
    float* d32;
    double tol;
    int maxit;
    double* red;       // 2 * 2 * gridDim partials
    unsigned* bar;
    int* err;
    double* out;       // [0] iterations, [1] relres, [2] status, [3] refinement residual passes
    double* acc;       // optional running totals (see solve_accumulate)
    double bytes_it;   // algorithmic bytes per CG iteration (for acc)
    double bytes_res;  // algorithmic bytes per residual pass (for acc)
    const int* gate;   // optional: the component counters (CC_*); see gate_closed
    // optional: the solution also goes to the vertex values (uv, float-float
    // uvf) of the row's vertex scat_row[r]
    const int* scat_row;
    double* scat_uv;
    float2* scat_uvf;
};

// whole-system kernels launched behind the component solve return at once
// unless some component is too large for it (and the search succeeded)
__device__ __forceinline__ bool gate_closed(const SolveArgs& A) {
    return A.gate && (A.gate[CC_NBIG] == 0 || A.gate[CC_ERR] != 0);
}

// Running totals of solves whose results are not read back one by one:
// acc[0] CG iterations, [1] largest relative residual, [2] first failing
// status, [3] solves, [4] algorithmic bytes.  Kernels on one stream run one
// after another, so the single writing thread needs no atomics.
__device__ __forceinline__ void solve_accumulate(const SolveArgs& A, int iters, double relres, int status, int nres) {
    if (!A.acc) return;
    A.acc[0] += iters;
    if (relres > A.acc[1]) A.acc[1] = relres;
    if (status != FEM_OK && A.acc[2] == 0.0) A.acc[2] = status;
    A.acc[3] += 1.0;
    A.acc[4] += A.bytes_it * iters + A.bytes_res * nres;
}

// Reductions are written for GB300's FP64 rate (about 2 FP64 FMAs per clock
// per SM, 1/64 of FP32): FP32 partials are summed per warp in FP32 and only
// the warp sums are combined in FP64; FP64 partials are combined through
// shared memory by a single warp instead of a shuffle tree in every warp.
template <int BT>
__device__ __forceinline__ void block_sum2_f(float a, float b, double& ra, double& rb) {
    __shared__ double wa[BT / 32], wb[BT / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) { wa[w] = (double)a; wb[w] = (double)b; }
    __syncthreads();
    if (w == 0) {
        double ta = lane < BT / 32 ? wa[lane] : 0.0, tb = lane < BT / 32 ? wb[lane] : 0.0;
        ta = warp_sum(ta);
        tb = warp_sum(tb);
        if (lane == 0) { wa[0] = ta; wb[0] = tb; }
    }
    __syncthreads();
    ra = wa[0];
    rb = wb[0];
    __syncthreads();
}

template <int BT>
__device__ __forceinline__ void block_sum2_d(double& a, double& b) {
    __shared__ double sa[BT], sb[BT];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    if (w == 0) {
        double ta = 0.0, tb = 0.0;
        for (int i = lane; i < BT; i += 32) { ta += sa[i]; tb += sb[i]; }
        ta = warp_sum(ta);
        tb = warp_sum(tb);
        if (lane == 0) { sa[0] = ta; sb[0] = tb; }
    }
    __syncthreads();
    a = sa[0];
    b = sb[0];
    __syncthreads();
}

// Synchronisation policies.  GridSync: a cooperative grid of 256-thread
// blocks with bounded device-wide barriers; data written by other blocks is
// read through L2 (__ldcg) because L1 is not coherent across SMs.
// BlockSync: one 1024-thread block; barriers are __syncthreads and plain
// loads see the block's own writes.
struct GridSync {
    static constexpr int BT = kSolveThreads;
    __device__ static bool barrier(const SolveArgs& A) { return grid_barrier(A.bar, A.err); }
    // block sums -> per-block partials -> every block adds them in the same
    // order; `parity` alternates buffers so that slow readers are never overwritten
    __device__ static bool combine(double& a, double& b, const SolveArgs& A, int& parity) {
        int nb = gridDim.x;
        double* buf = A.red + (size_t)parity * 2 * nb;
        if (threadIdx.x == 0) { buf[2 * blockIdx.x] = a; buf[2 * blockIdx.x + 1] = b; }
        parity ^= 1;
        if (!grid_barrier(A.bar, A.err)) return false;
        double ta = 0.0, tb = 0.0;
        for (int k = threadIdx.x; k < nb; k += blockDim.x) {
            ta += __ldcg(&buf[2 * k]);
            tb += __ldcg(&buf[2 * k + 1]);
        }
        block_sum2_d<BT>(ta, tb);
        a = ta;
        b = tb;
        return true;
    }
    __device__ static bool sum2f(float a, float b, double& ra, double& rb, const SolveArgs& A, int& parity) {
        block_sum2_f<BT>(a, b, ra, rb);
        return combine(ra, rb, A, parity);
    }
    __device__ static bool sum2d(double& a, double& b, const SolveArgs& A, int& parity) {
        block_sum2_d<BT>(a, b);
        return combine(a, b, A, parity);
    }
    template <class T>
    __device__ static T ld(const T* p) { return __ldcg(p); }
};

struct BlockSync {
    static constexpr int BT = kSingleThreads;
    __device__ static bool barrier(const SolveArgs&) {
        __syncthreads();
        return true;
    }
    __device__ static bool sum2f(float a, float b, double& ra, double& rb, const SolveArgs&, int&) {
        block_sum2_f<BT>(a, b, ra, rb);
        return true;
    }
    __device__ static bool sum2d(double& a, double& b, const SolveArgs&, int&) {
        block_sum2_d<BT>(a, b);
        return true;
    }
    template <class T>
    __device__ static T ld(const T* p) { return *p; }
};

// y = A_UU v over this thread's rows; returns the thread's part of v.y
template <class T, class S>
__device__ __forceinline__ T spmv_rows(const SolveArgs& A, const T* __restrict__ v, T* __restrict__ y) {
    T dot = 0;
    int n = A.n;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        T vr = S::ld(&v[r]);
        T s = (T)A.diag[r] * vr;
        int c = A.cnt[r];
        for (int k = 0; k < c; ++k) s += (T)A.val[k * n + r] * S::ld(&v[A.col[k * n + r]]);
        y[r] = s;
        dot += vr * s;
    }
    return dot;
}

// FP32 Jacobi-PCG on A d = rhs from the start in d; stops when
// ||r|| <= eta ||rhs|| or after maxit iterations.  FP32 arithmetic
// throughout; only the scalars of the recurrences are kept in FP64.  Every
// branch depends on grid-uniform values, so all blocks take the same path.
template <class S>
__device__ bool pcg32(const SolveArgs& A, const float* rhs, float* d, float* r, float* z, float* p, float* q,
                      double eta, int maxit, int& iters, int& parity) {
    int n = A.n;
    int stride = gridDim.x * blockDim.x;
    int tid0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (!S::barrier(A)) return false;  // d and rhs complete
    spmv_rows<float, S>(A, d, q);
    float rz_t = 0.f, rr_t = 0.f, bb_t = 0.f;
    for (int i = tid0; i < n; i += stride) {
        float ri = rhs[i] - q[i];
        r[i] = ri;
        float zi = ri * A.dinv[i];
        z[i] = zi;
        p[i] = zi;
        rz_t += ri * zi;
        rr_t += ri * ri;
        bb_t += rhs[i] * rhs[i];
    }
    double rz, rr, bb, dm;
    if (!S::sum2f(rz_t, rr_t, rz, rr, A, parity)) return false;
    if (!S::sum2f(bb_t, 0.f, bb, dm, A, parity)) return false;
    // CG scalars in FP32: every thread computes them, and an FP64 division
    // replicated over a block costs microseconds on GB300's FP64 pipe
    float lim = (float)eta * (float)eta * (float)bb;
    float rzf = (float)rz, rrf = (float)rr;
    iters = 0;
    while (rrf > lim && iters < maxit) {
        float pq_t = spmv_rows<float, S>(A, p, q);
        double pq;
        if (!S::sum2f(pq_t, 0.f, pq, dm, A, parity)) return false;
        float pqf = (float)pq;
        if (!(pqf > 0.f)) break;  // breakdown guard
        float alpha = rzf / pqf;
        float rz1_t = 0.f, rr1_t = 0.f;
        for (int i = tid0; i < n; i += stride) {
            d[i] += alpha * p[i];
            float ri = r[i] - alpha * q[i];
            r[i] = ri;
            float zi = ri * A.dinv[i];
            z[i] = zi;
            rz1_t += ri * zi;
            rr1_t += ri * ri;
        }
        double rz1;
        if (!S::sum2f(rz1_t, rr1_t, rz1, rr, A, parity)) return false;
        iters++;
        float rz1f = (float)rz1;
        rrf = (float)rr;
        float beta = rz1f / rzf;
        rzf = rz1f;
        for (int i = tid0; i < n; i += stride) p[i] = z[i] + beta * p[i];
        if (!S::barrier(A)) return false;  // p complete before the next SpMV
    }
    return true;
}

// a scalar computed by thread 0 and broadcast (keeps FP64 divisions off the
// other 1023 threads' FP64 pipe time)
__device__ __forceinline__ double bcast_div(double num, double den) {
    __shared__ double s_v;
    if (threadIdx.x == 0) s_v = num / den;
    __syncthreads();
    double v = s_v;
    __syncthreads();
    return v;
}

// Plain FP64 Jacobi-PCG on A x = b from the start in x (the FP64 comparator).
template <class S>
__device__ bool pcg64(const SolveArgs& A, double eta, int maxit, int& iters, int& parity) {
    int n = A.n;
    int stride = gridDim.x * blockDim.x;
    int tid0 = blockIdx.x * blockDim.x + threadIdx.x;
    double *x = A.x, *r = A.r64, *z = A.z64, *p = A.p64, *q = A.q64;
    if (!S::barrier(A)) return false;
    spmv_rows<double, S>(A, x, q);
    double rz = 0.0, rr = 0.0, bb = 0.0, dm = 0.0;
    for (int i = tid0; i < n; i += stride) {
        double ri = A.b[i] - q[i];
        r[i] = ri;
        double zi = ri * A.dinv64[i];
        z[i] = zi;
        p[i] = zi;
        rz += ri * zi;
        rr += ri * ri;
        bb += A.b[i] * A.b[i];
    }
    if (!S::sum2d(rz, rr, A, parity)) return false;
    if (!S::sum2d(bb, dm, A, parity)) return false;
    double lim = eta * eta * bb;
    iters = 0;
    while (rr > lim && iters < maxit) {
        double pq = spmv_rows<double, S>(A, p, q);
        dm = 0.0;
        if (!S::sum2d(pq, dm, A, parity)) return false;
        if (!(pq > 0.0)) break;
        double alpha = bcast_div(rz, pq);
        double rz1 = 0.0, rr1 = 0.0;
        for (int i = tid0; i < n; i += stride) {
            x[i] += alpha * p[i];
            double ri = r[i] - alpha * q[i];
            r[i] = ri;
            double zi = ri * A.dinv64[i];
            z[i] = zi;
            rz1 += ri * zi;
            rr1 += ri * ri;
        }
        if (!S::sum2d(rz1, rr1, A, parity)) return false;
        iters++;
        rr = rr1;
        double beta = bcast_div(rz1, rz);
        rz = rz1;
        for (int i = tid0; i < n; i += stride) p[i] = z[i] + beta * p[i];
        if (!S::barrier(A)) return false;
    }
    return true;
}

// FP64 residual r = b - A x over the used entries of each row; returns
// (||r||^2, ||b||^2) grid-wide
template <class S>
__device__ bool residual64(const SolveArgs& A, double& rr, double& bb, int& parity) {
    if (!S::barrier(A)) return false;  // x complete
    int n = A.n;
    rr = 0.0;
    bb = 0.0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        double s = (double)A.diag[r] * S::ld(&A.x[r]);
        int c = A.cnt[r];
        for (int k = 0; k < c; ++k) s += (double)A.val[k * n + r] * S::ld(&A.x[A.col[k * n + r]]);
        double ri = A.b[r] - s;
        A.r64[r] = ri;
        rr += ri * ri;
        bb += A.b[r] * A.b[r];
    }
    return S::sum2d(rr, bb, A, parity);
}

template <bool FP64_ONLY, class S>
__device__ __forceinline__ void solve_body(const SolveArgs& A) {
    int parity = 0;
    int n = A.n;
    int stride = gridDim.x * blockDim.x;
    int tid0 = blockIdx.x * blockDim.x + threadIdx.x;
    int total_it = 0, n_res = 1;
    double rr = 0.0, bb = 0.0;
    int status = FEM_E_NOT_CONVERGED;
    if (!residual64<S>(A, rr, bb, parity)) goto fail;
    if (bb == 0.0) {
        for (int i = tid0; i < n; i += stride) A.x[i] = 0.0;
        rr = 0.0;
        status = FEM_OK;
        goto done;
    }
    if (FP64_ONLY) {
        for (int attempt = 0; attempt < 4; ++attempt) {
            if (rr <= A.tol * A.tol * bb) { status = FEM_OK; break; }
            if (total_it >= A.maxit) break;
            int it = 0;
            if (!pcg64<S>(A, A.tol, A.maxit - total_it, it, parity)) goto fail;
            total_it += it;
            n_res++;
            if (!residual64<S>(A, rr, bb, parity)) goto fail;
        }
        if (rr <= A.tol * A.tol * bb) status = FEM_OK;
    } else {
        for (int step = 0; step < 64; ++step) {
            if (rr <= A.tol * A.tol * bb) { status = FEM_OK; break; }
            if (total_it >= A.maxit) break;
            // normalise the residual; any scale works as long as the step is
            // scaled back by its inverse (FP32 scalars, see pcg32)
            float sc = rsqrtf((float)rr), back = 1.0f / sc;
            for (int i = tid0; i < n; i += stride) {
                A.r32[i] = (float)A.r64[i] * sc;
                A.d32[i] = 0.0f;
            }
            int it = 0;
            int cap = A.maxit - total_it;
            if (cap > kInnerCap) cap = kInnerCap;
            if (!pcg32<S>(A, A.r32, A.d32, A.z32 /*r*/, A.q32 /*z*/, A.p32, A.q32 + n /*q*/, kInnerEta, cap, it,
                          parity))
                goto fail;
            total_it += it;
            for (int i = tid0; i < n; i += stride) A.x[i] += (double)(back * A.d32[i]);
            n_res++;
            if (!residual64<S>(A, rr, bb, parity)) goto fail;
        }
        if (rr <= A.tol * A.tol * bb) status = FEM_OK;
    }
done:
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.out[0] = total_it;
        A.out[1] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        A.out[2] = status;
        A.out[3] = n_res;
        A.out[4] = (double)total_it * A.n;
        A.out[5] = (double)n_res * A.n;
        solve_accumulate(A, total_it, A.out[1], status, n_res);
    }
    return;
fail:
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.out[0] = total_it;
        A.out[1] = -1.0;
        A.out[2] = FEM_E_TIMEOUT;
        A.out[3] = n_res;
        A.out[4] = (double)total_it * A.n;
        A.out[5] = (double)n_res * A.n;
        solve_accumulate(A, total_it, 1.0, FEM_E_TIMEOUT, n_res);
    }
}

template <bool FP64_ONLY>
__global__ void __launch_bounds__(kSolveThreads) k_solve(SolveArgs A) {
    pdl_wait();
    if (gate_closed(A)) return;
    solve_body<FP64_ONLY, GridSync>(A);
}

template <bool FP64_ONLY>
__global__ void __launch_bounds__(kSingleThreads) k_solve_single(SolveArgs A) {
    pdl_wait();
    if (gate_closed(A)) return;
    solve_body<FP64_ONLY, BlockSync>(A);
}

// ---------------------------------------------------------------------------
// One-block FP32-IR solve for up to kBlockMaxRows unknowns, with no FP64
// arithmetic in its loops:
//  * A_UU's off-diagonal entries are -1/2 or -1 and its diagonal a multiple
//    of 1/2 up to 8: the kernel builds a CSR copy in shared memory with
//    16-bit entries ((column << 1) | (entry == -1)) and the diagonal as a
//    byte (twice its value; 1/diag from a 17-entry table);
//  * x and b are float-float (about 48 bits), scaled by an exact power of
//    two so that max |b| is about 1 and FP32 squares of 1e-12 residuals stay
//    normal; the refinement residual b - A x is computed in float-float;
//  * the inner CG is FP32 with two block barriers per iteration: each
//    reduction is one barrier over double-buffered warp slots, and the search
//    direction p_new = D^{-1} r + beta p_old is formed inside the next SpMV
//    (at neighbours on the fly, p double-buffered).
// The five CG vectors and the CSR copy live in shared memory when they fit
// (about 8k unknowns at 1.7 entries per row); otherwise the same code runs on
// global buffers (generic pointers), decided on the device.
constexpr int kBlockMaxRows = 16384;
constexpr int kBlockSmemBytes = 200 * 1024;

struct BlockRed {
    float4 slot[2][kSingleThreads / 32];
};

// sums of up to three floats over the block with one barrier: warps reduce
// by shuffles, lane 0 writes the warp sums to the current slot buffer, and
// after the barrier every warp reduces the 32 warp sums again by shuffles and
// takes lane 0's value, so all threads see the same bits
__device__ __forceinline__ float3 block_sum3(BlockRed& R, int& par, float a, float b, float c) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    if (lane == 0) R.slot[par][w] = make_float4(a, b, c, 0.f);
    __syncthreads();
    float4 v = R.slot[par][lane];
    float sa = warp_sum(v.x), sb = warp_sum(v.y), sc = warp_sum(v.z);
    sa = __shfl_sync(0xffffffffu, sa, 0);
    sb = __shfl_sync(0xffffffffu, sb, 0);
    sc = __shfl_sync(0xffffffffu, sc, 0);
    par ^= 1;
    return make_float3(sa, sb, sc);
}

__device__ __forceinline__ float ent_val(unsigned short e) { return (e & 1u) ? -1.0f : -0.5f; }

struct BlockScratch {
    float* vec;             // 5 n floats (global fallback)
    int* rowptr;            // n + 1 (global fallback)
    unsigned short* ent;    // 8 n (global fallback)
    unsigned char* dg2;     // n (global fallback)
    float2* xff;            // n float-float iterate
    float2* bff;            // n float-float right-hand side
};

// The solve proper.  SMEM selects where the CG vectors and the CSR copy
// live; each instantiation derives its pointers from one address space only,
// so the shared-memory one compiles to shared-memory instructions.
template <bool SMEM>
__device__ __forceinline__ void block_solve_core(const SolveArgs& A, const BlockScratch& G, unsigned char* sm_raw,
                                                 int nnz, float bm, BlockRed& R, const float* s_lut, int* s_wsum) {
    const int n = A.n, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // layout: floats (5n) | int rowptr (n+1) | u16 entries (nnz) | u8 diag (n)
    float* fv = SMEM ? (float*)sm_raw : G.vec;
    int* rowptr = SMEM ? (int*)(sm_raw + (size_t)20 * n) : G.rowptr;
    unsigned short* ent = SMEM ? (unsigned short*)(sm_raw + (size_t)24 * n + 4) : G.ent;
    unsigned char* dg2 = SMEM ? (sm_raw + (size_t)24 * n + 4 + (size_t)2 * nnz) : G.dg2;
    float *d = fv, *r = fv + n, *p0 = fv + 2 * n, *p1 = fv + 3 * n, *q = fv + 4 * n;
    // CSR row starts: contiguous chunks per thread, block exclusive scan
    int chunk = (n + kSingleThreads - 1) / kSingleThreads;
    int lo = tid * chunk, hi = min(n, lo + chunk), loc = 0;
    for (int i = lo; i < hi; ++i) loc += A.cnt[i];
    int incl = loc;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) s_wsum[wid] = incl;
    __syncthreads();
    int wbase = 0;
    for (int i = 0; i < wid; ++i) wbase += s_wsum[i];
    int run = wbase + incl - loc;
    for (int i = lo; i < hi; ++i) {
        rowptr[i] = run;
        int c = A.cnt[i];
        for (int k = 0; k < c; ++k)
            ent[run + k] = (unsigned short)((A.col[k * n + i] << 1) | (A.val[k * n + i] == -1.0f ? 1 : 0));
        dg2[i] = (unsigned char)(2.0f * A.diag[i]);
        run += c;
    }
    if (tid == kSingleThreads - 1) rowptr[n] = nnz;
    int total_it = 0, n_res = 0, status = FEM_E_NOT_CONVERGED, par = 0;
    float rr = 0.f, bb = 0.f;
    if (bm == 0.f) {
        for (int i = tid; i < n; i += kSingleThreads) A.x[i] = 0.0;
        status = FEM_OK;
    } else {
        // exact power-of-two normalisation: max |b| in [1, 2)
        int e = ilogbf(bm);
        float sigma = ldexpf(1.0f, -e);
        double inv_sigma = ldexp(1.0, e);
        for (int i = tid; i < n; i += kSingleThreads) {
            ff bi = ff_scale_pow2(ff_from_double(A.b[i]), sigma);
            ff xi = ff_scale_pow2(ff_from_double(A.x[i]), sigma);
            G.bff[i] = make_float2(bi.hi, bi.lo);
            G.xff[i] = make_float2(xi.hi, xi.lo);
        }
        __syncthreads();
        float tol2 = (float)(A.tol * A.tol);
        for (int step = 0; step < 64; ++step) {
            // refinement residual r = b - A x in float-float, rounded to FP32
            float rr_t = 0.f, bb_t = 0.f, rz_t = 0.f;
            for (int i = tid; i < n; i += kSingleThreads) {
                float2 xv = G.xff[i];
                int dd = dg2[i];
                ff s = ff_mul_f(ff{xv.x, xv.y}, 0.5f * (float)dd);
                for (int k = rowptr[i], k1 = rowptr[i + 1]; k < k1; ++k) {
                    unsigned short en = ent[k];
                    float2 xc = G.xff[en >> 1];
                    s = ff_add(s, ff_scale_pow2(ff{xc.x, xc.y}, ent_val(en)));
                }
                float2 bv = G.bff[i];
                ff res = ff_sub(ff{bv.x, bv.y}, s);
                float ri = __fadd_rn(res.hi, res.lo);
                r[i] = ri;
                d[i] = 0.f;
                p0[i] = 0.f;
                rr_t += ri * ri;
                rz_t += ri * ri * s_lut[dd];
                bb_t += bv.x * bv.x;
            }
            float3 red = block_sum3(R, par, rr_t, bb_t, rz_t);
            n_res++;
            rr = red.x;
            bb = red.y;
            if (rr <= tol2 * bb) { status = FEM_OK; break; }
            if (total_it >= A.maxit) break;
            // FP32 PCG on A d = r from d = 0; p_old = p0 = 0, beta = 0
            float rz = red.z, rr_in = rr, lim = (float)(kInnerEta * kInnerEta) * rr, beta = 0.f;
            int cap = A.maxit - total_it;
            if (cap > kInnerCap) cap = kInnerCap;
            int it = 0;
            float *pold = p0, *pnew = p1;
            while (rr_in > lim && it < cap) {
                // p_new = D^-1 r + beta p_old and q = A p_new (neighbours on the fly)
                float pq_t = 0.f;
                for (int i = tid; i < n; i += kSingleThreads) {
                    int dd = dg2[i];
                    float pi = fmaf(beta, pold[i], s_lut[dd] * r[i]);
                    pnew[i] = pi;
                    float sacc = 0.5f * (float)dd * pi;
                    for (int k = rowptr[i], k1 = rowptr[i + 1]; k < k1; ++k) {
                        unsigned short en = ent[k];
                        int col = en >> 1;
                        sacc = fmaf(ent_val(en), fmaf(beta, pold[col], s_lut[dg2[col]] * r[col]), sacc);
                    }
                    q[i] = sacc;
                    pq_t += pi * sacc;
                }
                float pq = block_sum3(R, par, pq_t, 0.f, 0.f).x;
                if (!(pq > 0.f)) break;  // breakdown guard (uniform over the block)
                float alpha = rz / pq;
                float rz_t2 = 0.f, rr_t2 = 0.f;
                for (int i = tid; i < n; i += kSingleThreads) {
                    d[i] = fmaf(alpha, pnew[i], d[i]);
                    float ri = fmaf(-alpha, q[i], r[i]);
                    r[i] = ri;
                    rz_t2 += ri * ri * s_lut[dg2[i]];
                    rr_t2 += ri * ri;
                }
                float3 s2 = block_sum3(R, par, rz_t2, rr_t2, 0.f);
                it++;
                beta = s2.x / rz;
                rz = s2.x;
                rr_in = s2.y;
                float* t = pold;
                pold = pnew;
                pnew = t;
            }
            total_it += it;
            for (int i = tid; i < n; i += kSingleThreads) {
                float2 xv = G.xff[i];
                ff xi = ff_add_f(ff{xv.x, xv.y}, d[i]);
                G.xff[i] = make_float2(xi.hi, xi.lo);
            }
            __syncthreads();
        }
        for (int i = tid; i < n; i += kSingleThreads) {
            float2 xv = G.xff[i];
            A.x[i] = ff_to_double(ff{xv.x, xv.y}) * inv_sigma;
        }
    }
    if (tid == 0) {
        A.out[0] = total_it;
        A.out[1] = bb > 0.f ? sqrt((double)rr / (double)bb) : 0.0;
        A.out[2] = status;
        A.out[3] = n_res;
        A.out[4] = (double)total_it * A.n;
        A.out[5] = (double)n_res * A.n;
        solve_accumulate(A, total_it, A.out[1], status, n_res);
    }
}

__global__ void __launch_bounds__(kSingleThreads) k_solve_block(SolveArgs A, BlockScratch G, int smem_bytes) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ BlockRed R;
    __shared__ float s_lut[17];
    __shared__ int s_wsum[kSingleThreads / 32];
    __shared__ float s_bmax[kSingleThreads / 32];
    if (gate_closed(A)) return;
    const int n = A.n, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid < 17) s_lut[tid] = tid ? 1.0f / (0.5f * (float)tid) : 0.0f;
    // number of off-diagonal entries, and max |b|
    int cnt_t = 0;
    float bm = 0.f;
    for (int i = tid; i < n; i += kSingleThreads) {
        cnt_t += A.cnt[i];
        bm = fmaxf(bm, fabsf((float)A.b[i]));
    }
    cnt_t = warp_sum(cnt_t);
    for (int o = 16; o > 0; o >>= 1) bm = fmaxf(bm, __shfl_xor_sync(0xffffffffu, bm, o));
    if (lane == 0) { s_wsum[wid] = cnt_t; s_bmax[wid] = bm; }
    __syncthreads();
    int nnz = 0;
    bm = 0.f;
    for (int i = 0; i < kSingleThreads / 32; ++i) { nnz += s_wsum[i]; bm = fmaxf(bm, s_bmax[i]); }
    size_t need = (size_t)20 * n + (size_t)4 * (n + 1) + (size_t)2 * nnz + (size_t)n;
    (void)lane;
    (void)wid;
    if (need <= (size_t)smem_bytes)
        block_solve_core<true>(A, G, sm_raw, nnz, bm, R, s_lut, s_wsum);
    else
        block_solve_core<false>(A, G, sm_raw, nnz, bm, R, s_lut, s_wsum);
    if (A.scat_uv) {
        __syncthreads();
        for (int i = tid; i < n; i += kSingleThreads) {
            const double v = A.x[i];
            const int vi = A.scat_row[i];
            A.scat_uv[vi] = v;
            const ff q = ff_from_double(v);
            A.scat_uvf[vi] = make_float2(q.hi, q.lo);
        }
    }
}

// ---------------------------------------------------------------------------
// Grid version of the FP64-free FP32-IR solve for systems above
// kBlockMaxRows: the same algorithm as k_solve_block on a cooperative grid.
// A_UU is read from the ELL arrays in global memory, x and b are float-float
// global vectors, data written by other blocks is read through L2 (__ldcg),
// and each reduction is a block reduction plus one bounded grid barrier
// (two barriers per CG iteration).
constexpr int kGridThreads = 512;

// Parities of the double-buffered partial slots: per-thread registers that
// advance identically in every thread (one flip per reduction).
struct GridPar {
    int par;   // block-level slot buffer
    int gpar;  // grid-level partial buffer
};

// totals of three floats over the grid (same bits in every thread)
__device__ __forceinline__ bool grid_sum3(const SolveArgs& A, BlockRed& R, GridPar& P, float a, float b, float c,
                                          float3& out) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    if (lane == 0) R.slot[P.par][w] = make_float4(a, b, c, 0.f);
    __syncthreads();
    float4 v = lane < kGridThreads / 32 ? R.slot[P.par][lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    P.par ^= 1;
    float ba = warp_sum(v.x), bb = warp_sum(v.y), bc = warp_sum(v.z);
    int nb = gridDim.x;
    float4* buf = (float4*)A.red + (size_t)P.gpar * nb;
    if (threadIdx.x == 0) buf[blockIdx.x] = make_float4(ba, bb, bc, 0.f);
    P.gpar ^= 1;
    if (!grid_barrier(A.bar, A.err)) return false;
    float sa = 0.f, sb = 0.f, sc = 0.f;
    for (int k = lane; k < nb; k += 32) {
        float4 u = __ldcg(&buf[k]);
        sa += u.x;
        sb += u.y;
        sc += u.z;
    }
    sa = __shfl_sync(0xffffffffu, warp_sum(sa), 0);
    sb = __shfl_sync(0xffffffffu, warp_sum(sb), 0);
    sc = __shfl_sync(0xffffffffu, warp_sum(sc), 0);
    out = make_float3(sa, sb, sc);
    return true;
}

__global__ void __launch_bounds__(kGridThreads) k_solve_grid(SolveArgs A, BlockScratch G) {
    pdl_wait();
    __shared__ BlockRed R;
    if (gate_closed(A)) return;
    GridPar P{0, 0};
    const int n = A.n, stride = gridDim.x * blockDim.x, tid0 = blockIdx.x * blockDim.x + threadIdx.x;
    float* d = G.vec;
    float *r = d + n, *p0 = d + 2 * n, *p1 = d + 3 * n, *q = d + 4 * n;
    int total_it = 0, n_res = 0, status = FEM_E_NOT_CONVERGED;
    float rr = 0.f, bb = 0.f;
    // max |b| over the grid (as a sum of per-block maxima is not a max, use
    // the three-value reduction on squares' maxima through an exact trick:
    // a max is order-independent, so each block contributes its max and the
    // grid takes the max of the partials)
    float bm = 0.f;
    for (int i = tid0; i < n; i += stride) bm = fmaxf(bm, fabsf((float)A.b[i]));
    for (int o = 16; o > 0; o >>= 1) bm = fmaxf(bm, __shfl_xor_sync(0xffffffffu, bm, o));
    {
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) R.slot[P.par][w] = make_float4(bm, 0.f, 0.f, 0.f);
        __syncthreads();
        float m = 0.f;
        for (int i = 0; i < kGridThreads / 32; ++i) m = fmaxf(m, R.slot[P.par][i].x);
        P.par ^= 1;
        float4* buf = (float4*)A.red + (size_t)P.gpar * gridDim.x;
        if (threadIdx.x == 0) buf[blockIdx.x] = make_float4(m, 0.f, 0.f, 0.f);
        P.gpar ^= 1;
        if (!grid_barrier(A.bar, A.err)) goto fail;
        m = 0.f;
        for (int k = 0; k < (int)gridDim.x; ++k) m = fmaxf(m, __ldcg(&buf[k]).x);
        bm = m;
    }
    if (bm == 0.f) {
        for (int i = tid0; i < n; i += stride) A.x[i] = 0.0;
        status = FEM_OK;
    } else {
        int e = ilogbf(bm);
        float sigma = ldexpf(1.0f, -e);
        double inv_sigma = ldexp(1.0, e);
        for (int i = tid0; i < n; i += stride) {
            ff bi = ff_scale_pow2(ff_from_double(A.b[i]), sigma);
            ff xi = ff_scale_pow2(ff_from_double(A.x[i]), sigma);
            G.bff[i] = make_float2(bi.hi, bi.lo);
            G.xff[i] = make_float2(xi.hi, xi.lo);
        }
        if (!grid_barrier(A.bar, A.err)) goto fail;
        float tol2 = (float)(A.tol * A.tol);
        for (int step = 0; step < 64; ++step) {
            float rr_t = 0.f, bb_t = 0.f, rz_t = 0.f;
            for (int i = tid0; i < n; i += stride) {
                float2 xv = __ldcg(&G.xff[i]);
                ff s2 = ff_mul_f(ff{xv.x, xv.y}, A.diag[i]);
                int c = A.cnt[i];
                for (int k = 0; k < c; ++k) {
                    float2 xc = __ldcg(&G.xff[A.col[k * n + i]]);
                    s2 = ff_add(s2, ff_scale_pow2(ff{xc.x, xc.y}, A.val[k * n + i]));
                }
                float2 bv = G.bff[i];
                ff res = ff_sub(ff{bv.x, bv.y}, s2);
                float ri = __fadd_rn(res.hi, res.lo);
                r[i] = ri;
                d[i] = 0.f;
                p0[i] = 0.f;
                rr_t += ri * ri;
                rz_t += ri * ri * A.dinv[i];
                bb_t += bv.x * bv.x;
            }
            float3 red;
            if (!grid_sum3(A, R, P, rr_t, bb_t, rz_t, red)) goto fail;
            n_res++;
            rr = red.x;
            bb = red.y;
            if (rr <= tol2 * bb) { status = FEM_OK; break; }
            if (total_it >= A.maxit) break;
            float rz = red.z, rr_in = rr, lim = (float)(kInnerEta * kInnerEta) * rr, beta = 0.f;
            int cap = A.maxit - total_it;
            if (cap > kInnerCap) cap = kInnerCap;
            int it = 0;
            float *pold = p0, *pnew = p1;
            while (rr_in > lim && it < cap) {
                float pq_t = 0.f;
                for (int i = tid0; i < n; i += stride) {
                    float pi = fmaf(beta, __ldcg(&pold[i]), A.dinv[i] * __ldcg(&r[i]));
                    pnew[i] = pi;
                    float sacc = A.diag[i] * pi;
                    int c = A.cnt[i];
                    for (int k = 0; k < c; ++k) {
                        int col = A.col[k * n + i];
                        sacc = fmaf(A.val[k * n + i], fmaf(beta, __ldcg(&pold[col]), A.dinv[col] * __ldcg(&r[col])),
                                    sacc);
                    }
                    q[i] = sacc;
                    pq_t += pi * sacc;
                }
                float3 s1;
                if (!grid_sum3(A, R, P, pq_t, 0.f, 0.f, s1)) goto fail;
                float pq = s1.x;
                if (!(pq > 0.f)) break;
                float alpha = rz / pq;
                float rz_t2 = 0.f, rr_t2 = 0.f;
                for (int i = tid0; i < n; i += stride) {
                    d[i] = fmaf(alpha, pnew[i], d[i]);
                    float ri = fmaf(-alpha, q[i], r[i]);
                    r[i] = ri;
                    rz_t2 += ri * ri * A.dinv[i];
                    rr_t2 += ri * ri;
                }
                float3 s2;
                if (!grid_sum3(A, R, P, rz_t2, rr_t2, 0.f, s2)) goto fail;
                it++;
                beta = s2.x / rz;
                rz = s2.x;
                rr_in = s2.y;
                float* t = pold;
                pold = pnew;
                pnew = t;
            }
            total_it += it;
            for (int i = tid0; i < n; i += stride) {
                float2 xv = G.xff[i];
                ff xi = ff_add_f(ff{xv.x, xv.y}, d[i]);
                G.xff[i] = make_float2(xi.hi, xi.lo);
            }
            if (!grid_barrier(A.bar, A.err)) goto fail;
        }
        for (int i = tid0; i < n; i += stride) {
            float2 xv = G.xff[i];
            A.x[i] = ff_to_double(ff{xv.x, xv.y}) * inv_sigma;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.out[0] = total_it;
        A.out[1] = bb > 0.f ? sqrt((double)rr / (double)bb) : 0.0;
        A.out[2] = status;
        A.out[3] = n_res;
        A.out[4] = (double)total_it * A.n;
        A.out[5] = (double)n_res * A.n;
        solve_accumulate(A, total_it, A.out[1], status, n_res);
    }
    return;
fail:
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.out[0] = total_it;
        A.out[1] = -1.0;
        A.out[2] = FEM_E_TIMEOUT;
        A.out[3] = n_res;
        A.out[4] = (double)total_it * A.n;
        A.out[5] = (double)n_res * A.n;
        solve_accumulate(A, total_it, 1.0, FEM_E_TIMEOUT, n_res);
    }
}

static int occupancy(const void* func, int threads) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, func, threads, 0);
    return nb > 0 ? nb : 1;
}

static int coop_blocks(const void* func, int n, int num_sms) {
    static const int occ64 = occupancy((const void*)k_solve<true>, kSolveThreads);
    static const int occ32 = occupancy((const void*)k_solve<false>, kSolveThreads);
    int maxb = (func == (const void*)k_solve<true> ? occ64 : occ32) * num_sms;
    int want = (n + 4 * kSolveThreads - 1) / (4 * kSolveThreads);
    if (want < 1) want = 1;
    return want < maxb ? want : maxb;
}

// Solve A_UU x = b (device vectors of length nU; x holds the start).
fem_status run_solve(fem_mesh* m, const double* b, double* x, bool use_fp64, double tol, int maxit, cudaStream_t s,
                     int* iters_out, double* relres_out, bool deferred, bool scatter) {
    FEM_TRY(build_system(m, s));
    int nU = m->nU;
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    if (nU == 0) return FEM_OK;
    size_t n = nU;
    FEM_TRY(ensure(m->r64, n, s));
    if (use_fp64) {
        FEM_TRY(ensure(m->p64, n, s));
        FEM_TRY(ensure(m->q64, n, s));
        FEM_TRY(ensure(m->z64, n, s));
    } else {
        FEM_TRY(ensure(m->r32, n, s));
        FEM_TRY(ensure(m->p32, n, s));
        FEM_TRY(ensure(m->q32, 2 * n, s));
        FEM_TRY(ensure(m->z32, n, s));
        FEM_TRY(ensure(m->d32, n, s));
    }
    bool single = nU <= kSingleMaxRows;
    const void* func = use_fp64 ? (const void*)k_solve<true> : (const void*)k_solve<false>;
    int grid = single ? 1 : coop_blocks(func, nU, m->num_sms);
    FEM_TRY(ensure(m->red, (size_t)4 * grid + 8, s));
    SolveArgs A;
    A.n = nU;
    A.col = m->ucol.p;
    A.val = m->uval32.p;
    A.cnt = m->ucnt.p;
    A.diag = m->udiag.p;
    A.dinv = m->dinv32.p;
    A.dinv64 = m->dinv64.p;
    A.b = b;
    A.x = x;
    A.r64 = m->r64.p;
    A.p64 = m->p64.p; A.q64 = m->q64.p; A.z64 = m->z64.p;
    A.r32 = m->r32.p; A.p32 = m->p32.p; A.q32 = m->q32.p; A.z32 = m->z32.p; A.d32 = m->d32.p;
    A.tol = tol;
    A.maxit = maxit;
    A.red = m->red.p;
    A.bar = m->bar.p;
    A.err = m->dflag.p + 1;
    A.out = m->dscal.p;
    // Algorithmic bytes per row: ELL matrix (8 columns + 8 values + diagonal,
    // 68 B) per SpMV; FP32 CG iteration = SpMV 76 B + updates 44 B; FP64 CG
    // iteration = SpMV 84 B + updates 84 B; FP64 residual pass 92 B; each FP32
    // refinement step adds 36 B of conversions and the FP64 update.
    A.bytes_it = (double)nU * (use_fp64 ? 168.0 : 120.0);
    A.bytes_res = (double)nU * (92.0 + (use_fp64 ? 0.0 : 36.0));
    A.acc = deferred ? m->dscal.p + 64 : nullptr;
    A.scat_row = scatter ? m->urow_vertex.p : nullptr;
    A.scat_uv = scatter ? m->uv.p : nullptr;
    A.scat_uvf = scatter ? m->uvf.p : nullptr;
    // Components of at most kBlockComp rows are solved independently, all at
    // once; when a component is larger, that kernel returns at once and the
    // whole-system solver below (gated on the same device counter) runs.
    // The component kernel also clears the error word of that solver.
    FEM_TRY(solve_components(m, b, x, use_fp64, tol, maxit, deferred, scatter, m->dflag.p + 1, s));
    A.gate = m->ccount.p;
    // With at most kBlockComp unknowns no component can be larger, so the
    // whole-system solvers (and their scatter) would return at once: they
    // are not launched.
    const bool whole_system = nU > kBlockComp;
    if (!whole_system) {
        // nothing more to launch
    } else if (!use_fp64 && nU <= kBlockMaxRows) {
        static const bool attr_set = [] {
            return cudaFuncSetAttribute(k_solve_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kBlockSmemBytes) == cudaSuccess;
        }();
        (void)attr_set;
        FEM_TRY(ensure(m->bvec, (size_t)5 * nU, s));
        FEM_TRY(ensure(m->browptr, (size_t)nU + 1, s));
        FEM_TRY(ensure(m->bent, (size_t)8 * nU, s));
        FEM_TRY(ensure(m->bdg2, (size_t)nU, s));
        FEM_TRY(ensure(m->bxff, (size_t)nU, s));
        FEM_TRY(ensure(m->bbff, (size_t)nU, s));
        BlockScratch G{m->bvec.p, m->browptr.p, m->bent.p, m->bdg2.p, m->bxff.p, m->bbff.p};
        FEM_LAUNCH(F_CG, s, k_solve_block, 1, kSingleThreads, (size_t)kBlockSmemBytes, A, G, kBlockSmemBytes);
    } else if (!use_fp64) {
        static const int occ = occupancy((const void*)k_solve_grid, kGridThreads);
        int gb = (nU + 2 * kGridThreads - 1) / (2 * kGridThreads);
        gb = std::max(1, std::min(gb, occ * m->num_sms));
        FEM_TRY(ensure(m->red, (size_t)4 * gb + 8, s));
        A.red = m->red.p;
        FEM_TRY(ensure(m->bvec, (size_t)5 * nU, s));
        FEM_TRY(ensure(m->bxff, (size_t)nU, s));
        FEM_TRY(ensure(m->bbff, (size_t)nU, s));
        BlockScratch G{m->bvec.p, nullptr, nullptr, nullptr, m->bxff.p, m->bbff.p};
        void* args[] = {&A, &G};
        FEM_TRY(launch_coop(F_CG, (const void*)k_solve_grid, gb, kGridThreads, 0, s, args, "k_solve_grid"));
    } else if (single) {
        FEM_LAUNCH(F_CG, s, k_solve_single<true>, 1, kSingleThreads, 0, A);
    } else {
        void* args[] = {&A};
        FEM_TRY(launch_coop(F_CG, func, grid, kSolveThreads, 0, s, args, "k_solve<fp64>"));
    }
    if (scatter && whole_system && !(!use_fp64 && nU <= kBlockMaxRows)) {
        // these whole-system solvers leave the scatter to a kernel of its own
        // (it repeats what the component solver wrote when that one solved)
        FEM_LAUNCH(F_CG, s, k_scatter_solution, (nU + 255) / 256, 256, 0, nU, m->V, (const int*)m->urow_vertex.p,
                   (const double*)x, m->uv.p, m->uvf.p, (const int*)m->ccount.p);
    }
    if (deferred) {
        if (profiling(F_CG)) note_bytes(F_CG, 0.0);  // bytes are added from the device totals at the end
        return FEM_OK;
    }
    double* hs = (double*)m->host_stage;
    FEM_CUDA(cudaMemcpyAsync(hs, m->dscal.p, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    int its = (int)hs[0];
    double rel = hs[1];
    int st = (int)hs[2];
    // bytes from row-iterations and row-residual passes (out[4], out[5])
    note_bytes(F_CG, (use_fp64 ? 168.0 : 120.0) * hs[4] + (use_fp64 ? 92.0 : 128.0) * hs[5]);
    m->stats.cg_iters += its;
    m->stats.solves += 1;
    m->stats.relres = rel;
    if (iters_out) *iters_out = its;
    if (relres_out) *relres_out = rel;
    if (st == FEM_E_TIMEOUT) {
        reset_coop_state(m, s);
        set_error("Laplace solve: a grid barrier wait ran out");
        return FEM_E_TIMEOUT;
    }
    if (st == FEM_E_INVALID) {
        set_error("Laplace solve: the component search of A_UU failed (unknown count does not match the mesh)");
        return FEM_E_INVALID;
    }
    if (st != FEM_OK) {
        set_error("Laplace solve: iteration cap reached, relative residual " + std::to_string(rel));
        return FEM_E_NOT_CONVERGED;
    }
    return FEM_OK;
}

// Start / finish a sequence of deferred solves (running totals on the device).
fem_status solve_totals_reset(fem_mesh* m, cudaStream_t s) {
    FEM_CUDA(cudaMemsetAsync(m->dscal.p + 64, 0, 8 * sizeof(double), s));
    return FEM_OK;
}

fem_status solve_totals_read(fem_mesh* m, cudaStream_t s) {
    double* hs = (double*)m->host_stage;
    FEM_CUDA(cudaMemcpyAsync(hs, m->dscal.p + 64, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    m->stats.cg_iters += (long long)hs[0];
    m->stats.solves += (int)hs[3];
    m->stats.relres = hs[1];
    note_bytes(F_CG, hs[4]);
    int st = (int)hs[2];
    if (st == FEM_E_TIMEOUT) {
        reset_coop_state(m, s);
        set_error("Laplace solve: a grid barrier wait ran out");
        return FEM_E_TIMEOUT;
    }
    if (st == FEM_E_INVALID) {
        set_error("Laplace solve: the component search of A_UU failed (unknown count does not match the mesh)");
        return FEM_E_INVALID;
    }
    if (st != FEM_OK) {
        set_error("Laplace solve: iteration cap reached, largest relative residual " + std::to_string(hs[1]));
        return FEM_E_NOT_CONVERGED;
    }
    return FEM_OK;
}

// Laplace solve for the current vertex values: the entries of m->uv at K are
// the Dirichlet data, those at U the start; the solution is written back.
fem_status solve_laplace(fem_mesh* m, bool use_fp64, double tol, int maxit, cudaStream_t s, int* iters_out,
                         double* relres_out, bool deferred) {
    Nvtx range("laplace solve");
    bool rhs_done = true;  // filled by the ELL kernel when the system is rebuilt here
    FEM_TRY(build_system_rhs(m, s, &rhs_done));
    int nU = m->nU;
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    if (nU == 0) return FEM_OK;
    FEM_TRY(ensure(m->b64, (size_t)nU, s));
    FEM_TRY(ensure(m->x64, (size_t)nU, s));
    int b = (nU + 255) / 256;
    if (!rhs_done)
        FEM_LAUNCH(F_CG, s, k_rhs_and_start, b, 256, 0, nU, m->V, m->urow_vertex.p, m->nbr.p, m->coefA.p, m->mask.p,
                   m->uv.p, m->b64.p, m->x64.p);
    // the solvers write the solution back to the vertex values themselves
    return run_solve(m, m->b64.p, m->x64.p, use_fp64, tol, maxit, s, iters_out, relres_out, deferred, true);
}

// ------------------------------------------------------- vertex data setup
__global__ void k_uv_from_g(const unsigned char* __restrict__ mask, const int* __restrict__ kidx, int V,
                            const float* __restrict__ g, double* __restrict__ uv) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < V && mask[i]) uv[i] = (double)g[kidx[i]];
}

__global__ void k_uv_from_f(const unsigned char* __restrict__ mask, const int2* __restrict__ vxy, int V, int N,
                            const float* __restrict__ f, double* __restrict__ uv, float2* __restrict__ uvf) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < V && mask[i]) {
        int2 p = vxy[i];
        float v = f[(long long)p.y * N + p.x];
        uv[i] = (double)v;
        uvf[i] = make_float2(v, 0.0f);
    }
}

__global__ void k_gather_mask(const int* __restrict__ kvert, const int2* __restrict__ vxy, int nK, int N,
                              const float* __restrict__ f, float* __restrict__ g) {
    pdl_wait();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nK) return;
    int2 p = vxy[kvert[k]];
    g[k] = f[(long long)p.y * N + p.x];
}

fem_status set_uv_from_g(fem_mesh* m, const float* g_dev, cudaStream_t s) {
    FEM_TRY(build_system(m, s));
    FEM_LAUNCH(F_OTHER, s, k_uv_from_g, (m->V + 255) / 256, 256, 0, m->mask.p, m->kidx.p, m->V, g_dev, m->uv.p);
    return FEM_OK;
}

fem_status set_uv_from_f(fem_mesh* m, const float* f_dev, cudaStream_t s) {
    FEM_LAUNCH(F_OTHER, s, k_uv_from_f, (m->V + 255) / 256, 256, 0, m->mask.p, m->vxy.p, m->V, m->N, f_dev, m->uv.p,
               m->uvf.p);
    return FEM_OK;
}

}  // namespace fem

using namespace fem;

extern "C" fem_status fem_gather_mask(fem_mesh* m, const float* f_dev, float* g_dev, void* stream) {
    if (!m || !f_dev || !g_dev) {
        set_error("fem_gather_mask: null argument");
        return FEM_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    m->last_stream = s;
    FEM_TRY(build_system(m, s));
    FEM_TRY(domain_image(m, f_dev, s, &f_dev));
    if (m->nK > 0)
        FEM_LAUNCH(F_OTHER, s, k_gather_mask, (m->nK + 255) / 256, 256, 0, m->kvert.p, m->vxy.p, m->nK, m->N, f_dev,
                   g_dev);
    return FEM_OK;
}

extern "C" fem_status fem_inpaint(fem_mesh* m, const float* g_dev, float* u_dev, double* uv_dev, const fem_params* p,
                                  void* stream) {
    Nvtx range("fem_inpaint");
    if (!m || !g_dev) {
        set_error("fem_inpaint: null argument");
        return FEM_E_INVALID;
    }
    fem_params d;
    fem_params_default(&d);
    if (!p) p = &d;
    cudaStream_t s = (cudaStream_t)stream;
    m->last_stream = s;
    m->stats = fem_stats{};
    FEM_TRY(set_uv_from_g(m, g_dev, s));
    int it = 0;
    double rel = 0.0;
    fem_status st = solve_laplace(m, p->precision == FEM_PREC_FP64, p->tol, p->maxit, s, &it, &rel);
    if (st != FEM_OK && st != FEM_E_NOT_CONVERGED) return st;
    if (u_dev) FEM_TRY(raster_image(m, m->uv.p, u_dev, nullptr, s));
    if (uv_dev) FEM_CUDA(cudaMemcpyAsync(uv_dev, m->uv.p, sizeof(double) * m->V, cudaMemcpyDeviceToDevice, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    return st;
}
