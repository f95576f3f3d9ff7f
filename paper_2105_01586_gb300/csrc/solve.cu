// solve.cu -- P1 stiffness assembly and the Laplace solve on the unknown
// vertices (Sec. 2.2): A_UU x_U = -A_UK g_K by Jacobi-preconditioned CG.
//
// Every triangle of a newest-vertex-bisection mesh of the pixel square is a
// right isosceles triangle, so its P1 stiffness matrix is the same for all
// sizes: with c at the right angle, K_cc = 1, K_aa = K_bb = 1/2,
// K_ac = K_bc = -1/2, K_ab = 0.  All entries of A are multiples of 1/2 and
// exact in FP32.  All edges point in one of 8 lattice directions, so A is
// stored per vertex and direction (ELL with 8 slots, slot-major).
//
// The solve is one cooperative kernel with bounded grid barriers:
//   FP32_IR: repeat { r = b - A x in FP64; stop if ||r|| <= tol ||b||;
//                     solve A d = r/||r|| by FP32 PCG to relative 1e-5;
//                     x += ||r|| d (FP64) }
//   FP64:    PCG in FP64 from the warm start until ||r|| <= tol ||b||, then
//            the residual is recomputed from scratch to confirm.
#include <cmath>
#include <vector>

#include "fem_internal.cuh"

namespace fem {

constexpr int kSolveThreads = 256;
constexpr double kInnerEta = 1e-5;

// ---------------------------------------------------------------- assembly
__global__ void k_assemble(const int4* __restrict__ tri, const int2* __restrict__ vxy, int T, int V,
                           int* __restrict__ nbr, float* __restrict__ coef, float* __restrict__ diag) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    int4 tr = tri[t];
    int a = tr.x, b = tr.y, c = tr.z;
    int2 pa = vxy[a], pb = vxy[b], pc = vxy[c];
    // legs (c,a) and (c,b)
    int d;
    d = dir_index(pa.x - pc.x, pa.y - pc.y);
    nbr[d * V + c] = a; atomicAdd(&coef[d * V + c], -0.5f);
    d = (d + 4) & 7;
    nbr[d * V + a] = c; atomicAdd(&coef[d * V + a], -0.5f);
    d = dir_index(pb.x - pc.x, pb.y - pc.y);
    nbr[d * V + c] = b; atomicAdd(&coef[d * V + c], -0.5f);
    d = (d + 4) & 7;
    nbr[d * V + b] = c; atomicAdd(&coef[d * V + b], -0.5f);
    // hypotenuse (a,b): adjacency only, zero stiffness
    d = dir_index(pb.x - pa.x, pb.y - pa.y);
    nbr[d * V + a] = b;
    nbr[((d + 4) & 7) * V + b] = a;
    atomicAdd(&diag[c], 1.0f);
    atomicAdd(&diag[a], 0.5f);
    atomicAdd(&diag[b], 0.5f);
}

__global__ void k_unknown_flags(const unsigned char* __restrict__ mask, int V, int* __restrict__ flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < V) flag[i] = mask[i] ? 0 : 1;
}

__global__ void k_index_maps(const unsigned char* __restrict__ mask, int V, int* __restrict__ uidx,
                             int* __restrict__ kidx, int* __restrict__ urow_vertex, int* __restrict__ kvert) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V) return;
    int u = uidx[i];  // exclusive count of unknowns before i
    if (mask[i]) {
        int k = i - u;
        kidx[i] = k;
        kvert[k] = i;
        uidx[i] = -1;
    } else {
        kidx[i] = -1;
        urow_vertex[u] = i;
    }
}

__global__ void k_build_ell(int nU, int V, const int* __restrict__ urow_vertex, const int* __restrict__ nbr,
                            const float* __restrict__ coef, const float* __restrict__ diag,
                            const int* __restrict__ uidx, int* __restrict__ ucol, float* __restrict__ uval,
                            float* __restrict__ udiag) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nU) return;
    int i = urow_vertex[r];
    int s = 0;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        int j = nbr[d * V + i];
        float c = coef[d * V + i];
        if (j >= 0 && c != 0.0f) {
            int uj = uidx[j];
            if (uj >= 0) {
                ucol[s * nU + r] = uj;
                uval[s * nU + r] = c;
                s++;
            }
        }
    }
    for (; s < 8; ++s) {
        ucol[s * nU + r] = r;
        uval[s * nU + r] = 0.0f;
    }
    udiag[r] = diag[i];
}

// b_r = -sum over mask neighbours j of A_ij uv_j;  x_r = uv of the row's vertex
__global__ void k_rhs_and_start(int nU, int V, const int* __restrict__ urow_vertex, const int* __restrict__ nbr,
                                const float* __restrict__ coef, const unsigned char* __restrict__ mask,
                                const double* __restrict__ uv, double* __restrict__ b, double* __restrict__ x) {
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

__global__ void k_scatter_solution(int nU, const int* __restrict__ urow_vertex, const double* __restrict__ x,
                                   double* __restrict__ uv) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nU) uv[urow_vertex[r]] = x[r];
}

fem_status build_system(fem_mesh* m, cudaStream_t s) {
    if (m->sys_version == m->mesh_version) return FEM_OK;
    int V = m->V, T = m->T;
    FEM_TRY(ensure(m->nbr, (size_t)8 * V, s));
    FEM_TRY(ensure(m->coefA, (size_t)8 * V, s));
    FEM_TRY(ensure(m->diagA, V, s));
    FEM_TRY(ensure(m->uidx, V, s));
    FEM_TRY(ensure(m->kidx, V, s));
    FEM_TRY(ensure(m->flags, (size_t)V + 1, s));
    FEM_TRY(ensure(m->urow_vertex, V, s));
    FEM_TRY(ensure(m->kvert, V, s));
    FEM_CUDA(cudaMemsetAsync(m->nbr.p, 0xff, sizeof(int) * 8 * V, s));
    FEM_CUDA(cudaMemsetAsync(m->coefA.p, 0, sizeof(float) * 8 * V, s));
    FEM_CUDA(cudaMemsetAsync(m->diagA.p, 0, sizeof(float) * V, s));
    FEM_LAUNCH(F_ASSEMBLY, s, k_assemble, (T + 255) / 256, 256, 0, m->tri.p, m->vxy.p, T, V, m->nbr.p, m->coefA.p,
               m->diagA.p);
    int vb = (V + 255) / 256;
    FEM_LAUNCH(F_ASSEMBLY, s, k_unknown_flags, vb, 256, 0, m->mask.p, V, m->flags.p);
    int* nU_dev = m->dcount.p + 1;
    FEM_TRY(exclusive_scan_i32(m->flags.p, m->uidx.p, V, s, nU_dev));
    FEM_LAUNCH(F_ASSEMBLY, s, k_index_maps, vb, 256, 0, m->mask.p, V, m->uidx.p, m->kidx.p, m->urow_vertex.p,
               m->kvert.p);
    int nU = 0;
    FEM_CUDA(cudaMemcpyAsync(m->host_stage, nU_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    nU = *(int*)m->host_stage;
    m->nU = nU;
    m->nK = V - nU;
    size_t n = nU > 0 ? nU : 1;
    FEM_TRY(ensure(m->ucol, 8 * n, s));
    FEM_TRY(ensure(m->uval32, 8 * n, s));
    FEM_TRY(ensure(m->dinv32, n, s));  // holds the diagonal of A_UU
    if (nU > 0)
        FEM_LAUNCH(F_ASSEMBLY, s, k_build_ell, (nU + 255) / 256, 256, 0, nU, V, m->urow_vertex.p, m->nbr.p,
                   m->coefA.p, m->diagA.p, m->uidx.p, m->ucol.p, m->uval32.p, m->dinv32.p);
    m->sys_version = m->mesh_version;
    return FEM_OK;
}

// ------------------------------------------------------------ device solve
struct SolveArgs {
    int n;
    const int* col;
    const float* val;
    const float* diag;
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
    double* out;       // [0] iterations, [1] relres, [2] status
};

// block-wide sum of two doubles; result valid in all threads
__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double s_a[kSolveThreads / 32], s_b[kSolveThreads / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    __syncthreads();
    if (lane == 0) { s_a[w] = a; s_b[w] = b; }
    __syncthreads();
    double ta = 0.0, tb = 0.0;
#pragma unroll
    for (int i = 0; i < kSolveThreads / 32; ++i) { ta += s_a[i]; tb += s_b[i]; }
    a = ta;
    b = tb;
}

// grid-wide deterministic sum of two doubles (same result in every block).
// `parity` alternates between calls so that slow readers are never overwritten.
__device__ __forceinline__ bool grid_sum2(double& a, double& b, double* red, unsigned* bar, int* err, int& parity) {
    block_sum2(a, b);
    int nb = gridDim.x;
    double* buf = red + (size_t)parity * 2 * nb;
    if (threadIdx.x == 0) { buf[2 * blockIdx.x] = a; buf[2 * blockIdx.x + 1] = b; }
    parity ^= 1;
    if (!grid_barrier(bar, err)) return false;
    double ta = 0.0, tb = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        ta += __ldcg(&buf[2 * k]);
        tb += __ldcg(&buf[2 * k + 1]);
    }
    block_sum2(ta, tb);
    a = ta;
    b = tb;
    return true;
}

// y = A_UU v for rows of this thread (grid-stride); returns sum of v_r * y_r
template <class T>
__device__ __forceinline__ double spmv_rows(const SolveArgs& A, const T* __restrict__ v, T* __restrict__ y) {
    double dot = 0.0;
    int n = A.n;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        T vr = __ldcg(&v[r]);
        T s = (T)A.diag[r] * vr;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            int c = A.col[k * n + r];
            T w = (T)A.val[k * n + r];
            s += w * __ldcg(&v[c]);
        }
        y[r] = s;
        dot += (double)vr * (double)s;
    }
    return dot;
}

// PCG on A d = rhs from d = d0 (in: d), precision T.  Stops when
// ||r|| <= eta ||rhs||.  Returns false on a barrier failure.
template <class T>
__device__ bool pcg(const SolveArgs& A, const T* rhs, T* d, T* r, T* z, T* p, T* q, double eta, int maxit,
                    int& iters, double& rr_out, double& bb_out, int& parity) {
    int n = A.n;
    int stride = gridDim.x * blockDim.x;
    int tid0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (!grid_barrier(A.bar, A.err)) return false;  // d and rhs complete
    spmv_rows<T>(A, d, q);
    double rz = 0.0, bb = 0.0;
    for (int i = tid0; i < n; i += stride) {
        T ri = rhs[i] - q[i];
        r[i] = ri;
        T zi = ri / (T)A.diag[i];
        z[i] = zi;
        p[i] = zi;
        rz += (double)ri * (double)zi;
        double bi = (double)rhs[i];
        bb += bi * bi;
    }
    if (!grid_sum2(rz, bb, A.red, A.bar, A.err, parity)) return false;
    double rr = 0.0, dummy = 0.0;
    for (int i = tid0; i < n; i += stride) rr += (double)r[i] * (double)r[i];
    if (!grid_sum2(rr, dummy, A.red, A.bar, A.err, parity)) return false;
    bb_out = bb;
    double lim = eta * eta * bb;
    iters = 0;
    while (rr > lim && iters < maxit) {
        double pq = spmv_rows<T>(A, p, q), dm = 0.0;
        if (!grid_sum2(pq, dm, A.red, A.bar, A.err, parity)) return false;
        if (!(pq > 0.0)) break;  // breakdown guard (exact solution or loss of SPD in rounding)
        T alpha = (T)(rz / pq);
        double rz1 = 0.0, rr1 = 0.0;
        for (int i = tid0; i < n; i += stride) {
            d[i] += alpha * p[i];
            T ri = r[i] - alpha * q[i];
            r[i] = ri;
            T zi = ri / (T)A.diag[i];
            z[i] = zi;
            rz1 += (double)ri * (double)zi;
            rr1 += (double)ri * (double)ri;
        }
        if (!grid_sum2(rz1, rr1, A.red, A.bar, A.err, parity)) return false;
        iters++;
        rr = rr1;
        T beta = (T)(rz1 / rz);
        rz = rz1;
        for (int i = tid0; i < n; i += stride) p[i] = z[i] + beta * p[i];
        if (!grid_barrier(A.bar, A.err)) return false;  // p complete before the next SpMV
    }
    rr_out = rr;
    return true;
}

// FP64 residual r = b - A x; returns (||r||^2, ||b||^2) grid-wide
__device__ bool residual64(const SolveArgs& A, double& rr, double& bb, int& parity) {
    if (!grid_barrier(A.bar, A.err)) return false;  // x complete
    int n = A.n;
    rr = 0.0;
    bb = 0.0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        double s = (double)A.diag[r] * __ldcg(&A.x[r]);
#pragma unroll
        for (int k = 0; k < 8; ++k) s += (double)A.val[k * n + r] * __ldcg(&A.x[A.col[k * n + r]]);
        double ri = A.b[r] - s;
        A.r64[r] = ri;
        rr += ri * ri;
        bb += A.b[r] * A.b[r];
    }
    return grid_sum2(rr, bb, A.red, A.bar, A.err, parity);
}

template <bool FP64_ONLY>
__global__ void __launch_bounds__(kSolveThreads) k_solve(SolveArgs A) {
    int parity = 0;
    int n = A.n;
    int stride = gridDim.x * blockDim.x;
    int tid0 = blockIdx.x * blockDim.x + threadIdx.x;
    int total_it = 0, n_res = 1;
    double rr = 0.0, bb = 0.0;
    int status = FEM_E_NOT_CONVERGED;
    if (!residual64(A, rr, bb, parity)) goto fail;
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
            // solve A x = b from the current x: d = x, rhs = b
            int it = 0;
            double rr_in = 0.0, bb_in = 0.0;
            if (!pcg<double>(A, A.b, A.x, A.r64, A.z64, A.p64, A.q64, A.tol, A.maxit - total_it, it, rr_in, bb_in,
                             parity))
                goto fail;
            total_it += it;
            n_res++;
            if (!residual64(A, rr, bb, parity)) goto fail;
        }
        if (rr <= A.tol * A.tol * bb) status = FEM_OK;
    } else {
        for (int step = 0; step < 64; ++step) {
            if (rr <= A.tol * A.tol * bb) { status = FEM_OK; break; }
            if (total_it >= A.maxit) break;
            double scale = 1.0 / sqrt(rr);
            for (int i = tid0; i < n; i += stride) {
                A.r32[i] = (float)(A.r64[i] * scale);
                A.d32[i] = 0.0f;
            }
            int it = 0;
            double rr_in = 0.0, bb_in = 0.0;
            if (!pcg<float>(A, A.r32, A.d32, A.z32 /*r*/, A.q32 /*z*/, A.p32, A.q32 + n /*q*/, kInnerEta,
                            A.maxit - total_it, it, rr_in, bb_in, parity))
                goto fail;
            total_it += it;
            double back = sqrt(rr);
            for (int i = tid0; i < n; i += stride) A.x[i] += back * (double)A.d32[i];
            n_res++;
            if (!residual64(A, rr, bb, parity)) goto fail;
        }
        if (rr <= A.tol * A.tol * bb) status = FEM_OK;
    }
done:
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.out[0] = total_it;
        A.out[1] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        A.out[2] = status;
        A.out[3] = n_res;
    }
    return;
fail:
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.out[0] = total_it;
        A.out[1] = -1.0;
        A.out[2] = FEM_E_TIMEOUT;
        A.out[3] = n_res;
    }
}

static int coop_blocks(const void* func, int n, int num_sms) {
    static int occ[2] = {0, 0};
    int which = func == (const void*)k_solve<true> ? 1 : 0;
    if (!occ[which]) {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, func, kSolveThreads, 0);
        occ[which] = nb > 0 ? nb : 1;
    }
    int maxb = occ[which] * num_sms;
    int want = (n + 4 * kSolveThreads - 1) / (4 * kSolveThreads);
    if (want < 1) want = 1;
    return want < maxb ? want : maxb;
}

// Solve A_UU x = b (device vectors of length nU; x holds the start).
fem_status run_solve(fem_mesh* m, const double* b, double* x, bool use_fp64, double tol, int maxit, cudaStream_t s,
                     int* iters_out, double* relres_out) {
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
    const void* func = use_fp64 ? (const void*)k_solve<true> : (const void*)k_solve<false>;
    int grid = coop_blocks(func, nU, m->num_sms);
    FEM_TRY(ensure(m->red, (size_t)4 * grid + 8, s));
    SolveArgs A;
    A.n = nU;
    A.col = m->ucol.p;
    A.val = m->uval32.p;
    A.diag = m->dinv32.p;
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
    FEM_CUDA(cudaMemsetAsync(m->dflag.p + 1, 0, sizeof(int), s));
    void* args[] = {&A};
    FEM_TRY(launch_coop(F_CG, func, grid, kSolveThreads, 0, s, args, use_fp64 ? "k_solve<fp64>" : "k_solve<fp32ir>"));
    double* hs = (double*)m->host_stage;
    FEM_CUDA(cudaMemcpyAsync(hs, m->dscal.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    int its = (int)hs[0];
    double rel = hs[1];
    int st = (int)hs[2];
    int nres = (int)hs[3];
    // Algorithmic bytes per row: ELL matrix (8 columns + 8 values + diagonal,
    // 68 B) per SpMV; FP32 CG iteration = SpMV 76 B + updates 44 B; FP64 CG
    // iteration = SpMV 84 B + updates 84 B; FP64 residual pass 92 B; each FP32
    // refinement step adds 36 B of conversions and the FP64 update.
    double per_it = use_fp64 ? 168.0 : 120.0;
    double per_res = 92.0 + (use_fp64 ? 0.0 : 36.0);
    note_bytes(F_CG, (double)nU * (per_it * its + per_res * nres));
    m->stats.cg_iters += its;
    m->stats.solves += 1;
    m->stats.relres = rel;
    if (iters_out) *iters_out = its;
    if (relres_out) *relres_out = rel;
    if (st == FEM_E_TIMEOUT) {
        cudaMemsetAsync(m->bar.p, 0, 2 * sizeof(unsigned), s);
        set_error("Laplace solve: a grid barrier wait ran out");
        return FEM_E_TIMEOUT;
    }
    if (st != FEM_OK) {
        set_error("Laplace solve: iteration cap reached, relative residual " + std::to_string(rel));
        return FEM_E_NOT_CONVERGED;
    }
    return FEM_OK;
}

// Laplace solve for the current vertex values: the entries of m->uv at K are
// the Dirichlet data, those at U the start; the solution is written back.
fem_status solve_laplace(fem_mesh* m, bool use_fp64, double tol, int maxit, cudaStream_t s, int* iters_out,
                         double* relres_out) {
    FEM_TRY(build_system(m, s));
    int nU = m->nU;
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    if (nU == 0) return FEM_OK;
    FEM_TRY(ensure(m->b64, (size_t)nU, s));
    FEM_TRY(ensure(m->x64, (size_t)nU, s));
    int b = (nU + 255) / 256;
    FEM_LAUNCH(F_CG, s, k_rhs_and_start, b, 256, 0, nU, m->V, m->urow_vertex.p, m->nbr.p, m->coefA.p, m->mask.p,
               m->uv.p, m->b64.p, m->x64.p);
    fem_status st = run_solve(m, m->b64.p, m->x64.p, use_fp64, tol, maxit, s, iters_out, relres_out);
    if (st != FEM_OK && st != FEM_E_NOT_CONVERGED) return st;
    FEM_LAUNCH(F_CG, s, k_scatter_solution, b, 256, 0, nU, m->urow_vertex.p, m->x64.p, m->uv.p);
    return st;
}

// ------------------------------------------------------- vertex data setup
__global__ void k_uv_from_g(const unsigned char* __restrict__ mask, const int* __restrict__ kidx, int V,
                            const float* __restrict__ g, double* __restrict__ uv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < V && mask[i]) uv[i] = (double)g[kidx[i]];
}

__global__ void k_uv_from_f(const unsigned char* __restrict__ mask, const int2* __restrict__ vxy, int V, int N,
                            const float* __restrict__ f, double* __restrict__ uv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < V && mask[i]) {
        int2 p = vxy[i];
        uv[i] = (double)f[(long long)p.y * N + p.x];
    }
}

__global__ void k_gather_mask(const int* __restrict__ kvert, const int2* __restrict__ vxy, int nK, int N,
                              const float* __restrict__ f, float* __restrict__ g) {
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
    FEM_LAUNCH(F_OTHER, s, k_uv_from_f, (m->V + 255) / 256, 256, 0, m->mask.p, m->vxy.p, m->V, m->N, f_dev, m->uv.p);
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
    if (m->nK > 0)
        FEM_LAUNCH(F_OTHER, s, k_gather_mask, (m->nK + 255) / 256, 256, 0, m->kvert.p, m->vxy.p, m->nK, m->N, f_dev,
                   g_dev);
    return FEM_OK;
}

extern "C" fem_status fem_inpaint(fem_mesh* m, const float* g_dev, float* u_dev, double* uv_dev, const fem_params* p,
                                  void* stream) {
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
