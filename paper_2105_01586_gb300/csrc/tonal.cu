// tonal.cu -- tonal optimisation (Sec. 4, eqs. 4-5) and the adjoint B^T.
//
// u = B g with B = P E: E g is the vertex vector with g at the mask vertices
// and -A_UU^{-1} A_UK g at the unknown ones (an inpainting solve), P the
// pixel interpolation.  The normal equations B^T B g = B^T f are solved by
// CG; B^T B p = E^T (P^T P) (E p).  P^T P =: M is a sparse V x V matrix with
// the mesh's graph (a pixel couples only the three vertices of its owner),
// so it is assembled once per mesh from one pass over the pixels, and each
// outer iteration costs one forward solve, one sparse product with M and one
// adjoint solve (E^T y = y_K - A_KU A_UU^{-1} y_U); no pixel is read inside
// the iteration.  B itself is never formed.  The iteration has the form of
// CGLS: its residual recursion runs on y = P^T (f - B g), and the normal
// residual E^T y is formed afresh each iteration.
//
// Per-vertex sums are gathered over the (at most 8) triangles around a
// vertex in a fixed order of their angular sector, so results do not depend
// on scheduling.
#include <cmath>
#include <vector>

#include <cstring>

#include "fem_internal.cuh"

namespace fem {

constexpr int kVecThreads = 256;

// Sector (octant) k of a nonzero direction: its angle lies in
// [k*45deg, (k+1)*45deg).  A triangle's sector at one of its vertices is the
// sector of the sum of its two edge vectors there: strictly inside a 45-degree
// corner, and on the bisector of a right-angle corner, i.e. on the boundary
// between its two sectors, where the half-open rule picks the upper one.
// Either way the sector is covered by no other triangle around the vertex.
__device__ __forceinline__ int octant(int dx, int dy) {
    if (dy >= 0) {
        if (dx > 0) return dy < dx ? 0 : 1;
        if (dy == 0) return 4;
        return dy > -dx ? 2 : 3;
    }
    if (dx < 0) return dy > dx ? 4 : 5;
    return dx < -dy ? 6 : 7;
}

__global__ void k_incidence(const int4* __restrict__ tri, const int2* __restrict__ vxy, int T, int V,
                            int* __restrict__ inc) {
    pdl_wait();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    int4 tr = tri[t];
    int id[3] = {tr.x, tr.y, tr.z};
    int2 p[3] = {vxy[tr.x], vxy[tr.y], vxy[tr.z]};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        int j = (r + 1) % 3, k = (r + 2) % 3;
        int dx = (p[j].x - p[r].x) + (p[k].x - p[r].x);
        int dy = (p[j].y - p[r].y) + (p[k].y - p[r].y);
        inc[octant(dx, dy) * V + id[r]] = 3 * t + r;
    }
}

// local pixel-mass entries of triangle t: [aa, bb, cc, ab, bc, ca]
__device__ __forceinline__ int mass_diag_slot(int r) { return r; }
__device__ __forceinline__ int mass_off_slot(int r, int s) {
    int lo = min(r, s), hi = max(r, s);
    return lo == 0 ? (hi == 1 ? 3 : 5) : 4;
}

__global__ void k_gather_mass(int V, const int* __restrict__ inc, const int4* __restrict__ tri,
                              const int2* __restrict__ vxy, const double* __restrict__ loc6,
                              double* __restrict__ Mdiag, double* __restrict__ Moff) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V) return;
    double dsum = 0.0, off[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) off[d] = 0.0;
    int2 pi = vxy[i];
    for (int o = 0; o < 8; ++o) {
        int e = inc[o * V + i];
        if (e < 0) continue;
        int t = e / 3, r = e % 3;
        int4 tr = tri[t];
        int id[3] = {tr.x, tr.y, tr.z};
        dsum += loc6[6 * t + mass_diag_slot(r)];
#pragma unroll
        for (int q = 1; q < 3; ++q) {
            int s = (r + q) % 3;
            int2 pj = vxy[id[s]];
            int d = dir_index(pj.x - pi.x, pj.y - pi.y);
            off[d] += loc6[6 * t + mass_off_slot(r, s)];
        }
    }
    Mdiag[i] = dsum;
#pragma unroll
    for (int d = 0; d < 8; ++d) Moff[d * V + i] = off[d];
}

// s_i = sum over the triangles around i of their local scatter sums
__global__ void k_gather_scatter(int V, const int* __restrict__ inc, const double* __restrict__ loc3,
                                 double* __restrict__ s) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V) return;
    double acc = 0.0;
    for (int o = 0; o < 8; ++o) {
        int e = inc[o * V + i];
        if (e >= 0) acc += loc3[e];  // loc3[3t + r]
    }
    s[i] = acc;
}

// b_r = -sum over mask neighbours j of A_ij p[kidx[j]]
__global__ void k_fwd_rhs(int nU, int V, const int* __restrict__ urow_vertex, const int* __restrict__ nbr,
                          const float* __restrict__ coef, const unsigned char* __restrict__ mask,
                          const int* __restrict__ kidx, const double* __restrict__ p, double* __restrict__ b,
                          double* __restrict__ x) {
    pdl_wait();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nU) return;
    int i = urow_vertex[r];
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        int j = nbr[d * V + i];
        float c = coef[d * V + i];
        if (j >= 0 && c != 0.0f && mask[j]) s -= (double)c * p[kidx[j]];
    }
    b[r] = s;
    x[r] = 0.0;
}

// v = E p given the unknown-vertex solution x
__global__ void k_assemble_v(int V, const unsigned char* __restrict__ mask, const int* __restrict__ kidx,
                             const int* __restrict__ uidx, const double* __restrict__ p, const double* __restrict__ x,
                             double* __restrict__ v) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V) return;
    v[i] = mask[i] ? p[kidx[i]] : x[uidx[i]];
}

// y = M v, and per-block partial sums of v.y
__global__ void k_mass_spmv(int V, const double* __restrict__ Mdiag, const double* __restrict__ Moff,
                            const int* __restrict__ nbr, const double* __restrict__ v, double* __restrict__ y,
                            double* __restrict__ partial) {
    pdl_wait();
    double dot = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
        double vi = v[i];
        double s = Mdiag[i] * vi;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            int j = nbr[d * V + i];
            if (j >= 0) s += Moff[d * V + i] * v[j];
        }
        y[i] = s;
        dot += vi * s;
    }
    __shared__ double sh[kVecThreads / 32];
    dot = warp_sum(dot);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = dot;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kVecThreads / 32; ++w) t += sh[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void k_gather_U(int nU, const int* __restrict__ urow_vertex, const double* __restrict__ y,
                           double* __restrict__ b, double* __restrict__ x) {
    pdl_wait();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nU) return;
    b[r] = y[urow_vertex[r]];
    x[r] = 0.0;
}

// w_k = y_k - sum over unknown neighbours j of A_kj z_j   (E^T y)
__global__ void k_adj_combine(int nK, int V, const int* __restrict__ kvert, const int* __restrict__ nbr,
                              const float* __restrict__ coef, const int* __restrict__ uidx,
                              const double* __restrict__ y, const double* __restrict__ z, double* __restrict__ w) {
    pdl_wait();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nK) return;
    int i = kvert[k];
    double s = y[i];
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        int j = nbr[d * V + i];
        float c = coef[d * V + i];
        if (j >= 0 && c != 0.0f) {
            int u = uidx[j];
            if (u >= 0) s -= (double)c * z[u];
        }
    }
    w[k] = s;
}

// scalars of the outer CG on the device (dscal + 32): |c|^2, p.N p, gamma =
// r.r, the previous gamma, the stop threshold tol |c| (compared with
// sqrt(gamma)), the stop flag and the number of completed iterations
struct CgScalars {
    double cc, pNp, gamma, gamma_old, thr, stop, iters;
};

__global__ void k_final_sum(int n, const double* __restrict__ partial, double* __restrict__ out) {
    pdl_wait();
    __shared__ double sh[kVecThreads / 32];
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t += partial[i];
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kVecThreads / 32; ++w) s += sh[w];
        *out = s;
    }
}

// end of a CG update (mode 1): gamma_old = gamma, gamma = sum of the
// partials, one more iteration, stop when sqrt(gamma) <= thr; a breakdown
// (pNp <= 0) stops without an update
__global__ void k_cg_update_sum(int nb, const double* __restrict__ partial, CgScalars* __restrict__ cg) {
    pdl_wait();
    __shared__ double sh[kVecThreads / 32];
    if (cg->stop != 0.0) return;
    if (!(cg->pNp > 0.0)) {
        if (threadIdx.x == 0) cg->stop = 1.0;
        return;
    }
    double t = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) t += partial[i];
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double g = 0.0;
        for (int w = 0; w < kVecThreads / 32; ++w) g += sh[w];
        cg->gamma_old = cg->gamma;
        cg->gamma = g;
        cg->iters += 1.0;
        if (sqrt(g) <= cg->thr) cg->stop = 1.0;
    }
}

// mode 0: partial of x.y; mode 1: g += a p, r -= a w, partial of r.r;
// mode 2: p = r + b p; mode 3: r = c - w (r = c when w is null), p = r,
// partial r.r.
// cg (optional, the outer CG's device scalars, see CgScalars): modes 1 and
// 2 take a = gamma / pNp and b = gamma / gamma_old from it and do nothing
// once the iteration has stopped, so no scalar is read back per iteration.

__global__ void k_vec(int mode, int n, double a, double* __restrict__ x, double* __restrict__ y,
                      double* __restrict__ z, const double* __restrict__ w, double* __restrict__ partial,
                      const CgScalars* __restrict__ cg = nullptr) {
    pdl_wait();
    if (cg) {
        if (cg->stop != 0.0) return;
        if (mode == 1) {
            if (!(cg->pNp > 0.0)) return;
            a = cg->gamma / cg->pNp;
        } else if (mode == 2) {
            a = cg->gamma / cg->gamma_old;
        }
    }
    double dot = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (mode == 0) {
            dot += x[i] * y[i];
        } else if (mode == 1) {  // x = g, y = p, z = r
            x[i] += a * y[i];
            double r = z[i] - a * w[i];
            z[i] = r;
            dot += r * r;
        } else if (mode == 2) {  // x = p, z = r
            x[i] = z[i] + a * x[i];
        } else {  // x = r, y = p, z = c (w null: r = c)
            double r = w ? z[i] - w[i] : z[i];
            x[i] = r;
            y[i] = r;
            dot += r * r;
        }
    }
    if (mode == 2) return;
    __shared__ double sh[kVecThreads / 32];
    dot = warp_sum(dot);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = dot;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w2 = 0; w2 < kVecThreads / 32; ++w2) t += sh[w2];
        partial[blockIdx.x] = t;
    }
}

// One step of the outer iteration (modes of the CgScalars): a = gamma / pNp,
// g += a p over the nK mask values and y -= a (M E p) over the V vertices;
// nothing once the iteration has stopped or broken down (pNp <= 0).
__global__ void k_tonal_step(int nK, int V, double* __restrict__ g, const double* __restrict__ p,
                             double* __restrict__ y, const double* __restrict__ My, const CgScalars* __restrict__ cg) {
    pdl_wait();
    if (cg->stop != 0.0 || !(cg->pNp > 0.0)) return;
    const double a = cg->gamma / cg->pNp;
    const int n = max(nK, V);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i < nK) g[i] += a * p[i];
        if (i < V) y[i] -= a * My[i];
    }
}

// y = y - x
__global__ void k_sub_into(int n, const double* __restrict__ x, double* __restrict__ y) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] -= x[i];
}

__global__ void k_f2d(int n, const float* __restrict__ a, double* __restrict__ b) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

__global__ void k_d2f(int n, const double* __restrict__ a, float* __restrict__ b) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// b = a - b
__global__ void k_sub_from(int n, const double* __restrict__ a, double* __restrict__ b) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i] - b[i];
}

// per-block partial sums of x (grid-stride, fixed order within a block)
__global__ void k_sum_partial(long long n, const double* __restrict__ x, double* __restrict__ partial) {
    pdl_wait();
    __shared__ double sh[kVecThreads / 32];
    double t = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        t += x[i];
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kVecThreads / 32; ++w) s += sh[w];
        partial[blockIdx.x] = s;
    }
}

// *out = scale * (sum of the n partials), one block
__global__ void k_final_sum_scaled(int n, const double* __restrict__ partial, double scale, double* __restrict__ out) {
    pdl_wait();
    __shared__ double sh[kVecThreads / 32];
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t += partial[i];
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kVecThreads / 32; ++w) s += sh[w];
        *out = scale * s;
    }
}

static int vec_grid(fem_mesh* m) { return 2 * m->num_sms; }

// read one device double (synchronises the stream)
static fem_status read_scalar(fem_mesh* m, const double* d, double* out, cudaStream_t s) {
    FEM_CUDA(cudaMemcpyAsync(m->host_stage, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    *out = *(double*)m->host_stage;
    return FEM_OK;
}

// Incidence by sector and the pixel-mass matrix M = P^T P (once per mesh).
static fem_status prepare_tonal(fem_mesh* m, cudaStream_t s) {
    FEM_TRY(build_system(m, s));
    int V = m->V, T = m->T;
    if (m->tonal_version == m->mesh_version) return FEM_OK;
    FEM_TRY(ensure(m->inc, (size_t)8 * V, s));
    FEM_TRY(ensure(m->Moff, (size_t)8 * V, s));
    FEM_TRY(ensure(m->Mdiag, (size_t)V, s));
    FEM_CUDA(cudaMemsetAsync(m->inc.p, 0xff, sizeof(int) * 8 * V, s));
    FEM_LAUNCH(F_TONAL, s, k_incidence, (T + 255) / 256, 256, 0, m->tri.p, m->vxy.p, T, V, m->inc.p);
    FEM_TRY(raster_local(m, 2 /*R_MASS*/, nullptr, s));
    FEM_LAUNCH(F_TONAL, s, k_gather_mass, (V + 255) / 256, 256, 0, V, m->inc.p, m->tri.p, m->vxy.p, m->loc.p,
               m->Mdiag.p, m->Moff.p);
    m->tonal_version = m->mesh_version;
    return FEM_OK;
}

static fem_status ensure_tonal_vectors(fem_mesh* m, cudaStream_t s) {
    size_t V = m->V, nK = m->nK > 0 ? m->nK : 1, nU = m->nU > 0 ? m->nU : 1;
    FEM_TRY(ensure(m->tv, V, s));
    FEM_TRY(ensure(m->ty, V, s));
    FEM_TRY(ensure(m->tz, nU, s));
    FEM_TRY(ensure(m->b64, nU, s));
    FEM_TRY(ensure(m->x64, nU, s));
    FEM_TRY(ensure(m->tg, nK, s));
    FEM_TRY(ensure(m->tr, nK, s));
    FEM_TRY(ensure(m->tp, nK, s));
    FEM_TRY(ensure(m->tw, nK, s));
    FEM_TRY(ensure(m->tc, nK, s));
    FEM_TRY(ensure(m->tyr, V, s));
    FEM_TRY(ensure(m->red, (size_t)vec_grid(m) + 8, s));
    return FEM_OK;
}

struct InnerCfg {
    bool fp64;
    double tol;
    int maxit;
    bool deferred;  // statistics stay on the device (solve_totals_*); no read-back per solve
};

// w = E^T y for the vertex vector y (m->ty); uses m->b64 / m->tz
static fem_status apply_ET(fem_mesh* m, const double* y, double* w, const InnerCfg& c, cudaStream_t s) {
    int nU = m->nU, nK = m->nK;
    if (nU > 0) {
        FEM_LAUNCH(F_TONAL, s, k_gather_U, (nU + 255) / 256, 256, 0, nU, m->urow_vertex.p, y, m->b64.p, m->tz.p);
        fem_status st = run_solve(m, m->b64.p, m->tz.p, c.fp64, c.tol, c.maxit, s, nullptr, nullptr, c.deferred);
        if (st != FEM_OK) return st;
    }
    FEM_LAUNCH(F_TONAL, s, k_adj_combine, (nK + 255) / 256, 256, 0, nK, m->V, m->kvert.p, m->nbr.p, m->coefA.p,
               m->uidx.p, y, m->tz.p, w);
    return FEM_OK;
}

// ty = M E p (V entries) and *pNp_dev = (E p) . M (E p) = ||B p||^2
static fem_status apply_EM(fem_mesh* m, const double* p, double* pNp_dev, const InnerCfg& c, cudaStream_t s) {
    int nU = m->nU, V = m->V;
    if (nU > 0) {
        FEM_LAUNCH(F_TONAL, s, k_fwd_rhs, (nU + 255) / 256, 256, 0, nU, V, m->urow_vertex.p, m->nbr.p, m->coefA.p,
                   m->mask.p, m->kidx.p, p, m->b64.p, m->x64.p);
        fem_status st = run_solve(m, m->b64.p, m->x64.p, c.fp64, c.tol, c.maxit, s, nullptr, nullptr, c.deferred);
        if (st != FEM_OK) return st;
    }
    FEM_LAUNCH(F_TONAL, s, k_assemble_v, (V + 255) / 256, 256, 0, V, m->mask.p, m->kidx.p, m->uidx.p, p, m->x64.p,
               m->tv.p);
    int G = vec_grid(m);
    FEM_LAUNCH(F_TONAL, s, k_mass_spmv, G, kVecThreads, 0, V, m->Mdiag.p, m->Moff.p, m->nbr.p, m->tv.p, m->ty.p,
               m->red.p);
    FEM_LAUNCH(F_TONAL, s, k_final_sum, 1, kVecThreads, 0, G, m->red.p, pNp_dev);
    return FEM_OK;
}

static fem_status vec_op(fem_mesh* m, int mode, int n, double a, double* x, double* y, double* z, const double* w,
                         double* out_dev, cudaStream_t s) {
    int G = vec_grid(m);
    FEM_LAUNCH(F_TONAL, s, k_vec, G, kVecThreads, 0, mode, n, a, x, y, z, w, m->red.p, nullptr);
    if (mode != 2) FEM_LAUNCH(F_TONAL, s, k_final_sum, 1, kVecThreads, 0, G, m->red.p, out_dev);
    return FEM_OK;
}

// s = P^T r into m->ty (V entries)
static fem_status scatter_PT(fem_mesh* m, const float* r, cudaStream_t s) {
    FEM_TRY(raster_local(m, 3 /*R_SCAT*/, r, s));
    FEM_LAUNCH(F_TONAL, s, k_gather_scatter, (m->V + 255) / 256, 256, 0, m->V, m->inc.p, m->loc.p, m->ty.p);
    return FEM_OK;
}

}  // namespace fem

using namespace fem;

// The tonal optimisation's CG (below) on the least-squares problem
// min_g |B g - f|^2, or with `weighted` the weighted one
// min_g sum_p w_p ((B g)_p - f_p)^2: then the caller has put P^T W P into the
// pixel-mass matrix (prepare_weighted) and passes rhs = W f.  rhs is a
// domain image.  g_dev holds the start and receives the result.
static fem_status tonal_cg(fem_mesh* m, const float* rhs, float* g_dev, const fem_params* p, cudaStream_t s,
                           bool weighted) {
    m->stats = fem_stats{};
    if (!weighted) FEM_TRY(prepare_tonal(m, s));
    FEM_TRY(ensure_tonal_vectors(m, s));
    int nK = m->nK;
    // inner solves keep their statistics on the device (read once at the end)
    InnerCfg c{p->precision == FEM_PREC_FP64, p->inner_tol, p->maxit, true};
    FEM_TRY(solve_totals_reset(m, s));
    CgScalars* cg = (CgScalars*)(m->dscal.p + 32);
    double* sc = m->dscal.p + 32;  // [0] |c|^2 [1] pNp [2] gamma (the CgScalars layout)
    // The outer iteration is CG on the normal equations in the form of CGLS:
    // the recursion runs on y = P^T (f - B g) (the pixel residual seen through
    // P^T, a vertex vector: y -= a M E p), and the normal residual
    // s = B^T (f - B g) = E^T y is formed from it each iteration by the
    // adjoint solve.  Updating s itself (s -= a B^T B p) would lose accuracy
    // with the square of B's condition number.
    // c = B^T f = E^T P^T f, and y = P^T f - M E g for the start g
    FEM_TRY(scatter_PT(m, rhs, s));
    FEM_CUDA(cudaMemcpyAsync(m->tyr.p, m->ty.p, sizeof(double) * m->V, cudaMemcpyDeviceToDevice, s));
    FEM_TRY(apply_ET(m, m->ty.p, m->tc.p, c, s));
    FEM_TRY(vec_op(m, 0, nK, 0.0, m->tc.p, m->tc.p, nullptr, nullptr, sc + 0, s));
    FEM_LAUNCH(F_TONAL, s, k_f2d, (nK + 255) / 256, 256, 0, nK, g_dev, m->tg.p);
    FEM_TRY(apply_EM(m, m->tg.p, sc + 1, c, s));
    FEM_LAUNCH(F_TONAL, s, k_sub_into, (m->V + 255) / 256, 256, 0, m->V, (const double*)m->ty.p, m->tyr.p);
    // s = E^T y (into tw), r = s, p = s, gamma = |s|^2
    FEM_TRY(apply_ET(m, m->tyr.p, m->tw.p, c, s));
    FEM_TRY(vec_op(m, 3, nK, 0.0, m->tr.p, m->tp.p, m->tw.p, nullptr, sc + 2, s));
    double cc = 0.0, gamma = 0.0;
    FEM_TRY(read_scalar(m, sc + 0, &cc, s));
    FEM_TRY(read_scalar(m, sc + 2, &gamma, s));
    double cnorm = sqrt(cc);
    int it = 0;
    fem_status st = FEM_E_NOT_CONVERGED;
    if (cnorm == 0.0 || sqrt(gamma) <= p->tonal_tol * cnorm) {
        st = FEM_OK;
    } else if (p->tonal_maxit > 0) {
        // Outer CG with its scalars on the device: alpha = gamma / pNp and
        // beta = gamma / gamma_old are formed by the vector kernels, the stop
        // test (sqrt(gamma) <= tonal_tol |c|, or a breakdown pNp <= 0) by the
        // update's reduction, after which the vector kernels do nothing.  The
        // host reads the stop flag two iterations behind, so the GPU never
        // waits for it; the one or two iterations enqueued beyond the stop
        // leave g unchanged.
        double* hs = (double*)m->host_stage;
        // thr holds tol |c| and is compared with sqrt(gamma) (as above)
        double init[4] = {gamma, p->tonal_tol * cnorm, 0.0, 0.0};  // gamma_old, thr, stop, iters
        std::memcpy(hs, init, sizeof(init));
        FEM_CUDA(cudaMemcpyAsync(&cg->gamma_old, hs, sizeof(init), cudaMemcpyHostToDevice, s));
        cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
        fem_status lst = FEM_OK;
        for (int q = 0; q < 3 && lst == FEM_OK; ++q) {
            cudaError_t e = cudaEventCreateWithFlags(&ev[q], cudaEventDisableTiming);
            if (e != cudaSuccess) lst = cuda_fail(e, "cudaEventCreate");
        }
        double* slot = hs + 8;  // three pinned (stop, iters) pairs
        int G = vec_grid(m);
        for (int k = 0; lst == FEM_OK && k < p->tonal_maxit; ++k) {
            Nvtx it_range("tonal iteration");
            lst = check_cancel(m);
            if (lst != FEM_OK) break;
            // ||B p||^2 and M E p; g += a p, y -= a M E p; r = E^T y
            lst = apply_EM(m, m->tp.p, &cg->pNp, c, s);
            if (lst != FEM_OK) break;
            note_launch_begin(F_TONAL, s);
            k_tonal_step<<<G, kVecThreads, 0, s>>>(nK, m->V, m->tg.p, m->tp.p, m->tyr.p, m->ty.p, cg);
            note_launch_end(F_TONAL, s);
            lst = apply_ET(m, m->tyr.p, m->tr.p, c, s);
            if (lst != FEM_OK) break;
            note_launch_begin(F_TONAL, s);
            k_vec<<<G, kVecThreads, 0, s>>>(0, nK, 0.0, m->tr.p, m->tr.p, nullptr, nullptr, m->red.p, cg);
            note_launch_end(F_TONAL, s);
            note_launch_begin(F_TONAL, s);
            k_cg_update_sum<<<1, kVecThreads, 0, s>>>(G, m->red.p, cg);
            note_launch_end(F_TONAL, s);
            note_launch_begin(F_TONAL, s);
            k_vec<<<G, kVecThreads, 0, s>>>(2, nK, 0.0, m->tp.p, nullptr, m->tr.p, nullptr, m->red.p, cg);
            note_launch_end(F_TONAL, s);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(slot + 2 * (k % 3), &cg->stop, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaEventRecord(ev[k % 3], s);
            if (e != cudaSuccess) { lst = cuda_fail(e, "tonal iteration"); break; }
            if (k >= 2) {
                e = cudaEventSynchronize(ev[(k - 2) % 3]);
                if (e != cudaSuccess) { lst = cuda_fail(e, "cudaEventSynchronize"); break; }
                if (slot[2 * ((k - 2) % 3)] != 0.0) break;
            }
        }
        for (int q = 0; q < 3; ++q)
            if (ev[q]) cudaEventDestroy(ev[q]);
        FEM_TRY(lst);
        double fin[7];
        FEM_CUDA(cudaMemcpyAsync(hs, cg, sizeof(fin), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaStreamSynchronize(s));
        std::memcpy(fin, hs, sizeof(fin));
        gamma = fin[2];
        it = (int)fin[6];
        if (fin[5] != 0.0) st = FEM_OK;
    }
    FEM_LAUNCH(F_TONAL, s, k_d2f, (nK + 255) / 256, 256, 0, nK, m->tg.p, g_dev);
    fem_status sst = solve_totals_read(m, s);  // synchronises; inner-solve failures
    m->stats.tonal_iters = it;
    m->stats.tonal_relres = cnorm > 0 ? sqrt(gamma) / cnorm : 0.0;
    if (sst != FEM_OK) return sst;
    if (st != FEM_OK) set_error("fem_tonal_opt: outer iteration cap reached");
    return st;
}

extern "C" fem_status fem_tonal_opt(fem_mesh* m, const float* f_dev, float* g_dev, const fem_params* p, void* stream) {
    Nvtx range("fem_tonal_opt");
    if (!m || !f_dev || !g_dev) {
        set_error("fem_tonal_opt: null argument");
        return FEM_E_INVALID;
    }
    fem_params dflt;
    fem_params_default(&dflt);
    if (!p) p = &dflt;
    cudaStream_t s = (cudaStream_t)stream;
    m->last_stream = s;
    FEM_TRY(domain_image(m, f_dev, s, &f_dev));
    return tonal_cg(m, f_dev, g_dev, p, s, false);
}

// P^T W P from the pixel weights w (domain layout) into the pixel-mass
// matrix; the unweighted one is rebuilt by the next unweighted call.
static fem_status prepare_weighted(fem_mesh* m, const float* w, cudaStream_t s) {
    FEM_TRY(prepare_tonal(m, s));  // system and incidence
    FEM_TRY(raster_local(m, 4 /*R_WMASS*/, w, s));
    FEM_LAUNCH(F_TONAL, s, k_gather_mass, (m->V + 255) / 256, 256, 0, m->V, m->inc.p, m->tri.p, m->vxy.p, m->loc.p,
               m->Mdiag.p, m->Moff.p);
    m->tonal_version = -1;
    return FEM_OK;
}

extern "C" fem_status fem_tonal_opt_l1(fem_mesh* m, const float* f_dev, float* g_dev, int irls, double eps,
                                       const fem_params* p, void* stream) {
    Nvtx range("fem_tonal_opt_l1");
    if (!m || !f_dev || !g_dev || irls < 0 || !(eps > 0.0)) {
        set_error("fem_tonal_opt_l1: null argument, irls < 0 or eps <= 0");
        return FEM_E_INVALID;
    }
    fem_params dflt;
    fem_params_default(&dflt);
    if (!p) p = &dflt;
    cudaStream_t s = (cudaStream_t)stream;
    m->last_stream = s;
    FEM_TRY(domain_image(m, f_dev, s, &f_dev));
    FEM_TRY(build_system(m, s));
    FEM_TRY(ensure(m->wimg, (size_t)m->P, s));
    FEM_TRY(ensure(m->wfimg, (size_t)m->P, s));
    const bool fp64 = p->precision == FEM_PREC_FP64;
    int iters = 0;
    fem_status st = FEM_OK;
    for (int k = 0; k < irls; ++k) {
        Nvtx step_range("IRLS step");
        FEM_TRY(check_cancel(m));
        // the weights from u = B g: g at the mask, the Laplace solve
        FEM_TRY(set_uv_from_g(m, g_dev, s));
        FEM_TRY(solve_laplace(m, fp64, p->tol, p->maxit, s, nullptr, nullptr));
        FEM_TRY(raster_weights(m, m->uv.p, f_dev, (float)eps, m->wimg.p, m->wfimg.p, s));
        FEM_TRY(prepare_weighted(m, m->wimg.p, s));
        st = tonal_cg(m, m->wfimg.p, g_dev, p, s, true);
        iters += m->stats.tonal_iters;
        if (st != FEM_OK && st != FEM_E_NOT_CONVERGED) return st;
    }
    m->stats.tonal_iters = iters;
    return st;
}

extern "C" fem_status fem_adjoint(fem_mesh* m, const float* r_dev, float* gbar_dev, const fem_params* p, void* stream) {
    Nvtx range("fem_adjoint");
    if (!m || !r_dev || !gbar_dev) {
        set_error("fem_adjoint: null argument");
        return FEM_E_INVALID;
    }
    fem_params dflt;
    fem_params_default(&dflt);
    if (!p) p = &dflt;
    cudaStream_t s = (cudaStream_t)stream;
    m->last_stream = s;
    m->stats = fem_stats{};
    FEM_TRY(prepare_tonal(m, s));
    FEM_TRY(ensure_tonal_vectors(m, s));
    InnerCfg c{p->precision == FEM_PREC_FP64, p->inner_tol, p->maxit, false};
    FEM_TRY(domain_image(m, r_dev, s, &r_dev));
    FEM_TRY(scatter_PT(m, r_dev, s));
    FEM_TRY(apply_ET(m, m->ty.p, m->tw.p, c, s));
    FEM_LAUNCH(F_TONAL, s, k_d2f, (m->nK + 255) / 256, 256, 0, m->nK, m->tw.p, gbar_dev);
    FEM_CUDA(cudaStreamSynchronize(s));
    return FEM_OK;
}

// Tonal loss of Sec. 4 (eq. 4) and its gradient, the left side of the normal
// equations (eq. 5):  L(g) = 1/2 ||B g - f||^2,  dL/dg = B^T (B g - f).
// v = E g comes from one inpainting solve.  L is half the sum of the
// per-triangle squared errors of the error pass (float-float per pixel,
// FP64 per triangle).  The gradient never forms the pixel residual:
// P^T (P v - f) = M v - P^T f with the pixel-mass matrix M = P^T P, then
// E^T (one adjoint solve) maps it to the mask vertices.
extern "C" fem_status fem_tonal_loss(fem_mesh* m, const float* g_dev, const float* f_dev, double* loss_dev,
                                     float* grad_dev, const fem_params* p, void* stream) {
    Nvtx range("fem_tonal_loss");
    if (!m || !g_dev || !f_dev || (!loss_dev && !grad_dev)) {
        set_error("fem_tonal_loss: null argument (g, f and at least one of loss, grad are required)");
        return FEM_E_INVALID;
    }
    fem_params dflt;
    fem_params_default(&dflt);
    if (!p) p = &dflt;
    cudaStream_t s = (cudaStream_t)stream;
    m->last_stream = s;
    m->stats = fem_stats{};
    const bool fp64 = p->precision == FEM_PREC_FP64;
    FEM_TRY(domain_image(m, f_dev, s, &f_dev));
    // v = E g: g at the mask vertices, the Laplace solution at the unknown ones
    FEM_TRY(set_uv_from_g(m, g_dev, s));
    int it = 0;
    double rel = 0.0;
    FEM_TRY(solve_laplace(m, fp64, p->tol, p->maxit, s, &it, &rel));
    if (loss_dev) {
        FEM_TRY(ensure(m->lossk, (size_t)m->T, s));
        FEM_TRY(sq_image(m, f_dev, s));
        FEM_TRY(raster_errors(m, m->uv.p, nullptr, m->lossk.p, s));
        const int G = vec_grid(m);
        FEM_TRY(ensure(m->lossred, (size_t)G, s));
        FEM_LAUNCH(F_TONAL, s, k_sum_partial, G, kVecThreads, 0, (long long)m->T, (const double*)m->lossk.p,
                   m->lossred.p);
        FEM_LAUNCH(F_TONAL, s, k_final_sum_scaled, 1, kVecThreads, 0, G, (const double*)m->lossred.p, 0.5, loss_dev);
    }
    if (grad_dev) {
        FEM_TRY(prepare_tonal(m, s));
        FEM_TRY(ensure_tonal_vectors(m, s));
        FEM_TRY(scatter_PT(m, f_dev, s));  // ty = P^T f
        const int G = vec_grid(m);
        FEM_LAUNCH(F_TONAL, s, k_mass_spmv, G, kVecThreads, 0, m->V, (const double*)m->Mdiag.p,
                   (const double*)m->Moff.p, (const int*)m->nbr.p, (const double*)m->uv.p, m->tv.p, m->red.p);
        FEM_LAUNCH(F_TONAL, s, k_sub_from, (m->V + 255) / 256, 256, 0, m->V, (const double*)m->tv.p, m->ty.p);
        InnerCfg c{fp64, p->inner_tol, p->maxit, false};
        FEM_TRY(apply_ET(m, m->ty.p, m->tw.p, c, s));
        FEM_LAUNCH(F_TONAL, s, k_d2f, (m->nK + 255) / 256, 256, 0, m->nK, (const double*)m->tw.p, grad_dev);
    }
    int e = 0;
    FEM_CUDA(cudaMemcpyAsync(&e, m->dflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    if (e) {
        cudaMemsetAsync(m->dflag.p, 0, sizeof(int), s);
        m->plan_version = -1;
        set_error("fem_tonal_loss: rasterisation plan overflow");
        return (fem_status)e;
    }
    return FEM_OK;
}
