// solve_comp.cu -- the Laplace solve A_UU x = b (Sec. 2.2) block by block.
//
// With the unknowns numbered by connected component (components.cu), A_UU is
// block diagonal and every block is an independent SPD system.  One kernel
// solves all of them at once over every SM: components above one warp are
// taken by 256-thread blocks (rows in registers, the search directions and
// the float-float iterate in shared memory, one block barrier per
// reduction), components of at most 32 rows by single warps (one row per
// lane, neighbours through register shuffles, no barrier at all).  There is
// no grid-wide synchronisation.
//
// Per component the FP32_IR arithmetic is the mixed-precision refinement of
// the one-block solver: x and b in float-float scaled by a power of two, the
// residual b - A x in float-float, FP32 Jacobi-PCG on A d = r down to a
// relative 1e-5, x += d; the component stops when ||r_c|| <= tol ||b_c||, so
// that all components together meet ||r|| <= tol ||b||.  The FP64 variant is
// plain FP64 Jacobi-PCG per component with the residual recomputed from
// scratch before it stops (the FP64 comparison path).
//
// One-row components (the most common kind) are solved directly, x = b / a,
// one per thread.
//
// Statistics: per component the iterations, residual passes and
// ||r_c||^2 / ||b_c||^2, combined per block in shared memory and then across
// blocks by integer atomics (maxima and integer sums: independent of
// scheduling).  Iterations: the largest over the components, i.e. the length
// of the critical path; relative residual: the largest over the components,
// which bounds the relative residual of the whole system.
// The kernel does nothing when some component is above kBlockComp rows: the
// grid-wide solver then runs on the whole system instead.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "fem_internal.cuh"
#include "ff.cuh"

namespace fem {

constexpr int kCompThreads = 256;
constexpr int kCompRows = kBlockComp / kCompThreads;  // rows per thread in a block component
constexpr double kCompInnerEta = 1e-5;
constexpr int kCompInnerCap = 4000;

struct CompArgs {
    int nU;
    const int* rowcomp;    // component size at its first row, else 0
    const int* blk_list;   // first rows of the components above one warp
    const int* warp_list;  // first rows of the components of 2..32 rows
    const int* cnt;  // CC_* counters (read)
    int* work;       // the same counters (work distribution)
    const int* col;
    const float* val;
    const float* diag;
    const double* b;
    double* x;
    double tol;
    int maxit;
    unsigned long long* gstats;  // [0] it max [1] nres max [2] worst [3] relmax bits [4] rowit [5] rowres (zero between launches)
    // per-component results are stored at the component's first row
    double* out;  // [0] iterations (critical path), [1] relres, [2] status, [3] residual passes, [4] row-iterations, [5] row-residual passes
    double* acc;  // optional running totals (as solve_accumulate)
    double bytes_row_it, bytes_row_res;
    // optional: the solution also goes to the vertex values (uv, float-float
    // uvf) of the row's vertex scat_row[r]
    const int* scat_row;
    double* scat_uv;
    float2* scat_uvf;
    int* clear_word;  // optional: set to 0 at the start (the next solver's error word)
};

__device__ __forceinline__ void comp_store(const CompArgs& A, int row, double v) {
    A.x[row] = v;
    if (A.scat_uv) {
        const int vi = A.scat_row[row];
        A.scat_uv[vi] = v;
        const ff q = ff_from_double(v);
        A.scat_uvf[vi] = make_float2(q.hi, q.lo);
    }
}

// exact power-of-two scale that brings max |b| to [1, 2), kept in the normal range
__device__ __forceinline__ int comp_scale_exp(float bm) {
    int e = ilogbf(bm);
    return e < -120 ? -120 : (e > 120 ? 120 : e);
}

// Statistics of the components a block solved, combined in shared memory
// (each component's record takes a few shared atomics), then once per block
// into the global totals: the largest iteration count and residual-pass
// count, the worst status, the largest ||r_c||^2 / ||b_c||^2, and the row
// sums of iterations and residual passes (for the byte count).  All are
// maxima or integer sums, so the totals do not depend on scheduling.
struct CompStats {
    int itmax, nresmax, worst, pad;
    unsigned long long relmax;  // bits of a non-negative double: ordered like the values
    unsigned long long rowit, rowres;
};

__device__ __forceinline__ void comp_record(CompStats* S, int rows, int it, int nres, int status, double rr,
                                            double bb) {
    atomicMax(&S->itmax, it);
    atomicMax(&S->nresmax, nres);
    if (status != FEM_OK) atomicMax(&S->worst, status);
    double q = bb > 0.0 ? rr / bb : 0.0;
    atomicMax(&S->relmax, (unsigned long long)__double_as_longlong(q));
    atomicAdd(&S->rowit, (unsigned long long)rows * (unsigned long long)it);
    atomicAdd(&S->rowres, (unsigned long long)rows * (unsigned long long)nres);
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ----------------------------------------------------------- one warp
// Component of m <= 32 rows: lane i holds row i; columns are lane indices.
template <bool FP64>
__device__ void warp_comp(const CompArgs& A, int s0, int m, CompStats* S) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool act = lane < m;
    const int row = s0 + (act ? lane : 0);
    int lc[8];
    float v[8];
    float dg = 0.f, dinv = 0.f;
    double b = 0.0, x = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        lc[k] = lane;
        v[k] = 0.f;
    }
    if (act) {
        dg = A.diag[row];
        dinv = 1.0f / dg;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float w = A.val[(size_t)k * A.nU + row];
            if (w != 0.f) {
                lc[k] = A.col[(size_t)k * A.nU + row] - s0;
                v[k] = w;
            }
        }
        b = A.b[row];
        x = A.x[row];
    }
    float bm = warp_max(fabsf((float)b));
    if (bm == 0.f) {
        if (act) comp_store(A, row, 0.0);
        if (lane == 0) comp_record(S, m, 0, 0, FEM_OK, 0.0, 0.0);
        return;
    }
    int total_it = 0, nres = 0, status = FEM_E_NOT_CONVERGED;
    if constexpr (!FP64) {
        const int e = comp_scale_exp(bm);
        const double sc = ldexp(1.0, -e), inv = ldexp(1.0, e);
        ff xf = ff_from_double(x * sc), bf = ff_from_double(b * sc);
        const float tol2 = (float)(A.tol * A.tol);
        float rr = 0.f, bb = 0.f;
        for (int step = 0; step < 64; ++step) {
            // refinement residual in float-float
            ff s = ff_mul_f(xf, dg);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                float h = __shfl_sync(FULL, xf.hi, lc[k]), l = __shfl_sync(FULL, xf.lo, lc[k]);
                s = ff_add(s, ff_scale_pow2(ff{h, l}, v[k]));
            }
            ff res = ff_sub(bf, s);
            float r = act ? __fadd_rn(res.hi, res.lo) : 0.f;
            rr = warp_sum(r * r);
            bb = warp_sum(bf.hi * bf.hi);
            nres++;
            if (rr <= tol2 * bb) { status = FEM_OK; break; }
            if (total_it >= A.maxit) break;
            // FP32 Jacobi-PCG on A d = r from d = 0 in the single-reduction
            // form of Chronopoulos and Gear: s = A p is kept by recurrence, so
            // each iteration has one SpMV (w = A z) and one fused reduction of
            // (r.z, w.z, r.r): three independent butterflies instead of two
            // dependent rounds
            float d = 0.f, z = dinv * r;
            float w = dg * z;
#pragma unroll
            for (int k = 0; k < 8; ++k) w = fmaf(v[k], __shfl_sync(FULL, z, lc[k]), w);
            float gamma = warp_sum(r * z), delta = warp_sum(w * z), rr_in = rr;
            const float lim = (float)(kCompInnerEta * kCompInnerEta) * rr;
            const int cap = min(A.maxit - total_it, kCompInnerCap);
            int it = 0;
            float alpha = delta > 0.f ? gamma / delta : 0.f, p = z, sv = w;
            while (delta > 0.f && rr_in > lim && it < cap) {
                d = fmaf(alpha, p, d);
                r = fmaf(-alpha, sv, r);
                it++;
                z = dinv * r;
                w = dg * z;
#pragma unroll
                for (int k = 0; k < 8; ++k) w = fmaf(v[k], __shfl_sync(FULL, z, lc[k]), w);
                float gn = warp_sum(r * z), dn = warp_sum(w * z);
                rr_in = warp_sum(r * r);
                float beta = gn / gamma;
                float den = dn - beta * gn / alpha;
                if (!(den > 0.f)) break;  // breakdown guard (uniform over the warp)
                alpha = gn / den;
                gamma = gn;
                p = fmaf(beta, p, z);
                sv = fmaf(beta, sv, w);
            }
            total_it += it;
            xf = ff_add_f(xf, d);
            if (it == 0) break;  // breakdown: no progress possible
        }
        if (act) comp_store(A, row, ff_to_double(xf) * inv);
        if (lane == 0) comp_record(S, m, total_it, nres, status, (double)rr * inv * inv, (double)bb * inv * inv);
    } else {
        const double tol2 = A.tol * A.tol;
        double bb = warp_sum(b * b), rr = 0.0;
        double ddinv = act ? 1.0 / (double)dg : 0.0;
        for (int pass = 0; pass < 64; ++pass) {
            // residual from scratch
            double ax = (double)dg * x;
#pragma unroll
            for (int k = 0; k < 8; ++k) ax = fma((double)v[k], __shfl_sync(FULL, x, lc[k]), ax);
            double r = act ? b - ax : 0.0;
            rr = warp_sum(r * r);
            nres++;
            if (rr <= tol2 * bb) { status = FEM_OK; break; }
            if (total_it >= A.maxit) break;
            double z = ddinv * r, p = z;
            double rz = warp_sum(r * z);
            int it = 0;
            const int cap = A.maxit - total_it;
            while (it < cap) {
                double q = (double)dg * p;
#pragma unroll
                for (int k = 0; k < 8; ++k) q = fma((double)v[k], __shfl_sync(FULL, p, lc[k]), q);
                double pq = warp_sum(p * q);
                if (!(pq > 0.0)) break;
                double alpha = rz / pq;
                x = fma(alpha, p, x);
                r = fma(-alpha, q, r);
                z = ddinv * r;
                double rz2 = warp_sum(r * z);
                rr = warp_sum(r * r);
                it++;
                if (rr <= tol2 * bb) break;
                double beta = rz2 / rz;
                rz = rz2;
                p = fma(beta, p, z);
            }
            total_it += it;
            if (it == 0) break;
        }
        if (act) comp_store(A, row, x);
        if (lane == 0) comp_record(S, m, total_it, nres, status, rr, bb);
    }
}

// ---------------------------------------------------------- one block
// Component of 32 < m <= kBlockComp rows: thread t holds rows t + 256 k.
// Shared memory: the local ELL ((local column << 2) | code, code 1: -1/2,
// 2: -1, 0: padding), the diagonal, z, two buffers for p (the new search
// direction p = z + beta p_old is formed at the neighbours on the fly, so a
// CG iteration needs two barriers), and the iterate for the residual.
constexpr int kCompSmemBytes = 46 * 1024;

struct CtaRed {
    double2 slot[2][kCompThreads / 32];
};

// Sums of two values over the block with one barrier, the same bits in
// every thread (warp sums added in a fixed order).  The FP32 path keeps the
// sums in FP32: with every thread adding the eight warp sums, FP64 adds
// would cost thousands of FP64 operations per reduction on this part.
template <class T>
__device__ __forceinline__ void cta_sum2(CtaRed& R, int& par, T& a, T& b) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    if constexpr (sizeof(T) == 4) {
        float2* sl = (float2*)R.slot[par];
        if (lane == 0) sl[w] = make_float2(a, b);
        __syncthreads();
        float sa = 0.f, sb = 0.f;
#pragma unroll
        for (int i = 0; i < kCompThreads / 32; ++i) {
            float2 t = sl[i];
            sa += t.x;
            sb += t.y;
        }
        a = sa;
        b = sb;
    } else {
        if (lane == 0) R.slot[par][w] = make_double2(a, b);
        __syncthreads();
        double sa = 0.0, sb = 0.0;
#pragma unroll
        for (int i = 0; i < kCompThreads / 32; ++i) {
            double2 t = R.slot[par][i];
            sa += t.x;
            sb += t.y;
        }
        a = sa;
        b = sb;
    }
    par ^= 1;
}

// three FP32 sums with one barrier (the same bits in every thread)
__device__ __forceinline__ void cta_sum3f(CtaRed& R, int& par, float& a, float& b, float& c) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    float4* sl = (float4*)R.slot[par];
    if (lane == 0) sl[w] = make_float4(a, b, c, 0.f);
    __syncthreads();
    float sa = 0.f, sb = 0.f, sc = 0.f;
#pragma unroll
    for (int i = 0; i < kCompThreads / 32; ++i) {
        float4 t = sl[i];
        sa += t.x;
        sb += t.y;
        sc += t.z;
    }
    a = sa;
    b = sb;
    c = sc;
    par ^= 1;
}

__device__ __forceinline__ float cta_max(CtaRed& R, int& par, float a) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a = warp_max(a);
    float* sl = (float*)R.slot[par];
    if (lane == 0) sl[w] = a;
    __syncthreads();
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < kCompThreads / 32; ++i) mx = fmaxf(mx, sl[i]);
    par ^= 1;
    return mx;
}

__device__ __forceinline__ float code_val(unsigned short e) {
    unsigned c = e & 3u;
    return c == 1u ? -0.5f : (c == 2u ? -1.0f : 0.0f);
}

template <bool FP64>
__device__ void cta_comp(const CompArgs& A, int s0, int m, unsigned char* raw, CtaRed& R, CompStats* S) {
    using Real = typename std::conditional<FP64, double, float>::type;
    const int tid = threadIdx.x;
    // shared layout: ent[8][kBlockComp] u16 | dg[kBlockComp] f32 | z | p[2] | x (float2, FP32_IR only)
    unsigned short* ent = (unsigned short*)raw;
    float* dg_s = (float*)(raw + 16 * kBlockComp);
    Real* z_s = (Real*)(raw + 20 * kBlockComp);
    Real* p_s0 = z_s + kBlockComp;
    Real* p_s1 = p_s0 + kBlockComp;
    float2* x_s = (float2*)(p_s1 + kBlockComp);
    int par = 0;
    float bmt = 0.f;
    double bl[kCompRows];
#pragma unroll
    for (int k = 0; k < kCompRows; ++k) {
        int i = tid + k * kCompThreads;
        bl[k] = 0.0;
        if (i < m) {
            int row = s0 + i;
            dg_s[i] = A.diag[row];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                float w = A.val[(size_t)e * A.nU + row];
                int lcol = A.col[(size_t)e * A.nU + row] - s0;
                ent[e * kBlockComp + i] =
                    w == 0.f ? (unsigned short)(i << 2) : (unsigned short)((lcol << 2) | (w == -1.0f ? 2 : 1));
            }
            bl[k] = A.b[row];
            bmt = fmaxf(bmt, fabsf((float)bl[k]));
        }
    }
    float bm = cta_max(R, par, bmt);  // its barrier also publishes ent and dg_s
    if (bm == 0.f) {
        for (int i = tid; i < m; i += kCompThreads) comp_store(A, s0 + i, 0.0);
        if (tid == 0) comp_record(S, m, 0, 0, FEM_OK, 0.0, 0.0);
        return;
    }
    int total_it = 0, nres = 0, status = FEM_E_NOT_CONVERGED;
    Real r[kCompRows], d[kCompRows];
    if constexpr (!FP64) {
        const int e = comp_scale_exp(bm);
        const double sc = ldexp(1.0, -e), inv = ldexp(1.0, e);
        ff bf[kCompRows];
        float dinv[kCompRows];
#pragma unroll
        for (int k = 0; k < kCompRows; ++k) {
            int i = tid + k * kCompThreads;
            bf[k] = ff_from_double(bl[k] * sc);
            dinv[k] = 0.f;
            if (i < m) {
                dinv[k] = 1.0f / dg_s[i];
                ff xi = ff_from_double(A.x[s0 + i] * sc);
                x_s[i] = make_float2(xi.hi, xi.lo);
            }
        }
        __syncthreads();
        const float tol2 = (float)(A.tol * A.tol);
        float rr = 0.f, bb = 0.f;
        for (int step = 0; step < 64; ++step) {
            float rr_t = 0.f, bb_t = 0.f;
#pragma unroll
            for (int k = 0; k < kCompRows; ++k) {
                int i = tid + k * kCompThreads;
                r[k] = 0.f;
                if (i < m) {
                    float2 xv = x_s[i];
                    ff s = ff_mul_f(ff{xv.x, xv.y}, dg_s[i]);
#pragma unroll
                    for (int e2 = 0; e2 < 8; ++e2) {
                        unsigned short en = ent[e2 * kBlockComp + i];
                        float2 xc = x_s[en >> 2];
                        s = ff_add(s, ff_scale_pow2(ff{xc.x, xc.y}, code_val(en)));
                    }
                    ff res = ff_sub(bf[k], s);
                    r[k] = __fadd_rn(res.hi, res.lo);
                    rr_t += r[k] * r[k];
                    bb_t += bf[k].hi * bf[k].hi;
                }
            }
            cta_sum2(R, par, rr_t, bb_t);
            rr = rr_t;
            bb = bb_t;
            nres++;
            if (rr <= tol2 * bb) { status = FEM_OK; break; }
            if (total_it >= A.maxit) break;
            // FP32 Jacobi-PCG on A d = r from d = 0 in the single-reduction
            // form of Chronopoulos and Gear (see warp_comp): per iteration one
            // barrier publishes z for the SpMV w = A z, one fused reduction of
            // (r.z, w.z, r.r) follows; s = A p by recurrence
            float* zf = (float*)z_s;
            float zk[kCompRows], wk[kCompRows], pk[kCompRows], sk[kCompRows];
#pragma unroll
            for (int k = 0; k < kCompRows; ++k) {
                int i = tid + k * kCompThreads;
                d[k] = 0.f;
                zk[k] = 0.f;
                if (i < m) {
                    zk[k] = r[k] * dinv[k];
                    zf[i] = zk[k];
                }
            }
            __syncthreads();
            float g_t = 0.f, d_t = 0.f, r_t = 0.f;
#pragma unroll
            for (int k = 0; k < kCompRows; ++k) {
                int i = tid + k * kCompThreads;
                wk[k] = 0.f;
                if (i < m) {
                    float sacc = dg_s[i] * zk[k];
#pragma unroll
                    for (int e2 = 0; e2 < 8; ++e2) {
                        unsigned short en = ent[e2 * kBlockComp + i];
                        sacc = fmaf(code_val(en), zf[en >> 2], sacc);
                    }
                    wk[k] = sacc;
                    g_t += r[k] * zk[k];
                    d_t += sacc * zk[k];
                }
            }
            cta_sum3f(R, par, g_t, d_t, r_t);
            float gamma = g_t, delta = d_t, rr_in = rr;
            const float lim = (float)(kCompInnerEta * kCompInnerEta) * rr;
            const int cap = min(A.maxit - total_it, kCompInnerCap);
            int it = 0;
            float alpha = delta > 0.f ? gamma / delta : 0.f;
#pragma unroll
            for (int k = 0; k < kCompRows; ++k) {
                pk[k] = zk[k];
                sk[k] = wk[k];
            }
            while (delta > 0.f && rr_in > lim && it < cap) {
#pragma unroll
                for (int k = 0; k < kCompRows; ++k) {
                    int i = tid + k * kCompThreads;
                    if (i < m) {
                        d[k] = fmaf(alpha, pk[k], d[k]);
                        r[k] = fmaf(-alpha, sk[k], r[k]);
                        zk[k] = r[k] * dinv[k];
                        zf[i] = zk[k];  // the last reads of z_s were before the previous reduction's barrier
                    }
                }
                it++;
                __syncthreads();
                g_t = 0.f;
                d_t = 0.f;
                r_t = 0.f;
#pragma unroll
                for (int k = 0; k < kCompRows; ++k) {
                    int i = tid + k * kCompThreads;
                    wk[k] = 0.f;
                    if (i < m) {
                        float sacc = dg_s[i] * zk[k];
#pragma unroll
                        for (int e2 = 0; e2 < 8; ++e2) {
                            unsigned short en = ent[e2 * kBlockComp + i];
                            sacc = fmaf(code_val(en), zf[en >> 2], sacc);
                        }
                        wk[k] = sacc;
                        g_t += r[k] * zk[k];
                        d_t += sacc * zk[k];
                        r_t += r[k] * r[k];
                    }
                }
                cta_sum3f(R, par, g_t, d_t, r_t);
                rr_in = r_t;
                float beta = g_t / gamma;
                float den = d_t - beta * g_t / alpha;
                if (!(den > 0.f)) break;  // breakdown guard (uniform over the block)
                alpha = g_t / den;
                gamma = g_t;
#pragma unroll
                for (int k = 0; k < kCompRows; ++k) {
                    pk[k] = fmaf(beta, pk[k], zk[k]);
                    sk[k] = fmaf(beta, sk[k], wk[k]);
                }
            }
            total_it += it;
#pragma unroll
            for (int k = 0; k < kCompRows; ++k) {
                int i = tid + k * kCompThreads;
                if (i < m) {
                    float2 xv = x_s[i];
                    ff xi = ff_add_f(ff{xv.x, xv.y}, d[k]);
                    x_s[i] = make_float2(xi.hi, xi.lo);
                }
            }
            __syncthreads();
            if (it == 0) break;
        }
        for (int i = tid; i < m; i += kCompThreads) {
            float2 xv = x_s[i];
            comp_store(A, s0 + i, ff_to_double(ff{xv.x, xv.y}) * inv);
        }
        if (tid == 0) comp_record(S, m, total_it, nres, status, (double)rr * inv * inv, (double)bb * inv * inv);
    } else {
        // plain FP64 PCG; the iterate stays in A.x (global memory, read back
        // through the block after a barrier for the residual passes)
        const double tol2 = A.tol * A.tol;
        double xk[kCompRows];
        double bb_t = 0.0, dmy = 0.0;
#pragma unroll
        for (int k = 0; k < kCompRows; ++k) {
            int i = tid + k * kCompThreads;
            xk[k] = i < m ? A.x[s0 + i] : 0.0;
            bb_t += bl[k] * bl[k];
        }
        cta_sum2(R, par, bb_t, dmy);
        const double bb = bb_t;
        double rr = 0.0;
        double* zd = (double*)z_s;
        double *pold = (double*)p_s0, *pnew = (double*)p_s1;
        for (int pass = 0; pass < 64; ++pass) {
            double rr_t = 0.0, rz_t = 0.0;
#pragma unroll
            for (int k = 0; k < kCompRows; ++k) {
                int i = tid + k * kCompThreads;
                r[k] = 0.0;
                if (i < m) {
                    double ax = (double)dg_s[i] * xk[k];
#pragma unroll
                    for (int e2 = 0; e2 < 8; ++e2) {
                        unsigned short en = ent[e2 * kBlockComp + i];
                        ax = fma((double)code_val(en), __ldcg(A.x + s0 + (en >> 2)), ax);
                    }
                    r[k] = bl[k] - ax;
                    double zi = r[k] / (double)dg_s[i];
                    zd[i] = zi;
                    pold[i] = 0.0;
                    rr_t += r[k] * r[k];
                    rz_t += r[k] * zi;
                }
            }
            cta_sum2(R, par, rr_t, rz_t);
            rr = rr_t;
            nres++;
            if (rr <= tol2 * bb) { status = FEM_OK; break; }
            if (total_it >= A.maxit) break;
            double rz = rz_t, beta = 0.0;
            int it = 0;
            const int cap = A.maxit - total_it;
            bool conv = false;
            while (it < cap) {
                double pq_t = 0.0, pk[kCompRows], qk[kCompRows];
#pragma unroll
                for (int k = 0; k < kCompRows; ++k) {
                    int i = tid + k * kCompThreads;
                    pk[k] = 0.0;
                    qk[k] = 0.0;
                    if (i < m) {
                        double pi = fma(beta, pold[i], zd[i]);
                        double sacc = (double)dg_s[i] * pi;
#pragma unroll
                        for (int e2 = 0; e2 < 8; ++e2) {
                            unsigned short en = ent[e2 * kBlockComp + i];
                            int j = en >> 2;
                            sacc = fma((double)code_val(en), fma(beta, pold[j], zd[j]), sacc);
                        }
                        pk[k] = pi;
                        qk[k] = sacc;
                        pq_t += pi * sacc;
                    }
                }
                double dmy2 = 0.0;
                cta_sum2(R, par, pq_t, dmy2);
                if (!(pq_t > 0.0)) break;
                double alpha = rz / pq_t;
                double rz_t2 = 0.0, rr_t2 = 0.0;
#pragma unroll
                for (int k = 0; k < kCompRows; ++k) {
                    int i = tid + k * kCompThreads;
                    if (i < m) {
                        pnew[i] = pk[k];
                        xk[k] = fma(alpha, pk[k], xk[k]);
                        r[k] = fma(-alpha, qk[k], r[k]);
                        double zi = r[k] / (double)dg_s[i];
                        zd[i] = zi;
                        rz_t2 += r[k] * zi;
                        rr_t2 += r[k] * r[k];
                    }
                }
                cta_sum2(R, par, rz_t2, rr_t2);
                it++;
                beta = rz_t2 / rz;
                rz = rz_t2;
                double* t = pold;
                pold = pnew;
                pnew = t;
                if (rr_t2 <= tol2 * bb) { conv = true; break; }
            }
            total_it += it;
#pragma unroll
            for (int k = 0; k < kCompRows; ++k) {
                int i = tid + k * kCompThreads;
                if (i < m) A.x[s0 + i] = xk[k];
            }
            __syncthreads();
            if (it == 0 && !conv) break;
        }
        if (A.scat_uv)  // the last pass stored x (read back after its barrier)
            for (int i = tid; i < m; i += kCompThreads) comp_store(A, s0 + i, A.x[s0 + i]);
        if (tid == 0) comp_record(S, m, total_it, nres, status, rr, bb);
    }
    __syncthreads();
}

// ------------------------------------------------------------- kernel
template <bool FP64>
__global__ void __launch_bounds__(kCompThreads) k_solve_comp(CompArgs A) {
    pdl_wait();
    __shared__ __align__(16) unsigned char raw[kCompSmemBytes];
    __shared__ CtaRed R;
    __shared__ int s_item, s_last;
    if (A.clear_word && blockIdx.x == 0 && threadIdx.x == 0) *A.clear_word = 0;
    if (A.cnt[CC_ERR] != 0) {  // the system build failed: report its code, solve nothing
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const int code = A.cnt[CC_ERR];
            A.out[0] = 0; A.out[1] = 0; A.out[2] = code; A.out[3] = 0; A.out[4] = 0; A.out[5] = 0;
            if (A.acc && A.acc[2] == 0.0) A.acc[2] = code;
        }
        return;
    }
    if (A.cnt[CC_NBIG] > 0) return;  // the grid-wide solver takes the system
    __shared__ CompStats S;
    if (threadIdx.x == 0) S = CompStats{0, 0, FEM_OK, 0, 0ull, 0ull, 0ull};
    __syncthreads();
    const int nblk = A.cnt[CC_NBLK], nwarp = A.cnt[CC_NWARP];
    // components above one warp: one block each, taken in turn
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(A.work + CC_WORK, 1);
        __syncthreads();
        int i = s_item;
        __syncthreads();
        if (i >= nblk) break;
        int s0 = A.blk_list[i];
        cta_comp<FP64>(A, s0, A.rowcomp[s0], raw, R, &S);
    }
    // components of 2..32 rows: one warp each
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = gw; i < nwarp; i += nw) {
        int s0 = A.warp_list[i];
        warp_comp<FP64>(A, s0, A.rowcomp[s0], &S);
    }
    // one-row components: x = b / a directly, one thread each
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < A.nU; p += gridDim.x * blockDim.x) {
        if (A.rowcomp[p] != 1) continue;
        double a = (double)A.diag[p], b = A.b[p];
        double x = b / a;
        double r = b - a * x;
        comp_store(A, p, x);
        comp_record(&S, 1, 0, 1, FEM_OK, r * r, b * b);
    }
    // block totals into the global totals; the last block to finish writes
    // the solve's statistics and clears the totals for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long* G = A.gstats;
        atomicMax(G + 0, (unsigned long long)S.itmax);
        atomicMax(G + 1, (unsigned long long)S.nresmax);
        atomicMax(G + 2, (unsigned long long)S.worst);
        atomicMax(G + 3, S.relmax);
        atomicAdd(G + 4, S.rowit);
        atomicAdd(G + 5, S.rowres);
        __threadfence();
        s_last = atomicAdd(A.work + CC_DONE, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    unsigned long long* G = A.gstats;
    int mit = (int)__ldcg(G + 0), mres = (int)__ldcg(G + 1), wst = (int)__ldcg(G + 2);
    double rel = sqrt(__longlong_as_double((long long)__ldcg(G + 3)));
    double tit = (double)__ldcg(G + 4), tres = (double)__ldcg(G + 5);
#pragma unroll
    for (int q = 0; q < 6; ++q) G[q] = 0ull;
    // work counters back to zero for the next launch (every block is done)
    A.work[CC_WORK] = 0;
    A.work[CC_DONE] = 0;
    A.out[0] = mit;
    A.out[1] = rel;  // largest ||r_c|| / ||b_c|| over the components (bounds the global one)
    A.out[2] = wst;
    A.out[3] = mres;
    A.out[4] = tit;
    A.out[5] = tres;
    if (A.acc) {
        A.acc[0] += mit;
        if (rel > A.acc[1]) A.acc[1] = rel;
        if (wst != FEM_OK && A.acc[2] == 0.0) A.acc[2] = wst;
        A.acc[3] += 1.0;
        A.acc[4] += A.bytes_row_it * tit + A.bytes_row_res * tres;
    }
}

// Launch the component solve (results in x, statistics in dscal / its totals).
fem_status solve_components(fem_mesh* m, const double* b, double* x, bool use_fp64, double tol, int maxit,
                            bool deferred, bool scatter, int* clear_word, cudaStream_t s) {
    int nU = m->nU;
    if (!m->comp_stats.p) {  // zero once; each launch's last block clears it again
        FEM_TRY(ensure(m->comp_stats, 8, s));
        FEM_CUDA(cudaMemsetAsync(m->comp_stats.p, 0, sizeof(unsigned long long) * m->comp_stats.n, s));
    }
    CompArgs A;
    A.nU = nU;
    A.rowcomp = m->rowcomp.p;
    A.blk_list = m->blk_list.p;
    A.warp_list = m->warp_list.p;
    A.cnt = m->ccount.p;
    A.work = m->ccount.p;
    A.col = m->ucol.p;
    A.val = m->uval32.p;
    A.diag = m->udiag.p;
    A.b = b;
    A.x = x;
    A.tol = tol;
    A.maxit = maxit;
    A.gstats = m->comp_stats.p;
    A.out = m->dscal.p;
    A.acc = deferred ? m->dscal.p + 64 : nullptr;
    // algorithmic bytes per row: as the grid-wide solver (ELL matrix 68 B per
    // SpMV; FP32 iteration 120 B, FP64 iteration 168 B; residual pass 92 B,
    // plus 36 B of conversions per FP32 refinement step)
    A.bytes_row_it = use_fp64 ? 168.0 : 120.0;
    A.bytes_row_res = use_fp64 ? 92.0 : 128.0;
    A.scat_row = scatter ? m->urow_vertex.p : nullptr;
    A.scat_uv = scatter ? m->uv.p : nullptr;
    A.scat_uvf = scatter ? m->uvf.p : nullptr;
    A.clear_word = clear_word;
    // CC_WORK / CC_DONE are zero here: cleared by the system build, and
    // again by the last block of every launch
    // about one component of 2..32 rows per warp (at most half the rows),
    // at most a few blocks per SM
    int grid = std::max(1, std::min(m->num_sms * 4, (nU / 2 + 7) / 8));
    if (use_fp64)
        FEM_LAUNCH(F_CG, s, k_solve_comp<true>, grid, kCompThreads, 0, A);
    else
        FEM_LAUNCH(F_CG, s, k_solve_comp<false>, grid, kCompThreads, 0, A);
    return FEM_OK;
}

}  // namespace fem
