// raster.cu -- pixel ownership, linear interpolation and per-triangle
// reductions on the pixel grid (Sec. 2.2 interpolation, Sec. 3 error map).
//
// Ownership: pixel (x, y) belongs to the triangle whose interior contains
// (x, y) + eps*(sx, delta*sy), 0 < delta << 1, eps -> 0+, sx = sy = +1 except
// -1 on the last column / row.  For a lattice triangle with edges of slope
// 0, +-1 or infinity this is: rows [ytop, ybot) (plus ybot on the last image
// row), and in row y the columns [L(y), R(y)) (plus R on the last image
// column when L < R), where [L, R] is the triangle's intersection with the row.
//
// Work decomposition: a triangle is cut into items of rpi consecutive rows
// (rpi = clamp(1024 / bbox width, 1, 32)), so an item holds about a thousand
// pixels at most.  One warp takes one item: lane i holds the span of the
// item's row i, a warp scan turns the spans into offsets, and the warp walks
// the item's pixels 32 at a time, each lane finding its row by a binary
// search over the lanes.  Consecutive lanes read consecutive pixels of a row.
// Per-item partial sums are added per triangle in item order, so results do
// not depend on scheduling.
#include <algorithm>
#include <climits>

#include "fem_internal.cuh"
#include "ff.cuh"
#include "raster_common.cuh"
#include "scan.cuh"

namespace fem {

// R_WMASS: the mass entries with a pixel weight (P^T W P of a weighted least
// squares step); R_WGT: the weights of an IRLS step of the L1 data term,
// w = 1 / max(|u - f|, eps), and w f, written per image pixel in domain
// layout (u in float-float, as in the error mode)
enum RasterMode { R_ERR = 0, R_IMG = 1, R_MASS = 2, R_SCAT = 3, R_WMASS = 4, R_WGT = 5 };
// Pixels per item (about 1024): fewer items mean less fixed cost per pixel.
// 256-pixel items at 1025^2, meant to shorten the longest item, measured
// slower (the fixed cost of four times as many items), so every size uses
// 1024; the plan and the kernels take the size as a parameter.
__host__ __device__ __forceinline__ int item_pixels_for(long long P) {
    (void)P;
    return 1024;
}
constexpr int kRasterThreads = 256;

// raster plan as one fused scan: the item count of triangle t is the input,
// the output records its first item and writes its item list
struct ItemCountIn {
    const int4* tri;
    const int2* vxy;
    int N;
    int item_px;
    int* cnt;
    __device__ __forceinline__ int operator()(long long lt) const {
        int t = (int)lt;
        TriGeom g = tri_geom(tri[t], vxy, N);
        int rows = g.yend - g.ytop + 1;
        int rpi = rows_per_item(g.maxw, item_px);
        int c = (rows > 0 && !is_small(g)) ? (rows + rpi - 1) / rpi : 0;
        cnt[t] = c;
        return c;
    }
};

struct ItemExpandOut {
    int* off;
    int* item_tri;
    int cap;
    int* err;
    __device__ __forceinline__ void operator()(long long lt, int o, int n) const {
        int t = (int)lt;
        off[t] = o;
        if (o + n > cap) {
            atomicCAS(err, 0, (int)FEM_E_INVALID);
            return;
        }
        for (int j = 0; j < n; ++j) item_tri[o + j] = t;
    }
};

// separate kernels of the plan (used by the allocation-free error pass)
__global__ void k_item_count(const int4* __restrict__ tri, const int2* __restrict__ vxy, int T, int N,
                             int* __restrict__ cnt, int item_px) {
    pdl_wait();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    TriGeom g = tri_geom(tri[t], vxy, N);
    int rows = g.yend - g.ytop + 1;
    int rpi = rows_per_item(g.maxw, item_px);
    cnt[t] = (rows > 0 && !is_small(g)) ? (rows + rpi - 1) / rpi : 0;
}

__global__ void k_item_expand(const int* __restrict__ cnt, const int* __restrict__ off, int T, int cap,
                              int* __restrict__ item_tri, int* __restrict__ err) {
    pdl_wait();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    int o = off[t], n = cnt[t];
    if (o + n > cap) {
        atomicCAS(err, 0, (int)FEM_E_INVALID);
        return;
    }
    for (int j = 0; j < n; ++j) item_tri[o + j] = t;
}

template <int MODE>
struct NAcc {
    static constexpr int n = MODE == R_ERR ? 1 : ((MODE == R_MASS || MODE == R_WMASS) ? 6 : (MODE == R_SCAT ? 3 : 0));
};

// Sum of a triangle's item partials (float-float) by one warp in a fixed
// order: lane j adds items j, j + 32, ...; then a butterfly.  All lanes
// return the same value.
__device__ __forceinline__ ff warp_sum_partials(const float2* partial, int o, int n) {
    ff s{0.f, 0.f};
    for (int j = (int)(threadIdx.x & 31); j < n; j += 32) {
        float2 v = __ldcg(&partial[o + j]);
        s = ff_add(s, ff{v.x, v.y});
    }
    return ff_warp_sum(s);
}

// Error and image modes evaluate the linear interpolant as a plane in
// float-float, u(x, y) = u_c + g_x (x - c_x) + g_y (y - c_y), with g the
// gradient ((a-c)(u_a-u_c) + (b-c)(u_b-u_c)) / |a-c|^2 (legs orthogonal and
// of equal length), and accumulate (u - f)^2 in float-float: about 48-bit
// precision on the FP32 pipes.  The mass and scatter modes (run once per
// tonal optimisation) use FP64 barycentric weights.
template <int MODE>
__global__ void __launch_bounds__(kRasterThreads) k_raster(
    const int4* __restrict__ tri, const int2* __restrict__ vxy, const double* __restrict__ uv,
    const float2* __restrict__ uvf, const float* __restrict__ img, Dom D, const int* __restrict__ item_tri,
    const int* __restrict__ item_off, const int* __restrict__ n_items_dev, int item_cap, int item_px,
    double* __restrict__ partial, float* __restrict__ u_out, int* __restrict__ owner_out,
    const int* __restrict__ plan_err, float* __restrict__ wf_out, float eps) {
    pdl_wait();
    // An overflowing plan left item slots unwritten (they may hold another
    // mesh's triangle ids): read none of them.  Every thread reads the same
    // word, so the whole grid returns or none of it does.
    if (plan_err && *plan_err) return;
    constexpr int NA = NAcc<MODE>::n;
    constexpr bool FF = (MODE == R_ERR || MODE == R_IMG || MODE == R_WGT);
    const unsigned FULL = 0xffffffffu;
    int lane = threadIdx.x & 31;
    long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    int n_items = min(*n_items_dev, item_cap);  // never past the capacity
    for (long long it = warp; it < n_items; it += nwarps) {
        int t = item_tri[it];
        int j = (int)(it - item_off[t]);
        int4 tr = tri[t];
        TriGeom g = tri_geom(tr, vxy, D.N);
        int rpi = rows_per_item(g.maxw, item_px);
        int r0 = g.ytop + j * rpi;
        int nr = min(rpi, g.yend + 1 - r0);
        int L = 0, len = 0;
        if (lane < nr) row_span(g, r0 + lane, D, L, len);

        int dax = g.ax - g.cx, day = g.ay - g.cy, dbx = g.bx - g.cx, dby = g.by - g.cy;
        long long l2 = (long long)dax * dax + (long long)day * day;
        bool pow2 = (l2 & (l2 - 1)) == 0;
        // plane of the interpolant (float-float), error accumulator
        ff uc{0.f, 0.f}, gx{0.f, 0.f}, gy{0.f, 0.f}, acc_ff{0.f, 0.f};
        double inv_l2 = 0.0;
        if (FF) {
            ff va = vertex_ff(uv, uvf, tr.x), vb = vertex_ff(uv, uvf, tr.y);
            uc = vertex_ff(uv, uvf, tr.z);
            ff da = ff_sub(va, uc), db = ff_sub(vb, uc);
            gx = ff_add(ff_mul_f(da, (float)dax), ff_mul_f(db, (float)dbx));
            gy = ff_add(ff_mul_f(da, (float)day), ff_mul_f(db, (float)dby));
            if (pow2) {
                // exact reciprocal of a power of two
                float inv = __int_as_float((127 - (63 - __clzll(l2))) << 23);
                gx = ff_scale_pow2(gx, inv);
                gy = ff_scale_pow2(gy, inv);
            } else {
                float inv = 1.0f / (float)l2;
                gx = ff_mul_f(gx, inv);
                gy = ff_mul_f(gy, inv);
            }
        } else {
            inv_l2 = pow2 ? __longlong_as_double((long long)(1023 - (63 - __clzll(l2))) << 52) : 1.0 / (double)l2;
        }
        double acc[NA > 0 ? NA : 1];
#pragma unroll
        for (int q = 0; q < (NA > 0 ? NA : 1); ++q) acc[q] = 0.0;

        // The item's rows are cut into chunks of 32 pixels (chunk c of row r
        // covers its pixels 32c .. 32c+31); lane r holds the first chunk of row
        // r.  A warp step takes one chunk: a ballot over the lanes' chunk
        // offsets gives its row, and lane l takes pixel 32c + l.  kPre chunks
        // are located and their image values loaded before any arithmetic.
        int ccnt = (len + 31) >> 5, cinc = ccnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL, cinc, o);
            if (lane >= o) cinc += y;
        }
        const int coff = cinc - ccnt;
        const int nchunks = __shfl_sync(FULL, cinc, 31);
        constexpr int kPre = 4;
        constexpr bool READS = (MODE == R_ERR || MODE == R_SCAT || MODE == R_WMASS || MODE == R_WGT);
        for (int q0 = 0; q0 < nchunks; q0 += kPre) {
            int px[kPre], py[kPre];
            float fv[kPre];
#pragma unroll
            for (int u = 0; u < kPre; ++u) {
                const int q = q0 + u;
                const unsigned bq = __ballot_sync(FULL, lane < nr && coff <= q);
                const int r = bq ? 31 - __clz(bq) : 0;
                const int Lr = __shfl_sync(FULL, L, r), lr = __shfl_sync(FULL, len, r),
                          cr = __shfl_sync(FULL, coff, r);
                const int c = ((q - cr) << 5) + lane;
                const bool ok = q < nchunks && c < lr;
                px[u] = ok ? Lr + c : -1;
                py[u] = r0 + r;
                fv[u] = (READS && ok) ? img[(long long)py[u] * D.N + px[u]] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kPre; ++u) {
            if (px[u] >= 0) {
                int x = px[u], y = py[u];
                long long p = (long long)y * D.W + x;  // outputs are W x H
                if (FF) {
                    float dx = (float)(x - g.cx), dy = (float)(y - g.cy);
                    ff u_ = ff_add(ff_add(uc, ff_mul_f(gx, dx)), ff_mul_f(gy, dy));
                    if (MODE == R_ERR) {
                        ff d = ff_add_f(u_, -fv[u]);
                        acc_ff = ff_add(acc_ff, ff_sqr(d));
                    } else if (MODE == R_WGT) {
                        const ff d = ff_add_f(u_, -fv[u]);
                        const float w = 1.0f / fmaxf(fabsf(__fadd_rn(d.hi, d.lo)), eps);
                        const long long pd = (long long)y * D.N + x;  // domain layout
                        u_out[pd] = w;
                        wf_out[pd] = w * fv[u];
                    } else {
                        if (u_out) u_out[p] = __fadd_rn(u_.hi, u_.lo);
                        if (owner_out) owner_out[p] = t;
                    }
                } else {
                    long long dxp = x - g.cx, dyp = y - g.cy;
                    double la = (double)(dxp * dax + dyp * day) * inv_l2;
                    double lb = (double)(dxp * dbx + dyp * dby) * inv_l2;
                    double lc = 1.0 - la - lb;
                    if (MODE == R_MASS || MODE == R_WMASS) {
                        const double wt = MODE == R_WMASS ? (double)fv[u] : 1.0;
                        const double wa = wt * la, wb = wt * lb, wc = wt * lc;
                        acc[0] = fma(wa, la, acc[0]);
                        acc[1] = fma(wb, lb, acc[1]);
                        acc[2] = fma(wc, lc, acc[2]);
                        acc[3] = fma(wa, lb, acc[3]);
                        acc[4] = fma(wb, lc, acc[4]);
                        acc[5] = fma(wc, la, acc[5]);
                    } else if (MODE == R_SCAT) {
                        double r = (double)fv[u];
                        acc[0] = fma(la, r, acc[0]);
                        acc[1] = fma(lb, r, acc[1]);
                        acc[2] = fma(lc, r, acc[2]);
                    }
                }
            }
            }
        }
        if (MODE == R_ERR) {
            ff tot = ff_warp_sum(acc_ff);
            if (lane == 0) ((float2*)partial)[it] = make_float2(tot.hi, tot.lo);
        } else if (NA > 0) {
#pragma unroll
            for (int q = 0; q < (NA > 0 ? NA : 1); ++q) {
                double v = warp_sum(acc[q]);
                if (lane == 0) partial[it * NA + q] = v;
            }
        }
    }
}

// per-triangle error from float-float item partials, one warp per
// triangle (the summation of the fused path in k_raster); keyc (optional):
// composite selection key, eligible triangles (refinement-edge midpoint on
// the pixel grid) get the FP64 key bits with the top bit set, the others 0,
// so that unsigned order = selection order
__global__ void k_finalize_err(const int* __restrict__ cnt, const int* __restrict__ off,
                               const float2* __restrict__ partial, int T, const int4* __restrict__ tri,
                               const int2* __restrict__ vxy, double* __restrict__ out,
                               unsigned long long* __restrict__ keyc, int item_cap, const int* __restrict__ plan_err,
                               Dom D) {
    pdl_wait();
    if (plan_err && *plan_err) return;  // the plan overflowed: no partial is valid
    long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long tt = gw; tt < T; tt += nw) {
        int t = (int)tt;
        int o = off[t], n = cnt[t];
        if (n == 0) continue;  // small triangle: written by the small-triangle kernel
        if ((long long)o + n > item_cap) continue;  // never past the partials' capacity
        ff s = warp_sum_partials(partial, o, n);
        if ((threadIdx.x & 31) == 0) {
            double key = ff_to_double(s);
            out[t] = key;
            if (keyc) {
                int4 tr = tri[t];
                int2 a = vxy[tr.x], b = vxy[tr.y], c = vxy[tr.z];
                bool eligible = dom_eligible(a.x, a.y, b.x, b.y, c.x, c.y, D);
                keyc[t] = eligible ? ((unsigned long long)__double_as_longlong(key) | (1ull << 63)) : 0ull;
            }
        }
    }
}

template <int NA>
__global__ void k_finalize(const int* __restrict__ cnt, const int* __restrict__ off, const double* __restrict__ partial,
                           int T, double* __restrict__ out) {
    pdl_wait();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    int o = off[t], n = cnt[t];
    if (n == 0) return;  // small triangle: written by k_raster_small
    double s[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) s[q] = 0.0;
    for (int j = 0; j < n; ++j)
#pragma unroll
        for (int q = 0; q < NA; ++q) s[q] += partial[(long long)(o + j) * NA + q];
#pragma unroll
    for (int q = 0; q < NA; ++q) out[(long long)t * NA + q] = s[q];
}

// One small triangle per thread, threads in curve order (order == nullptr:
// id order), so that neighbouring threads read neighbouring pixels.  Rows are
// walked left to right; in the error and image modes the float-float
// interpolant advances by the exact gradient g_x per pixel.
template <int MODE>
__global__ void __launch_bounds__(256) k_raster_small(const int* __restrict__ order, const int4* __restrict__ tri,
                                                      const int2* __restrict__ vxy, const double* __restrict__ uv,
                                                      const float2* __restrict__ uvf, const float* __restrict__ img,
                                                      Dom D, int T, double* __restrict__ out,
                                                      unsigned long long* __restrict__ keyc,
                                                      float* __restrict__ u_out, int* __restrict__ owner_out,
                                                      const int* __restrict__ n_dev, float* __restrict__ wf_out,
                                                      float eps) {
    pdl_wait();
    // n_dev: the order list has *n_dev entries (a device-side count, at most T)
    const int Tn = n_dev ? min(*n_dev, T) : T;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Tn; i += gridDim.x * blockDim.x) {
        int t = order ? order[i] : i;
        int4 tr = tri[t];
        TriGeom g = tri_geom(tr, vxy, D.N);
        if (!is_small(g)) continue;
        int dax = g.ax - g.cx, day = g.ay - g.cy, dbx = g.bx - g.cx, dby = g.by - g.cy;
        long long l2 = (long long)dax * dax + (long long)day * day;
        bool pow2 = (l2 & (l2 - 1)) == 0;
        if (MODE == R_ERR || MODE == R_IMG || MODE == R_WGT) {
            ff va = vertex_ff(uv, uvf, tr.x), vb = vertex_ff(uv, uvf, tr.y), uc = vertex_ff(uv, uvf, tr.z);
            ff da = ff_sub(va, uc), db = ff_sub(vb, uc);
            ff gx = ff_add(ff_mul_f(da, (float)dax), ff_mul_f(db, (float)dbx));
            ff gy = ff_add(ff_mul_f(da, (float)day), ff_mul_f(db, (float)dby));
            if (pow2) {
                float inv = __int_as_float((127 - (63 - __clzll(l2))) << 23);
                gx = ff_scale_pow2(gx, inv);
                gy = ff_scale_pow2(gy, inv);
            } else {
                float inv = 1.0f / (float)l2;
                gx = ff_mul_f(gx, inv);
                gy = ff_mul_f(gy, inv);
            }
            ff acc{0.f, 0.f};
            for (int y = g.ytop; y <= g.yend; ++y) {
                int L, len;
                row_span(g, y, D, L, len);
                if (len <= 0) continue;
                ff u = ff_add(ff_add(uc, ff_mul_f(gx, (float)(L - g.cx))), ff_mul_f(gy, (float)(y - g.cy)));
                const long long p0 = (long long)y * D.N + L;  // the domain image
                const long long q0 = (long long)y * D.W + L;  // the W x H outputs
#pragma unroll 4
                for (int k = 0; k < len; ++k) {
                    if (MODE == R_ERR) {
                        ff d = ff_add_f(u, -img[p0 + k]);
                        acc = ff_add(acc, ff_sqr(d));
                    } else if (MODE == R_WGT) {
                        const float fv = img[p0 + k];
                        const ff d = ff_add_f(u, -fv);
                        const float w = 1.0f / fmaxf(fabsf(__fadd_rn(d.hi, d.lo)), eps);
                        u_out[p0 + k] = w;  // domain layout
                        wf_out[p0 + k] = w * fv;
                    } else {
                        if (u_out) u_out[q0 + k] = __fadd_rn(u.hi, u.lo);
                        if (owner_out) owner_out[q0 + k] = t;
                    }
                    u = ff_add(u, gx);
                }
            }
            if (MODE == R_ERR) {
                double key = ff_to_double(acc);
                out[t] = key;
                if (keyc) {
                    bool eligible = tri_eligible(g, D);
                    keyc[t] = eligible ? ((unsigned long long)__double_as_longlong(key) | (1ull << 63)) : 0ull;
                }
            }
        } else {
            double inv_l2 = pow2 ? __longlong_as_double((long long)(1023 - (63 - __clzll(l2))) << 52) : 1.0 / (double)l2;
            double acc[6] = {0, 0, 0, 0, 0, 0};
            for (int y = g.ytop; y <= g.yend; ++y) {
                int L, len;
                row_span(g, y, D, L, len);
                for (int k = 0; k < len; ++k) {
                    int x = L + k;
                    long long dxp = x - g.cx, dyp = y - g.cy;
                    double la = (double)(dxp * dax + dyp * day) * inv_l2;
                    double lb = (double)(dxp * dbx + dyp * dby) * inv_l2;
                    double lc = 1.0 - la - lb;
                    if (MODE == R_MASS || MODE == R_WMASS) {
                        const double wt = MODE == R_WMASS ? (double)img[(long long)y * D.N + x] : 1.0;
                        const double wa = wt * la, wb = wt * lb, wc = wt * lc;
                        acc[0] = fma(wa, la, acc[0]);
                        acc[1] = fma(wb, lb, acc[1]);
                        acc[2] = fma(wc, lc, acc[2]);
                        acc[3] = fma(wa, lb, acc[3]);
                        acc[4] = fma(wb, lc, acc[4]);
                        acc[5] = fma(wc, la, acc[5]);
                    } else {
                        double r = (double)img[(long long)y * D.N + x];
                        acc[0] = fma(la, r, acc[0]);
                        acc[1] = fma(lb, r, acc[1]);
                        acc[2] = fma(lc, r, acc[2]);
                    }
                }
            }
            constexpr int NA = (MODE == R_MASS || MODE == R_WMASS) ? 6 : 3;
#pragma unroll
            for (int q = 0; q < NA; ++q) out[(long long)t * NA + q] = acc[q];
        }
    }
}

static int small_grid(fem_mesh* m) { return std::max(1, std::min((m->T + 255) / 256, m->num_sms * 8)); }

static int raster_grid(fem_mesh* m) { return m->num_sms * (2048 / kRasterThreads); }

fem_status raster_plan(fem_mesh* m, cudaStream_t s) {
    if (m->plan_version == m->mesh_version) return FEM_OK;
    int T = m->T;
    size_t cap = (size_t)3 * T + (size_t)(m->P / 128) + 1024;
    FEM_TRY(ensure(m->item_cnt, T + 1, s));
    FEM_TRY(ensure(m->item_off, T + 1, s));
    FEM_TRY(ensure(m->item_tri, cap, s));
    FEM_TRY(ensure(m->partial, cap * 6, s));
    int* n_items_dev = m->dcount.p + 0;
    // overflow flag: sticky until a host check reads it (and clears it)
    int* err = m->dflag.p + 0;
    FEM_TRY(scan_fused(m, ItemCountIn{m->tri.p, m->vxy.p, m->N, item_pixels_for(m->P), m->item_cnt.p},
                       ItemExpandOut{m->item_off.p, m->item_tri.p, (int)m->item_tri.n, err}, T, s, n_items_dev,
                       F_RASTER));
    m->plan_version = m->mesh_version;
    return FEM_OK;
}

// Exact keys of every triangle by the square-tiled pass (raster_sq.cu);
// the image must have been laid out in squares (sq_image) for this call.
fem_status raster_errors(fem_mesh* m, const double* uv, const float2* uvf, double* err_out, cudaStream_t s,
                         unsigned long long* keyc_out) {
    return sq_keys_exact(m, uv, uvf, err_out, keyc_out, nullptr, nullptr, nullptr, 0, s);
}

fem_status raster_image(fem_mesh* m, const double* uv, float* u, int* owner, cudaStream_t s) {
    FEM_TRY(raster_plan(m, s));
    note_bytes(F_RASTER, (u ? 4.0 * (double)m->P : 0.0) + (owner ? 4.0 * (double)m->P : 0.0) + 16.0 * m->T +
                             16.0 * m->V);
    FEM_LAUNCH(F_RASTER, s, k_raster<R_IMG>, raster_grid(m), kRasterThreads, 0, m->tri.p, m->vxy.p, uv,
               (const float2*)nullptr, (const float*)nullptr, dom_of(m), m->item_tri.p, m->item_off.p, m->dcount.p + 0, (int)m->item_tri.n, item_pixels_for(m->P), m->partial.p, u, owner,
               (const int*)(m->dflag.p + 0), (float*)nullptr, 0.0f);
    FEM_LAUNCH(F_RASTER, s, k_raster_small<R_IMG>, small_grid(m), 256, 0, m->order.p, m->tri.p, m->vxy.p, uv,
               (const float2*)nullptr, (const float*)nullptr, dom_of(m), m->T, (double*)nullptr,
               (unsigned long long*)nullptr, u, owner, nullptr, (float*)nullptr, 0.0f);
    return FEM_OK;
}

// mode R_MASS: loc[6t..6t+5] = sums of la^2, lb^2, lc^2, la lb, lb lc, lc la
// mode R_SCAT: loc[3t..3t+2] = sums of la r, lb r, lc r
fem_status raster_local(fem_mesh* m, int mode, const float* r, cudaStream_t s) {
    FEM_TRY(raster_plan(m, s));
    FEM_TRY(ensure(m->loc, (size_t)6 * m->T + 6, s));
    int blocks = (m->T + 255) / 256;
    note_bytes(F_RASTER, (mode == R_MASS ? 64.0 * m->T : 4.0 * (double)m->P + 40.0 * m->T) + 8.0 * m->V);
    if (mode == R_MASS) {
        FEM_LAUNCH(F_RASTER, s, k_raster<R_MASS>, raster_grid(m), kRasterThreads, 0, m->tri.p, m->vxy.p,
                   (const double*)nullptr, (const float2*)nullptr, (const float*)nullptr, dom_of(m), m->item_tri.p, m->item_off.p, m->dcount.p + 0,
                   (int)m->item_tri.n, item_pixels_for(m->P), m->partial.p, (float*)nullptr, (int*)nullptr,
                   (const int*)(m->dflag.p + 0), (float*)nullptr, 0.0f);
        FEM_LAUNCH(F_RASTER, s, k_finalize<6>, blocks, 256, 0, m->item_cnt.p, m->item_off.p, m->partial.p, m->T,
                   m->loc.p);
        FEM_LAUNCH(F_RASTER, s, k_raster_small<R_MASS>, small_grid(m), 256, 0, m->order.p, m->tri.p, m->vxy.p,
                   (const double*)nullptr, (const float2*)nullptr, (const float*)nullptr, dom_of(m), m->T, m->loc.p,
                   (unsigned long long*)nullptr, (float*)nullptr, (int*)nullptr, nullptr, (float*)nullptr, 0.0f);
    } else if (mode == R_WMASS) {
        // r: the pixel weights (domain layout)
        FEM_LAUNCH(F_RASTER, s, k_raster<R_WMASS>, raster_grid(m), kRasterThreads, 0, m->tri.p, m->vxy.p,
                   (const double*)nullptr, (const float2*)nullptr, r, dom_of(m), m->item_tri.p, m->item_off.p,
                   m->dcount.p + 0, (int)m->item_tri.n, item_pixels_for(m->P), m->partial.p, (float*)nullptr,
                   (int*)nullptr, (const int*)(m->dflag.p + 0), (float*)nullptr, 0.0f);
        FEM_LAUNCH(F_RASTER, s, k_finalize<6>, blocks, 256, 0, m->item_cnt.p, m->item_off.p, m->partial.p, m->T,
                   m->loc.p);
        FEM_LAUNCH(F_RASTER, s, k_raster_small<R_WMASS>, small_grid(m), 256, 0, m->order.p, m->tri.p, m->vxy.p,
                   (const double*)nullptr, (const float2*)nullptr, r, dom_of(m), m->T, m->loc.p,
                   (unsigned long long*)nullptr, (float*)nullptr, (int*)nullptr, nullptr, (float*)nullptr, 0.0f);
    } else {
        FEM_LAUNCH(F_RASTER, s, k_raster<R_SCAT>, raster_grid(m), kRasterThreads, 0, m->tri.p, m->vxy.p,
                   (const double*)nullptr, (const float2*)nullptr, r, dom_of(m), m->item_tri.p, m->item_off.p, m->dcount.p + 0, (int)m->item_tri.n, item_pixels_for(m->P),
                   m->partial.p, (float*)nullptr, (int*)nullptr,
                   (const int*)(m->dflag.p + 0), (float*)nullptr, 0.0f);
        FEM_LAUNCH(F_RASTER, s, k_finalize<3>, blocks, 256, 0, m->item_cnt.p, m->item_off.p, m->partial.p, m->T,
                   m->loc.p);
        FEM_LAUNCH(F_RASTER, s, k_raster_small<R_SCAT>, small_grid(m), 256, 0, m->order.p, m->tri.p, m->vxy.p,
                   (const double*)nullptr, (const float2*)nullptr, r, dom_of(m), m->T, m->loc.p,
                   (unsigned long long*)nullptr, (float*)nullptr, (int*)nullptr, nullptr, (float*)nullptr, 0.0f);
    }
    return FEM_OK;
}

// The weights of an IRLS step of the L1 data term from the vertex values uv
// and the domain image f: w = 1 / max(|u - f|, eps) and w f at every image
// pixel, in domain layout (w_dom, wf_dom: N^2 floats; other pixels are not
// written and never read).
fem_status raster_weights(fem_mesh* m, const double* uv, const float* f, float eps, float* w_dom, float* wf_dom,
                          cudaStream_t s) {
    FEM_TRY(raster_plan(m, s));
    note_bytes(F_RASTER, 12.0 * (double)m->PI + 16.0 * m->T + 8.0 * m->V);
    FEM_LAUNCH(F_RASTER, s, k_raster<R_WGT>, raster_grid(m), kRasterThreads, 0, m->tri.p, m->vxy.p, uv,
               (const float2*)nullptr, f, dom_of(m), m->item_tri.p, m->item_off.p, m->dcount.p + 0,
               (int)m->item_tri.n, item_pixels_for(m->P), m->partial.p, w_dom, (int*)nullptr,
               (const int*)(m->dflag.p + 0), wf_dom, eps);
    FEM_LAUNCH(F_RASTER, s, k_raster_small<R_WGT>, small_grid(m), 256, 0, m->order.p, m->tri.p, m->vxy.p, uv,
               (const float2*)nullptr, f, dom_of(m), m->T, (double*)nullptr, (unsigned long long*)nullptr, w_dom,
               (int*)nullptr, nullptr, wf_dom, eps);
    return FEM_OK;
}

// Error pass on caller-described mesh arrays with caller-provided scratch
// (no allocation).  Same kernels as raster_errors.
fem_status raster_errors_scratch(const int4* tri, const int2* vxy, int T, int N, const double* uv, const float* f,
                                 double* err_out, cudaStream_t s, const RasterScratch& w) {
    int* n_items_dev = w.counters + 0;
    int* err = w.counters + 1;
    int blocks = (T + 255) / 256;
    FEM_LAUNCH(F_RASTER, s, k_item_count, blocks, 256, 0, tri, vxy, T, N, w.item_cnt, item_pixels_for((long long)N * N));
    FEM_TRY(exclusive_scan_i32_scratch(w.item_cnt, w.item_off, T, s, n_items_dev, w.scan_tmp, w.scan_tmp_n));
    FEM_LAUNCH(F_RASTER, s, k_item_expand, blocks, 256, 0, w.item_cnt, w.item_off, T, w.item_cap, w.item_tri, err);
    const Dom D{N, N, N};  // the allocation-free pass takes square images only
    FEM_LAUNCH(F_RASTER, s, k_raster<R_ERR>, w.grid, kRasterThreads, 0, tri, vxy, uv, (const float2*)nullptr, f, D,
               w.item_tri, w.item_off, n_items_dev, w.item_cap, item_pixels_for((long long)N * N), w.partial, (float*)nullptr,
               (int*)nullptr, (const int*)err, (float*)nullptr, 0.0f);
    FEM_LAUNCH(F_RASTER, s, k_finalize_err, std::max(1, std::min(w.grid, (T + 7) / 8)), 256, 0, w.item_cnt,
               w.item_off, (const float2*)w.partial, T, tri, vxy, err_out, (unsigned long long*)nullptr, w.item_cap,
               (const int*)err, D);
    FEM_LAUNCH(F_RASTER, s, k_raster_small<R_ERR>, std::max(1, std::min(blocks, w.grid / 2)), 256, 0, (const int*)nullptr,
               tri, vxy, uv, (const float2*)nullptr, f, D, T, err_out, (unsigned long long*)nullptr, (float*)nullptr,
               (int*)nullptr, nullptr, (float*)nullptr, 0.0f);
    return FEM_OK;
}

}  // namespace fem

using namespace fem;

extern "C" {

fem_status fem_triangle_errors(fem_mesh* m, const double* uv_dev, const float* f_dev, double* err_dev, void* stream) {
    if (!m || !uv_dev || !f_dev || !err_dev) {
        set_error("fem_triangle_errors: null argument");
        return FEM_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    m->last_stream = s;
    const float* fd = nullptr;
    FEM_TRY(domain_image(m, f_dev, s, &fd));
    FEM_TRY(sq_image(m, fd, s));
    FEM_TRY(raster_errors(m, uv_dev, nullptr, err_dev, s));
    int e = 0;
    FEM_CUDA(cudaMemcpyAsync(&e, m->dflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    if (e) {
        cudaMemsetAsync(m->dflag.p, 0, sizeof(int), s);
        m->plan_version = -1;
        set_error("fem_triangle_errors: a square holds more large triangles than the pass can list (is it a valid mesh?)");
        return (fem_status)e;
    }
    return FEM_OK;
}

fem_status fem_rasterize(fem_mesh* m, const double* uv_dev, float* u_dev, int* owner_dev, void* stream) {
    if (!m || !uv_dev) {
        set_error("fem_rasterize: null argument");
        return FEM_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    m->last_stream = s;
    FEM_TRY(raster_image(m, uv_dev, u_dev, owner_dev, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    return FEM_OK;
}

}  // extern "C"

namespace fem {

// ===================================================================== fast keys
// FP32 keys with a rigorous error bound, for the selection of the spatial
// optimisation on large images.
//
// Per triangle the FP32 pass returns S (the sum of FP32 squares) and an
// interval [lo, hi] that contains the float-float key K of the exact pass:
//  * u is evaluated in FP32 from the FP32-rounded plane (u_c, g_x, g_y) with
//    at most three roundings, so |u - u*| <= delta = 5 u M with u = 2^-24 and
//    M = |u_c| + |g_x| W_x + |g_y| W_y (W = the largest |x - c_x|, |y - c_y|
//    over the vertices, which bounds it over the triangle);
//  * d = fl(u - f) adds at most u |d|;
//  * each partial sum is a chain of at most H FP32 additions of non-negative
//    terms: |S - sum d^2| <= gamma_H sum d^2, gamma_H = H u / (1 - H u);
//  * |sum d^2 - sum (u* - f)^2| <= 2 delta sqrt(n D) + 2.0001 u D + 2 n delta^2,
//    D = S / (1 - gamma_H) >= sum d^2 (Cauchy-Schwarz on sum |d|);
//  * K itself is within 2^-40 of the real sum (float-float keys).
// The bound is widened by 1 %.  A histogram of the float bit patterns of lo
// (rounded down) and hi (rounded up) brackets the k-th largest key between
// two bin edges; triangles whose interval overlaps the bracket (the band)
// get their exact float-float key, the others keep lo (surely selected:
// lo above the upper edge) or hi (surely not: hi below the lower edge).
// Selecting the k largest of these keys with ties by id gives the same set
// as selecting on the exact keys: a surely selected key exceeds the k-th
// exact key, a surely rejected one is below it, and the band is exact.
// The bracket: k = max(1, ceil(frac T)) capped by the eligible count (the
// histogram total) and V* - V; the bin of the k-th largest lo gives the
// lower edge, the bin of the k-th largest hi the upper edge.  One block:
// lane l of warp w holds the 32 bins starting kFastBins - 1 - 32 (32 w + l)
// downwards; a warp scan and a scan over the 32 warp totals give every
// lane the count above its bins, and the lane whose bins reach k walks them.
constexpr int kBracketThreads = 1024;
constexpr int kBinsPerThread = kFastBins / kBracketThreads;

__global__ void __launch_bounds__(kBracketThreads) k_fast_bracket(const unsigned* __restrict__ hlo,
                                                                   const unsigned* __restrict__ hhi, int T,
                                                                   double frac, long long vcap, int* __restrict__ kdev,
                                                                   double* __restrict__ tau) {
    pdl_wait();
    __shared__ int s_wl[kBracketThreads / 32], s_wh[kBracketThreads / 32];
    __shared__ int s_blo, s_bhi;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int top = kFastBins - 1 - tid * kBinsPerThread;
    int ml = 0, mh = 0;
    {
        // the thread's 32 bins are contiguous: top - 31 .. top
        const uint4* vl = (const uint4*)(hlo + top - (kBinsPerThread - 1));
        const uint4* vh = (const uint4*)(hhi + top - (kBinsPerThread - 1));
#pragma unroll
        for (int q = 0; q < kBinsPerThread / 4; ++q) {
            uint4 a = vl[q], b = vh[q];
            ml += (int)(a.x + a.y + a.z + a.w);
            mh += (int)(b.x + b.y + b.z + b.w);
        }
    }
    int il = ml, ih = mh;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int a = __shfl_up_sync(0xffffffffu, il, o), c = __shfl_up_sync(0xffffffffu, ih, o);
        if (lane >= o) { il += a; ih += c; }
    }
    if (lane == 31) { s_wl[w] = il; s_wh[w] = ih; }
    if (tid == 0) { s_blo = 0; s_bhi = 0; }
    __syncthreads();
    int bl = 0, bh = 0, tot = 0;
#pragma unroll
    for (int q = 0; q < kBracketThreads / 32; ++q) {
        int vl = s_wl[q], vh = s_wh[q];
        bl += q < w ? vl : 0;
        bh += q < w ? vh : 0;
        tot += vl;
    }
    const int exl = bl + il - ml, exh = bh + ih - mh;
    long long k = (long long)ceil(frac * (double)T);
    if (k < 1) k = 1;
    if (k > tot) k = tot;
    if (k > vcap) k = vcap;
    if (k < 0) k = 0;
    if (k > 0 && exl < k && exl + ml >= k) {
        long long cum = exl;
        for (int q = 0; q < kBinsPerThread; ++q) {
            cum += hlo[top - q];
            if (cum >= k) { s_blo = top - q; break; }
        }
    }
    if (k > 0 && exh < k && exh + mh >= k) {
        long long cum = exh;
        for (int q = 0; q < kBinsPerThread; ++q) {
            cum += hhi[top - q];
            if (cum >= k) { s_bhi = top - q; break; }
        }
    }
    __syncthreads();
    if (tid == 0) {
        *kdev = (int)k;
        tau[0] = (double)__uint_as_float((unsigned)s_blo << 16);
        tau[1] = (double)__uint_as_float((unsigned)(s_bhi + 1) << 16);
    }
}

// Classify every triangle against the bracket: surely selected (key := lo),
// surely not (key := hi; the largest such composite is kept for the margin),
// or band (listed, sel[t] = 1, and the square of a band triangle below the
// square level marked for the exact pass; bands of larger triangles are
// found from the node tables).
__global__ void k_fast_classify(const int4* __restrict__ tri, const int2* __restrict__ vxy, int T, SqGeo G,
                                const float* __restrict__ lo, const float* __restrict__ hi,
                                const double* __restrict__ tau, double* __restrict__ keys,
                                unsigned long long* __restrict__ keyc, int* __restrict__ band,
                                unsigned char* __restrict__ sel, unsigned char* __restrict__ sq_mark,
                                const int* __restrict__ pos, int* __restrict__ band_coarse, int* __restrict__ cnt,
                                unsigned long long* __restrict__ max_out) {
    pdl_wait();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int cls = 0;  // 0 ineligible / outside, 1 in, 2 out, 3 band
    unsigned long long comp_out = 0ull;
    if (t < T) {
        const int4 tr = tri[t];
        TriGeom g = tri_geom(tr, vxy, G.N);
        const double l = (double)lo[t], h = (double)hi[t];
        if (!tri_eligible(g, sq_dom(G))) {
            keys[t] = l;
            keyc[t] = 0ull;
        } else if (l > tau[1]) {
            cls = 1;
            keys[t] = l;
            keyc[t] = (unsigned long long)__double_as_longlong(l) | (1ull << 63);
        } else if (h < tau[0]) {
            cls = 2;
            comp_out = (unsigned long long)__double_as_longlong(h) | (1ull << 63);
            keys[t] = h;
            keyc[t] = comp_out;
        } else {
            cls = 3;
            const int2 a = make_int2(g.ax, g.ay), b = make_int2(g.bx, g.by), c = make_int2(g.cx, g.cy);
            if (leg2(a, c) <= (long long)G.s * G.s)
                sq_mark[sq_node_at((long long)a.x + b.x + c.x, (long long)a.y + b.y + c.y, G) >> 1] = 1;
            else
                band_coarse[atomicAdd(cnt + FC_BAND_COARSE, 1)] = pos[t];  // its exact key needs its node sums
        }
        sel[t] = cls == 3 ? 1 : 0;
    }
    // warp-combined counters
    unsigned in_mask = __ballot_sync(FULL, cls == 1);
    if (lane == 0 && in_mask) atomicAdd(cnt + 0, __popc(in_mask));
    unsigned long long mo = comp_out;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(FULL, mo, o);
        mo = v > mo ? v : mo;
    }
    if (lane == 0 && mo) atomicMax(max_out, mo);
    unsigned band_mask = __ballot_sync(FULL, cls == 3);
    int base = 0;
    if (lane == 0 && band_mask) base = atomicAdd(cnt + 1, __popc(band_mask));
    base = __shfl_sync(FULL, base, 0);
    if (cls == 3) band[base + __popc(band_mask & ((1u << lane) - 1u))] = t;
}

// Keys of the spatial optimisation by the fast path: on return keys[] and
// keyc[] hold, for every triangle, the exact key (band) or the substituted
// bound (outside the band), kdev the total k, and the band list with its
// counts for the selection (refine_round).  The image must have been laid
// out in squares (sq_image) for this call.  incremental: the mesh is the
// previous call's refined by one round on the same image (the FP32 pass
// then recomputes only what the round can have changed).
fem_status raster_keys_fast(fem_mesh* m, const double* uv, const float2* uvf, double frac, long long vcap,
                            cudaStream_t s, bool incremental) {
    FEM_TRY(sq_plan(m, s));
    const int T = m->T;
    const SqGeo G = sq_geo(m);
    const size_t keep = incremental && m->inc_ok ? (size_t)m->inc_T : 0;
    FEM_TRY(ensure(m->keys_lo, (size_t)T, s, keep));
    FEM_TRY(ensure(m->keys_hi, (size_t)T, s, keep));
    FEM_TRY(ensure(m->band, (size_t)T, s));
    FEM_TRY(ensure(m->bsel, (size_t)T, s));
    if (!m->sq_mark.p || m->sq_mark.n < (size_t)G.Q * G.Q) {
        FEM_TRY(ensure(m->sq_mark, (size_t)G.Q * G.Q, s));
        FEM_CUDA(cudaMemsetAsync(m->sq_mark.p, 0, m->sq_mark.n, s));  // cleared by each round's band list after
    }
    FEM_TRY(ensure(m->fast_hist, (size_t)2 * kFastBins + 8, s));
    unsigned* hist = m->fast_hist.p;
    int* cnt = (int*)(hist + 2 * kFastBins);  // [0] in, [1] band, [2] band squares, [3] coarse band triangles
    FEM_TRY(ensure(m->sq_bcoarse, (size_t)T, s));
    unsigned long long* max_out = (unsigned long long*)(m->dscal.p + 18);
    double* tau = m->dscal.p + 16;
    int* kdev = m->dcount.p + 2;
    // the histograms are cleared (full pass) or kept up to date by the pass
    FEM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned) * 8, s));
    FEM_CUDA(cudaMemsetAsync(max_out, 0, sizeof(unsigned long long), s));
    // all pixels in FP32 with error intervals
    FEM_TRY(sq_keys_fast(m, uv, uvf, FastOut{m->keys_lo.p, m->keys_hi.p, hist, hist + kFastBins}, s, incremental));
    // bracket and classification
    FEM_LAUNCH(F_TOPK, s, k_fast_bracket, 1, kBracketThreads, 0, hist, hist + kFastBins, T, frac, vcap, kdev, tau);
    FEM_LAUNCH(F_TOPK, s, k_fast_classify, (T + 255) / 256, 256, 0, m->tri.p, m->vxy.p, T, G, m->keys_lo.p,
               m->keys_hi.p, tau, m->keys.p, m->keyc.p, m->band.p, m->bsel.p, m->sq_mark.p, (const int*)m->sq_pos.p,
               m->sq_bcoarse.p, cnt, max_out);
    // exact float-float keys of the band, over the squares that hold it
    return sq_band_exact(m, uv, uvf, cnt + 2, s);
}

// the FP32 intervals as the FP64 arrays of the public call (exact)
__global__ void k_bounds_out(int T, const float* __restrict__ lo, const float* __restrict__ hi, double* __restrict__ lo_out,
                             double* __restrict__ hi_out) {
    pdl_wait();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T) {
        lo_out[t] = (double)lo[t];
        hi_out[t] = (double)hi[t];
    }
}

}  // namespace fem

using namespace fem;

extern "C" fem_status fem_triangle_error_bounds(fem_mesh* m, const double* uv_dev, const float* f_dev, double* lo_dev,
                                                double* hi_dev, void* stream) {
    if (!m || !uv_dev || !f_dev || !lo_dev || !hi_dev) {
        set_error("fem_triangle_error_bounds: null argument");
        return FEM_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    m->last_stream = s;
    const float* fd = nullptr;
    FEM_TRY(domain_image(m, f_dev, s, &fd));
    FEM_TRY(sq_image(m, fd, s));
    FEM_TRY(ensure(m->fast_hist, (size_t)2 * kFastBins + 8, s));
    FEM_TRY(ensure(m->keys_lo, (size_t)m->T, s));
    FEM_TRY(ensure(m->keys_hi, (size_t)m->T, s));
    FEM_CUDA(cudaMemsetAsync(m->fast_hist.p, 0, sizeof(unsigned) * (2 * kFastBins + 8), s));
    FEM_TRY(sq_keys_fast(m, uv_dev, nullptr, FastOut{m->keys_lo.p, m->keys_hi.p, m->fast_hist.p,
                                                     m->fast_hist.p + kFastBins}, s));
    FEM_LAUNCH(F_RASTER, s, k_bounds_out, (m->T + 255) / 256, 256, 0, m->T, (const float*)m->keys_lo.p,
               (const float*)m->keys_hi.p, lo_dev, hi_dev);
    int e = 0;
    FEM_CUDA(cudaMemcpyAsync(&e, m->dflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    if (e) {
        cudaMemsetAsync(m->dflag.p, 0, sizeof(int), s);
        m->plan_version = -1;
        set_error("fem_triangle_error_bounds: a square holds more large triangles than the pass can list (is it a valid mesh?)");
        return (fem_status)e;
    }
    return FEM_OK;
}
