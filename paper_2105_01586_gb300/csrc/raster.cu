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
#include "scan.cuh"

namespace fem {

enum RasterMode { R_ERR = 0, R_IMG = 1, R_MASS = 2, R_SCAT = 3 };
// Pixels per item (about 1024): fewer items mean less fixed cost per pixel.
// 256-pixel items at 1025^2, meant to shorten the longest item, measured
// slower (the fixed cost of four times as many items), so every size uses
// 1024; the plan and the kernels take the size as a parameter.
__host__ __device__ __forceinline__ int item_pixels_for(long long P) {
    (void)P;
    return 1024;
}
constexpr int kRasterThreads = 256;

struct TriGeom {
    int ax, ay, bx, by, cx, cy;
    int ytop, yend;  // owned rows ytop..yend (inclusive)
    int maxw;        // bounding-box width in pixels
};

__device__ __forceinline__ TriGeom tri_geom(int4 tr, const int2* __restrict__ vxy, int N) {
    TriGeom g;
    int2 a = vxy[tr.x], b = vxy[tr.y], c = vxy[tr.z];
    g.ax = a.x; g.ay = a.y; g.bx = b.x; g.by = b.y; g.cx = c.x; g.cy = c.y;
    int ytop = min(a.y, min(b.y, c.y)), ybot = max(a.y, max(b.y, c.y));
    g.ytop = ytop;
    g.yend = (ybot == N - 1) ? ybot : ybot - 1;
    g.maxw = max(a.x, max(b.x, c.x)) - min(a.x, min(b.x, c.x)) + 1;
    return g;
}

__device__ __forceinline__ int rows_per_item(int maxw, int item_px) {
    int r = item_px / maxw;
    return r < 1 ? 1 : (r > 32 ? 32 : r);
}

__device__ __forceinline__ void edge_x(int px, int py, int qx, int qy, int y, int& L, int& R) {
    if (py == qy) return;
    int lo = min(py, qy), hi = max(py, qy);
    if (y < lo || y > hi) return;
    int s = (qx == px) ? 0 : (((qx > px) == (qy > py)) ? 1 : -1);
    int x = px + (y - py) * s;
    L = min(L, x);
    R = max(R, x);
}

// owned columns of row y: [L, L + len)
__device__ __forceinline__ void row_span(const TriGeom& g, int y, int N, int& L, int& len) {
    int l = INT_MAX, r = INT_MIN;
    edge_x(g.ax, g.ay, g.bx, g.by, y, l, r);
    edge_x(g.bx, g.by, g.cx, g.cy, y, l, r);
    edge_x(g.cx, g.cy, g.ax, g.ay, y, l, r);
    int n = r - l + ((r == N - 1 && l < r) ? 1 : 0);
    L = l;
    len = n > 0 ? n : 0;
}

// Small triangles (bounding box at most kSmallSide pixels each way, at most
// 153 pixels) are rasterised one per thread along the space-filling curve
// (k_raster_small); only the larger ones are cut into warp items.
constexpr int kSmallSide = 17;

__device__ __forceinline__ bool is_small(const TriGeom& g) {
    return g.maxw <= kSmallSide && (g.yend - g.ytop + 1) <= kSmallSide;
}

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
    static constexpr int n = MODE == R_ERR ? 1 : (MODE == R_MASS ? 6 : (MODE == R_SCAT ? 3 : 0));
};

// vertex value as float-float: from the float-float copy when there is one,
// else split from FP64
__device__ __forceinline__ ff vertex_ff(const double* __restrict__ uv, const float2* __restrict__ uvf, int i) {
    if (uvf) {
        float2 v = uvf[i];
        return ff{v.x, v.y};
    }
    return ff_from_double(uv[i]);
}

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
    const float2* __restrict__ uvf, const float* __restrict__ img, int N, const int* __restrict__ item_tri,
    const int* __restrict__ item_off, const int* __restrict__ n_items_dev, int item_cap, int item_px,
    double* __restrict__ partial, float* __restrict__ u_out, int* __restrict__ owner_out,
    const int* __restrict__ item_cnt = nullptr, int* __restrict__ item_done = nullptr,
    double* __restrict__ key_out = nullptr, unsigned long long* __restrict__ keyc_out = nullptr,
    const int* __restrict__ item_list = nullptr, const int* __restrict__ plan_err = nullptr) {
    pdl_wait();
    // An overflowing plan left item slots unwritten (they may hold another
    // mesh's triangle ids): read none of them.  Every thread reads the same
    // word, so the whole grid returns or none of it does.
    if (plan_err && *plan_err) return;
    constexpr int NA = NAcc<MODE>::n;
    constexpr bool FF = (MODE == R_ERR || MODE == R_IMG);
    const unsigned FULL = 0xffffffffu;
    int lane = threadIdx.x & 31;
    long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    int n_items = min(*n_items_dev, item_cap);  // never past the capacity
    for (long long ii = warp; ii < n_items; ii += nwarps) {
        // item_list: a subset of the plan's items (the band of the fast keys)
        long long it = item_list ? item_list[ii] : ii;
        int t = item_tri[it];
        int j = (int)(it - item_off[t]);
        int4 tr = tri[t];
        TriGeom g = tri_geom(tr, vxy, N);
        int rpi = rows_per_item(g.maxw, item_px);
        int r0 = g.ytop + j * rpi;
        int nr = min(rpi, g.yend + 1 - r0);
        int L = 0, len = 0;
        if (lane < nr) row_span(g, r0 + lane, N, L, len);

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
        constexpr bool READS = (MODE == R_ERR || MODE == R_SCAT);
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
                fv[u] = (READS && ok) ? img[(long long)py[u] * N + px[u]] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kPre; ++u) {
            if (px[u] >= 0) {
                int x = px[u], y = py[u];
                long long p = (long long)y * N + x;
                if (FF) {
                    float dx = (float)(x - g.cx), dy = (float)(y - g.cy);
                    ff u_ = ff_add(ff_add(uc, ff_mul_f(gx, dx)), ff_mul_f(gy, dy));
                    if (MODE == R_ERR) {
                        ff d = ff_add_f(u_, -fv[u]);
                        acc_ff = ff_add(acc_ff, ff_sqr(d));
                    } else {
                        if (u_out) u_out[p] = __fadd_rn(u_.hi, u_.lo);
                        if (owner_out) owner_out[p] = t;
                    }
                } else {
                    long long dxp = x - g.cx, dyp = y - g.cy;
                    double la = (double)(dxp * dax + dyp * day) * inv_l2;
                    double lb = (double)(dxp * dbx + dyp * dby) * inv_l2;
                    double lc = 1.0 - la - lb;
                    if (MODE == R_MASS) {
                        acc[0] = fma(la, la, acc[0]);
                        acc[1] = fma(lb, lb, acc[1]);
                        acc[2] = fma(lc, lc, acc[2]);
                        acc[3] = fma(la, lb, acc[3]);
                        acc[4] = fma(lb, lc, acc[4]);
                        acc[5] = fma(lc, la, acc[5]);
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
            if (!item_done) {
                if (lane == 0) ((float2*)partial)[it] = make_float2(tot.hi, tot.lo);
            } else {
                // fused finalisation: the warp that completes a triangle's
                // items sums its partials and writes the key
                const int nit = item_cnt[t];
                int last = 0;
                if (nit > 1 && lane == 0) {
                    ((float2*)partial)[it] = make_float2(tot.hi, tot.lo);
                    __threadfence();
                    last = atomicAdd(item_done + t, 1) == nit - 1;
                }
                last = nit == 1 ? 1 : __shfl_sync(FULL, last, 0);
                if (last) {
                    ff sum = tot;  // one item: its own sum (what the warp sum of one partial gives)
                    if (nit > 1) {
                        __threadfence();
                        sum = warp_sum_partials((const float2*)partial, item_off[t], nit);
                    }
                    if (lane == 0) {
                        double key = ff_to_double(sum);
                        key_out[t] = key;
                        if (keyc_out) {
                            bool eligible = (((g.ax + g.bx) | (g.ay + g.by)) & 1) == 0;
                            keyc_out[t] = eligible ? ((unsigned long long)__double_as_longlong(key) | (1ull << 63)) : 0ull;
                        }
                        if (nit > 1) item_done[t] = 0;  // ready for the next pass
                    }
                }
            }
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
                               unsigned long long* __restrict__ keyc, int item_cap, const int* __restrict__ plan_err) {
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
                int2 a = vxy[tr.x], b = vxy[tr.y];
                bool eligible = (((a.x + b.x) | (a.y + b.y)) & 1) == 0;
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
                                                      int N, int T, double* __restrict__ out,
                                                      unsigned long long* __restrict__ keyc,
                                                      float* __restrict__ u_out, int* __restrict__ owner_out,
                                                      const int* __restrict__ n_dev = nullptr) {
    pdl_wait();
    // n_dev: the order list has *n_dev entries (a device-side count, at most T)
    const int Tn = n_dev ? min(*n_dev, T) : T;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Tn; i += gridDim.x * blockDim.x) {
        int t = order ? order[i] : i;
        int4 tr = tri[t];
        TriGeom g = tri_geom(tr, vxy, N);
        if (!is_small(g)) continue;
        int dax = g.ax - g.cx, day = g.ay - g.cy, dbx = g.bx - g.cx, dby = g.by - g.cy;
        long long l2 = (long long)dax * dax + (long long)day * day;
        bool pow2 = (l2 & (l2 - 1)) == 0;
        if (MODE == R_ERR || MODE == R_IMG) {
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
                row_span(g, y, N, L, len);
                if (len <= 0) continue;
                ff u = ff_add(ff_add(uc, ff_mul_f(gx, (float)(L - g.cx))), ff_mul_f(gy, (float)(y - g.cy)));
                long long p0 = (long long)y * N + L;
#pragma unroll 4
                for (int k = 0; k < len; ++k) {
                    if (MODE == R_ERR) {
                        ff d = ff_add_f(u, -img[p0 + k]);
                        acc = ff_add(acc, ff_sqr(d));
                    } else {
                        if (u_out) u_out[p0 + k] = __fadd_rn(u.hi, u.lo);
                        if (owner_out) owner_out[p0 + k] = t;
                    }
                    u = ff_add(u, gx);
                }
            }
            if (MODE == R_ERR) {
                double key = ff_to_double(acc);
                out[t] = key;
                if (keyc) {
                    bool eligible = (((g.ax + g.bx) | (g.ay + g.by)) & 1) == 0;
                    keyc[t] = eligible ? ((unsigned long long)__double_as_longlong(key) | (1ull << 63)) : 0ull;
                }
            }
        } else {
            double inv_l2 = pow2 ? __longlong_as_double((long long)(1023 - (63 - __clzll(l2))) << 52) : 1.0 / (double)l2;
            double acc[6] = {0, 0, 0, 0, 0, 0};
            for (int y = g.ytop; y <= g.yend; ++y) {
                int L, len;
                row_span(g, y, N, L, len);
                for (int k = 0; k < len; ++k) {
                    int x = L + k;
                    long long dxp = x - g.cx, dyp = y - g.cy;
                    double la = (double)(dxp * dax + dyp * day) * inv_l2;
                    double lb = (double)(dxp * dbx + dyp * dby) * inv_l2;
                    double lc = 1.0 - la - lb;
                    if (MODE == R_MASS) {
                        acc[0] = fma(la, la, acc[0]);
                        acc[1] = fma(lb, lb, acc[1]);
                        acc[2] = fma(lc, lc, acc[2]);
                        acc[3] = fma(la, lb, acc[3]);
                        acc[4] = fma(lb, lc, acc[4]);
                        acc[5] = fma(lc, la, acc[5]);
                    } else {
                        double r = (double)img[(long long)y * N + x];
                        acc[0] = fma(la, r, acc[0]);
                        acc[1] = fma(lb, r, acc[1]);
                        acc[2] = fma(lc, r, acc[2]);
                    }
                }
            }
            constexpr int NA = MODE == R_MASS ? 6 : 3;
#pragma unroll
            for (int q = 0; q < NA; ++q) out[(long long)t * NA + q] = acc[q];
        }
    }
}

// Error pass over the small triangles with the image staged in shared
// memory.  A block takes 16 consecutive entries of the curve order (a
// compact patch of the image), copies the bounding box of its small
// triangles into shared memory with asynchronous copies (cp.async, all in
// flight at once), and eight lanes share each triangle: lane j of a group
// walks rows ytop + j, ytop + j + 8, ..., so no lane serialises more than
// three rows of at most 17 pixels.  The eight float-float row sums are
// combined by a fixed butterfly.  A block whose box exceeds the tile reads
// the image directly.
constexpr int kTileThreads = 128;
constexpr int kTileTris = kTileThreads / 8;
constexpr int kTileCap = 4096;  // floats (16 KB)

__global__ void __launch_bounds__(kTileThreads) k_raster_small_err_tiled(
    const int* __restrict__ order, const int4* __restrict__ tri, const int2* __restrict__ vxy,
    const double* __restrict__ uv, const float2* __restrict__ uvf, const float* __restrict__ img, int N, int T,
    double* __restrict__ out, unsigned long long* __restrict__ keyc) {
    pdl_wait();
    __shared__ float s_img[kTileCap];
    __shared__ int s_red[4][kTileThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, sub = lane & 7;
    const int i = blockIdx.x * kTileTris + (tid >> 3);
    int t = -1;
    TriGeom g{};
    bool act = false;
    if (i < T) {
        t = order ? order[i] : i;
        g = tri_geom(tri[t], vxy, N);
        act = is_small(g);
    }
    int x0 = INT_MAX, y0 = INT_MAX, x1 = INT_MIN, y1 = INT_MIN;
    if (act) {
        x0 = min(g.ax, min(g.bx, g.cx));
        x1 = max(g.ax, max(g.bx, g.cx));
        y0 = g.ytop;
        y1 = g.yend;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x0 = min(x0, __shfl_xor_sync(0xffffffffu, x0, o));
        y0 = min(y0, __shfl_xor_sync(0xffffffffu, y0, o));
        x1 = max(x1, __shfl_xor_sync(0xffffffffu, x1, o));
        y1 = max(y1, __shfl_xor_sync(0xffffffffu, y1, o));
    }
    if (lane == 0) { s_red[0][w] = x0; s_red[1][w] = y0; s_red[2][w] = x1; s_red[3][w] = y1; }
    __syncthreads();
    x0 = INT_MAX; y0 = INT_MAX; x1 = INT_MIN; y1 = INT_MIN;
#pragma unroll
    for (int k = 0; k < kTileThreads / 32; ++k) {
        x0 = min(x0, s_red[0][k]);
        y0 = min(y0, s_red[1][k]);
        x1 = max(x1, s_red[2][k]);
        y1 = max(y1, s_red[3][k]);
    }
    if (x1 < x0) return;  // no small triangle in this block (uniform)
    const int W = x1 - x0 + 1, H = y1 - y0 + 1;
    const bool staged = (long long)W * H <= kTileCap;
    if (staged) {
        for (int r = w; r < H; r += kTileThreads / 32) {
            const float* src = img + (long long)(y0 + r) * N + x0;
            unsigned dst = (unsigned)__cvta_generic_to_shared(s_img + r * W);
            for (int c = lane; c < W; c += 32)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst + 4u * c), "l"(src + c) : "memory");
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
        __syncthreads();
    }
    ff acc{0.f, 0.f};
    if (act) {
        int dax = g.ax - g.cx, day = g.ay - g.cy, dbx = g.bx - g.cx, dby = g.by - g.cy;
        long long l2 = (long long)dax * dax + (long long)day * day;
        bool pow2 = (l2 & (l2 - 1)) == 0;
        int4 tr = tri[t];
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
        for (int y = g.ytop + sub; y <= g.yend; y += 8) {
            int L, len;
            row_span(g, y, N, L, len);
            if (len <= 0) continue;
            ff u = ff_add(ff_add(uc, ff_mul_f(gx, (float)(L - g.cx))), ff_mul_f(gy, (float)(y - g.cy)));
            const float* rowp = staged ? s_img + (y - y0) * W + (L - x0) : img + (long long)y * N + L;
#pragma unroll 4
            for (int k = 0; k < len; ++k) {
                ff d = ff_add_f(u, -rowp[k]);
                acc = ff_add(acc, ff_sqr(d));
                u = ff_add(u, gx);
            }
        }
    }
    // the eight lanes of a triangle: fixed butterfly (all lanes take part)
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) acc = ff_add(acc, ff_shfl_xor(acc, o));
    if (act && sub == 0) {
        double key = ff_to_double(acc);
        out[t] = key;
        if (keyc) {
            bool eligible = (((g.ax + g.bx) | (g.ay + g.by)) & 1) == 0;
            keyc[t] = eligible ? ((unsigned long long)__double_as_longlong(key) | (1ull << 63)) : 0ull;
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

// algorithmic bytes of one error pass: f once (4 B/px), triangles (16 B),
// vertex positions and values (8 + 8 B), one key out (8 B per triangle)
static double raster_err_bytes(const fem_mesh* m) {
    return 4.0 * (double)m->P + 24.0 * m->T + 16.0 * m->V;
}

fem_status raster_errors(fem_mesh* m, const double* uv, const float2* uvf, const float* f, double* err_out,
                         cudaStream_t s, unsigned long long* keyc_out) {
    FEM_TRY(raster_plan(m, s));
    // per-triangle completion counters, zero between passes (each triangle's
    // last warp resets its counter)
    if (m->item_done.n < (size_t)m->T || !m->item_done.p) {
        FEM_TRY(ensure(m->item_done, (size_t)m->T, s));
        FEM_CUDA(cudaMemsetAsync(m->item_done.p, 0, sizeof(int) * m->item_done.n, s));
    }
    note_bytes(F_RASTER, raster_err_bytes(m));
    FEM_LAUNCH(F_RASTER, s, k_raster<R_ERR>, raster_grid(m), kRasterThreads, 0, m->tri.p, m->vxy.p, uv, uvf, f, m->N,
               m->item_tri.p, m->item_off.p, m->dcount.p + 0, (int)m->item_tri.n, item_pixels_for(m->P), m->partial.p,
               (float*)nullptr, (int*)nullptr, m->item_cnt.p, m->item_done.p, err_out, keyc_out, nullptr,
               (const int*)(m->dflag.p + 0));
    // Few small triangles: eight lanes each over staged tiles, which shortens
    // the longest thread.  Many (above about 1k per SM): one thread each,
    // which avoids the eight-fold plane setup once every SM is full anyway.
    if (m->T <= m->num_sms * 1024)
        FEM_LAUNCH(F_RASTER, s, k_raster_small_err_tiled, (m->T + kTileTris - 1) / kTileTris, kTileThreads, 0,
                   m->order.p, m->tri.p, m->vxy.p, uv, uvf, f, m->N, m->T, err_out, keyc_out);
    else
        FEM_LAUNCH(F_RASTER, s, k_raster_small<R_ERR>, small_grid(m), 256, 0, m->order.p, m->tri.p, m->vxy.p, uv,
                   uvf, f, m->N, m->T, err_out, keyc_out, (float*)nullptr, (int*)nullptr, nullptr);
    return FEM_OK;
}

fem_status raster_image(fem_mesh* m, const double* uv, float* u, int* owner, cudaStream_t s) {
    FEM_TRY(raster_plan(m, s));
    note_bytes(F_RASTER, (u ? 4.0 * (double)m->P : 0.0) + (owner ? 4.0 * (double)m->P : 0.0) + 16.0 * m->T +
                             16.0 * m->V);
    FEM_LAUNCH(F_RASTER, s, k_raster<R_IMG>, raster_grid(m), kRasterThreads, 0, m->tri.p, m->vxy.p, uv,
               (const float2*)nullptr, (const float*)nullptr, m->N, m->item_tri.p, m->item_off.p, m->dcount.p + 0, (int)m->item_tri.n, item_pixels_for(m->P), m->partial.p, u, owner, nullptr, nullptr, nullptr, nullptr, nullptr,
               (const int*)(m->dflag.p + 0));
    FEM_LAUNCH(F_RASTER, s, k_raster_small<R_IMG>, small_grid(m), 256, 0, m->order.p, m->tri.p, m->vxy.p, uv,
               (const float2*)nullptr, (const float*)nullptr, m->N, m->T, (double*)nullptr,
               (unsigned long long*)nullptr, u, owner, nullptr);
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
                   (const double*)nullptr, (const float2*)nullptr, (const float*)nullptr, m->N, m->item_tri.p, m->item_off.p, m->dcount.p + 0,
                   (int)m->item_tri.n, item_pixels_for(m->P), m->partial.p, (float*)nullptr, (int*)nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                   (const int*)(m->dflag.p + 0));
        FEM_LAUNCH(F_RASTER, s, k_finalize<6>, blocks, 256, 0, m->item_cnt.p, m->item_off.p, m->partial.p, m->T,
                   m->loc.p);
        FEM_LAUNCH(F_RASTER, s, k_raster_small<R_MASS>, small_grid(m), 256, 0, m->order.p, m->tri.p, m->vxy.p,
                   (const double*)nullptr, (const float2*)nullptr, (const float*)nullptr, m->N, m->T, m->loc.p,
                   (unsigned long long*)nullptr, (float*)nullptr, (int*)nullptr, nullptr);
    } else {
        FEM_LAUNCH(F_RASTER, s, k_raster<R_SCAT>, raster_grid(m), kRasterThreads, 0, m->tri.p, m->vxy.p,
                   (const double*)nullptr, (const float2*)nullptr, r, m->N, m->item_tri.p, m->item_off.p, m->dcount.p + 0, (int)m->item_tri.n, item_pixels_for(m->P),
                   m->partial.p, (float*)nullptr, (int*)nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                   (const int*)(m->dflag.p + 0));
        FEM_LAUNCH(F_RASTER, s, k_finalize<3>, blocks, 256, 0, m->item_cnt.p, m->item_off.p, m->partial.p, m->T,
                   m->loc.p);
        FEM_LAUNCH(F_RASTER, s, k_raster_small<R_SCAT>, small_grid(m), 256, 0, m->order.p, m->tri.p, m->vxy.p,
                   (const double*)nullptr, (const float2*)nullptr, r, m->N, m->T, m->loc.p,
                   (unsigned long long*)nullptr, (float*)nullptr, (int*)nullptr, nullptr);
    }
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
    FEM_LAUNCH(F_RASTER, s, k_raster<R_ERR>, w.grid, kRasterThreads, 0, tri, vxy, uv, (const float2*)nullptr, f, N,
               w.item_tri, w.item_off, n_items_dev, w.item_cap, item_pixels_for((long long)N * N), w.partial, (float*)nullptr,
               (int*)nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, (const int*)err);
    FEM_LAUNCH(F_RASTER, s, k_finalize_err, std::max(1, std::min(w.grid, (T + 7) / 8)), 256, 0, w.item_cnt,
               w.item_off, (const float2*)w.partial, T, tri, vxy, err_out, (unsigned long long*)nullptr, w.item_cap,
               (const int*)err);
    FEM_LAUNCH(F_RASTER, s, k_raster_small<R_ERR>, std::max(1, std::min(blocks, w.grid / 2)), 256, 0, (const int*)nullptr,
               tri, vxy, uv, (const float2*)nullptr, f, N, T, err_out, (unsigned long long*)nullptr, (float*)nullptr,
               (int*)nullptr, nullptr);
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
    FEM_TRY(raster_errors(m, uv_dev, nullptr, f_dev, err_dev, s));
    int e = 0;
    FEM_CUDA(cudaMemcpyAsync(&e, m->dflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    if (e) {
        cudaMemsetAsync(m->dflag.p, 0, sizeof(int), s);
        m->plan_version = -1;
        set_error("fem_triangle_errors: rasterisation plan overflow");
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
// In the fast path triangles with a bounding box up to kFastSide pixels each
// way are summed one per thread, the larger ones by items (the split of the
// exact pass).  A wider split (64) was measured slower at 2049^2 and no
// faster at 8193^2: one thread walking a medium triangle issues a warp load
// over 32 different rows per pixel.
constexpr int kFastSide = kSmallSide;

__device__ __forceinline__ bool fast_small(const TriGeom& g) {
    return g.maxw <= kFastSide && (g.yend - g.ytop + 1) <= kFastSide;
}

struct FastOut {
    double* lo;
    double* hi;
    unsigned* hlo;
    unsigned* hhi;
};

// The bound in FP32 (GB300's FP64 rate would make a per-triangle FP64
// evaluation, with its divisions and square root, cost more than the pixels
// of a small triangle).  Every division is replaced by an upper bound
// (H u / (1 - H u) <= H u (1 + 2 H u) and S / (1 - g) <= S (1 + 2 g) for
// H u, g <= 1/4), and the about 12 FP32 roundings of the expression (each at
// most 2^-24 relative, all terms non-negative) are covered by the 2 %
// widening.
__device__ __forceinline__ void fast_interval(double S, float n, float M, float H, double& lo, double& hi) {
    const float u = 5.9604645e-08f;  // 2^-24
    float hu = H * u;
    float gam = hu * (1.0f + 2.0f * hu);
    float D = (float)S * (1.0f + 2.0f * gam) * (1.0f + 2.0f * u);  // (float)S may round down
    float delta = 5.0f * u * M;
    float B = gam * D + 2.0f * delta * sqrtf(n * D) + 2.0001f * u * D + 2.0f * n * delta * delta;
    B = 1.02f * B + 9.094947e-13f * (D + B) + 1e-30f;  // + 2^-40 (D + B)
    lo = fmax(0.0, S - (double)B);
    hi = S + (double)B;
}

__device__ __forceinline__ unsigned fast_bin_lo(double lo) { return __float_as_uint(__double2float_rd(lo)) >> 16; }
__device__ __forceinline__ unsigned fast_bin_hi(double hi) { return __float_as_uint(__double2float_ru(hi)) >> 16; }

// M of the error bound from the plane and the triangle's extent (FP32; its
// own rounding is covered by the widening of the bound)
__device__ __forceinline__ float fast_M(const TriGeom& g, float ucf, float gxf, float gyf) {
    float wx = (float)max(abs(g.ax - g.cx), abs(g.bx - g.cx));
    float wy = (float)max(abs(g.ay - g.cy), abs(g.by - g.cy));
    return (fabsf(ucf) + fabsf(gxf) * wx + fabsf(gyf) * wy) * (1.0f + 1e-6f);
}

// float-float plane of the interpolant (as in the exact kernels)
__device__ __forceinline__ void tri_plane(const TriGeom& g, int4 tr, const double* uv, const float2* uvf, ff& uc,
                                          ff& gx, ff& gy) {
    int dax = g.ax - g.cx, day = g.ay - g.cy, dbx = g.bx - g.cx, dby = g.by - g.cy;
    long long l2 = (long long)dax * dax + (long long)day * day;
    bool pow2 = (l2 & (l2 - 1)) == 0;
    ff va = vertex_ff(uv, uvf, tr.x), vb = vertex_ff(uv, uvf, tr.y);
    uc = vertex_ff(uv, uvf, tr.z);
    ff da = ff_sub(va, uc), db = ff_sub(vb, uc);
    gx = ff_add(ff_mul_f(da, (float)dax), ff_mul_f(db, (float)dbx));
    gy = ff_add(ff_mul_f(da, (float)day), ff_mul_f(db, (float)dby));
    if (pow2) {
        float inv = __int_as_float((127 - (63 - __clzll(l2))) << 23);
        gx = ff_scale_pow2(gx, inv);
        gy = ff_scale_pow2(gy, inv);
    } else {
        float inv = 1.0f / (float)l2;
        gx = ff_mul_f(gx, inv);
        gy = ff_mul_f(gy, inv);
    }
}

__device__ __forceinline__ bool tri_eligible(const TriGeom& g) { return (((g.ax + g.bx) | (g.ay + g.by)) & 1) == 0; }

// Large triangles: the item decomposition of k_raster in FP32.  Item
// partials are (sum, pixel count); the warp that completes a triangle
// combines them (float-float sum, integer count) and writes its interval.
__global__ void __launch_bounds__(kRasterThreads) k_raster_fast(
    const int4* __restrict__ tri, const int2* __restrict__ vxy, const double* __restrict__ uv,
    const float2* __restrict__ uvf, const float* __restrict__ img, int N, const int* __restrict__ item_tri,
    const int* __restrict__ item_off, const int* __restrict__ item_cnt, const int* __restrict__ n_items_dev,
    int item_cap, int item_px, float2* __restrict__ partial, int* __restrict__ item_done, FastOut F,
    const int* __restrict__ plan_err) {
    pdl_wait();
    if (plan_err && *plan_err) return;  // an overflowing plan: as in k_raster
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int n_items = min(*n_items_dev, item_cap);
    for (long long it = warp; it < n_items; it += nwarps) {
        int t = item_tri[it];
        int j = (int)(it - item_off[t]);
        int4 tr = tri[t];
        TriGeom g = tri_geom(tr, vxy, N);
        if (fast_small(g)) continue;  // summed by k_raster_small_fast (uniform over the warp)
        int rpi = rows_per_item(g.maxw, item_px);
        int r0 = g.ytop + j * rpi;
        int nr = min(rpi, g.yend + 1 - r0);
        int L = 0, len = 0;
        if (lane < nr) row_span(g, r0 + lane, N, L, len);
        int total = warp_sum(len);
        // chunks of 32 pixels per row, located by a ballot (as in k_raster)
        int ccnt = (len + 31) >> 5, cinc = ccnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL, cinc, o);
            if (lane >= o) cinc += y;
        }
        const int coff = cinc - ccnt;
        const int nchunks = __shfl_sync(FULL, cinc, 31);
        ff uc, gx, gy;
        tri_plane(g, tr, uv, uvf, uc, gx, gy);
        const float ucf = __fadd_rn(uc.hi, uc.lo), gxf = __fadd_rn(gx.hi, gx.lo), gyf = __fadd_rn(gy.hi, gy.lo);
        float acc = 0.f;
        constexpr int kPre = 4;
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
                fv[u] = ok ? img[(long long)py[u] * N + px[u]] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kPre; ++u) {
                if (px[u] >= 0) {
                    float uu = fmaf(gyf, (float)(py[u] - g.cy), fmaf(gxf, (float)(px[u] - g.cx), ucf));
                    float d = uu - fv[u];
                    acc = fmaf(d, d, acc);
                }
            }
        }
        float tot = warp_sum(acc);
        const int nit = item_cnt[t];
        int last = 0;
        if (nit > 1 && lane == 0) {
            partial[it] = make_float2(tot, __int_as_float(total));
            __threadfence();
            last = atomicAdd(item_done + t, 1) == nit - 1;
        }
        last = nit == 1 ? 1 : __shfl_sync(FULL, last, 0);
        if (last) {
            ff s{tot, 0.f};
            long long cnt = total;
            if (nit > 1) {
                __threadfence();
                const int o = item_off[t];
                s = ff{0.f, 0.f};
                cnt = 0;
                for (int q = lane; q < nit; q += 32) {
                    float2 v = __ldcg(&partial[o + q]);
                    s = ff_add_f(s, v.x);
                    cnt += __float_as_int(v.y);
                }
                s = ff_warp_sum(s);
                cnt = warp_sum(cnt);
            }
            if (lane == 0) {
                // per lane at most 64 chunk pixels per item (32 rows plus 1024
                // pixels in chunks), a 5-level butterfly, then the float-float
                // combination of the items
                double lo, hi;
                fast_interval(ff_to_double(s), (float)cnt, fast_M(g, ucf, gxf, gyf), 64.0f + 5.0f + 2.0f, lo, hi);
                F.lo[t] = lo;
                F.hi[t] = hi;
                if (tri_eligible(g)) {
                    atomicAdd(F.hlo + fast_bin_lo(lo), 1u);
                    atomicAdd(F.hhi + fast_bin_hi(hi), 1u);
                }
                if (nit > 1) item_done[t] = 0;
            }
        }
    }
}

// Small triangles: one thread each along the curve order, FP32 with the
// plane evaluated afresh per pixel (u = g_x k + u_row, no running sum).
// Histogram updates are combined per warp for equal bins.
__global__ void __launch_bounds__(256) k_raster_small_fast(const int* __restrict__ order, const int4* __restrict__ tri,
                                                           const int2* __restrict__ vxy, const double* __restrict__ uv,
                                                           const float2* __restrict__ uvf,
                                                           const float* __restrict__ img, int N, int T, FastOut F) {
    pdl_wait();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T; i += gridDim.x * blockDim.x) {
        int t = order ? order[i] : i;
        int4 tr = tri[t];
        TriGeom g = tri_geom(tr, vxy, N);
        bool small = fast_small(g);
        unsigned blo = 0xffffffffu, bhi = 0xffffffffu;
        if (small) {
            ff uc, gx, gy;
            tri_plane(g, tr, uv, uvf, uc, gx, gy);
            const float ucf = __fadd_rn(uc.hi, uc.lo), gxf = __fadd_rn(gx.hi, gx.lo),
                        gyf = __fadd_rn(gy.hi, gy.lo);
            // row sums (at most kFastSide + 1 terms each), then the sum of the
            // rows (at most kFastSide + 1 terms): chains of at most
            // 2 (kFastSide + 1) additions
            float acc = 0.f;
            int n = 0;
            for (int y = g.ytop; y <= g.yend; ++y) {
                int L, len;
                row_span(g, y, N, L, len);
                if (len <= 0) continue;
                float urow = fmaf(gyf, (float)(y - g.cy), fmaf(gxf, (float)(L - g.cx), ucf));
                const float* rowp = img + (long long)y * N + L;
                float racc = 0.f;
#pragma unroll 4
                for (int k = 0; k < len; ++k) {
                    float u = fmaf(gxf, (float)k, urow);
                    float d = u - rowp[k];
                    racc = fmaf(d, d, racc);
                }
                acc += racc;
                n += len;
            }
            double lo, hi;
            fast_interval((double)acc, (float)n, fast_M(g, ucf, gxf, gyf), 2.0f * (kFastSide + 1) + 2.0f, lo, hi);
            F.lo[t] = lo;
            F.hi[t] = hi;
            if (tri_eligible(g)) {
                blo = fast_bin_lo(lo);
                bhi = fast_bin_hi(hi);
            }
        }
        // histogram: one atomic per distinct bin among the converged lanes
        unsigned act = __activemask();
        unsigned peers = __match_any_sync(act, blo);
        if (blo != 0xffffffffu && (__ffs(peers) - 1) == (int)(threadIdx.x & 31))
            atomicAdd(F.hlo + blo, (unsigned)__popc(peers));
        peers = __match_any_sync(act, bhi);
        if (bhi != 0xffffffffu && (__ffs(peers) - 1) == (int)(threadIdx.x & 31))
            atomicAdd(F.hhi + bhi, (unsigned)__popc(peers));
    }
}

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
// or band (listed; large ones by their items, small ones by id).
__global__ void k_fast_classify(const int4* __restrict__ tri, const int2* __restrict__ vxy, int T, int N,
                                const double* __restrict__ lo, const double* __restrict__ hi,
                                const double* __restrict__ tau, const int* __restrict__ item_cnt,
                                const int* __restrict__ item_off, double* __restrict__ keys,
                                unsigned long long* __restrict__ keyc, int* __restrict__ band,
                                int* __restrict__ band_items, int* __restrict__ band_small, int* __restrict__ cnt,
                                unsigned long long* __restrict__ max_out) {
    pdl_wait();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int cls = 0;  // 0 ineligible / outside, 1 in, 2 out, 3 band
    unsigned long long comp_out = 0ull;
    if (t < T) {
        TriGeom g = tri_geom(tri[t], vxy, N);
        double l = lo[t], h = hi[t];
        if (!tri_eligible(g)) {
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
        }
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
    if (cls == 3) {
        band[base + __popc(band_mask & ((1u << lane) - 1u))] = t;
        int nc = item_cnt[t];
        if (nc > 0) {
            int ip = atomicAdd(cnt + 2, nc);
            for (int q = 0; q < nc; ++q) band_items[ip + q] = item_off[t] + q;
        } else {
            band_small[atomicAdd(cnt + 3, 1)] = t;
        }
    }
}

// Keys of the spatial optimisation by the fast path: on return keys[] and
// keyc[] hold, for every triangle, the exact key (band) or the substituted
// bound (outside the band), kdev the total k, and the band list with its
// counts for the selection (refine_round).
fem_status raster_keys_fast(fem_mesh* m, const double* uv, const float2* uvf, const float* f, double frac,
                            long long vcap, cudaStream_t s) {
    FEM_TRY(raster_plan(m, s));
    int T = m->T;
    if (m->item_done.n < (size_t)T || !m->item_done.p) {
        FEM_TRY(ensure(m->item_done, (size_t)T, s));
        FEM_CUDA(cudaMemsetAsync(m->item_done.p, 0, sizeof(int) * m->item_done.n, s));
    }
    FEM_TRY(ensure(m->keys_lo, (size_t)T, s));
    FEM_TRY(ensure(m->keys_hi, (size_t)T, s));
    FEM_TRY(ensure(m->band, (size_t)T, s));
    FEM_TRY(ensure(m->band_small, (size_t)T, s));
    FEM_TRY(ensure(m->band_items, m->item_tri.n, s));
    FEM_TRY(ensure(m->fast_hist, (size_t)2 * kFastBins + 8, s));
    unsigned* hist = m->fast_hist.p;
    int* cnt = (int*)(hist + 2 * kFastBins);  // [0] in, [1] band, [2] band items, [3] band small
    unsigned long long* max_out = (unsigned long long*)(m->dscal.p + 18);
    double* tau = m->dscal.p + 16;
    int* kdev = m->dcount.p + 2;
    FEM_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned) * (2 * kFastBins + 8), s));
    FEM_CUDA(cudaMemsetAsync(max_out, 0, sizeof(unsigned long long), s));
    FastOut F{m->keys_lo.p, m->keys_hi.p, hist, hist + kFastBins};
    // all pixels in FP32
    note_bytes(F_RASTER, raster_err_bytes(m));
    FEM_LAUNCH(F_RASTER, s, k_raster_fast, raster_grid(m), kRasterThreads, 0, m->tri.p, m->vxy.p, uv, uvf, f, m->N,
               m->item_tri.p, m->item_off.p, m->item_cnt.p, m->dcount.p + 0, (int)m->item_tri.n, item_pixels_for(m->P),
               (float2*)m->partial.p, m->item_done.p, F, (const int*)(m->dflag.p + 0));
    FEM_LAUNCH(F_RASTER, s, k_raster_small_fast, small_grid(m), 256, 0, m->order.p, m->tri.p, m->vxy.p, uv, uvf, f,
               m->N, T, F);
    // bracket and classification
    FEM_LAUNCH(F_TOPK, s, k_fast_bracket, 1, kBracketThreads, 0, hist, hist + kFastBins, T, frac, vcap, kdev, tau);
    FEM_LAUNCH(F_TOPK, s, k_fast_classify, (T + 255) / 256, 256, 0, m->tri.p, m->vxy.p, T, m->N, m->keys_lo.p,
               m->keys_hi.p, tau, m->item_cnt.p, m->item_off.p, m->keys.p, m->keyc.p, m->band.p, m->band_items.p,
               m->band_small.p, cnt, max_out);
    // exact float-float keys of the band
    FEM_LAUNCH(F_RASTER, s, k_raster<R_ERR>, raster_grid(m), kRasterThreads, 0, m->tri.p, m->vxy.p, uv, uvf, f, m->N,
               m->item_tri.p, m->item_off.p, cnt + 2, (int)m->band_items.n, item_pixels_for(m->P), m->partial.p,
               (float*)nullptr, (int*)nullptr, m->item_cnt.p, m->item_done.p, m->keys.p, m->keyc.p, m->band_items.p,
               (const int*)(m->dflag.p + 0));
    FEM_LAUNCH(F_RASTER, s, k_raster_small<R_ERR>, small_grid(m), 256, 0, m->band_small.p, m->tri.p, m->vxy.p, uv,
               uvf, f, m->N, T, m->keys.p, m->keyc.p, (float*)nullptr, (int*)nullptr, cnt + 3);
    return FEM_OK;
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
    FEM_TRY(raster_plan(m, s));
    int T = m->T;
    if (m->item_done.n < (size_t)T || !m->item_done.p) {
        FEM_TRY(ensure(m->item_done, (size_t)T, s));
        FEM_CUDA(cudaMemsetAsync(m->item_done.p, 0, sizeof(int) * m->item_done.n, s));
    }
    FEM_TRY(ensure(m->fast_hist, (size_t)2 * kFastBins + 8, s));
    FEM_CUDA(cudaMemsetAsync(m->fast_hist.p, 0, sizeof(unsigned) * (2 * kFastBins + 8), s));
    FastOut F{lo_dev, hi_dev, m->fast_hist.p, m->fast_hist.p + kFastBins};
    FEM_LAUNCH(F_RASTER, s, k_raster_fast, raster_grid(m), kRasterThreads, 0, m->tri.p, m->vxy.p, uv_dev,
               (const float2*)nullptr, f_dev, m->N, m->item_tri.p, m->item_off.p, m->item_cnt.p, m->dcount.p + 0,
               (int)m->item_tri.n, item_pixels_for(m->P), (float2*)m->partial.p, m->item_done.p, F,
               (const int*)(m->dflag.p + 0));
    FEM_LAUNCH(F_RASTER, s, k_raster_small_fast, small_grid(m), 256, 0, (const int*)nullptr, m->tri.p, m->vxy.p,
               uv_dev, (const float2*)nullptr, f_dev, m->N, T, F);
    int e = 0;
    FEM_CUDA(cudaMemcpyAsync(&e, m->dflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    if (e) {
        cudaMemsetAsync(m->dflag.p, 0, sizeof(int), s);
        m->plan_version = -1;
        set_error("fem_triangle_error_bounds: rasterisation plan overflow");
        return (fem_status)e;
    }
    return FEM_OK;
}
