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
constexpr int kItemPixels = 1024;
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

__device__ __forceinline__ int rows_per_item(int maxw) {
    int r = kItemPixels / maxw;
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
    int* cnt;
    __device__ __forceinline__ int operator()(long long lt) const {
        int t = (int)lt;
        TriGeom g = tri_geom(tri[t], vxy, N);
        int rows = g.yend - g.ytop + 1;
        int rpi = rows_per_item(g.maxw);
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
                             int* __restrict__ cnt) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    TriGeom g = tri_geom(tri[t], vxy, N);
    int rows = g.yend - g.ytop + 1;
    int rpi = rows_per_item(g.maxw);
    cnt[t] = (rows > 0 && !is_small(g)) ? (rows + rpi - 1) / rpi : 0;
}

__global__ void k_item_expand(const int* __restrict__ cnt, const int* __restrict__ off, int T, int cap,
                              int* __restrict__ item_tri, int* __restrict__ err) {
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
    const int* __restrict__ item_off, const int* __restrict__ n_items_dev, int item_cap,
    double* __restrict__ partial, float* __restrict__ u_out, int* __restrict__ owner_out,
    const int* __restrict__ item_cnt = nullptr, int* __restrict__ item_done = nullptr,
    double* __restrict__ key_out = nullptr, unsigned long long* __restrict__ keyc_out = nullptr) {
    constexpr int NA = NAcc<MODE>::n;
    constexpr bool FF = (MODE == R_ERR || MODE == R_IMG);
    const unsigned FULL = 0xffffffffu;
    int lane = threadIdx.x & 31;
    long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    int n_items = min(*n_items_dev, item_cap);  // never past the plan's capacity
    for (long long it = warp; it < n_items; it += nwarps) {
        int t = item_tri[it];
        int j = (int)(it - item_off[t]);
        int4 tr = tri[t];
        TriGeom g = tri_geom(tr, vxy, N);
        int rpi = rows_per_item(g.maxw);
        int r0 = g.ytop + j * rpi;
        int nr = min(rpi, g.yend + 1 - r0);
        int L = 0, len = 0;
        if (lane < nr) row_span(g, r0 + lane, N, L, len);
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        int off = incl - len;
        int total = __shfl_sync(FULL, incl, 31);

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

        // pixels are taken kPre chunks of 32 at a time: positions and image
        // values of all chunks first (kPre loads in flight per lane), then
        // the arithmetic
        constexpr int kPre = 4;
        constexpr bool READS = (MODE == R_ERR || MODE == R_SCAT);
        for (int base0 = 0; base0 < total; base0 += 32 * kPre) {
            int px[kPre], py[kPre];
            float fv[kPre];
#pragma unroll
            for (int u = 0; u < kPre; ++u) {
                int jj = base0 + 32 * u + lane;
                int k = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    int cand = k + step;
                    int oc = __shfl_sync(FULL, off, cand & 31);
                    if (cand < nr && oc <= jj) k = cand;
                }
                int Lk = __shfl_sync(FULL, L, k);
                int okk = __shfl_sync(FULL, off, k);
                px[u] = jj < total ? Lk + (jj - okk) : -1;
                py[u] = r0 + k;
                fv[u] = (READS && jj < total) ? img[(long long)py[u] * N + px[u]] : 0.f;
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
                int last = 0;
                if (lane == 0) {
                    ((float2*)partial)[it] = make_float2(tot.hi, tot.lo);
                    __threadfence();
                    last = atomicAdd(item_done + t, 1) == item_cnt[t] - 1;
                }
                last = __shfl_sync(FULL, last, 0);
                if (last) {
                    __threadfence();
                    ff sum = warp_sum_partials((const float2*)partial, item_off[t], item_cnt[t]);
                    if (lane == 0) {
                        double key = ff_to_double(sum);
                        key_out[t] = key;
                        if (keyc_out) {
                            bool eligible = (((g.ax + g.bx) | (g.ay + g.by)) & 1) == 0;
                            keyc_out[t] = eligible ? ((unsigned long long)__double_as_longlong(key) | (1ull << 63)) : 0ull;
                        }
                        item_done[t] = 0;  // ready for the next pass
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
                               unsigned long long* __restrict__ keyc) {
    long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long tt = gw; tt < T; tt += nw) {
        int t = (int)tt;
        int o = off[t], n = cnt[t];
        if (n == 0) continue;  // small triangle: written by the small-triangle kernel
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
                                                      float* __restrict__ u_out, int* __restrict__ owner_out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T; i += gridDim.x * blockDim.x) {
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
    int* err = m->dflag.p + 0;
    FEM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    FEM_TRY(scan_fused(m, ItemCountIn{m->tri.p, m->vxy.p, m->N, m->item_cnt.p},
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
               m->item_tri.p, m->item_off.p, m->dcount.p + 0, (int)m->item_tri.n, m->partial.p, (float*)nullptr,
               (int*)nullptr, m->item_cnt.p, m->item_done.p, err_out, keyc_out);
    // Few small triangles: eight lanes each over staged tiles, which shortens
    // the longest thread.  Many (above about 1k per SM): one thread each,
    // which avoids the eight-fold plane setup once every SM is full anyway.
    if (m->T <= m->num_sms * 1024)
        FEM_LAUNCH(F_RASTER, s, k_raster_small_err_tiled, (m->T + kTileTris - 1) / kTileTris, kTileThreads, 0,
                   m->order.p, m->tri.p, m->vxy.p, uv, uvf, f, m->N, m->T, err_out, keyc_out);
    else
        FEM_LAUNCH(F_RASTER, s, k_raster_small<R_ERR>, small_grid(m), 256, 0, m->order.p, m->tri.p, m->vxy.p, uv,
                   uvf, f, m->N, m->T, err_out, keyc_out, (float*)nullptr, (int*)nullptr);
    return FEM_OK;
}

fem_status raster_image(fem_mesh* m, const double* uv, float* u, int* owner, cudaStream_t s) {
    FEM_TRY(raster_plan(m, s));
    note_bytes(F_RASTER, (u ? 4.0 * (double)m->P : 0.0) + (owner ? 4.0 * (double)m->P : 0.0) + 16.0 * m->T +
                             16.0 * m->V);
    FEM_LAUNCH(F_RASTER, s, k_raster<R_IMG>, raster_grid(m), kRasterThreads, 0, m->tri.p, m->vxy.p, uv,
               (const float2*)nullptr, (const float*)nullptr, m->N, m->item_tri.p, m->item_off.p, m->dcount.p + 0, (int)m->item_tri.n, m->partial.p, u, owner);
    FEM_LAUNCH(F_RASTER, s, k_raster_small<R_IMG>, small_grid(m), 256, 0, m->order.p, m->tri.p, m->vxy.p, uv,
               (const float2*)nullptr, (const float*)nullptr, m->N, m->T, (double*)nullptr,
               (unsigned long long*)nullptr, u, owner);
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
                   (int)m->item_tri.n, m->partial.p, (float*)nullptr, (int*)nullptr);
        FEM_LAUNCH(F_RASTER, s, k_finalize<6>, blocks, 256, 0, m->item_cnt.p, m->item_off.p, m->partial.p, m->T,
                   m->loc.p);
        FEM_LAUNCH(F_RASTER, s, k_raster_small<R_MASS>, small_grid(m), 256, 0, m->order.p, m->tri.p, m->vxy.p,
                   (const double*)nullptr, (const float2*)nullptr, (const float*)nullptr, m->N, m->T, m->loc.p,
                   (unsigned long long*)nullptr, (float*)nullptr, (int*)nullptr);
    } else {
        FEM_LAUNCH(F_RASTER, s, k_raster<R_SCAT>, raster_grid(m), kRasterThreads, 0, m->tri.p, m->vxy.p,
                   (const double*)nullptr, (const float2*)nullptr, r, m->N, m->item_tri.p, m->item_off.p, m->dcount.p + 0, (int)m->item_tri.n, m->partial.p,
                   (float*)nullptr, (int*)nullptr);
        FEM_LAUNCH(F_RASTER, s, k_finalize<3>, blocks, 256, 0, m->item_cnt.p, m->item_off.p, m->partial.p, m->T,
                   m->loc.p);
        FEM_LAUNCH(F_RASTER, s, k_raster_small<R_SCAT>, small_grid(m), 256, 0, m->order.p, m->tri.p, m->vxy.p,
                   (const double*)nullptr, (const float2*)nullptr, r, m->N, m->T, m->loc.p,
                   (unsigned long long*)nullptr, (float*)nullptr, (int*)nullptr);
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
    FEM_LAUNCH(F_RASTER, s, k_item_count, blocks, 256, 0, tri, vxy, T, N, w.item_cnt);
    FEM_TRY(exclusive_scan_i32_scratch(w.item_cnt, w.item_off, T, s, n_items_dev, w.scan_tmp, w.scan_tmp_n));
    FEM_LAUNCH(F_RASTER, s, k_item_expand, blocks, 256, 0, w.item_cnt, w.item_off, T, w.item_cap, w.item_tri, err);
    FEM_LAUNCH(F_RASTER, s, k_raster<R_ERR>, w.grid, kRasterThreads, 0, tri, vxy, uv, (const float2*)nullptr, f, N,
               w.item_tri, w.item_off, n_items_dev, w.item_cap, w.partial, (float*)nullptr, (int*)nullptr);
    FEM_LAUNCH(F_RASTER, s, k_finalize_err, std::max(1, std::min(w.grid, (T + 7) / 8)), 256, 0, w.item_cnt,
               w.item_off, (const float2*)w.partial, T, tri, vxy, err_out, (unsigned long long*)nullptr);
    FEM_LAUNCH(F_RASTER, s, k_raster_small<R_ERR>, std::max(1, std::min(blocks, w.grid / 2)), 256, 0, (const int*)nullptr,
               tri, vxy, uv, (const float2*)nullptr, f, N, T, err_out, (unsigned long long*)nullptr, (float*)nullptr,
               (int*)nullptr);
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
