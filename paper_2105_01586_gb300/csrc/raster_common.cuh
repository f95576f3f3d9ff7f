// raster_common.cuh -- device helpers shared by the rasterisation kernels:
// the lattice-triangle geometry and pixel ownership (Sec. 2.2), the plane
// of the linear interpolant, and the FP32 error intervals of the fast
// selection keys (Sec. 3 error map).
#pragma once
#include <climits>

#include "fem_internal.cuh"
#include "ff.cuh"

namespace fem {

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

// the part of a row's span [L, L + len) inside the image (nothing below it)
__device__ __forceinline__ void clip_span(int y, const Dom& D, int L, int& len) {
    const int e = min(L + len, D.W);
    len = (y < D.H && e > L) ? e - L : 0;
}

// owned columns of row y: [L, L + len), within the image
__device__ __forceinline__ void row_span(const TriGeom& g, int y, const Dom& D, int& L, int& len) {
    int l = INT_MAX, r = INT_MIN;
    edge_x(g.ax, g.ay, g.bx, g.by, y, l, r);
    edge_x(g.bx, g.by, g.cx, g.cy, y, l, r);
    edge_x(g.cx, g.cy, g.ax, g.ay, y, l, r);
    int n = r - l + ((r == D.N - 1 && l < r) ? 1 : 0);
    L = l;
    len = n > 0 ? n : 0;
    clip_span(y, D, L, len);
}

// Row spans in closed form.  Every edge of the mesh's triangles is
// horizontal, vertical or diagonal, so with the corners sorted by y (v0, v1,
// v2) row y meets the long edge v0-v2 at x0 + (y - y0) s02 and the short
// edges at x0 + (y - y0) s01 (y < y1) or x1 + (y - y1) s12, where s is the
// edge's step in x per row (0 or +-1).  The span [min, max) of the two, with
// the image's last column added as in row_span, equals row_span's for every
// owned row, at a few operations per row instead of three edge tests.
struct RowGeo {
    int y0, y1, x0, x1;
    int sl;  // (s02 + 1) | (s01 + 1) << 2 | (s12 + 1) << 4
};

__device__ __forceinline__ int step_sign(int d) { return (d > 0) - (d < 0); }

__device__ __forceinline__ RowGeo row_geo(const TriGeom& g) {
    int ax = g.ax, ay = g.ay, bx = g.bx, by = g.by, cx = g.cx, cy = g.cy, t;
    if (by < ay) { t = ax; ax = bx; bx = t; t = ay; ay = by; by = t; }
    if (cy < by) { t = bx; bx = cx; cx = t; t = by; by = cy; cy = t; }
    if (by < ay) { t = ax; ax = bx; bx = t; t = ay; ay = by; by = t; }
    RowGeo r;
    r.y0 = ay; r.y1 = by; r.x0 = ax; r.x1 = bx;
    r.sl = (step_sign(cx - ax) + 1) | ((step_sign(bx - ax) + 1) << 2) | ((step_sign(cx - bx) + 1) << 4);
    return r;
}

__device__ __forceinline__ void row_span_geo(const RowGeo& r, int y, const Dom& D, int& L, int& len) {
    const int s02 = (r.sl & 3) - 1, s01 = ((r.sl >> 2) & 3) - 1, s12 = ((r.sl >> 4) & 3) - 1;
    const int xl = r.x0 + (y - r.y0) * s02;
    const int xs = y < r.y1 ? r.x0 + (y - r.y0) * s01 : r.x1 + (y - r.y1) * s12;
    const int l = min(xl, xs), rr = max(xl, xs);
    const int n = rr - l + ((rr == D.N - 1 && l < rr) ? 1 : 0);
    L = l;
    len = n > 0 ? n : 0;
    clip_span(y, D, L, len);
}

// Small triangles (bounding box at most kSmallSide pixels each way, at most
// 153 pixels) are rasterised one per thread along the space-filling curve
// (k_raster_small); only the larger ones are cut into warp items.
constexpr int kSmallSide = 17;

__device__ __forceinline__ bool is_small(const TriGeom& g) {
    return g.maxw <= kSmallSide && (g.yend - g.ytop + 1) <= kSmallSide;
}

// vertex value as float-float: from the float-float copy when there is one,
// else split from FP64
__device__ __forceinline__ ff vertex_ff(const double* __restrict__ uv, const float2* __restrict__ uvf, int i) {
    if (uvf) {
        float2 v = uvf[i];
        return ff{v.x, v.y};
    }
    return ff_from_double(uv[i]);
}

// Outputs of the FP32 pass: an interval [lo, hi] per triangle (FP32, rounded
// outwards) and the histograms of the bit patterns of lo and hi.
struct FastOut {
    float* lo;
    float* hi;
    unsigned* hlo;
    unsigned* hhi;
};

// The bound in FP32, rounded outwards (GB300's FP64 rate would make a
// per-triangle FP64 evaluation, with its divisions and square root, cost
// more than the pixels of a small triangle).  S is the sum as a float-float
// pair (an FP32 sum has lo = 0).  Every division is replaced by an upper
// bound (H u / (1 - H u) <= H u (1 + 2 H u) and S / (1 - g) <= S (1 + 2 g)
// for H u, g <= 1/4), and the about 12 FP32 roundings of the expression
// (each at most 2^-24 relative, all terms non-negative) are covered by the
// 2 % widening.
__device__ __forceinline__ void fast_interval(ff S, float n, float M, float H, float& lo, float& hi) {
    const float u = 5.9604645e-08f;  // 2^-24
    const float Sd = __fadd_rd(S.hi, S.lo), Su = __fadd_ru(S.hi, S.lo);
    float hu = H * u;
    float gam = hu * (1.0f + 2.0f * hu);
    float D = Su * (1.0f + 2.0f * gam) * (1.0f + 2.0f * u);
    float delta = 5.0f * u * M;
    float B = gam * D + 2.0f * delta * sqrtf(n * D) + 2.0001f * u * D + 2.0f * n * delta * delta;
    B = 1.02f * B + 9.094947e-13f * (D + B) + 1e-30f;  // + 2^-40 (D + B)
    lo = fmaxf(0.0f, __fsub_rd(Sd, B));
    hi = __fadd_ru(Su, B);
}

// histogram bins: the top 16 bits of a non-negative float
__device__ __forceinline__ unsigned fast_bin(float v) { return __float_as_uint(v) >> 16; }

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

// eligible for selection (dom_eligible)
__device__ __forceinline__ bool tri_eligible(const TriGeom& g, const Dom& D) {
    return dom_eligible(g.ax, g.ay, g.bx, g.by, g.cx, g.cy, D);
}

// Squares of the image for the square-tiled pass (raster_sq.cu): side s =
// min(64, N - 1), Q x Q of them; node 2q + h is half h of square q.
struct SqGeo {
    int N, s, Q;
    int W, H;  // the image within the domain
};

__device__ __forceinline__ Dom sq_dom(const SqGeo& G) { return Dom{G.N, G.W, G.H}; }

// node of the point with three times the coordinates (X3, Y3), a point
// strictly inside a node (the centroid of a triangle below the node level):
// the square's diagonal runs top-left to bottom-right when I + J is even,
// else top-right to bottom-left; half 0 holds the square's left side
__device__ __forceinline__ int sq_node_at(long long X3, long long Y3, const SqGeo& G) {
    const long long s3 = 3LL * G.s;
    const int I = (int)(Y3 / s3), J = (int)(X3 / s3);
    const long long u3 = X3 - s3 * J, v3 = Y3 - s3 * I;
    const int h = ((I + J) & 1) == 0 ? (v3 > u3 ? 0 : 1) : (u3 + v3 < s3 ? 0 : 1);
    return ((I * G.Q + J) << 1) | h;
}

__device__ __forceinline__ long long leg2(int2 a, int2 c) {
    const long long dx = a.x - c.x, dy = a.y - c.y;
    return dx * dx + dy * dy;
}

// A fine triangle for the FP32 pass, stored at its curve position so that a
// square's triangles are read with coalesced loads: its vertices, its id and
// the FP32 plane of the interpolant (u_c, g_x, g_y rounded from float-float).
struct __align__(16) SqRec {
    unsigned short ax, ay, bx, by, cx, cy;
    int t;
    float ucf, gxf, gyf, pad;
};

// square-tiled pass (raster_sq.cu)
int sq_side(int N);
SqGeo sq_geo(const fem_mesh* m);
fem_status sq_plan(fem_mesh* m, cudaStream_t s);
fem_status sq_keys_fast(fem_mesh* m, const double* uv, const float2* uvf, FastOut F, cudaStream_t s,
                        bool incremental = false);
// coarse (optional): the coarse triangles to finish, by curve position
// (default: all of them)
fem_status sq_keys_exact(fem_mesh* m, const double* uv, const float2* uvf, double* keys, unsigned long long* keyc,
                         const unsigned char* sel, const int* list, const int* n_list, int n_max, cudaStream_t s,
                         const int* coarse = nullptr, const int* n_coarse = nullptr);
fem_status sq_band_exact(fem_mesh* m, const double* uv, const float2* uvf, int* n_list_dev, cudaStream_t s);

}  // namespace fem
