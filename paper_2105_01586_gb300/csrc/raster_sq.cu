// raster_sq.cu -- the per-triangle squared errors of the spatial
// optimisation (Sec. 3 error map, with the linear interpolation of Sec. 2.2)
// as one pass over the image in squares.
//
// Squares and nodes.  The image side is N = 2^L + 1, so with s = min(32,
// N - 1) the pixels split into Q x Q squares of s x s (the squares of the
// last row and column also hold the image's last row and column).  Every
// square is the union of two triangles of the bisection tree ("nodes"): its
// diagonal runs from top-left to bottom-right when I + J is even and from
// top-right to bottom-left when it is odd (each level of the uniform
// newest-vertex refinement splits a square through its parent's centre).
// Node h = 0 is the half that holds the square's left side.  Because the
// mesh is the leaf set of the bisection tree, every node is either inside
// one mesh triangle (a "coarse" triangle, leg^2 > s^2) or the union of the
// mesh triangles below it ("fine" triangles), and those are consecutive on
// the space-filling curve that the mesh keeps its triangles in.  The plan of
// a mesh therefore needs no sorting: one scan over the curve gives every
// node its covering triangle or its segment of the curve.
//
// The pass.  The image is laid out once per call as squares of s rows of
// s + 1 floats (fem_mesh::fsq; the extra column is the first pixel of the
// next square, which the last column of squares needs for the image's last
// column), so a square is one contiguous block of 4 s (s + 1) bytes.  Each
// warp of a persistent grid takes squares in turn, with two shared-memory
// buffers of its own: the next square is copied in by one bulk asynchronous
// copy (completion on an mbarrier) while the current one is processed, so
// the image is read from HBM once (plus the 1/s of the extra column) with
// many bytes in flight per SM, and no warp waits for another.  The image's
// last row is loaded by the last row of squares.  In a square:
//   * a square inside one triangle is summed as a dense block (lanes over
//     its columns);
//   * fine triangles with a bounding box of at most 17 x 17 pixels are summed
//     one per lane, walking their rows in shared memory;
//   * nodes inside coarse triangles (with the coarse triangle's plane) are
//     swept together over the square's full rows, and larger fine triangles
//     over their bounding box: lane r finds the span of row r, then the
//     lanes take the columns of each row;
//   * the sums of coarse triangles go to per-node slots, and k_sq_final adds
//     each coarse triangle's slots in a fixed order, one warp per triangle.
// Squares that hold only small triangles are left to k_sq_small (one thread
// per triangle along the curve, pixels from the squared image in global
// memory); the plan lists the other squares for k_sq.
// Every triangle's result is formed in a fixed order of operations, so the
// pass is deterministic.
//
// Two modes.  FAST: FP32 sums with a rigorous error interval (the fast keys
// of raster.cu: per-lane chains of at most kSqChain FP32 additions of
// non-negative terms, lanes added by an FP32 butterfly, nodes in
// float-float), planes from per-triangle records.  EXACT: float-float per
// pixel (the keys of the selection), over all triangles or only the
// selected ones (the band of the fast keys), on all squares or a list.
#include <algorithm>
#include <climits>

#include "fem_internal.cuh"
#include "ff.cuh"
#include "raster_common.cuh"
#include "scan.cuh"

namespace fem {

constexpr int kSqMax = 32;             // square side
// one staged square: s + 1 rows (with the image's last row) of s + 1 floats,
// rounded up to 16 bytes so that the second buffer starts aligned
constexpr int kSqBuf = ((kSqMax + 1) * (kSqMax + 1) + 3) / 4 * 4;
constexpr int kSqThreads = 128;        // four warps, each with its own squares
constexpr int kSqWarps = kSqThreads / 32;
// larger fine triangles of one square: a bounding box above 17 pixels means
// at least 81 pixels, so at most 1089 / 81 = 13
constexpr int kSqBigCap = 32;
// Longest FP32 addition chain of one lane in the FAST mode: a small triangle
// summed by one lane has at most 153 pixels; with the lanes over the columns
// a lane takes at most 2 pixels in each of at most 33 rows.  Lanes are
// combined in float-float.
constexpr float kSqChain = 153.0f + 7.0f;
constexpr unsigned long long kSqWaitLimitNs = 1000000000ull;

int sq_side(int N) { return std::min(N - 1, kSqMax); }

__device__ __forceinline__ TriGeom geom_xy(int2 a, int2 b, int2 c, int N) {
    TriGeom g;
    g.ax = a.x; g.ay = a.y; g.bx = b.x; g.by = b.y; g.cx = c.x; g.cy = c.y;
    int ytop = min(a.y, min(b.y, c.y)), ybot = max(a.y, max(b.y, c.y));
    g.ytop = ytop;
    g.yend = (ybot == N - 1) ? ybot : ybot - 1;
    g.maxw = max(a.x, max(b.x, c.x)) - min(a.x, min(b.x, c.x)) + 1;
    return g;
}

// the node's triangle: (a, b) its diagonal, c the right-angle corner
__device__ __forceinline__ void sq_node_tri(int n, const SqGeo& G, int2& a, int2& b, int2& c) {
    const int sq = n >> 1, h = n & 1, I = sq / G.Q, J = sq - I * G.Q;
    const int x0 = J * G.s, y0 = I * G.s, x1 = x0 + G.s, y1 = y0 + G.s;
    if (((I + J) & 1) == 0) {
        a = make_int2(x0, y0);
        b = make_int2(x1, y1);
        c = h == 0 ? make_int2(x0, y1) : make_int2(x1, y0);
    } else {
        a = make_int2(x1, y0);
        b = make_int2(x0, y1);
        c = h == 0 ? make_int2(x0, y0) : make_int2(x1, y1);
    }
}

// strictly inside the positively oriented triangle (a, b, c) (3x coordinates)
__device__ __forceinline__ bool inside3(long long px, long long py, int2 a, int2 b, int2 c) {
    const long long ax = 3LL * a.x, ay = 3LL * a.y, bx = 3LL * b.x, by = 3LL * b.y, cx = 3LL * c.x, cy = 3LL * c.y;
    const long long e0 = (bx - ax) * (py - ay) - (by - ay) * (px - ax);
    const long long e1 = (cx - bx) * (py - by) - (cy - by) * (px - bx);
    const long long e2 = (ax - cx) * (py - cy) - (ay - cy) * (px - cx);
    return e0 > 0 && e1 > 0 && e2 > 0;
}

// ------------------------------------------------------------------ plan
// Producer of the plan's scan over the curve: a fine triangle records its
// node and counts 0; a coarse one records -1 and counts the squares of its
// bounding box (its vertices lie on the square grid).
struct SqCountIn {
    const int* order;
    const int4* tri;
    const int2* vxy;
    SqGeo G;
    int* nodeof;
    int* pos;             // curve position of each triangle
    unsigned char* flag;  // squares that the staged pass takes (a fine triangle larger than small)
    __device__ __forceinline__ int operator()(long long i) const {
        const int t = order[i];
        pos[t] = (int)i;
        const int4 tr = tri[t];
        const int2 a = vxy[tr.x], b = vxy[tr.y], c = vxy[tr.z];
        if (leg2(a, c) <= (long long)G.s * G.s) {
            const int n = sq_node_at((long long)a.x + b.x + c.x, (long long)a.y + b.y + c.y, G);
            nodeof[i] = n;
            if (!is_small(geom_xy(a, b, c, G.N))) flag[n >> 1] = 1;
            return 0;
        }
        nodeof[i] = -1;
        const int w = max(a.x, max(b.x, c.x)) - min(a.x, min(b.x, c.x));
        const int h = max(a.y, max(b.y, c.y)) - min(a.y, min(b.y, c.y));
        return (w / G.s) * (h / G.s);
    }
};

// Node tables: a fine node gets its curve segment [start, end) and ncov =
// -1; a node inside a coarse triangle gets the triangle's curve position
// and its partial-sum slot 2w + h (w: the square's index among the coarse
// triangle's bounding-box squares).  Slots of bounding-box halves outside
// the triangle are zeroed, so a triangle's slots can be added unconditionally.
__global__ void k_sq_nodes(const int* __restrict__ order, const int4* __restrict__ tri, const int2* __restrict__ vxy,
                           const int* __restrict__ nodeof, const int* __restrict__ sqoff, const int* __restrict__ W_dev,
                           int T, SqGeo G, int* __restrict__ ncov, int2* __restrict__ nseg, int* __restrict__ nslot,
                           float4* __restrict__ partial, long long part_cap, int* __restrict__ err,
                           int* __restrict__ coarse, int* __restrict__ n_coarse, unsigned char* __restrict__ flag) {
    pdl_wait();
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    // every thread of the grid runs the same number of iterations of this
    // loop (the bound is rounded up to the grid), so the warp-aggregated
    // append below sees full warps
    const long long Tr = (T + stride - 1) / stride * stride;
    for (long long i = i0; i < Tr; i += stride) {
        const int n = i < T ? nodeof[i] : 0;
        const bool is_coarse = n < 0;
        const unsigned bal = __ballot_sync(0xffffffffu, is_coarse);
        int base = 0;
        if ((threadIdx.x & 31) == 0 && bal) base = atomicAdd(n_coarse, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (is_coarse) coarse[base + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u))] = (int)i;
        if (i >= T || n < 0) continue;
        if (i == 0 || nodeof[i - 1] != n) {
            nseg[n].x = (int)i;
            ncov[n] = -1;
        }
        if (i == T - 1 || nodeof[i + 1] != n) nseg[n].y = (int)i + 1;
    }
    const int W = *W_dev;
    if (2LL * W > part_cap) {
        // more bounding-box squares than a conforming mesh can have: nothing
        // is written past the slots, the call reports the mesh as invalid
        if (i0 == 0) atomicCAS(err, 0, (int)FEM_E_INVALID);
        return;
    }
    for (long long w = i0; w < W; w += stride) {
        // the coarse triangle whose bounding-box squares hold w: the last
        // curve position c with sqoff[c] <= w
        int lo = 0, hi = T;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (sqoff[mid] <= w) lo = mid; else hi = mid;
        }
        const int c = lo;
        const int4 tr = tri[order[c]];
        const int2 a = vxy[tr.x], b = vxy[tr.y], cc = vxy[tr.z];
        const int xmin = min(a.x, min(b.x, cc.x)), xmax = max(a.x, max(b.x, cc.x));
        const int ymin = min(a.y, min(b.y, cc.y));
        const int bw = (xmax - xmin) / G.s;
        const int j = (int)(w - sqoff[c]);
        const int I = ymin / G.s + j / bw, J = xmin / G.s + j % bw;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int n = ((I * G.Q + J) << 1) | h;
            int2 na, nb, nc;
            sq_node_tri(n, G, na, nb, nc);
            if (inside3((long long)na.x + nb.x + nc.x, (long long)na.y + nb.y + nc.y, a, b, cc)) {
                ncov[n] = c;
                nslot[n] = (int)(2 * w + h);
                flag[n >> 1] = 1;
            } else {
                partial[2 * w + h] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    }
}

// ------------------------------------------------------------------ pass
enum SqMode { SQ_FAST = 0, SQ_EXACT = 1 };

struct SqArgs {
    const float* fsq;   // Q*Q squares of s rows of s + 1 floats
    const float* frow;  // N floats: the image's last row
    SqGeo G;
    const int* order;
    const int4* tri;
    const int2* vxy;
    const double* uv;
    const float2* uvf;
    const int* ncov;
    const int2* nseg;
    const int* nslot;
    const int* sqoff;
    const SqRec* rec;           // SQ_FAST: fine-triangle records by curve position
    float4* partial;
    long long part_cap;         // slots in partial
    FastOut F;                  // SQ_FAST: intervals and histograms
    double* keys;               // SQ_EXACT: keys
    unsigned long long* keyc;   // SQ_EXACT: composite selection keys, or null
    const unsigned char* sel;   // SQ_EXACT: only triangles with sel[t] != 0 (null: all)
    const int* sq_list;         // squares to process (null: all Q*Q)
    const int* n_sq;            // their number (device)
    int* err;
};

struct SqPlane {
    ff uc, gx, gy;
    float ucf, gxf, gyf;
};

__device__ __forceinline__ SqPlane sq_plane(const TriGeom& g, int4 tr, const double* uv, const float2* uvf) {
    SqPlane p;
    tri_plane(g, tr, uv, uvf, p.uc, p.gx, p.gy);
    p.ucf = __fadd_rn(p.uc.hi, p.uc.lo);
    p.gxf = __fadd_rn(p.gx.hi, p.gx.lo);
    p.gyf = __fadd_rn(p.gy.hi, p.gy.lo);
    return p;
}

template <int MODE>
__device__ __forceinline__ bool sq_want(const SqArgs& A, int t) {
    return MODE == SQ_FAST || !A.sel || A.sel[t];
}

// the selection key of an eligible triangle (flag bit over the FP64 key bits)
__device__ __forceinline__ unsigned long long sq_keyc(const TriGeom& g, double key) {
    return tri_eligible(g) ? ((unsigned long long)__double_as_longlong(key) | (1ull << 63)) : 0ull;
}

// FAST: interval and histogram of triangle t from its sum S and pixel
// count; EXACT: key.  One thread.
template <int MODE>
__device__ __forceinline__ void sq_finish(const SqArgs& A, int t, const TriGeom& g, const SqPlane& P, ff S, long long n) {
    if (MODE == SQ_FAST) {
        float lo, hi;
        fast_interval(S, (float)n, fast_M(g, P.ucf, P.gxf, P.gyf), kSqChain, lo, hi);
        A.F.lo[t] = lo;
        A.F.hi[t] = hi;
        if (tri_eligible(g)) {
            atomicAdd(A.F.hlo + fast_bin(lo), 1u);
            atomicAdd(A.F.hhi + fast_bin(hi), 1u);
        }
    } else {
        const double key = ff_to_double(S);
        A.keys[t] = key;
        if (A.keyc) A.keyc[t] = sq_keyc(g, key);
    }
}

// One lane, one small fine triangle, pixels from the staged square.  Along a
// row u = g_x k + u_row is evaluated afresh per pixel (FAST; k counted in
// floats, exact) or advanced by the exact float-float g_x (EXACT).  FAST
// returns the histogram bins (0xffffffff: none) for warp aggregation.
template <int MODE>
__device__ __forceinline__ void sq_small(const SqArgs& A, const float* img, int x0, int y0, int pitch, int t,
                                         const TriGeom& g, const SqPlane& P, unsigned& blo, unsigned& bhi) {
    const int N = A.G.N;
    if (MODE == SQ_FAST) {
        float acc = 0.f;
        int n = 0;
        for (int y = g.ytop; y <= g.yend; ++y) {
            int L, len;
            row_span(g, y, N, L, len);
            if (len <= 0) continue;
            const float* rowp = img + (y - y0) * pitch + (L - x0);
            const float urow = fmaf(P.gyf, (float)(y - g.cy), fmaf(P.gxf, (float)(L - g.cx), P.ucf));
            float fk = 0.f;
#pragma unroll 4
            for (int k = 0; k < len; ++k) {
                const float d = fmaf(P.gxf, fk, urow) - rowp[k];
                acc = fmaf(d, d, acc);
                fk += 1.0f;
            }
            n += len;
        }
        float lo, hi;
        fast_interval(ff{acc, 0.f}, (float)n, fast_M(g, P.ucf, P.gxf, P.gyf), kSqChain, lo, hi);
        A.F.lo[t] = lo;
        A.F.hi[t] = hi;
        if (tri_eligible(g)) {
            blo = fast_bin(lo);
            bhi = fast_bin(hi);
        }
    } else {
        ff acc{0.f, 0.f};
        for (int y = g.ytop; y <= g.yend; ++y) {
            int L, len;
            row_span(g, y, N, L, len);
            if (len <= 0) continue;
            const float* rowp = img + (y - y0) * pitch + (L - x0);
            ff u = ff_add(ff_add(P.uc, ff_mul_f(P.gx, (float)(L - g.cx))), ff_mul_f(P.gy, (float)(y - g.cy)));
#pragma unroll 4
            for (int k = 0; k < len; ++k) {
                const ff d = ff_add_f(u, -rowp[k]);
                acc = ff_add(acc, ff_sqr(d));
                u = ff_add(u, P.gx);
            }
        }
        const double key = ff_to_double(acc);
        A.keys[t] = key;
        if (A.keyc) A.keyc[t] = sq_keyc(g, key);
    }
}

// The warp's sum of the lanes' sums: FAST adds the FP32 sums by a butterfly
// (five more additions in each lane's chain, within kSqChain), EXACT the
// float-float sums.  Every lane returns the same value.
template <int MODE>
__device__ __forceinline__ ff sq_warp_total(float accf, ff acc) {
    if (MODE == SQ_FAST) return ff{warp_sum(accf), 0.f};
    return ff_warp_sum(acc);
}

// Row spans of region g for a sweep of up to 33 rows from row y (the first
// row of the sweep): lane r holds the span of row y + r, lane 0 also of row
// y + 32; rows outside the region's rows get an empty span.
__device__ __forceinline__ void sq_spans(const TriGeom& g, int y, int R, int N, int& La, int& na, int& Lb, int& nb) {
    const int lane = threadIdx.x & 31;
    La = 0; na = 0; Lb = 0; nb = 0;
    const int ya = y + lane, yb = y + 32;
    if (lane < R && ya >= g.ytop && ya <= g.yend) row_span(g, ya, N, La, na);
    if (lane == 0 && R > 32 && yb >= g.ytop && yb <= g.yend) row_span(g, yb, N, Lb, nb);
}

// A pixel's contribution: FAST adds d^2 to an FP32 sum, EXACT to a float-float
// sum (u from the float-float plane, urow = u_c + g_y dy).
template <int MODE>
__device__ __forceinline__ void sq_px(const SqPlane& P, float fx, float urowf, const ff& urow, float v, float& accf,
                                      ff& acc) {
    if (MODE == SQ_FAST) {
        const float d = fmaf(P.gxf, fx, urowf) - v;
        accf = fmaf(d, d, accf);
    } else {
        acc = ff_add(acc, ff_sqr(ff_add_f(ff_add(urow, ff_mul_f(P.gx, fx)), -v)));
    }
}

// The coarse nodes of a square in one sweep over its w x h staged pixels,
// lanes over the columns.  A pixel belongs to node 0 when it lies in node
// 0's span of its row (g0), else to node 1; node j is summed when want_j,
// with plane Pj of a triangle with right-angle corner (cxj, cyj).  Returns
// the two sums (every lane) and node 0's pixel count.
template <int MODE>
__device__ __forceinline__ void sq_sweep2(const TriGeom& g0, bool want0, const SqPlane& P0, int cx0, int cy0,
                                          bool want1, const SqPlane& P1, int cx1, int cy1, const float* img, int x0,
                                          int y0, int w, int h, int pitch, int N, ff& S0, ff& S1, long long& n0) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int La, na, Lb, nb;
    sq_spans(g0, y0, h, N, La, na, Lb, nb);
    n0 = (long long)warp_sum(na) + __shfl_sync(FULL, nb, 0);
    const bool two = lane + 32 < w, one = lane < w;
    const int xa = x0 + lane, xb = xa + 32;
    const float f0a = (float)(xa - cx0), f0b = f0a + 32.0f, f1a = (float)(xa - cx1), f1b = f1a + 32.0f;
    float fy0 = (float)(y0 - cy0), fy1 = (float)(y0 - cy1);
    float a0 = 0.f, a1 = 0.f;
    ff e0{0.f, 0.f}, e1{0.f, 0.f};
    for (int r = 0; r < h; ++r) {
        // rows 0..31 take their span from lane r, row 32 from lane 0's second
        const int src = r < 32 ? r : 0;
        const int L = __shfl_sync(FULL, r < 32 ? La : Lb, src);
        const int n = __shfl_sync(FULL, r < 32 ? na : nb, src);
        const float* rowp = img + r * pitch;
        const float u0f = fmaf(P0.gyf, fy0, P0.ucf), u1f = fmaf(P1.gyf, fy1, P1.ucf);
        ff u0{0.f, 0.f}, u1{0.f, 0.f};
        if (MODE == SQ_EXACT) {
            u0 = ff_add(P0.uc, ff_mul_f(P0.gy, fy0));
            u1 = ff_add(P1.uc, ff_mul_f(P1.gy, fy1));
        }
        if (one) {
            const bool in0 = (unsigned)(xa - L) < (unsigned)n;
            if (in0 ? want0 : want1) {
                if (in0) sq_px<MODE>(P0, f0a, u0f, u0, rowp[lane], a0, e0);
                else sq_px<MODE>(P1, f1a, u1f, u1, rowp[lane], a1, e1);
            }
        }
        if (two) {
            const bool in0 = (unsigned)(xb - L) < (unsigned)n;
            if (in0 ? want0 : want1) {
                if (in0) sq_px<MODE>(P0, f0b, u0f, u0, rowp[lane + 32], a0, e0);
                else sq_px<MODE>(P1, f1b, u1f, u1, rowp[lane + 32], a1, e1);
            }
        }
        fy0 += 1.0f;
        fy1 += 1.0f;
    }
    S0 = sq_warp_total<MODE>(a0, e0);
    S1 = sq_warp_total<MODE>(a1, e1);
}

// A larger fine triangle over its bounding box (at most 33 x 33 pixels of the
// staged square), lanes over the columns, each pixel tested against its
// row's span.  Returns the warp's sum (every lane) and the pixel count.
template <int MODE>
__device__ __forceinline__ ff sq_bbox(const TriGeom& g, const SqPlane& P, const float* img, int x0, int y0, int pitch,
                                      int N, long long& npix) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int R = g.yend - g.ytop + 1;
    int La, na, Lb, nb;
    sq_spans(g, g.ytop, R, N, La, na, Lb, nb);
    npix = (long long)warp_sum(na) + __shfl_sync(FULL, nb, 0);
    const int xmin = min(g.ax, min(g.bx, g.cx));
    const bool two = lane + 32 < g.maxw, one = lane < g.maxw;
    const int xa = xmin + lane, xb = xa + 32;
    const float fa = (float)(xa - g.cx), fb = fa + 32.0f;
    float fy = (float)(g.ytop - g.cy);
    float af = 0.f;
    ff e{0.f, 0.f};
    for (int r = 0; r < R; ++r) {
        const int src = r < 32 ? r : 0;
        const int L = __shfl_sync(FULL, r < 32 ? La : Lb, src);
        const int n = __shfl_sync(FULL, r < 32 ? na : nb, src);
        const float* rowp = img + (g.ytop + r - y0) * pitch - x0;
        const float uf = fmaf(P.gyf, fy, P.ucf);
        ff u{0.f, 0.f};
        if (MODE == SQ_EXACT) u = ff_add(P.uc, ff_mul_f(P.gy, fy));
        if (one && (unsigned)(xa - L) < (unsigned)n) sq_px<MODE>(P, fa, uf, u, rowp[xa], af, e);
        if (two && (unsigned)(xb - L) < (unsigned)n) sq_px<MODE>(P, fb, uf, u, rowp[xb], af, e);
        fy += 1.0f;
    }
    return sq_warp_total<MODE>(af, e);
}

// A square inside one triangle: every staged pixel, lanes over columns.
template <int MODE>
__device__ __forceinline__ ff sq_full(const SqPlane& P, int pcx, int pcy, const float* img, int x0, int y0, int w,
                                      int h, int pitch) {
    const int lane = threadIdx.x & 31;
    const float fxa = (float)(x0 + lane - pcx), fxb = fxa + 32.0f;
    const bool two = lane + 32 < w;
    float accf = 0.f;
    ff acc{0.f, 0.f};
    ff gxa{0.f, 0.f}, gxb{0.f, 0.f};
    if (MODE == SQ_EXACT) {
        gxa = ff_mul_f(P.gx, fxa);
        gxb = ff_mul_f(P.gx, fxb);
    }
    float dy = (float)(y0 - pcy);
    for (int r = 0; r < h; ++r, dy += 1.0f) {
        const float* rowp = img + r * pitch;
        if (MODE == SQ_FAST) {
            const float urow = fmaf(P.gyf, dy, P.ucf);
            if (lane < w) {
                const float d = fmaf(P.gxf, fxa, urow) - rowp[lane];
                accf = fmaf(d, d, accf);
            }
            if (two) {
                const float d = fmaf(P.gxf, fxb, urow) - rowp[lane + 32];
                accf = fmaf(d, d, accf);
            }
        } else {
            const ff urow = ff_add(P.uc, ff_mul_f(P.gy, dy));
            if (lane < w) acc = ff_add(acc, ff_sqr(ff_add_f(ff_add(urow, gxa), -rowp[lane])));
            if (two) acc = ff_add(acc, ff_sqr(ff_add_f(ff_add(urow, gxb), -rowp[lane + 32])));
        }
    }
    return sq_warp_total<MODE>(accf, acc);
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// bounded wait for the phase with the given parity; false when the limit ran out
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    const unsigned addr = smem_u32(bar);
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
        if (globaltimer_ns() - t0 > kSqWaitLimitNs) return false;
    }
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* bar,
                                          unsigned long long policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// Issue the copy of square q into buffer `img` (one lane).  A bulk copy
// needs a size that is a multiple of 16 bytes: 4 s (s + 1) is for s >= 4;
// smaller images are loaded by the warp when the square is processed.
__device__ __forceinline__ void sq_issue(const SqArgs& A, int q, float* img, unsigned long long* bar,
                                         unsigned long long policy) {
    const int s = A.G.s;
    const unsigned bytes = (unsigned)(4 * s * (s + 1));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, bytes);
    bulk_copy(img, A.fsq + (long long)q * s * (s + 1), bytes, bar, policy);
}

// The records of the triangles for the FP32 pass, one thread per curve
// position; all gathers of the pass happen here, in a fully parallel kernel,
// and the pass reads each square's records contiguously (fine triangles) or
// one record per covered node (coarse ones).
__global__ void k_sq_records(const int* __restrict__ order, const int4* __restrict__ tri, const int2* __restrict__ vxy,
                             const double* __restrict__ uv, const float2* __restrict__ uvf,
                             const int* __restrict__ nodeof, int T, int N, SqRec* __restrict__ rec) {
    pdl_wait();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T; i += gridDim.x * blockDim.x) {
        const int t = order[i];
        const int4 tr = tri[t];
        const TriGeom g = tri_geom(tr, vxy, N);
        ff uc, gx, gy;
        tri_plane(g, tr, uv, uvf, uc, gx, gy);
        SqRec r;
        r.ax = (unsigned short)g.ax; r.ay = (unsigned short)g.ay;
        r.bx = (unsigned short)g.bx; r.by = (unsigned short)g.by;
        r.cx = (unsigned short)g.cx; r.cy = (unsigned short)g.cy;
        r.t = t;
        r.ucf = __fadd_rn(uc.hi, uc.lo);
        r.gxf = __fadd_rn(gx.hi, gx.lo);
        r.gyf = __fadd_rn(gy.hi, gy.lo);
        r.pad = 0.f;
        rec[i] = r;
    }
}

// Squares for the staged pass: those flagged by the plan (a node inside a
// coarse triangle, or a fine triangle larger than small); staged[q] records
// the decision for the small-triangle kernel, and the flags are cleared.
__global__ void k_sq_stage_list(int nsq, unsigned char* __restrict__ flag, unsigned char* __restrict__ staged,
                                int* __restrict__ list, int* __restrict__ n_list) {
    pdl_wait();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    bool on = false;
    if (q < nsq) {
        on = flag[q] != 0;
        flag[q] = 0;
        staged[q] = on ? 1 : 0;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, on);
    int base = 0;
    if ((threadIdx.x & 31) == 0 && bal) base = atomicAdd(n_list, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (on) list[base + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u))] = q;
}

__device__ __forceinline__ TriGeom rec_geom(const SqRec& r, int N) {
    return geom_xy(make_int2(r.ax, r.ay), make_int2(r.bx, r.by), make_int2(r.cx, r.cy), N);
}

__device__ __forceinline__ SqPlane rec_plane(const SqRec& r) {
    SqPlane P{};
    P.ucf = r.ucf;
    P.gxf = r.gxf;
    P.gyf = r.gyf;
    return P;
}

// The FP32 pass over the squares that hold only small triangles: one thread
// per triangle along the curve (neighbouring threads read neighbouring
// pixels), each walking its rows in the image laid out in squares (global
// memory).  The triangles of staged squares are left to k_sq.
__global__ void __launch_bounds__(256) k_sq_small(const SqRec* __restrict__ rec, const int* __restrict__ nodeof,
                                                  const unsigned char* __restrict__ staged, int T, SqGeo G,
                                                  const float* __restrict__ fsq, const float* __restrict__ frow,
                                                  FastOut F) {
    pdl_wait();
    const int N = G.N, s = G.s, Q = G.Q, pitch = s + 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T; i += gridDim.x * blockDim.x) {
        const int n = nodeof[i];
        unsigned blo = 0xffffffffu, bhi = 0xffffffffu;
        if (n >= 0 && !staged[n >> 1]) {
            const SqRec R = rec[i];
            const TriGeom g = rec_geom(R, N);
            const int q = n >> 1, I = q / Q, J = q - I * Q;
            const int x0 = J * s, y0 = I * s;
            const float* sqp = fsq + (long long)q * s * pitch;
            float acc = 0.f;
            int cnt = 0;
            for (int y = g.ytop; y <= g.yend; ++y) {
                int L, len;
                row_span(g, y, N, L, len);
                if (len <= 0) continue;
                // rows of the square, or the image's last row
                const float* rowp = (y - y0 < s ? sqp + (y - y0) * pitch - x0 : frow) + L;
                const float urow = fmaf(R.gyf, (float)(y - g.cy), fmaf(R.gxf, (float)(L - g.cx), R.ucf));
                float fk = 0.f;
#pragma unroll 4
                for (int k = 0; k < len; ++k) {
                    const float d = fmaf(R.gxf, fk, urow) - rowp[k];
                    acc = fmaf(d, d, acc);
                    fk += 1.0f;
                }
                cnt += len;
            }
            float lo, hi;
            fast_interval(ff{acc, 0.f}, (float)cnt, fast_M(g, R.ucf, R.gxf, R.gyf), kSqChain, lo, hi);
            F.lo[R.t] = lo;
            F.hi[R.t] = hi;
            if (tri_eligible(g)) {
                blo = fast_bin(lo);
                bhi = fast_bin(hi);
            }
        }
        // histogram: one atomic per distinct bin among the converged lanes
        const unsigned act = __activemask();
        unsigned peers = __match_any_sync(act, blo);
        if (blo != 0xffffffffu && (__ffs(peers) - 1) == (int)(threadIdx.x & 31))
            atomicAdd(F.hlo + blo, (unsigned)__popc(peers));
        peers = __match_any_sync(act, bhi);
        if (bhi != 0xffffffffu && (__ffs(peers) - 1) == (int)(threadIdx.x & 31))
            atomicAdd(F.hhi + bhi, (unsigned)__popc(peers));
    }
}

// The plane and right-angle corner of the triangle at curve position c:
// FAST from its record, EXACT from the mesh (float-float plane).
template <int MODE>
__device__ __forceinline__ void sq_plane_at(const SqArgs& A, int c, int t, SqPlane& P, int& cx, int& cy) {
    if (MODE == SQ_FAST) {
        const SqRec R = A.rec[c];
        P = rec_plane(R);
        cx = R.cx;
        cy = R.cy;
    } else {
        const int4 tr = A.tri[t];
        const TriGeom gt = tri_geom(tr, A.vxy, A.G.N);
        P = sq_plane(gt, tr, A.uv, A.uvf);
        cx = gt.cx;
        cy = gt.cy;
    }
}

// Warp w of the grid takes squares w, w + W, ... (W warps); each warp stages
// its next square while it works on the current one, with its own two
// buffers and mbarriers, so warps never wait for one another.
template <int MODE>
__global__ void __launch_bounds__(kSqThreads) k_sq(SqArgs A) {
    pdl_wait();
    __shared__ __align__(128) float s_img[kSqWarps][2][kSqBuf];
    __shared__ __align__(8) unsigned long long s_bar[kSqWarps][2];
    __shared__ int s_big[kSqWarps][kSqBigCap];
    __shared__ int s_nbig[kSqWarps];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    const int gw = blockIdx.x * kSqWarps + wb, nw = gridDim.x * kSqWarps;
    const SqGeo G = A.G;
    const int N = G.N, s = G.s, Q = G.Q, pitch = s + 1;
    const bool bulk = s >= 4;
    const int nsq = A.sq_list ? *A.n_sq : Q * Q;
    unsigned long long* bar = s_bar[wb];
    unsigned long long policy = 0;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (bulk && lane == 0 && gw < nsq) sq_issue(A, A.sq_list ? A.sq_list[gw] : gw, s_img[wb][0], &bar[0], policy);
    unsigned phases = 0u;  // bit b: parity of buffer b's next phase
    int it = 0;
    for (int k = gw; k < nsq; k += nw, ++it) {
        const int b = it & 1;
        const int q = A.sq_list ? A.sq_list[k] : k;
        const int kn = k + nw;
        if (bulk && lane == 0 && kn < nsq)
            sq_issue(A, A.sq_list ? A.sq_list[kn] : kn, s_img[wb][b ^ 1], &bar[b ^ 1], policy);
        float* img = s_img[wb][b];
        const int I = q / Q, J = q - I * Q;
        const int x0 = J * s, y0 = I * s;
        if (!bulk)
            for (int e = lane; e < s * pitch; e += 32) img[e] = A.fsq[(long long)q * s * pitch + e];
        // the image's last row belongs to the last row of squares
        if (I == Q - 1)
            for (int c = lane; c <= s; c += 32) img[s * pitch + c] = A.frow[x0 + c];
        if (bulk) {
            const bool ok = mbar_wait(&bar[b], (phases >> b) & 1u);
            phases ^= 1u << b;
            if (__any_sync(FULL, !ok)) {
                // a copy never completed: wait (bounded) for the other
                // buffer's copy in flight, then stop
                if (lane == 0) atomicCAS(A.err, 0, (int)FEM_E_TIMEOUT);
                if (kn < nsq) mbar_wait(&bar[b ^ 1], (phases >> (b ^ 1)) & 1u);
                return;
            }
        }
        __syncwarp();
        const int n0 = q << 1;
        const int c0 = A.ncov[n0], c1 = A.ncov[n0 + 1];
        if (c0 >= 0 && c0 == c1) {
            // the whole square lies in one triangle
            const int t = MODE == SQ_FAST ? -1 : A.order[c0];
            if (MODE == SQ_FAST || sq_want<MODE>(A, t)) {
                SqPlane P;
                int cx, cy;
                sq_plane_at<MODE>(A, c0, t, P, cx, cy);
                const int w = s + (J == Q - 1 ? 1 : 0), h = s + (I == Q - 1 ? 1 : 0);
                const ff S = sq_full<MODE>(P, cx, cy, img, x0, y0, w, h, pitch);
                if (lane == 0) {
                    const int s0 = A.nslot[n0], s1 = A.nslot[n0 + 1];
                    if (s0 >= 0 && s0 < A.part_cap) A.partial[s0] = make_float4(S.hi, S.lo, __int_as_float(w * h), 0.f);
                    if (s1 >= 0 && s1 < A.part_cap) A.partial[s1] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        } else {
            // nodes inside coarse triangles: one sweep over the square
            const int t0 = c0 >= 0 && MODE == SQ_EXACT ? A.order[c0] : -1;
            const int t1 = c1 >= 0 && MODE == SQ_EXACT ? A.order[c1] : -1;
            const bool want0 = c0 >= 0 && (MODE == SQ_FAST || sq_want<MODE>(A, t0));
            const bool want1 = c1 >= 0 && (MODE == SQ_FAST || sq_want<MODE>(A, t1));
            if (want0 || want1) {
                SqPlane P0{}, P1{};
                int cx0 = 0, cy0 = 0, cx1 = 0, cy1 = 0;
                if (want0) sq_plane_at<MODE>(A, c0, t0, P0, cx0, cy0);
                if (want1) sq_plane_at<MODE>(A, c1, t1, P1, cx1, cy1);
                int2 na, nb, nc;
                sq_node_tri(n0, G, na, nb, nc);
                const int w = s + (J == Q - 1 ? 1 : 0), h = s + (I == Q - 1 ? 1 : 0);
                ff S0, S1;
                long long np0 = 0;
                sq_sweep2<MODE>(geom_xy(na, nb, nc, N), want0, P0, cx0, cy0, want1, P1, cx1, cy1, img, x0, y0, w, h,
                                pitch, N, S0, S1, np0);
                if (lane == 0) {
                    const int s0 = A.nslot[n0], s1 = A.nslot[n0 + 1];
                    if (want0 && s0 >= 0 && s0 < A.part_cap)
                        A.partial[s0] = make_float4(S0.hi, S0.lo, __int_as_float((int)np0), 0.f);
                    if (want1 && s1 >= 0 && s1 < A.part_cap)
                        A.partial[s1] = make_float4(S1.hi, S1.lo, __int_as_float(w * h - (int)np0), 0.f);
                }
            }
            // fine triangles: small ones by one lane each, larger ones listed
            const int2 sg0 = A.nseg[n0], sg1 = A.nseg[n0 + 1];
            const int len0 = c0 < 0 ? sg0.y - sg0.x : 0, len1 = c1 < 0 ? sg1.y - sg1.x : 0;
            if (lane == 0) s_nbig[wb] = 0;
            __syncwarp();
            for (int e = lane; e < len0 + len1; e += 32) {
                const int c = e < len0 ? sg0.x + e : sg1.x + (e - len0);
                unsigned blo = 0xffffffffu, bhi = 0xffffffffu;
                bool big = false;
                if (MODE == SQ_FAST) {
                    const SqRec R = A.rec[c];
                    const TriGeom g = rec_geom(R, N);
                    if (is_small(g)) sq_small<MODE>(A, img, x0, y0, pitch, R.t, g, rec_plane(R), blo, bhi);
                    else big = true;
                } else {
                    const int t = A.order[c];
                    if (sq_want<MODE>(A, t)) {
                        const int4 tr = A.tri[t];
                        const TriGeom g = tri_geom(tr, A.vxy, N);
                        if (is_small(g)) sq_small<MODE>(A, img, x0, y0, pitch, t, g, sq_plane(g, tr, A.uv, A.uvf), blo, bhi);
                        else big = true;
                    }
                }
                if (big) {
                    // listed by curve position
                    const int slot = atomicAdd(&s_nbig[wb], 1);
                    if (slot < kSqBigCap) s_big[wb][slot] = c;
                    else atomicCAS(A.err, 0, (int)FEM_E_INVALID);
                }
                if (MODE == SQ_FAST) {
                    // histogram: one atomic per distinct bin among the converged lanes
                    const unsigned act = __activemask();
                    unsigned peers = __match_any_sync(act, blo);
                    if (blo != 0xffffffffu && (__ffs(peers) - 1) == lane) atomicAdd(A.F.hlo + blo, (unsigned)__popc(peers));
                    peers = __match_any_sync(act, bhi);
                    if (bhi != 0xffffffffu && (__ffs(peers) - 1) == lane) atomicAdd(A.F.hhi + bhi, (unsigned)__popc(peers));
                }
            }
            __syncwarp();
            const int nbig = min(s_nbig[wb], kSqBigCap);
            for (int e = 0; e < nbig; ++e) {
                const int c = s_big[wb][e];
                int t;
                TriGeom g;
                SqPlane P;
                if (MODE == SQ_FAST) {
                    const SqRec R = A.rec[c];
                    t = R.t;
                    g = rec_geom(R, N);
                    P = rec_plane(R);
                } else {
                    t = A.order[c];
                    const int4 tr = A.tri[t];
                    g = tri_geom(tr, A.vxy, N);
                    P = sq_plane(g, tr, A.uv, A.uvf);
                }
                long long np = 0;
                const ff S = sq_bbox<MODE>(g, P, img, x0, y0, pitch, N, np);
                if (lane == 0) sq_finish<MODE>(A, t, g, P, S, np);
            }
        }
        __syncwarp();
    }
}

// The coarse triangles: one warp each adds the triangle's node slots (all
// of its bounding-box slots; those outside it hold zero) in a fixed order
// and finishes its interval (FAST) or key (EXACT).  coarse[0 .. *n_coarse)
// are curve positions; many warps in flight hide the loads of each.
template <int MODE>
__global__ void __launch_bounds__(256) k_sq_final(SqArgs A, const int* __restrict__ coarse,
                                                  const int* __restrict__ n_coarse) {
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    const int n = *n_coarse;
    const int s = A.G.s;
    for (int k = gw; k < n; k += nw) {
        const int c = coarse[k];
        int t;
        TriGeom gt;
        int4 tr = make_int4(0, 0, 0, 0);
        SqRec R{};
        if (MODE == SQ_FAST) {
            R = A.rec[c];
            t = R.t;
            gt = rec_geom(R, A.G.N);
        } else {
            t = A.order[c];
            if (A.sel && !A.sel[t]) continue;  // the same for the whole warp
            tr = A.tri[t];
            gt = tri_geom(tr, A.vxy, A.G.N);
        }
        const int w = (gt.maxw - 1) / s, h = (max(gt.ay, max(gt.by, gt.cy)) - gt.ytop) / s;
        const long long o = 2LL * A.sqoff[c];
        const long long cnt = o + 2LL * w * h <= A.part_cap ? 2LL * w * h : 0;
        ff S{0.f, 0.f};
        int np = 0;
        // four independent loads in flight per lane, added in a fixed order
        for (long long e0 = lane; e0 < cnt; e0 += 4 * 32) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long e = e0 + 32LL * u;
                v[u] = e < cnt ? A.partial[o + e] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                S = ff_add(S, ff{v[u].x, v[u].y});
                np += __float_as_int(v[u].z);
            }
        }
        S = ff_warp_sum(S);
        np = warp_sum(np);
        if (lane == 0) sq_finish<MODE>(A, t, gt, MODE == SQ_FAST ? rec_plane(R) : sq_plane(gt, tr, A.uv, A.uvf), S, np);
    }
}

// The image as squares of s rows of s + 1 floats (row r of square (I, J):
// pixels x0 .. x0 + s of image row y0 + r), plus the image's last row.
__global__ void k_sq_image(const float* __restrict__ f, int N, SqGeo G, float* __restrict__ fsq,
                           float* __restrict__ frow) {
    pdl_wait();
    const int s = G.s, w = s + 1;
    const long long n = (long long)G.Q * G.Q * s * w;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n + N;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < n) {
            const long long q = e / ((long long)s * w);
            const int r = (int)((e / w) % s), c = (int)(e % w);
            const int I = (int)(q / G.Q), J = (int)(q % G.Q);
            fsq[e] = f[(long long)(I * s + r) * N + J * s + c];
        } else {
            const int x = (int)(e - n);
            frow[x] = f[(long long)(N - 1) * N + x];
        }
    }
}

// ------------------------------------------------------------------ host
SqGeo sq_geo(const fem_mesh* m) {
    SqGeo G;
    G.N = m->N;
    G.s = sq_side(m->N);
    G.Q = (m->N - 1) / G.s;
    return G;
}

fem_status sq_image(fem_mesh* m, const float* f, cudaStream_t s) {
    const SqGeo G = sq_geo(m);
    const long long n = (long long)G.Q * G.Q * G.s * (G.s + 1);
    FEM_TRY(ensure(m->fsq, (size_t)n, s));
    FEM_TRY(ensure(m->fedge, (size_t)m->N, s));
    const long long work = n + m->N;
    const int grid = (int)std::min<long long>((work + 255) / 256, (long long)m->num_sms * 16);
    note_bytes(F_RASTER, 8.0 * (double)work);
    FEM_LAUNCH(F_RASTER, s, k_sq_image, grid, 256, 0, f, m->N, G, m->fsq.p, m->fedge.p);
    return FEM_OK;
}

fem_status sq_plan(fem_mesh* m, cudaStream_t s) {
    if (m->sq_plan_version == m->mesh_version) return FEM_OK;
    const SqGeo G = sq_geo(m);
    const int T = m->T;
    const size_t nodes = (size_t)2 * G.Q * G.Q;
    FEM_TRY(ensure(m->sq_nodeof, (size_t)T, s));
    FEM_TRY(ensure(m->sq_off, (size_t)T + 1, s));
    FEM_TRY(ensure(m->sq_cov, nodes, s));
    FEM_TRY(ensure(m->sq_seg, nodes, s));
    FEM_TRY(ensure(m->sq_slot, nodes, s));
    // bounding-box squares of the coarse triangles: at most twice their
    // area each, so at most 2 Q^2 in all; two slots per square
    FEM_TRY(ensure(m->sq_part, (size_t)4 * G.Q * G.Q + 8, s));
    FEM_TRY(ensure(m->sq_coarse, (size_t)T, s));
    FEM_TRY(ensure(m->sq_ctr, 8, s));
    const int nsq = G.Q * G.Q;
    FEM_TRY(ensure(m->sq_stage, (size_t)nsq, s));
    FEM_TRY(ensure(m->sq_staged, (size_t)nsq, s));
    if (!m->sq_flag.p || m->sq_flag.n < (size_t)nsq) {
        FEM_TRY(ensure(m->sq_flag, (size_t)nsq, s));
        FEM_CUDA(cudaMemsetAsync(m->sq_flag.p, 0, m->sq_flag.n, s));  // cleared by each plan's stage list after
    }
    int* W = m->sq_ctr.p + 0;         // bounding-box squares of the coarse triangles
    int* n_coarse = m->sq_ctr.p + 1;  // coarse triangles listed
    FEM_CUDA(cudaMemsetAsync(n_coarse, 0, sizeof(int), s));
    // nodes that no triangle claims (only in a mesh with holes) read as
    // fine with an empty segment
    FEM_CUDA(cudaMemsetAsync(m->sq_cov.p, 0xff, sizeof(int) * nodes, s));
    FEM_CUDA(cudaMemsetAsync(m->sq_seg.p, 0xff, sizeof(int2) * nodes, s));
    FEM_TRY(ensure(m->sq_pos, (size_t)T, s));
    FEM_TRY(scan_fused(m, SqCountIn{m->order.p, m->tri.p, m->vxy.p, G, m->sq_nodeof.p, m->sq_pos.p, m->sq_flag.p},
                       ScanStore{m->sq_off.p}, T, s, W, F_RASTER));
    // work: T curve positions, then at most 2 Q^2 bounding-box squares
    const long long work = std::max<long long>(T, 2LL * G.Q * G.Q);
    const int grid = (int)std::max<long long>(1, std::min<long long>((work + 255) / 256, (long long)m->num_sms * 8));
    FEM_LAUNCH(F_RASTER, s, k_sq_nodes, grid, 256, 0, m->order.p, m->tri.p, m->vxy.p, (const int*)m->sq_nodeof.p,
               (const int*)m->sq_off.p, (const int*)W, T, G, m->sq_cov.p, m->sq_seg.p, m->sq_slot.p, m->sq_part.p,
               (long long)m->sq_part.n, m->dflag.p + 0, m->sq_coarse.p, n_coarse, m->sq_flag.p);
    FEM_CUDA(cudaMemsetAsync(m->sq_ctr.p + 2, 0, sizeof(int), s));
    FEM_LAUNCH(F_RASTER, s, k_sq_stage_list, (nsq + 255) / 256, 256, 0, nsq, m->sq_flag.p, m->sq_staged.p,
               m->sq_stage.p, m->sq_ctr.p + 2);
    m->sq_plan_version = m->mesh_version;
    return FEM_OK;
}

static int sq_grid(const fem_mesh* m, long long squares) {
    static const int per_sm = [] {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sq<SQ_FAST>, kSqThreads, 0);
        return nb < 1 ? 1 : nb;
    }();
    return (int)std::max<long long>(1, std::min<long long>(squares, (long long)m->num_sms * per_sm));
}

static SqArgs sq_args(fem_mesh* m, const double* uv, const float2* uvf) {
    SqArgs A{};
    A.fsq = m->fsq.p;
    A.frow = m->fedge.p;
    A.G = sq_geo(m);
    A.order = m->order.p;
    A.tri = m->tri.p;
    A.vxy = m->vxy.p;
    A.uv = uv;
    A.uvf = uvf;
    A.ncov = m->sq_cov.p;
    A.nseg = m->sq_seg.p;
    A.nslot = m->sq_slot.p;
    A.sqoff = m->sq_off.p;
    A.partial = m->sq_part.p;
    A.part_cap = (long long)m->sq_part.n;
    A.err = m->dflag.p + 0;
    return A;
}

// algorithmic bytes of one pass over all squares: the image once (4 B/px),
// the triangles (16 B) and their keys or intervals out (8 or 16 B), vertex
// positions and values (8 + 8 B)
static double sq_bytes(const fem_mesh* m, bool fast) {
    return 4.0 * (double)m->P + (fast ? 32.0 : 24.0) * m->T + 16.0 * m->V;
}

fem_status sq_keys_fast(fem_mesh* m, const double* uv, const float2* uvf, FastOut F, cudaStream_t s) {
    FEM_TRY(sq_plan(m, s));
    FEM_TRY(ensure(m->sq_rec, (size_t)2 * m->T, s));
    const int grid = std::max(1, std::min((m->T + 255) / 256, m->num_sms * 16));
    FEM_LAUNCH(F_RASTER, s, k_sq_records, grid, 256, 0, m->order.p, m->tri.p, m->vxy.p, uv, uvf,
               (const int*)m->sq_nodeof.p, m->T, m->N, (SqRec*)m->sq_rec.p);
    SqArgs A = sq_args(m, uv, uvf);
    A.F = F;
    A.rec = (const SqRec*)m->sq_rec.p;
    A.sq_list = m->sq_stage.p;
    A.n_sq = m->sq_ctr.p + 2;
    const int Q = A.G.Q;
    // the pass is two kernels that each read their share of the pixels once:
    // the staged squares (k_sq), then the small triangles of the others
    note_bytes(F_SQPASS, sq_bytes(m, true));
    FEM_LAUNCH(F_SQPASS, s, k_sq<SQ_FAST>, sq_grid(m, (long long)Q * Q), kSqThreads, 0, A);
    FEM_LAUNCH(F_SQPASS, s, k_sq_small, std::max(1, std::min((m->T + 255) / 256, m->num_sms * 16)), 256, 0,
               (const SqRec*)m->sq_rec.p, (const int*)m->sq_nodeof.p, (const unsigned char*)m->sq_staged.p, m->T,
               A.G, (const float*)m->fsq.p, (const float*)m->fedge.p, F);
    FEM_LAUNCH(F_RASTER, s, k_sq_final<SQ_FAST>, m->num_sms * 8, 256, 0, A, (const int*)m->sq_coarse.p,
               (const int*)(m->sq_ctr.p + 1));
    return FEM_OK;
}

// Exact keys: of every triangle (sel == null) over all squares, or of the
// selected triangles over the squares in list[0 .. *n_list) (n_max: the
// list's capacity, for the grid).
fem_status sq_keys_exact(fem_mesh* m, const double* uv, const float2* uvf, double* keys, unsigned long long* keyc,
                         const unsigned char* sel, const int* list, const int* n_list, int n_max, cudaStream_t s,
                         const int* coarse, const int* n_coarse) {
    FEM_TRY(sq_plan(m, s));
    SqArgs A = sq_args(m, uv, uvf);
    A.keys = keys;
    A.keyc = keyc;
    A.sel = sel;
    A.sq_list = list;
    A.n_sq = n_list;
    const int Q = A.G.Q;
    const int fam = list ? F_RASTER : F_SQPASS;
    if (!list) note_bytes(F_SQPASS, sq_bytes(m, false));
    FEM_LAUNCH(fam, s, k_sq<SQ_EXACT>, sq_grid(m, list ? (long long)n_max : (long long)Q * Q), kSqThreads, 0, A);
    // the coarse triangles to finish: the given list, else all of them
    FEM_LAUNCH(F_RASTER, s, k_sq_final<SQ_EXACT>, m->num_sms * 8, 256, 0, A, coarse ? coarse : (const int*)m->sq_coarse.p,
               n_coarse ? n_coarse : (const int*)(m->sq_ctr.p + 1));
    return FEM_OK;
}

// Squares that hold a selected triangle, listed for the exact pass: a
// square is listed when a fine triangle in it was marked (sq_mark, set by
// the classification) or one of its nodes lies in a selected coarse
// triangle.  The marks are cleared for the next round.
__global__ void k_sq_band_list(int nsq, const int* __restrict__ order, const int* __restrict__ ncov,
                               const unsigned char* __restrict__ sel, unsigned char* __restrict__ mark,
                               int* __restrict__ list, int* __restrict__ n_list) {
    pdl_wait();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    bool on = false;
    if (q < nsq) {
        on = mark[q] != 0;
        mark[q] = 0;
        const int c0 = ncov[2 * q], c1 = ncov[2 * q + 1];
        if (c0 >= 0 && sel[order[c0]]) on = true;
        if (c1 >= 0 && sel[order[c1]]) on = true;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, on);
    int base = 0;
    if ((threadIdx.x & 31) == 0 && bal) base = atomicAdd(n_list, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (on) list[base + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u))] = q;
}

fem_status sq_band_exact(fem_mesh* m, const double* uv, const float2* uvf, int* n_list_dev, cudaStream_t s) {
    const int Q = sq_geo(m).Q;
    const int nsq = Q * Q;
    FEM_TRY(ensure(m->sq_list, (size_t)nsq, s));
    FEM_CUDA(cudaMemsetAsync(n_list_dev, 0, sizeof(int), s));
    FEM_LAUNCH(F_TOPK, s, k_sq_band_list, (nsq + 255) / 256, 256, 0, nsq, (const int*)m->order.p,
               (const int*)m->sq_cov.p, (const unsigned char*)m->bsel.p, m->sq_mark.p, m->sq_list.p, n_list_dev);
    int* fc = (int*)(m->fast_hist.p + 2 * kFastBins);
    return sq_keys_exact(m, uv, uvf, m->keys.p, m->keyc.p, m->bsel.p, m->sq_list.p, n_list_dev, nsq, s,
                         (const int*)m->sq_bcoarse.p, (const int*)(fc + FC_BAND_COARSE));
}

}  // namespace fem
