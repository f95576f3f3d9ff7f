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
//   * nodes inside coarse triangles (with the coarse triangle's plane) are
//     swept together over the square's full rows: lane r finds the span of
//     row r, then the lanes take the columns of each row;
//   * fine triangles, FAST mode: one triangle row per lane (sq_fine_rows),
//     rows of a triangle combined by a segmented warp scan, so the lanes
//     stay busy for any mix of sizes;
//   * fine triangles, EXACT mode: those with a bounding box of at most
//     17 x 17 pixels one per lane, larger ones over their bounding box with
//     the lanes over the columns;
//   * the sums of coarse triangles go to per-node slots, and k_sq_final adds
//     each coarse triangle's slots in a fixed order, one warp per triangle.
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
// Bound on the FP32 additions any term of a FAST sum passes through: a row
// of a fine triangle is one lane's chain of at most 33 additions, then at
// most 5 levels of the segmented scan and 3 batches (41 in all); with the
// lanes over the columns of a coarse node a lane takes at most 2 pixels in
// each of at most 33 rows, then 5 levels of the butterfly.  Kept at the
// 153-pixel chain of a triangle summed by one lane, which covers both.
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

// columns (rows) of square J (I) that hold image pixels: s, one more for the
// domain's last column (row), clipped to the image (0 outside it)
__device__ __forceinline__ int sq_extent(int s, int J, int Q, int x0, int W) {
    return max(0, min(s + (J == Q - 1 ? 1 : 0), W - x0));
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
    __device__ __forceinline__ int operator()(long long i) const {
        const int t = order[i];
        pos[t] = (int)i;
        const int4 tr = tri[t];
        const int2 a = vxy[tr.x], b = vxy[tr.y], c = vxy[tr.z];
        if (leg2(a, c) <= (long long)G.s * G.s) {
            const int n = sq_node_at((long long)a.x + b.x + c.x, (long long)a.y + b.y + c.y, G);
            nodeof[i] = n;
            return 0;
        }
        nodeof[i] = -1;
        const int w = max(a.x, max(b.x, c.x)) - min(a.x, min(b.x, c.x));
        const int h = max(a.y, max(b.y, c.y)) - min(a.y, min(b.y, c.y));
        return (w / G.s) * (h / G.s);
    }
};

// Coarse triangles with more than kSqPiece node slots ("long": the large
// triangles of the early rounds) are summed in pieces of kSqPiece slots, one
// block per piece, so that no single warp reads a large triangle's slots
// alone.  longs[L] = (curve position, first piece, pieces, slots); piece[p] =
// (L, index of the piece in its triangle); psum[p] the piece's sum; pdone[L]
// counts the finished pieces (the block that finishes the last one adds them
// up and resets it to zero).
constexpr int kSqPiece = 4096;
struct SqLong {
    int4* longs;
    int2* piece;
    float4* psum;
    int* pdone;
    int* n_long;
    int* n_pieces;
    int cap_long, cap_pieces;
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
                           int* __restrict__ coarse, int* __restrict__ n_coarse, SqLong LG) {
    pdl_wait();
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int W = *W_dev;
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
        if (is_coarse) {
            coarse[base + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u))] = (int)i;
            // a long triangle is also listed with its pieces
            const int cnt = 2 * ((i + 1 < T ? sqoff[i + 1] : W) - sqoff[i]);
            if (cnt > kSqPiece) {
                const int np = (cnt + kSqPiece - 1) / kSqPiece;
                const int L = atomicAdd(LG.n_long, 1);
                const int pb = atomicAdd(LG.n_pieces, np);
                if (L < LG.cap_long && pb + np <= LG.cap_pieces) {
                    LG.longs[L] = make_int4((int)i, pb, np, cnt);
                    for (int j = 0; j < np; ++j) LG.piece[pb + j] = make_int2(L, j);
                } else {
                    atomicCAS(err, 0, (int)FEM_E_INVALID);
                }
            }
        }
        if (i >= T || n < 0) continue;
        if (i == 0 || nodeof[i - 1] != n) {
            nseg[n].x = (int)i;
            ncov[n] = -1;
        }
        if (i == T - 1 || nodeof[i + 1] != n) nseg[n].y = (int)i + 1;
    }
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
    const unsigned char* tdirty;  // SQ_FAST: finish only triangles with tdirty[t] != 0 (null: all)
    unsigned char* hcnt;          // SQ_FAST: per finished triangle, 1 when counted in the histograms
    SqLong LG;                  // long coarse triangles and their pieces
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
__device__ __forceinline__ unsigned long long sq_keyc(const Dom& D, const TriGeom& g, double key) {
    return tri_eligible(g, D) ? ((unsigned long long)__double_as_longlong(key) | (1ull << 63)) : 0ull;
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
        const bool el = tri_eligible(g, sq_dom(A.G));
        if (el) {
            atomicAdd(A.F.hlo + fast_bin(lo), 1u);
            atomicAdd(A.F.hhi + fast_bin(hi), 1u);
        }
        A.hcnt[t] = el ? 1 : 0;
    } else {
        const double key = ff_to_double(S);
        A.keys[t] = key;
        if (A.keyc) A.keyc[t] = sq_keyc(sq_dom(A.G), g, key);
    }
}

// EXACT: one lane, one small fine triangle, pixels from the staged square;
// along a row u is advanced by the exact float-float g_x.
__device__ __forceinline__ void sq_small(const SqArgs& A, const float* img, int x0, int y0, int pitch, int t,
                                         const TriGeom& g, const SqPlane& P) {
    const Dom D = sq_dom(A.G);
    ff acc{0.f, 0.f};
    for (int y = g.ytop; y <= g.yend; ++y) {
        int L, len;
        row_span(g, y, D, L, len);
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
    if (A.keyc) A.keyc[t] = sq_keyc(sq_dom(A.G), g, key);
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
__device__ __forceinline__ void sq_spans(const TriGeom& g, int y, int R, const Dom& D, int& La, int& na, int& Lb,
                                         int& nb) {
    const int lane = threadIdx.x & 31;
    La = 0; na = 0; Lb = 0; nb = 0;
    const int ya = y + lane, yb = y + 32;
    if (lane < R && ya >= g.ytop && ya <= g.yend) row_span(g, ya, D, La, na);
    if (lane == 0 && R > 32 && yb >= g.ytop && yb <= g.yend) row_span(g, yb, D, Lb, nb);
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
                                          int y0, int w, int h, int pitch, const Dom& D, ff& S0, ff& S1,
                                          long long& n0) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int La, na, Lb, nb;
    sq_spans(g0, y0, h, D, La, na, Lb, nb);
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
                                      const Dom& D, long long& npix) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int R = g.yend - g.ytop + 1;
    int La, na, Lb, nb;
    sq_spans(g, g.ytop, R, D, La, na, Lb, nb);
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
// A square with no image pixel (only where the image is smaller than the
// domain) is not copied: its arrival expects no bytes, so the phase
// completes at once, and its clamped extents read none of its pixels.
__device__ __forceinline__ void sq_issue(const SqArgs& A, int q, float* img, unsigned long long* bar,
                                         unsigned long long policy) {
    const int s = A.G.s;
    const int I = q / A.G.Q, J = q - I * A.G.Q;
    const bool outside = J * s >= A.G.W || I * s >= A.G.H;
    const unsigned bytes = outside ? 0u : (unsigned)(4 * s * (s + 1));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, bytes);
    if (!outside) bulk_copy(img, A.fsq + (long long)q * s * (s + 1), bytes, bar, policy);
}

// Incremental FP32 pass.  A triangle's interval depends only on its
// corners, its vertex values, the image and the fine triangles that share
// its square (they fix the order of the FP32 additions), and the pass forms
// it in a fixed order.  So after a refinement round only the intervals of
// "dirty" triangles can change: those the bisection made or rewrote, and
// those with a vertex whose value changed (new vertices, re-solved
// unknowns).  Only the squares that hold a dirty triangle are passed over;
// there every fine triangle comes out as a full pass would give it, the
// dirty ones are stored, and every other triangle keeps its interval, which
// a full pass would reproduce bit for bit.  The histograms of the intervals
// are kept too: a dirty triangle that was counted takes its old bins out
// (here) and the pass counts its new ones.
struct SqInc {
    const unsigned char* vchg;  // per vertex: value changed since the kept intervals (null: full pass)
    unsigned char* tchg;        // per triangle: rewritten by the bisection since (cleared here)
    int Tk;                     // triangles at the kept intervals: ids >= Tk are new
    unsigned char* tdirty;      // out: per triangle
    unsigned char* dmark;       // out: per square, holds a dirty fine triangle
    const float* lo;            // the kept intervals
    const float* hi;
    const unsigned char* hcnt;  // per triangle below Tk: its kept interval is counted
    unsigned* hlo;              // histograms
    unsigned* hhi;
};

// The records of the triangles for the FP32 pass, one thread per curve
// position; all gathers of the pass happen here, in a fully parallel kernel,
// and the pass reads each square's records contiguously (fine triangles) or
// one record per covered node (coarse ones).  With I.vchg the kernel also
// classifies every triangle dirty or clean (above), marks the squares of the
// dirty fine ones, and takes the old bins of the counted dirty ones out of
// the histograms (a few per cent of the triangles, spread over the bins, so
// plain atomics).
__global__ void k_sq_records(const int* __restrict__ order, const int4* __restrict__ tri, const int2* __restrict__ vxy,
                             const double* __restrict__ uv, const float2* __restrict__ uvf,
                             const int* __restrict__ nodeof, int T, int N, SqRec* __restrict__ rec, SqInc I) {
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
        if (I.vchg) {
            // flags are written only where they change: a few per cent of
            // the triangles, instead of scattered byte stores for all
            const unsigned char tc = t < I.Tk ? I.tchg[t] : 1;  // a new id's flag is not yet cleared
            const bool d = tc || I.vchg[tr.x] || I.vchg[tr.y] || I.vchg[tr.z];
            if (tc) I.tchg[t] = 0;
            if (I.tdirty[t] != (unsigned char)d) I.tdirty[t] = d ? 1 : 0;
            if (d) {
                const int nd = nodeof[i];
                if (nd >= 0) I.dmark[nd >> 1] = 1;
                if (t < I.Tk && I.hcnt[t]) {
                    atomicSub(I.hlo + fast_bin(I.lo[t]), 1u);
                    atomicSub(I.hhi + fast_bin(I.hi[t]), 1u);
                }
            }
        } else if (I.tchg) {
            I.tchg[t] = 0;
        }
    }
}

// Per vertex: has the value (FP64 and float-float copy) changed since the
// kept intervals were formed?  Vertices from Vk on are new.  The kept copy
// follows the current values.
__global__ void k_vchanged(int V, int Vk, const double* __restrict__ uv, const float2* __restrict__ uvf,
                           double* __restrict__ uvk, float2* __restrict__ uvfk, unsigned char* __restrict__ vchg) {
    pdl_wait();
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        const double x = uv[v];
        bool c = v >= Vk || __double_as_longlong(x) != __double_as_longlong(uvk[v]);
        float2 y = make_float2(0.f, 0.f);
        if (uvf) {
            y = uvf[v];
            if (!c) {
                const float2 z = uvfk[v];
                c = __float_as_uint(y.x) != __float_as_uint(z.x) || __float_as_uint(y.y) != __float_as_uint(z.y);
            }
        }
        vchg[v] = c ? 1 : 0;
        if (c) {
            uvk[v] = x;
            if (uvf) uvfk[v] = y;
        }
    }
}

// Algorithmic bytes of the incremental passes, when asked for (profiling):
// per listed square its image block (4 B per pixel), its two node entries
// (32 B), the record of each fine triangle in it (32 B) with its interval
// (8 B), and the record of each covering coarse triangle (32 B).
__device__ unsigned long long g_sq_inc_bytes;

// The squares of the incremental pass: a square is listed when one of its
// fine triangles is dirty (marked by k_sq_records) or one of its nodes lies
// in a dirty coarse triangle.  The marks are cleared for the next round.
__global__ void k_sq_dirty_list(int nsq, const int* __restrict__ order, const int* __restrict__ ncov,
                                const int2* __restrict__ nseg, const unsigned char* __restrict__ tdirty,
                                unsigned char* __restrict__ mark, int* __restrict__ list, int* __restrict__ n_list,
                                SqGeo G, bool count_bytes) {
    pdl_wait();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    bool on = false;
    unsigned long long bytes = 0;
    if (q < nsq) {
        on = mark[q] != 0;
        mark[q] = 0;
        const int c0 = ncov[2 * q], c1 = ncov[2 * q + 1];
        if (c0 >= 0 && tdirty[order[c0]]) on = true;
        if (c1 >= 0 && tdirty[order[c1]]) on = true;
        if (on && count_bytes) {
            const int I = q / G.Q, J = q - I * G.Q;
            const long long px = (long long)sq_extent(G.s, J, G.Q, J * G.s, G.W) * sq_extent(G.s, I, G.Q, I * G.s, G.H);
            long long fine = 0;
            if (c0 < 0) { const int2 sg = nseg[2 * q]; fine += max(0, sg.y - sg.x); }
            if (c1 < 0) { const int2 sg = nseg[2 * q + 1]; fine += max(0, sg.y - sg.x); }
            bytes = (unsigned long long)(4 * px + 32 + 40 * fine + 32 * ((c0 >= 0) + (c1 >= 0)));
        }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, on);
    int base = 0;
    if ((threadIdx.x & 31) == 0 && bal) base = atomicAdd(n_list, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (on) list[base + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u))] = q;
    if (count_bytes) {
        bytes = warp_sum(bytes);
        if ((threadIdx.x & 31) == 0 && bytes) atomicAdd(&g_sq_inc_bytes, bytes);
    }
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

// FAST: the interval of each lane's triangle from its FP32 sum and pixel
// count, and the histograms (one atomic per distinct bin).  Whole warp.
__device__ __forceinline__ void sq_fine_finish(const SqArgs& A, bool have, const SqRec& R, const TriGeom& g, float sum,
                                               int n) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    unsigned blo = 0xffffffffu, bhi = 0xffffffffu;
    if (have && (!A.tdirty || A.tdirty[R.t])) {
        float lo, hi;
        fast_interval(ff{sum, 0.f}, (float)n, fast_M(g, R.ucf, R.gxf, R.gyf), kSqChain, lo, hi);
        A.F.lo[R.t] = lo;
        A.F.hi[R.t] = hi;
        const bool el = tri_eligible(g, sq_dom(A.G));
        if (el) {
            blo = fast_bin(lo);
            bhi = fast_bin(hi);
        }
        A.hcnt[R.t] = el ? 1 : 0;
    }
    unsigned peers = __match_any_sync(FULL, blo);
    if (blo != 0xffffffffu && (__ffs(peers) - 1) == lane) atomicAdd(A.F.hlo + blo, (unsigned)__popc(peers));
    peers = __match_any_sync(FULL, bhi);
    if (bhi != 0xffffffffu && (__ffs(peers) - 1) == lane) atomicAdd(A.F.hhi + bhi, (unsigned)__popc(peers));
}

// FAST: the fine triangles of a square, one triangle row per lane.  The
// square's fine triangles (the curve segments of its two nodes) are taken
// 32 at a time in curve order, lane k holding triangle k of the chunk.  Their
// rows are numbered by an exclusive warp scan of the row counts, and in each
// batch lane i takes row item j0 + i: it finds its triangle from the batch's
// start bits, takes the triangle's corners and plane from that lane by
// shuffles, and sums the row's pixels from the staged square (one FP32 chain,
// at most 33 pixels).  A segmented scan over the lanes adds the rows of each
// triangle within the batch (5 levels), and the triangle's lane adds its
// batches in order (at most 3 for the at most 33 rows of a fine triangle).
// Every term thus passes through at most 33 + 5 + 3 additions of non-negative
// values, within kSqChain, and the order is fixed, so the pass stays
// deterministic.  Lanes take rows, not triangles, so a warp stays busy
// whatever the mix of triangle sizes in the square.  A chunk whose triangles
// are all small (bounding box at most 17 x 17) is summed one triangle per
// lane instead: there the exchanges of the row scheme would cost more than
// the lanes' uneven loads.
__device__ __forceinline__ void sq_fine_rows(const SqArgs& A, const float* img, int x0, int y0, int pitch, int2 sg0,
                                             int len0, int2 sg1, int len1) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int N = A.G.N;
    const Dom D = sq_dom(A.G);
    const int nf = len0 + len1;
    for (int e0 = 0; e0 < nf; e0 += 32) {
        const int e = e0 + lane;
        const bool have = e < nf;
        SqRec R{};
        TriGeom g{};
        int h = 0;
        if (have) {
            R = A.rec[e < len0 ? sg0.x + e : sg1.x + (e - len0)];
            g = rec_geom(R, N);
            h = g.yend - g.ytop + 1;
        }
        if (__all_sync(FULL, !have || is_small(g))) {
            // a chunk of small triangles: one lane each (a chain of at most
            // 153 pixels), no exchange between lanes
            float acc = 0.f;
            int n = 0;
            if (have) {
                const RowGeo rg = row_geo(g);
                for (int y = g.ytop; y <= g.yend; ++y) {
                    int L, len;
                    row_span_geo(rg, y, D, L, len);
                    if (len <= 0) continue;
                    const float* rowp = img + (y - y0) * pitch + (L - x0);
                    const float urow = fmaf(R.gyf, (float)(y - g.cy), fmaf(R.gxf, (float)(L - g.cx), R.ucf));
                    float fk = 0.f;
#pragma unroll 4
                    for (int q = 0; q < len; ++q) {
                        const float d = fmaf(R.gxf, fk, urow) - rowp[q];
                        acc = fmaf(d, d, acc);
                        fk += 1.0f;
                    }
                    n += len;
                }
            }
            sq_fine_finish(A, have, R, g, acc, n);
            continue;
        }
        // exclusive scan of the row counts: rows H .. Hn - 1 are triangle k's
        int Hn = h;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, Hn, o);
            if (lane >= o) Hn += v;
        }
        const int H = Hn - h;
        const int total = __shfl_sync(FULL, Hn, 31);
        const RowGeo rg = row_geo(g);
        float tot = 0.f;
        int cnt = 0;
        for (int j0 = 0; j0 < total; j0 += 32) {
            // triangle of item j0 + lane: the one holding item j0, plus the
            // triangles that start in (j0, j0 + lane]
            const unsigned starts = __reduce_or_sync(FULL, (have && H > j0 && H < j0 + 32) ? 1u << (H - j0) : 0u);
            const int k0 = __popc(__ballot_sync(FULL, have && H <= j0)) - 1;
            const int j = j0 + lane;
            const bool valid = j < total;
            const int k = valid ? k0 + __popc(starts & (FULL >> (31 - lane))) : 0;
            // triangle k's rows (its top row is y0 of its sorted corners), corner and plane
            RowGeo rk;
            rk.y0 = __shfl_sync(FULL, rg.y0, k); rk.y1 = __shfl_sync(FULL, rg.y1, k);
            rk.x0 = __shfl_sync(FULL, rg.x0, k); rk.x1 = __shfl_sync(FULL, rg.x1, k);
            rk.sl = __shfl_sync(FULL, rg.sl, k);
            const int Hk = __shfl_sync(FULL, H, k);
            const int ckx = __shfl_sync(FULL, g.cx, k), cky = __shfl_sync(FULL, g.cy, k);
            const float ucf = __shfl_sync(FULL, R.ucf, k), gxf = __shfl_sync(FULL, R.gxf, k);
            const float gyf = __shfl_sync(FULL, R.gyf, k);
            float acc = 0.f;
            int n = 0;
            if (valid) {
                const int y = rk.y0 + (j - Hk);
                int L, len;
                row_span_geo(rk, y, D, L, len);
                if (len > 0) {
                    const float* rowp = img + (y - y0) * pitch + (L - x0);
                    const float urow = fmaf(gyf, (float)(y - cky), fmaf(gxf, (float)(L - ckx), ucf));
                    float fk = 0.f;
#pragma unroll 4
                    for (int q = 0; q < len; ++q) {
                        const float d = fmaf(gxf, fk, urow) - rowp[q];
                        acc = fmaf(d, d, acc);
                        fk += 1.0f;
                    }
                    n = len;
                }
            }
            // the rows of one triangle are consecutive lanes: segmented scan
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float a = __shfl_up_sync(FULL, acc, o);
                const int m = __shfl_up_sync(FULL, n, o);
                const int ko = __shfl_up_sync(FULL, k, o);
                if (lane >= o && ko == k) {
                    acc += a;
                    n += m;
                }
            }
            // lane k takes its rows' total from the last of them in the batch
            const bool part = have && H < j0 + 32 && Hn > j0;
            const int last = part ? min(Hn, j0 + 32) - 1 - j0 : lane;
            const float a = __shfl_sync(FULL, acc, last);
            const int m = __shfl_sync(FULL, n, last);
            if (part) {
                tot += a;
                cnt += m;
            }
        }
        sq_fine_finish(A, have, R, g, tot, cnt);
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
                const int w = sq_extent(s, J, Q, x0, G.W), h = sq_extent(s, I, Q, y0, G.H);
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
                const int w = sq_extent(s, J, Q, x0, G.W), h = sq_extent(s, I, Q, y0, G.H);
                ff S0, S1;
                long long np0 = 0;
                sq_sweep2<MODE>(geom_xy(na, nb, nc, N), want0, P0, cx0, cy0, want1, P1, cx1, cy1, img, x0, y0, w, h,
                                pitch, sq_dom(G), S0, S1, np0);
                if (lane == 0) {
                    const int s0 = A.nslot[n0], s1 = A.nslot[n0 + 1];
                    if (want0 && s0 >= 0 && s0 < A.part_cap)
                        A.partial[s0] = make_float4(S0.hi, S0.lo, __int_as_float((int)np0), 0.f);
                    if (want1 && s1 >= 0 && s1 < A.part_cap)
                        A.partial[s1] = make_float4(S1.hi, S1.lo, __int_as_float(w * h - (int)np0), 0.f);
                }
            }
            // fine triangles.  FAST: one row per lane.  EXACT: small ones by
            // one lane each, larger ones listed
            const int2 sg0 = A.nseg[n0], sg1 = A.nseg[n0 + 1];
            const int len0 = c0 < 0 ? sg0.y - sg0.x : 0, len1 = c1 < 0 ? sg1.y - sg1.x : 0;
            if (MODE == SQ_FAST) {
                sq_fine_rows(A, img, x0, y0, pitch, sg0, len0, sg1, len1);
                __syncwarp();
                continue;
            }
            if (lane == 0) s_nbig[wb] = 0;
            __syncwarp();
            for (int e = lane; e < len0 + len1; e += 32) {
                const int c = e < len0 ? sg0.x + e : sg1.x + (e - len0);
                const int t = A.order[c];
                if (!sq_want<MODE>(A, t)) continue;
                const int4 tr = A.tri[t];
                const TriGeom g = tri_geom(tr, A.vxy, N);
                if (is_small(g)) {
                    sq_small(A, img, x0, y0, pitch, t, g, sq_plane(g, tr, A.uv, A.uvf));
                } else {
                    // listed by curve position
                    const int slot = atomicAdd(&s_nbig[wb], 1);
                    if (slot < kSqBigCap) s_big[wb][slot] = c;
                    else atomicCAS(A.err, 0, (int)FEM_E_INVALID);
                }
            }
            __syncwarp();
            const int nbig = min(s_nbig[wb], kSqBigCap);
            for (int e = 0; e < nbig; ++e) {
                const int c = s_big[wb][e];
                const int t = A.order[c];
                const int4 tr = A.tri[t];
                const TriGeom g = tri_geom(tr, A.vxy, N);
                const SqPlane P = sq_plane(g, tr, A.uv, A.uvf);
                long long np = 0;
                const ff S = sq_bbox<MODE>(g, P, img, x0, y0, pitch, sq_dom(G), np);
                if (lane == 0) sq_finish<MODE>(A, t, g, P, S, np);
            }
        }
        __syncwarp();
    }
}

// Finish coarse triangle c (curve position) from the sum S of its node slots
// and its pixel count: FAST interval or EXACT key.  One thread.
template <int MODE>
__device__ __forceinline__ void sq_coarse_finish(const SqArgs& A, int c, ff S, int np) {
    if (MODE == SQ_FAST) {
        const SqRec R = A.rec[c];
        sq_finish<MODE>(A, R.t, rec_geom(R, A.G.N), rec_plane(R), S, np);
    } else {
        const int t = A.order[c];
        const int4 tr = A.tri[t];
        const TriGeom gt = tri_geom(tr, A.vxy, A.G.N);
        sq_finish<MODE>(A, t, gt, sq_plane(gt, tr, A.uv, A.uvf), S, np);
    }
}

template <int MODE>
__device__ __forceinline__ bool sq_coarse_wanted(const SqArgs& A, int c) {
    if (MODE == SQ_FAST) return !A.tdirty || A.tdirty[A.order[c]];
    return !A.sel || A.sel[A.order[c]];
}

// The coarse triangles.  First the pieces of the long ones, one block per
// piece: the block adds the piece's slots in a fixed order (each thread a
// strided share, then the warps' butterflies, then the eight warps in
// order) and stores the piece's sum; the block that stores a triangle's last
// piece (counted by an atomic after a fence) adds its pieces in order and
// finishes the triangle.  Nothing waits.  Then the other coarse triangles,
// coarse[0 .. *n_coarse) (curve positions), one warp each: the triangle's
// node slots (all of its bounding-box slots; those outside it hold zero)
// added in a fixed order.  Both give the same sums on every run.
template <int MODE>
__global__ void __launch_bounds__(256) k_sq_final(SqArgs A, const int* __restrict__ coarse,
                                                  const int* __restrict__ n_coarse) {
    pdl_wait();
    __shared__ float2 s_sum[8];
    __shared__ int s_cnt[8];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    const int s = A.G.s;
    // after an overflow of the lists (only in a mesh the plan reported as
    // invalid) some entries were never written: no piece is read then
    const int nlong = *A.LG.n_long, npieces_all = *A.LG.n_pieces;
    const int npieces = (nlong <= A.LG.cap_long && npieces_all <= A.LG.cap_pieces) ? npieces_all : 0;
    for (int p = blockIdx.x; p < npieces; p += gridDim.x) {
        const int2 pc = A.LG.piece[p];
        const int4 L = A.LG.longs[pc.x];  // (curve position, first piece, pieces, slots)
        if (!sq_coarse_wanted<MODE>(A, L.x)) continue;  // the same for the whole block
        const long long o = 2LL * A.sqoff[L.x] + (long long)pc.y * kSqPiece;
        int len = min(kSqPiece, L.w - pc.y * kSqPiece);
        if (o + len > A.part_cap) len = 0;  // only in a mesh already reported invalid
        ff S{0.f, 0.f};
        int np = 0;
        for (int e0 = threadIdx.x; e0 < len; e0 += 4 * 256) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + 256 * u;
                v[u] = e < len ? A.partial[o + e] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                S = ff_add(S, ff{v[u].x, v[u].y});
                np += __float_as_int(v[u].z);
            }
        }
        S = ff_warp_sum(S);
        np = warp_sum(np);
        if (lane == 0) {
            s_sum[wb] = make_float2(S.hi, S.lo);
            s_cnt[wb] = np;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            ff T{0.f, 0.f};
            int n = 0;
            for (int w = 0; w < 8; ++w) {
                T = ff_add(T, ff{s_sum[w].x, s_sum[w].y});
                n += s_cnt[w];
            }
            A.LG.psum[p] = make_float4(T.hi, T.lo, __int_as_float(n), 0.f);
            __threadfence();
            s_last = atomicAdd(A.LG.pdone + pc.x, 1) == L.z - 1;
        }
        __syncthreads();
        if (s_last && wb == 0) {
            __threadfence();
            ff U{0.f, 0.f};
            int n = 0;
            for (int j = lane; j < L.z; j += 32) {
                const float4 v = __ldcg(A.LG.psum + L.y + j);
                U = ff_add(U, ff{v.x, v.y});
                n += __float_as_int(v.z);
            }
            U = ff_warp_sum(U);
            n = warp_sum(n);
            if (lane == 0) {
                A.LG.pdone[pc.x] = 0;
                sq_coarse_finish<MODE>(A, L.x, U, n);
            }
        }
        __syncthreads();
    }
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    const int n = *n_coarse;
    for (int k = gw; k < n; k += nw) {
        const int c = coarse[k];
        if (!sq_coarse_wanted<MODE>(A, c)) continue;  // the same for the whole warp
        TriGeom gt;
        if (MODE == SQ_FAST) {
            gt = rec_geom(A.rec[c], A.G.N);
        } else {
            gt = tri_geom(A.tri[A.order[c]], A.vxy, A.G.N);
        }
        const int w = (gt.maxw - 1) / s, h = (max(gt.ay, max(gt.by, gt.cy)) - gt.ytop) / s;
        if (2 * w * h > kSqPiece) continue;  // long: summed in pieces above
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
        if (lane == 0) sq_coarse_finish<MODE>(A, c, S, np);
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
    G.W = m->W;
    G.H = m->H;
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

static SqLong sq_long_args(fem_mesh* m) {
    SqLong LG;
    LG.longs = m->sq_long.p;
    LG.piece = m->sq_piece.p;
    LG.psum = m->sq_psum.p;
    LG.pdone = m->sq_pdone.p;
    LG.n_long = m->sq_ctr.p + 2;
    LG.n_pieces = m->sq_ctr.p + 3;
    LG.cap_long = (int)m->sq_long.n;
    LG.cap_pieces = (int)m->sq_piece.n;
    return LG;
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
    // long coarse triangles: each has more than kSqPiece of the at most
    // 4 Q^2 + 8 slots, and at most one piece more than its slots fill
    const int cap_long = (int)((4LL * G.Q * G.Q + 8) / kSqPiece + 2);
    FEM_TRY(ensure(m->sq_long, (size_t)cap_long, s));
    FEM_TRY(ensure(m->sq_pdone, (size_t)cap_long, s));
    FEM_TRY(ensure(m->sq_piece, (size_t)2 * cap_long, s));
    FEM_TRY(ensure(m->sq_psum, (size_t)2 * cap_long, s));
    FEM_CUDA(cudaMemsetAsync(m->sq_pdone.p, 0, sizeof(int) * cap_long, s));
    int* W = m->sq_ctr.p + 0;         // bounding-box squares of the coarse triangles
    int* n_coarse = m->sq_ctr.p + 1;  // coarse triangles listed
    // [1] coarse triangles, [2] long ones, [3] their pieces
    FEM_CUDA(cudaMemsetAsync(n_coarse, 0, 3 * sizeof(int), s));
    // nodes that no triangle claims (only in a mesh with holes) read as
    // fine with an empty segment
    FEM_CUDA(cudaMemsetAsync(m->sq_cov.p, 0xff, sizeof(int) * nodes, s));
    FEM_CUDA(cudaMemsetAsync(m->sq_seg.p, 0xff, sizeof(int2) * nodes, s));
    FEM_TRY(ensure(m->sq_pos, (size_t)T, s));
    FEM_TRY(scan_fused(m, SqCountIn{m->order.p, m->tri.p, m->vxy.p, G, m->sq_nodeof.p, m->sq_pos.p},
                       ScanStore{m->sq_off.p}, T, s, W, F_RASTER));
    // work: T curve positions, then at most 2 Q^2 bounding-box squares
    const long long work = std::max<long long>(T, 2LL * G.Q * G.Q);
    const int grid = (int)std::max<long long>(1, std::min<long long>((work + 255) / 256, (long long)m->num_sms * 8));
    FEM_LAUNCH(F_RASTER, s, k_sq_nodes, grid, 256, 0, m->order.p, m->tri.p, m->vxy.p, (const int*)m->sq_nodeof.p,
               (const int*)m->sq_off.p, (const int*)W, T, G, m->sq_cov.p, m->sq_seg.p, m->sq_slot.p, m->sq_part.p,
               (long long)m->sq_part.n, m->dflag.p + 0, m->sq_coarse.p, n_coarse, sq_long_args(m));
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
    A.LG = sq_long_args(m);
    A.err = m->dflag.p + 0;
    return A;
}

// algorithmic bytes of one pass over all squares: the image once (4 B/px),
// the triangles (16 B) and their keys or intervals out (8 or 16 B), vertex
// positions and values (8 + 8 B)
static double sq_bytes(const fem_mesh* m, bool fast) {
    return 4.0 * (double)m->PI + (fast ? 32.0 : 24.0) * m->T + 16.0 * m->V;
}

double sq_inc_bytes_take() {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_sq_inc_bytes, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0.0;
    }
    const unsigned long long z = 0;
    cudaMemcpyToSymbol(g_sq_inc_bytes, &z, sizeof(z));
    cudaGetLastError();
    return (double)v;
}

// incremental: the caller's intervals F.lo / F.hi and histograms F.hlo /
// F.hhi are those of the last pass on this mesh before the refinement round
// that made it (the spatial loop's rounds after its first); the pass then
// covers only the dirty triangles' squares.  Otherwise every square, with
// the histograms cleared first, and the kept state starts afresh.
fem_status sq_keys_fast(fem_mesh* m, const double* uv, const float2* uvf, FastOut F, cudaStream_t s,
                        bool incremental) {
    FEM_TRY(sq_plan(m, s));
    const int T = m->T, V = m->V;
    const SqGeo G = sq_geo(m);
    const int nsq = G.Q * G.Q;
    const bool inc = incremental && m->inc_ok && m->inc_T <= T && m->inc_V <= V;
    FEM_TRY(ensure(m->sq_rec, (size_t)2 * T, s));
    FEM_TRY(ensure(m->tchg, (size_t)T, s, inc ? (size_t)m->inc_T : 0));
    FEM_TRY(ensure(m->uvk, (size_t)V, s, inc ? (size_t)m->inc_V : 0));
    FEM_TRY(ensure(m->uvfk, (size_t)V, s, inc ? (size_t)m->inc_V : 0));
    FEM_TRY(ensure(m->hcnt, (size_t)T, s, inc ? (size_t)m->inc_T : 0));
    if (!inc) {
        FEM_CUDA(cudaMemsetAsync(F.hlo, 0, sizeof(unsigned) * kFastBins, s));
        FEM_CUDA(cudaMemsetAsync(F.hhi, 0, sizeof(unsigned) * kFastBins, s));
    }
    SqInc I{};
    I.tchg = m->tchg.p;
    if (inc) {
        FEM_TRY(ensure(m->vchg, (size_t)V, s));
        FEM_TRY(ensure(m->tdirty, (size_t)T, s, (size_t)m->inc_T));
        FEM_TRY(ensure(m->sq_dlist, (size_t)nsq + 1, s));
        if (!m->sq_dmark.p || m->sq_dmark.n < (size_t)nsq) {
            FEM_TRY(ensure(m->sq_dmark, (size_t)nsq, s));
            FEM_CUDA(cudaMemsetAsync(m->sq_dmark.p, 0, m->sq_dmark.n, s));  // cleared by each list after
        }
        const int vg = std::max(1, std::min((V + 255) / 256, m->num_sms * 8));
        FEM_LAUNCH(F_RASTER, s, k_vchanged, vg, 256, 0, V, m->inc_V, uv, uvf, m->uvk.p, uvf ? m->uvfk.p : nullptr,
                   m->vchg.p);
        I.vchg = m->vchg.p;
        I.Tk = m->inc_T;
        I.tdirty = m->tdirty.p;
        I.dmark = m->sq_dmark.p;
        I.lo = F.lo;
        I.hi = F.hi;
        I.hcnt = m->hcnt.p;
        I.hlo = F.hlo;
        I.hhi = F.hhi;
    }
    const int grid = std::max(1, std::min((T + 255) / 256, m->num_sms * 16));
    FEM_LAUNCH(F_RASTER, s, k_sq_records, grid, 256, 0, m->order.p, m->tri.p, m->vxy.p, uv, uvf,
               (const int*)m->sq_nodeof.p, T, m->N, (SqRec*)m->sq_rec.p, I);
    SqArgs A = sq_args(m, uv, uvf);
    A.F = F;
    A.rec = (const SqRec*)m->sq_rec.p;
    A.hcnt = m->hcnt.p;
    if (inc) {
        int* n_list = m->sq_dlist.p + nsq;
        FEM_CUDA(cudaMemsetAsync(n_list, 0, sizeof(int), s));
        FEM_LAUNCH(F_RASTER, s, k_sq_dirty_list, (nsq + 255) / 256, 256, 0, nsq, (const int*)m->order.p,
                   (const int*)m->sq_cov.p, (const int2*)m->sq_seg.p, (const unsigned char*)m->tdirty.p,
                   m->sq_dmark.p, m->sq_dlist.p, n_list, G, profiling(F_SQPASS));
        A.sq_list = m->sq_dlist.p;
        A.n_sq = n_list;
        A.tdirty = m->tdirty.p;
    } else {
        note_bytes(F_SQPASS, sq_bytes(m, true));
    }
    FEM_LAUNCH(F_SQPASS, s, k_sq<SQ_FAST>, sq_grid(m, (long long)nsq), kSqThreads, 0, A);
    FEM_LAUNCH(F_RASTER, s, k_sq_final<SQ_FAST>, m->num_sms * 8, 256, 0, A, (const int*)m->sq_coarse.p,
               (const int*)(m->sq_ctr.p + 1));
    if (!inc) {
        // the incremental passes that follow read and write only changes of
        // the dirty flags: they start from all clean
        FEM_TRY(ensure(m->tdirty, (size_t)T, s));
        FEM_CUDA(cudaMemsetAsync(m->tdirty.p, 0, (size_t)T, s));
        FEM_CUDA(cudaMemcpyAsync(m->uvk.p, uv, sizeof(double) * V, cudaMemcpyDeviceToDevice, s));
        if (uvf) FEM_CUDA(cudaMemcpyAsync(m->uvfk.p, uvf, sizeof(float2) * V, cudaMemcpyDeviceToDevice, s));
    }
    m->inc_ok = true;
    m->inc_V = V;
    m->inc_T = T;
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
