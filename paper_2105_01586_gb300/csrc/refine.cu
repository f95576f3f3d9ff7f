// refine.cu -- spatial optimisation (Sec. 3, adapted): top-k selection of
// the triangles with the largest squared error and their refinement by
// newest-vertex bisection (NVB).
//
// Edge marks.  Every edge that can be bisected has a midpoint on the pixel
// grid, and distinct edges have distinct midpoints, so a bitmap with one bit
// per pixel is a collision-free set of marked edges (bmM) and of the
// refinement edges of selected triangles (bmS).  No neighbour lists are kept.
// Closure: a triangle with a marked leg marks its refinement edge; sweeps
// repeat until nothing changes (marks only grow, so a sweep that adds none
// saw the fixpoint).
// Numbering.  The marked midpoints are exactly the new vertices; the id of
// the midpoint at pixel p is V + (number of set bits before p), i.e. new
// vertices are numbered by ascending pixel index.  One exclusive scan over
// the flags [gen-1 bisections | gen-2 of kept children | gen-2 of new
// children] gives every new triangle its id in (generation, parent id) order.
#include <cmath>
#include <utility>

#include "fem_internal.cuh"
#include "scan.cuh"

namespace fem {

constexpr int kTopkThreads = 256;

__device__ __forceinline__ bool lattice_mid(int2 p, int2 q) { return (((p.x + q.x) | (p.y + q.y)) & 1) == 0; }

__device__ __forceinline__ long long mid_pixel(int2 p, int2 q, int N) {
    return (long long)((p.y + q.y) >> 1) * N + ((p.x + q.x) >> 1);
}

__device__ __forceinline__ bool test_bit(const unsigned* bm, long long p) {
    return (__ldcg(&bm[p >> 5]) >> (p & 31)) & 1u;
}

// ------------------------------------------------------------------ top-k
struct TopkArgs {
    const double* keys;
    const int4* tri;
    const int2* vxy;
    int T;
    double frac;
    long long vcap;          // V* - V
    unsigned* hist;          // 12 * 256 counters, zeroed
    unsigned long long* below_max;  // zeroed
    unsigned* bar;
    int* err;
    int* out_k;              // k
    unsigned long long* out_thr;    // [0] hi, [1] lo of the k-th composite key
    double* red;
    double* out_margin;
    Dom D;  // the image within the domain (eligibility)
};

__device__ __forceinline__ unsigned long long comp_hi(const TopkArgs& A, int t) {
    int4 tr = A.tri[t];
    int2 a = A.vxy[tr.x], b = A.vxy[tr.y], c = A.vxy[tr.z];
    if (!dom_eligible(a.x, a.y, b.x, b.y, c.x, c.y, A.D)) return 0ull;
    return (unsigned long long)__double_as_longlong(A.keys[t]) | (1ull << 63);
}

// Bucket of the k-th largest element from a 256-bin histogram, by one warp:
// lane i holds bins 255-8i .. 248-8i (from the top), a warp scan gives the
// counts above each lane's group, and the lane whose group crosses krem
// walks its 8 bins.  Returns the bin; *above = elements in higher bins.
template <class Count>
__device__ __forceinline__ int warp_pick_bucket(const Count* hist, long long krem, long long* above) {
    const unsigned FULL = 0xffffffffu;
    int lane = threadIdx.x & 31;
    long long c[8], grp = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        c[j] = (long long)hist[255 - 8 * lane - j];
        grp += c[j];
    }
    long long incl = grp;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    long long excl = incl - grp;
    unsigned hit = __ballot_sync(FULL, excl < krem && incl >= krem);
    int chosen = 0;
    long long cum = 0;
    if (hit) {
        int l = __ffs(hit) - 1;
        if (lane == l) {
            cum = excl;
            int b = 255 - 8 * lane;
            for (int j = 0; j < 8; ++j, --b) {
                if (cum + c[j] >= krem) { chosen = b; break; }
                cum += c[j];
            }
        }
        chosen = __shfl_sync(FULL, chosen, l);
        cum = __shfl_sync(FULL, cum, l);
    }
    *above = cum;
    return chosen;
}

__device__ __forceinline__ unsigned digit_of(unsigned long long hi, unsigned lo, int d) {
    return d < 8 ? (unsigned)(hi >> (56 - 8 * d)) & 255u : (lo >> (24 - 8 * (d - 8))) & 255u;
}

__global__ void __launch_bounds__(kTopkThreads) k_topk(TopkArgs A) {
    pdl_wait();
    __shared__ unsigned s_hist[256];
    __shared__ unsigned long long s_pre_hi;
    __shared__ unsigned s_pre_lo;
    __shared__ long long s_krem;
    int tid0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    // eligible count -> k
    __shared__ unsigned s_ne;
    if (threadIdx.x == 0) s_ne = 0;
    __syncthreads();
    unsigned ne_loc = 0;
    for (int t = tid0; t < A.T; t += stride) ne_loc += comp_hi(A, t) ? 1u : 0u;
    ne_loc = warp_sum(ne_loc);
    if ((threadIdx.x & 31) == 0 && ne_loc) atomicAdd(&s_ne, ne_loc);
    __syncthreads();
    if (threadIdx.x == 0 && s_ne) atomicAdd(&A.hist[12 * 256], s_ne);  // slot after the histograms
    if (!grid_barrier(A.bar, A.err)) return;
    long long ne = (long long)__ldcg(&A.hist[12 * 256]);
    long long k = (long long)ceil(A.frac * (double)A.T);
    if (k < 1) k = 1;
    if (k > ne) k = ne;
    if (k > A.vcap) k = A.vcap;
    if (k < 0) k = 0;
    if (tid0 == 0) *A.out_k = (int)k;
    if (k == 0) return;
    if (threadIdx.x == 0) { s_pre_hi = 0; s_pre_lo = 0; s_krem = k; }
    __syncthreads();
    for (int d = 0; d < 12; ++d) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) s_hist[i] = 0;
        __syncthreads();
        unsigned long long pre_hi = s_pre_hi;
        unsigned pre_lo = s_pre_lo;
        // bits already decided: the top 8*d bits of the 96-bit composite
        unsigned long long mhi = d >= 8 ? ~0ull : (d == 0 ? 0ull : (~0ull << (64 - 8 * d)));
        unsigned mlo = d <= 8 ? 0u : (~0u << (32 - 8 * (d - 8)));
        for (int t = tid0; t < A.T; t += stride) {
            unsigned long long hi = comp_hi(A, t);
            unsigned lo = ~(unsigned)t;
            if ((hi & mhi) == pre_hi && (lo & mlo) == pre_lo) atomicAdd(&s_hist[digit_of(hi, lo, d)], 1u);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 256; i += blockDim.x)
            if (s_hist[i]) atomicAdd(&A.hist[d * 256 + i], s_hist[i]);
        if (!grid_barrier(A.bar, A.err)) return;
        if (threadIdx.x < 32) {
            for (int i = threadIdx.x; i < 256; i += 32) s_hist[i] = __ldcg(&A.hist[d * 256 + i]);
            __syncwarp();
            long long krem = s_krem, cum = 0;
            int chosen = warp_pick_bucket(s_hist, krem, &cum);
            if (threadIdx.x == 0) {
                s_krem = krem - cum;
                if (d < 8) s_pre_hi = pre_hi | ((unsigned long long)chosen << (56 - 8 * d));
                else s_pre_lo = pre_lo | ((unsigned)chosen << (24 - 8 * (d - 8)));
            }
        }
        __syncthreads();
    }
    unsigned long long thr_hi = s_pre_hi;
    unsigned thr_lo = s_pre_lo;
    if (tid0 == 0) { A.out_thr[0] = thr_hi; A.out_thr[1] = thr_lo; }
    // largest composite strictly below the threshold (for the decision margin)
    unsigned long long best = 0ull;
    for (int t = tid0; t < A.T; t += stride) {
        unsigned long long hi = comp_hi(A, t);
        unsigned lo = ~(unsigned)t;
        bool below = hi < thr_hi || (hi == thr_hi && lo < thr_lo);
        if (below && hi > best) best = hi;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
        best = v > best ? v : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(A.below_max, best);
    if (!grid_barrier(A.bar, A.err)) return;
    if (tid0 == 0) {
        unsigned long long bm = __ldcg(A.below_max);
        double kth = __longlong_as_double((long long)(thr_hi & ~(1ull << 63)));
        if (bm & (1ull << 63)) {
            double nxt = __longlong_as_double((long long)(bm & ~(1ull << 63)));
            *A.out_margin = kth > 0.0 ? (kth - nxt) / kth : 0.0;
        } else {
            *A.out_margin = INFINITY;
        }
    }
}

// Top-k for up to kTopkBlockMaxT triangles in one 1024-thread block (no
// device-wide barrier).  keyc holds the composite keys (0 = ineligible;
// else bit 63 set and the error's FP64 bits below it); the 96-bit order key
// is (keyc, ~id).  Radix select from the top, reading the global array until
// the current bucket fits in shared memory, then on the shared-memory
// candidate list; once the bucket holds at most kTopkRankCap keys, the
// threshold is found by counting.  The first digit is 12 bits wide (the
// flag and the 11 exponent bits), so one pass over the keys already splits
// them by binary order of magnitude; the other digits are 8 bits, the last 4.
constexpr int kTopkBlockThreads = 1024;
constexpr int kTopkCandCap = 12288;
constexpr int kTopkBlockMaxT = 1 << 20;
constexpr int kTopkBins0 = 4096;
constexpr int kTopkDigits = 12;
constexpr int kTopkRankCap = 1024;  // buckets up to this size are finished by counting
constexpr size_t kTopkBlockSmem = (size_t)kTopkCandCap * (sizeof(unsigned long long) + sizeof(unsigned));

// digit d covers key bits [tk_low(d), tk_low(d) + tk_width(d)) (bit 0 = bit 0 of lo)
__device__ __forceinline__ int tk_width(int d) { return d == 0 ? 12 : (d == kTopkDigits - 1 ? 4 : 8); }
__device__ __forceinline__ int tk_low(int d) { return d == kTopkDigits - 1 ? 0 : 84 - 8 * d; }

__device__ __forceinline__ unsigned tk_digit(unsigned long long hi, unsigned lo, int d) {
    const int low = tk_low(d);
    const unsigned long long v = low >= 32 ? hi >> (low - 32) : (hi << (32 - low)) | ((unsigned long long)lo >> low);
    return (unsigned)v & ((1u << tk_width(d)) - 1u);
}

// masks of the key bits at and above bit `low` (the prefix fixed so far)
__device__ __forceinline__ void tk_masks(int low, unsigned long long& mhi, unsigned& mlo) {
    const int P = 96 - low;  // fixed bits from the top
    mhi = P >= 64 ? ~0ull : (P <= 0 ? 0ull : ~0ull << (64 - P));
    const int lb = P - 64;
    mlo = lb <= 0 ? 0u : (lb >= 32 ? ~0u : ~0u << (32 - lb));
}

__device__ __forceinline__ void tk_set(unsigned long long& phi, unsigned& plo, int d, unsigned c) {
    const int low = tk_low(d);
    if (low >= 32) {
        phi |= (unsigned long long)c << (low - 32);
    } else {
        plo |= c << low;
        if (low + tk_width(d) > 32) phi |= (unsigned long long)(c >> (32 - low));
    }
}

// one increment of bin b (b == ~0u: none).  Aggregating equal bins per warp
// (__match_any_sync) measured slower here than plain shared atomics.
__device__ __forceinline__ void tk_hist_add(unsigned* hist, unsigned b) {
    if (b != ~0u) atomicAdd(&hist[b], 1u);
}

// Bucket of the krem-th largest key from the 4096-bin histogram, by the
// whole block: thread t holds bins 4095-4t .. 4092-4t (from the top); a
// block scan gives the count above each thread's group.
__device__ __forceinline__ void tk_block_pick(const unsigned* hist, long long krem, unsigned* s_w, int* s_bin,
                                              long long* s_above) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    unsigned c[4], grp = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        c[j] = hist[kTopkBins0 - 1 - 4 * tid - j];
        grp += c[j];
    }
    unsigned incl = grp;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const unsigned w = s_w[lane];
        unsigned wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        s_w[lane] = wi - w;
    }
    __syncthreads();
    const long long excl = (long long)s_w[wid] + (long long)(incl - grp);
    if (excl < krem && excl + (long long)grp >= krem) {
        long long cum = excl;
        int b = kTopkBins0 - 1 - 4 * tid;
        for (int j = 0; j < 4; ++j, --b) {
            if (cum + (long long)c[j] >= krem) break;
            cum += c[j];
        }
        *s_bin = b;
        *s_above = cum;
    }
    __syncthreads();
}

// Band mode (ids != nullptr): select among the *n_dev triangles ids[0..n)
// only, k = *k_total - *k_sub of them (the surely selected ones are already
// counted), out_k untouched; *extra_below (the largest key outside the
// band and below it) joins the margin.
__device__ __forceinline__ int topk_id(const int* ids, int i) { return ids ? ids[i] : i; }

__global__ void __launch_bounds__(kTopkBlockThreads) k_topk_block(const unsigned long long* __restrict__ keyc, int T,
                                                                  double frac, long long vcap, int* out_k,
                                                                  unsigned long long* out_thr, double* out_margin,
                                                                  const int* __restrict__ ids = nullptr,
                                                                  const int* __restrict__ n_dev = nullptr,
                                                                  const int* __restrict__ k_total = nullptr,
                                                                  const int* __restrict__ k_sub = nullptr,
                                                                  const unsigned long long* __restrict__ extra_below =
                                                                      nullptr) {
    pdl_wait();
    extern __shared__ unsigned char smem_raw[];
    unsigned long long* c_hi = (unsigned long long*)smem_raw;
    unsigned* c_lo = (unsigned*)(c_hi + kTopkCandCap);
    __shared__ unsigned hist[kTopkBins0];
    __shared__ unsigned long long s_pre_hi, s_best[32];
    __shared__ unsigned s_pre_lo, s_cnt32[32];
    __shared__ long long s_krem, s_above;
    __shared__ int s_n, s_cnt, s_smem, s_bin, s_m;
    __shared__ unsigned long long sv_hi[kTopkRankCap];
    __shared__ unsigned sv_lo[kTopkRankCap];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int U = 4;  // keys per thread per step of a pass over the global keys
    if (ids) T = min(*n_dev, T);
    // pass 1 over the keys: eligible count and the histogram of digit 0
    for (int i = tid; i < kTopkBins0; i += kTopkBlockThreads) hist[i] = 0;
    __syncthreads();
    unsigned ne = 0;
    for (int i0 = 0; i0 < T; i0 += U * kTopkBlockThreads) {
        unsigned long long h[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * kTopkBlockThreads + tid;
            h[u] = i < T ? keyc[topk_id(ids, i)] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ne += h[u] ? 1u : 0u;
            tk_hist_add(hist, h[u] ? tk_digit(h[u], 0u, 0) : ~0u);
        }
    }
    ne = warp_sum(ne);
    if (lane == 0) s_cnt32[wid] = ne;
    __syncthreads();
    if (tid == 0) {
        long long tot = 0;
        for (int w = 0; w < kTopkBlockThreads / 32; ++w) tot += s_cnt32[w];
        long long k;
        if (ids) {
            k = (long long)*k_total - (long long)*k_sub;
            if (k > tot) k = tot;
            if (k < 0) k = 0;
        } else {
            k = (long long)ceil(frac * (double)T);
            if (k < 1) k = 1;
            if (k > tot) k = tot;
            if (k > vcap) k = vcap;
            if (k < 0) k = 0;
            *out_k = (int)k;
        }
        s_krem = k;
        s_pre_hi = 0;
        s_pre_lo = 0;
        s_smem = 0;
        s_n = 0;
    }
    __syncthreads();
    if (s_krem == 0) return;
    // largest key below the bucket of the threshold, over the keys left
    // outside the shared-memory candidates (for the decision margin)
    unsigned long long best = extra_below ? *extra_below : 0ull;
    for (int d = 0; d < kTopkDigits; ++d) {
        const unsigned long long pre_hi = s_pre_hi;
        const unsigned pre_lo = s_pre_lo;
        if (d > 0) {  // digit 0's histogram came with the eligible count
            unsigned long long mhi;
            unsigned mlo;
            tk_masks(tk_low(d - 1), mhi, mlo);
            for (int i = tid; i < 256; i += kTopkBlockThreads) hist[i] = 0;
            __syncthreads();
            if (!s_smem) {
                for (int i0 = 0; i0 < T; i0 += U * kTopkBlockThreads) {
                    unsigned long long h[U];
                    unsigned l[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int i = i0 + u * kTopkBlockThreads + tid;
                        const int t = i < T ? topk_id(ids, i) : 0;
                        h[u] = i < T ? keyc[t] : 0ull;
                        l[u] = ~(unsigned)t;
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const bool in = h[u] && (h[u] & mhi) == pre_hi && (l[u] & mlo) == pre_lo;
                        tk_hist_add(hist, in ? tk_digit(h[u], l[u], d) : ~0u);
                    }
                }
            } else {
                const int n = s_n;
                for (int i0 = 0; i0 < n; i0 += kTopkBlockThreads) {
                    const int i = i0 + tid;
                    bool in = false;
                    unsigned b = ~0u;
                    if (i < n) {
                        const unsigned long long hi = c_hi[i];
                        const unsigned lo = c_lo[i];
                        in = (hi & mhi) == pre_hi && (lo & mlo) == pre_lo;
                        if (in) b = tk_digit(hi, lo, d);
                    }
                    tk_hist_add(hist, b);
                }
            }
            __syncthreads();
        }
        if (d == 0) {
            tk_block_pick(hist, s_krem, s_cnt32, &s_bin, &s_above);
        } else if (tid < 32) {
            long long cum = 0;
            const int chosen = warp_pick_bucket(hist, s_krem, &cum);
            if (tid == 0) {
                s_bin = chosen;
                s_above = cum;
            }
        }
        __syncthreads();
        if (tid == 0) {
            const unsigned c = (unsigned)s_bin;
            s_krem -= s_above;
            s_cnt = (int)hist[c];
            unsigned long long ph = pre_hi;
            unsigned pl = pre_lo;
            tk_set(ph, pl, d, c);
            s_pre_hi = ph;
            s_pre_lo = pl;
        }
        __syncthreads();
        if (!s_smem && d < kTopkDigits - 1 && s_cnt <= kTopkCandCap) {
            // collect the bucket; every key outside it lies wholly above or
            // wholly below it, and the largest below joins the margin
            const unsigned long long nh = s_pre_hi;
            const unsigned nl = s_pre_lo;
            unsigned long long mhi;
            unsigned mlo;
            tk_masks(tk_low(d), mhi, mlo);
            for (int i0 = 0; i0 < T; i0 += U * kTopkBlockThreads) {
                unsigned long long h[U];
                unsigned l[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = i0 + u * kTopkBlockThreads + tid;
                    const int t = i < T ? topk_id(ids, i) : 0;
                    h[u] = i < T ? keyc[t] : 0ull;
                    l[u] = ~(unsigned)t;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (!h[u]) continue;  // ineligible (or past the end)
                    const unsigned long long ph = h[u] & mhi;
                    const unsigned pl = l[u] & mlo;
                    if (ph == nh && pl == nl) {
                        const int pos = atomicAdd(&s_n, 1);
                        c_hi[pos] = h[u];
                        c_lo[pos] = l[u];
                    } else if ((ph < nh || (ph == nh && pl < nl)) && h[u] > best) {
                        best = h[u];
                    }
                }
            }
            __syncthreads();
            if (tid == 0) s_smem = 1;
            __syncthreads();
        }
        if (s_smem && s_cnt <= kTopkRankCap) {
            // few keys left in the bucket: copy them out of the candidates
            // and take the krem-th largest by counting, for each, the keys
            // above it (keys are distinct: the id is part of the key)
            const unsigned long long nh = s_pre_hi;
            const unsigned nl = s_pre_lo;
            unsigned long long mhi;
            unsigned mlo;
            tk_masks(tk_low(d), mhi, mlo);
            if (tid == 0) s_m = 0;
            __syncthreads();
            const int n = s_n;
            for (int i = tid; i < n; i += kTopkBlockThreads) {
                const unsigned long long hi = c_hi[i];
                const unsigned lo = c_lo[i];
                if ((hi & mhi) == nh && (lo & mlo) == nl) {
                    const int pos = atomicAdd(&s_m, 1);
                    if (pos < kTopkRankCap) {
                        sv_hi[pos] = hi;
                        sv_lo[pos] = lo;
                    }
                }
            }
            __syncthreads();
            const int m = min(s_m, kTopkRankCap);
            const long long krem = s_krem;
            if (tid < m) {
                const unsigned long long hi = sv_hi[tid];
                const unsigned lo = sv_lo[tid];
                int above = 0;
                for (int j = 0; j < m; ++j) {
                    const unsigned long long hj = sv_hi[j];
                    above += (hj > hi || (hj == hi && sv_lo[j] > lo)) ? 1 : 0;
                }
                if ((long long)above == krem - 1) {
                    s_pre_hi = hi;
                    s_pre_lo = lo;
                }
            }
            __syncthreads();
            break;
        }
    }
    const unsigned long long thr_hi = s_pre_hi;
    const unsigned thr_lo = s_pre_lo;
    // largest key strictly below the threshold among the candidates (or,
    // when they never fitted in shared memory, among all keys)
    if (s_smem) {
        for (int i = tid; i < s_n; i += kTopkBlockThreads) {
            const unsigned long long hi = c_hi[i];
            const unsigned lo = c_lo[i];
            if ((hi < thr_hi || (hi == thr_hi && lo < thr_lo)) && hi > best) best = hi;
        }
    } else {
        for (int i = tid; i < T; i += kTopkBlockThreads) {
            const int t = topk_id(ids, i);
            const unsigned long long hi = keyc[t];
            const unsigned lo = ~(unsigned)t;
            if ((hi < thr_hi || (hi == thr_hi && lo < thr_lo)) && hi > best) best = hi;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
        best = v > best ? v : best;
    }
    if (lane == 0) s_best[wid] = best;
    __syncthreads();
    if (tid == 0) {
        unsigned long long bm = 0;
        for (int w = 0; w < kTopkBlockThreads / 32; ++w) bm = s_best[w] > bm ? s_best[w] : bm;
        out_thr[0] = thr_hi;
        out_thr[1] = thr_lo;
        const double kth = __longlong_as_double((long long)(thr_hi & ~(1ull << 63)));
        if (bm & (1ull << 63)) {
            const double nxt = __longlong_as_double((long long)(bm & ~(1ull << 63)));
            *out_margin = kth > 0.0 ? (kth - nxt) / kth : 0.0;
        } else {
            *out_margin = INFINITY;
        }
    }
}

// mark the refinement edges of the selected triangles in bmM and bmS
__global__ void k_mark_selected(const double* __restrict__ keys, const int4* __restrict__ tri,
                                const int2* __restrict__ vxy, int T, Dom D, const unsigned long long* __restrict__ thr,
                                const int* __restrict__ kdev, unsigned* __restrict__ bmM, unsigned* __restrict__ bmS) {
    pdl_wait();
    const int N = D.N;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T || *kdev == 0) return;
    int4 tr = tri[t];
    int2 a = vxy[tr.x], b = vxy[tr.y], c = vxy[tr.z];
    if (!dom_eligible(a.x, a.y, b.x, b.y, c.x, c.y, D)) return;
    unsigned long long hi = (unsigned long long)__double_as_longlong(keys[t]) | (1ull << 63);
    unsigned lo = ~(unsigned)t;
    unsigned long long th = thr[0];
    unsigned tl = (unsigned)thr[1];
    if (hi > th || (hi == th && lo >= tl)) {
        long long p = mid_pixel(a, b, N);
        unsigned bit = 1u << (p & 31);
        atomicOr(&bmM[p >> 5], bit);
        atomicOr(&bmS[p >> 5], bit);
    }
}

// closure sweeps until a sweep adds no mark (cooperative, bounded)
__global__ void k_closure(const int4* __restrict__ tri, const int2* __restrict__ vxy, int T, int N,
                          unsigned* __restrict__ bmM, int* __restrict__ changed, int max_sweeps, unsigned* bar,
                          int* err, int* out_sweeps) {
    pdl_wait();
    int tid0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int sw = 0; sw < max_sweeps; ++sw) {
        int any = 0;
        for (int t = tid0; t < T; t += stride) {
            int4 tr = tri[t];
            int2 a = vxy[tr.x], b = vxy[tr.y], c = vxy[tr.z];
            if (!lattice_mid(a, b)) continue;  // unit triangles: never marked (no marked leg can exist)
            long long pr = mid_pixel(a, b, N);
            if (test_bit(bmM, pr)) continue;
            bool leg = (lattice_mid(b, c) && test_bit(bmM, mid_pixel(b, c, N))) ||
                       (lattice_mid(c, a) && test_bit(bmM, mid_pixel(c, a, N)));
            if (leg) {
                atomicOr(&bmM[pr >> 5], 1u << (pr & 31));
                any = 1;
            }
        }
        if (any) changed[sw] = 1;
        if (!grid_barrier(bar, err)) return;
        if (__ldcg(&changed[sw]) == 0) {
            if (tid0 == 0) *out_sweeps = sw + 1;
            return;
        }
    }
    if (tid0 == 0) {
        *out_sweeps = max_sweeps;
        atomicCAS(err, 0, (int)FEM_E_INVALID);
    }
}

// id of the new vertex at midpoint pixel p: V0 + marks before p
__device__ __forceinline__ int midpoint_id(const unsigned* __restrict__ bm, const int* __restrict__ wpre, int V0,
                                           long long p) {
    unsigned w = bm[p >> 5];
    unsigned below = w & ((1u << (p & 31)) - 1u);
    return V0 + wpre[p >> 5] + __popc(below);
}

// New vertices, numbered V0 + (marks before them) in ascending pixel order,
// with their positions and mask flags, and wpre[w] = the marks before word w
// (read by midpoint_id, which asks only for words with a mark).  The edge
// bitmaps alternate between two buffers by round, and the same pass clears
// the other round's words.  Up to kScanSmallN words (images up to about
// 2049^2) one fused scan runs over the words.  Larger bitmaps go through
// groups of 32 words (1024 pixels), a warp per group with a lane per word
// (coalesced): the groups' counts, a scan over them (1/32 of the length),
// and the numbering within each group that holds a mark (most hold none).
struct WordIn {
    const unsigned* bmM;
    unsigned* clearM;
    unsigned* clearS;
    __device__ __forceinline__ int operator()(long long w) const {
        clearM[w] = 0u;
        clearS[w] = 0u;
        return __popc(bmM[w]);
    }
};

struct NewVertexOut {
    const unsigned* bmM;
    const unsigned* bmS;
    int* wpre;
    int N, V0;
    int W, H;  // the image: every vertex outside it is a mask vertex
    int2* vxy;
    unsigned char* mask;
    int* n_new_mask;
    // the marks of word w, numbered from V0 + pre; returns the new mask vertices
    __device__ __forceinline__ int word(long long w, int pre) const {
        wpre[w] = pre;
        unsigned bits = bmM[w];
        const unsigned sbits = bmS[w];
        int id = V0 + pre, nm = 0;
        while (bits) {
            int b = __ffs(bits) - 1;
            bits &= bits - 1u;
            long long p = w * 32 + b;
            const int x = (int)(p % N), y = (int)(p / N);
            vxy[id] = make_int2(x, y);
            const int mk = (int)((sbits >> b) & 1u) | (x >= W || y >= H);
            mask[id] = (unsigned char)mk;
            nm += mk;
            id++;
        }
        return nm;
    }
    __device__ __forceinline__ void operator()(long long w, int pre, int cnt) const {
        if (cnt == 0) return;
        const int nm = word(w, pre);
        if (nm) atomicAdd(n_new_mask, nm);
    }
};

constexpr int kWordGroup = 32;

// a warp per group of 32 words: the group's marks, and the other round's
// words cleared
__global__ void k_group_count(const unsigned* __restrict__ bmM, unsigned* __restrict__ clearM,
                              unsigned* __restrict__ clearS, long long nw, int ngroups, int* __restrict__ gcnt) {
    pdl_wait();
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int g = (int)(gt >> 5), lane = threadIdx.x & 31;
    if (g >= ngroups) return;  // the same for the whole warp
    const long long w = (long long)g * kWordGroup + lane;
    int c = 0;
    if (w < nw) {
        c = __popc(bmM[w]);
        clearM[w] = 0u;
        clearS[w] = 0u;
    }
    c = warp_sum(c);
    if (lane == 0) gcnt[g] = c;
}

// a warp per group that holds a mark: each word's marks before it (the
// group's prefix plus a warp scan), then the word's new vertices
__global__ void k_group_number(NewVertexOut O, long long nw, int ngroups, const int* __restrict__ gcnt,
                               const int* __restrict__ gpre) {
    pdl_wait();
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int g = (int)(gt >> 5), lane = threadIdx.x & 31;
    if (g >= ngroups || gcnt[g] == 0) return;  // the same for the whole warp
    const long long w = (long long)g * kWordGroup + lane;
    const unsigned bits = w < nw ? O.bmM[w] : 0u;
    const int c = __popc(bits);
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    int nm = bits ? O.word(w, gpre[g] + inc - c) : 0;
    nm = warp_sum(nm);
    if (lane == 0 && nm) atomicAdd(O.n_new_mask, nm);
}

// Bisection flags [gen 1 | gen 2 of the kept child | gen 2 of the new
// child] as the input of one fused scan (the scan numbers the new
// triangles): element i of segment j = i / T belongs to triangle i - j T.
struct BisectFlagIn {
    const int4* tri;
    const int2* vxy;
    const unsigned* bmM;
    int T, N;
    int* flags;
    __device__ __forceinline__ int operator()(long long li) const {
        int seg = (int)(li / T), t = (int)(li - (long long)seg * T);
        int4 tr = tri[t];
        int2 a = vxy[tr.x], b = vxy[tr.y], c = vxy[tr.z];
        int e0 = lattice_mid(a, b) && test_bit(bmM, mid_pixel(a, b, N));
        int v = e0;
        if (seg == 1) v = e0 && lattice_mid(c, a) && test_bit(bmM, mid_pixel(c, a, N));
        if (seg == 2) v = e0 && lattice_mid(b, c) && test_bit(bmM, mid_pixel(b, c, N));
        flags[li] = v;
        return v;
    }
};

// Value of a new vertex: a new mask vertex takes the image value (g = f in
// the spatial optimisation; with its float-float copy), a new unknown the
// mean of the edge's end values as the start of the next solve.
__device__ __forceinline__ void new_vertex_value(int id, long long pix, int e0, int e1,
                                                 const unsigned char* __restrict__ mask, const float* __restrict__ f,
                                                 double* __restrict__ uv, float2* __restrict__ uvf) {
    if (mask[id]) {
        float v = f[pix];
        uv[id] = (double)v;
        uvf[id] = make_float2(v, 0.0f);
    } else {
        uv[id] = 0.5 * (uv[e0] + uv[e1]);
    }
}

__global__ void k_bisect(int4* __restrict__ tri, const int2* __restrict__ vxy, int T, int N,
                         const unsigned* __restrict__ bmM, const int* __restrict__ wpre, int V0,
                         const int* __restrict__ flags, const int* __restrict__ fscan,
                         const unsigned char* __restrict__ mask, const float* __restrict__ f, double* __restrict__ uv,
                         float2* __restrict__ uvf, const int* __restrict__ cnt, const int* __restrict__ scan_err,
                         const double* __restrict__ margin, int* __restrict__ stage, int* __restrict__ plan_err,
                         int* __restrict__ clear, unsigned char* __restrict__ tchg) {
    pdl_wait();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        // the round's counters are final (written by the kernels before
        // this one): hand them to the host (through mapped pinned memory,
        // else the host copies them) and clear the per-round counters
        // (new mask vertices, error flag, closure sweep flags) and the
        // rasterisation plan's overflow flag for the next round
        if (stage) {
#pragma unroll
            for (int i = 0; i < 8; ++i) stage[i] = cnt[i];
            stage[9] = *scan_err;
            stage[10] = *plan_err;
            *(double*)(stage + 16) = *margin;
        }
        if (clear) {
            for (int i = 6; i < 64; ++i) clear[i] = 0;
            *plan_err = 0;
        }
    }
    if (t >= T || !flags[t]) return;
    int4 tr = tri[t];
    int a = tr.x, b = tr.y, c = tr.z;
    int2 pa = vxy[a], pb = vxy[b], pc = vxy[c];
    long long pm = mid_pixel(pa, pb, N);
    int m = midpoint_id(bmM, wpre, V0, pm);
    new_vertex_value(m, pm, a, b, mask, f, uv, uvf);
    int id1 = T + fscan[t];
    int4 kept = make_int4(c, a, m, 0);   // (c, a, m) keeps id t
    int4 fresh = make_int4(b, c, m, 0);  // (b, c, m) new id
    if (flags[T + t]) {  // kept child's refinement edge (c, a) is marked
        long long p2 = mid_pixel(pc, pa, N);
        int m2 = midpoint_id(bmM, wpre, V0, p2);
        new_vertex_value(m2, p2, c, a, mask, f, uv, uvf);
        tri[T + fscan[T + t]] = make_int4(a, m, m2, 0);
        kept = make_int4(m, c, m2, 0);
    }
    if (flags[2 * T + t]) {  // new child's refinement edge (b, c) is marked
        long long p1 = mid_pixel(pb, pc, N);
        int m1 = midpoint_id(bmM, wpre, V0, p1);
        new_vertex_value(m1, p1, b, c, mask, f, uv, uvf);
        tri[T + fscan[2 * T + t]] = make_int4(c, m, m1, 0);
        fresh = make_int4(m, b, m1, 0);
    }
    tri[t] = kept;
    tri[id1] = fresh;
    if (tchg) tchg[t] = 1;  // id t now names the kept child (the other ids are new)
}

// Space-filling (Sierpinski) order of the triangles.  A newest-vertex
// bisection mesh is the leaf set of a binary tree whose natural traversal is
// a continuous curve: each triangle is entered at one end of its refinement
// edge and left at the other, and its two children are visited in the order
// that keeps the curve continuous.  With the two initial triangles entered at
// a, the entry end depends only on the triangle's type: right-angle legs
// along the axes -> entered at a, legs along the diagonals -> entered at b.
// When a triangle entered at a is bisected, (c,a,m) comes first and both
// children are entered at their b; entered at b, (b,c,m) comes first and both
// are entered at their a.  order[] lists triangle ids along the curve;
// refinement replaces each triangle by its children in curve order.
__device__ __forceinline__ int entered_at_b(int2 a, int2 c) { return (c.x != a.x && c.y != a.y) ? 1 : 0; }

// Curve order of the refined mesh as one fused scan: the input is the
// number of children that entry i of the order becomes, the output writes
// them in curve order.
struct OrderCountIn {
    const int* order;
    const int* flags;
    int T;
    __device__ __forceinline__ int operator()(long long i) const {
        int t = order[i];
        return 1 + flags[t] + flags[T + t] + flags[2 * T + t];
    }
};

// runs before k_bisect: reads the parents' geometry
struct OrderExpandOut {
    const int* order;
    const int* flags;
    const int* fscan;
    const int4* tri;
    const int2* vxy;
    int T;
    int* order_new;
    __device__ __forceinline__ void operator()(long long i, int o, int) const {
        int t = order[i];
        if (!flags[t]) {
            order_new[o] = t;
            return;
        }
        int4 tr = tri[t];
        int d = entered_at_b(vxy[tr.x], vxy[tr.z]);
        int kept = t, fresh = T + fscan[t];
        int e2 = flags[T + t], e1 = flags[2 * T + t];
        int kn = e2 ? T + fscan[T + t] : -1;      // second child of (c,a,m)
        int nn = e1 ? T + fscan[2 * T + t] : -1;  // second child of (b,c,m)
        if (d == 0) {
            // (c,a,m) part then (b,c,m) part; children are entered at b
            if (e2) { order_new[o++] = kn; order_new[o++] = kept; } else { order_new[o++] = kept; }
            if (e1) { order_new[o++] = nn; order_new[o++] = fresh; } else { order_new[o++] = fresh; }
        } else {
            // (b,c,m) part then (c,a,m) part; children are entered at a
            if (e1) { order_new[o++] = fresh; order_new[o++] = nn; } else { order_new[o++] = fresh; }
            if (e2) { order_new[o++] = kept; order_new[o++] = kn; } else { order_new[o++] = kept; }
        }
    }
};

// Up to this many triangles one block runs the closure sweeps (block
// barriers between sweeps instead of grid barriers).
constexpr int kClosureOneBlockT = 512;

// Cooperative grid: one thread per work item, at most the co-resident
// blocks (occupancy queried once per kernel).
static int coop_grid(const void* func, int threads, int work, int num_sms) {
    static const int nb_topk = [] {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)k_topk, kTopkThreads, 0);
        return nb < 1 ? 1 : nb;
    }();
    static const int nb_closure = [] {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)k_closure, 256, 0);
        return nb < 1 ? 1 : nb;
    }();
    int nb = func == (const void*)k_topk ? nb_topk : nb_closure;
    (void)threads;
    int maxb = nb * num_sms;
    int want = (work + threads - 1) / threads;
    if (want < 1) want = 1;
    return want < maxb ? want : maxb;
}

// One refinement round on the current keys (m->keys).  Returns k via k_out.
fem_status refine_round(fem_mesh* m, const float* f, double frac, long long vstar, cudaStream_t s, double* margin_out,
                        int* k_out, bool band) {
    int T = m->T, V = m->V, N = m->N;
    long long W = (m->P + 31) / 32;
    // two buffers per edge bitmap, alternating by round; fresh memory is
    // cleared once, afterwards the new-vertex scan clears the other round's
    // buffer
    if (!m->bm_clean || !m->bmM.p || !m->bmS.p || m->bmM.n < (size_t)(2 * W) || m->bmS.n < (size_t)(2 * W)) {
        FEM_TRY(ensure(m->bmM, (size_t)(2 * W), s));
        FEM_TRY(ensure(m->bmS, (size_t)(2 * W), s));
        FEM_CUDA(cudaMemsetAsync(m->bmM.p, 0, sizeof(unsigned) * m->bmM.n, s));
        FEM_CUDA(cudaMemsetAsync(m->bmS.p, 0, sizeof(unsigned) * m->bmS.n, s));
        m->bm_clean = true;
        m->bm_parity = 0;
    }
    m->bm_clean = false;  // until this round's clearing pass is known to have run
    unsigned* bmM = m->bmM.p + (m->bm_parity ? W : 0);
    unsigned* bmS = m->bmS.p + (m->bm_parity ? W : 0);
    unsigned* bmM_other = m->bmM.p + (m->bm_parity ? 0 : W);
    unsigned* bmS_other = m->bmS.p + (m->bm_parity ? 0 : W);
    FEM_TRY(ensure(m->wpre, (size_t)W + 1, s));
    FEM_TRY(ensure(m->topk_hist, (size_t)12 * 256 + 8, s));
    FEM_TRY(ensure(m->flags, (size_t)3 * T + 1, s));
    FEM_TRY(ensure(m->fscan, (size_t)3 * T + 1, s));
    // capacity: at most one new vertex per edge (E = V + T - 1), at most 4 children per triangle
    FEM_TRY(ensure_mesh_capacity(m, V + T + V + 4, 4 * T, s));
    unsigned* hist = m->topk_hist.p;
    int* kdev = m->dcount.p + 2;
    int* sweeps = m->dcount.p + 3;
    int* nnew = m->dcount.p + 4;
    int* ntri = m->dcount.p + 5;
    int* nmask_new = m->dcount.p + 6;
    int* changed = m->dcount.p + 16;  // 48 flags
    unsigned long long* thr = (unsigned long long*)(m->dscal.p + 8);
    unsigned long long* below = (unsigned long long*)(m->dscal.p + 10);
    double* margin = m->dscal.p + 11;
    int* err = m->dcount.p + 7;
    // counters 6..63 (new mask vertices, error flag, closure sweep flags)
    // are zero: cleared at creation and by the previous round's k_bisect,
    // or here when a round stopped before it
    if (!m->round_ctr_clear) FEM_CUDA(cudaMemsetAsync(m->dcount.p + 6, 0, sizeof(int) * 58, s));
    m->round_ctr_clear = false;

    TopkArgs A;
    A.keys = m->keys.p;
    A.tri = m->tri.p;
    A.vxy = m->vxy.p;
    A.T = T;
    A.frac = frac;
    A.vcap = vstar - V;
    A.hist = hist;
    A.below_max = below;
    A.bar = m->bar.p;
    A.err = err;
    A.out_k = kdev;
    A.out_thr = thr;
    A.red = m->red.p;
    A.out_margin = margin;
    A.D = dom_of(m);
    // set once per process (thread-safe static initialisation); a failure shows at the launch
    static const bool attr_set = [] {
        return cudaFuncSetAttribute(k_topk_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kTopkBlockSmem) == cudaSuccess;
    }();
    (void)attr_set;
    if (band) {
        // fast keys: k and the band were set by raster_keys_fast; the exact
        // selection runs over the band only
        int* fc = (int*)(m->fast_hist.p + 2 * kFastBins);
        FEM_LAUNCH(F_TOPK, s, k_topk_block, 1, kTopkBlockThreads, kTopkBlockSmem, m->keyc.p, T, frac, vstar - V,
                   (int*)nullptr, thr, margin, m->band.p, fc + FC_BAND, kdev, fc + FC_IN,
                   (const unsigned long long*)(m->dscal.p + 18));
    } else if (T <= kTopkBlockMaxT && m->keyc.p && m->keyc.n >= (size_t)T) {
        FEM_LAUNCH(F_TOPK, s, k_topk_block, 1, kTopkBlockThreads, kTopkBlockSmem, m->keyc.p, T, frac, vstar - V,
                   kdev, thr, margin, nullptr, nullptr, nullptr, nullptr, nullptr);
    } else {
        FEM_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned) * (12 * 256 + 1), s));
        FEM_CUDA(cudaMemsetAsync(below, 0, sizeof(unsigned long long), s));
        void* args[] = {&A};
        int grid = coop_grid((const void*)k_topk, kTopkThreads, T, m->num_sms);
        FEM_TRY(launch_coop(F_TOPK, (const void*)k_topk, grid, kTopkThreads, 0, s, args, "k_topk"));
    }
    int tb = (T + 255) / 256;
    FEM_LAUNCH(F_REFINE, s, k_mark_selected, tb, 256, 0, m->keys.p, m->tri.p, m->vxy.p, T, dom_of(m), thr, kdev, bmM,
               bmS);
    {
        int max_sweeps = 48;
        void* args[] = {(void*)&m->tri.p, (void*)&m->vxy.p, (void*)&T, (void*)&N, (void*)&bmM,
                        (void*)&changed, (void*)&max_sweeps, (void*)&m->bar.p, (void*)&err, (void*)&sweeps};
        int grid = T <= kClosureOneBlockT ? 1 : coop_grid((const void*)k_closure, 256, T, m->num_sms);
        FEM_TRY(launch_coop(F_REFINE, (const void*)k_closure, grid, 256, 0, s, args, "k_closure"));
    }
    int* stage_dev = m->host_stage_dev ? (int*)m->host_stage_dev + kRoundStageInts : nullptr;
    const NewVertexOut nvo{bmM, bmS, (int*)m->wpre.p, N, V, m->W, m->H, m->vxy.p, m->mask.p, nmask_new};
    if (W <= kScanSmallN) {
        FEM_TRY(scan_fused(m, WordIn{bmM, bmM_other, bmS_other}, nvo, (int)W, s, nnew, F_REFINE));
    } else {
        const int groups = (int)((W + kWordGroup - 1) / kWordGroup);
        FEM_TRY(ensure(m->gcnt, (size_t)2 * groups, s));
        int* gcnt = m->gcnt.p;
        int* gpre = m->gcnt.p + groups;
        const int gb = (int)(((long long)groups * 32 + 255) / 256);
        FEM_LAUNCH(F_REFINE, s, k_group_count, gb, 256, 0, (const unsigned*)bmM, bmM_other, bmS_other, (long long)W,
                   groups, gcnt);
        FEM_TRY(scan_fused(m, ScanLoad{gcnt}, ScanStoreTo{gpre}, groups, s, nnew, F_REFINE));
        FEM_LAUNCH(F_REFINE, s, k_group_number, gb, 256, 0, nvo, (long long)W, groups, (const int*)gcnt,
                   (const int*)gpre);
    }
    m->bm_parity ^= 1;
    FEM_TRY(scan_fused(m, BisectFlagIn{m->tri.p, m->vxy.p, bmM, T, N, m->flags.p}, ScanStore{m->fscan.p}, 3 * T, s,
                       ntri, F_REFINE));
    // curve order of the refined mesh (before k_bisect overwrites the parents)
    FEM_TRY(ensure(m->order_tmp, (size_t)4 * T, s));
    FEM_TRY(scan_fused(m, OrderCountIn{m->order.p, m->flags.p, T},
                       OrderExpandOut{m->order.p, m->flags.p, m->fscan.p, m->tri.p, m->vxy.p, T, m->order_tmp.p}, T,
                       s, nullptr, F_REFINE));
    FEM_LAUNCH(F_REFINE, s, k_bisect, tb, 256, 0, m->tri.p, m->vxy.p, T, N, bmM, (const int*)m->wpre.p, V,
               m->flags.p, m->fscan.p, m->mask.p, f, m->uv.p, m->uvf.p, (const int*)m->dcount.p,
               (const int*)(m->dflag.p + 8), (const double*)margin, m->host_stage_dev ? stage_dev : nullptr,
               m->dflag.p + 0, m->host_stage_dev ? m->dcount.p : nullptr,
               m->inc_ok && m->tchg.n >= (size_t)T ? m->tchg.p : nullptr);
    // k, sweeps, new counts, margin, errors: written by k_bisect into mapped
    // pinned memory, else copied (and the counters cleared here)
    int* hs = (int*)m->host_stage + kRoundStageInts;
    bool ahead = false;
    int Vcap = 0, Tcap = 0;
    if (!m->host_stage_dev) {
        FEM_CUDA(cudaMemcpyAsync(hs, m->dcount.p, 8 * sizeof(int), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaMemcpyAsync(hs + 9, m->dflag.p + 8, sizeof(int), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaMemcpyAsync(hs + 10, m->dflag.p + 0, sizeof(int), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaMemcpyAsync((double*)(hs + 16), margin, sizeof(double), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaMemsetAsync(m->dflag.p + 0, 0, sizeof(int), s));
        FEM_CUDA(cudaStreamSynchronize(s));
    } else {
        m->round_ctr_clear = true;
        // The next round starts with the system of the refined mesh: it is
        // launched behind k_bisect (it takes the refined counts from the
        // device), and the host waits for k_bisect alone, so the build runs
        // while the host reads the counts and prepares the next launches.
        if (!m->round_ev) FEM_CUDA(cudaEventCreateWithFlags(&m->round_ev, cudaEventDisableTiming));
        FEM_CUDA(cudaEventRecord(m->round_ev, s));
        fem_status st = build_system_ahead(m, s, V, T, stage_dev, &Vcap, &Tcap);
        if (st != FEM_OK) {
            // its arrays may have been reallocated: no system is valid now
            m->sys_version = -1;
            cudaEventSynchronize(m->round_ev);
            return st;
        }
        ahead = true;
        FEM_CUDA(cudaEventSynchronize(m->round_ev));
    }
    int k = hs[2], nn = hs[4], nt = hs[5], nkm = hs[6], e = hs[7] ? hs[7] : hs[9];
    if (ahead && (hs[10] || e || (k > 0 && nn <= 0))) m->sys_version = -1;  // the build saw another mesh
    if (hs[10]) {  // the rasterisation plan of this round overflowed: its keys are incomplete
        m->plan_version = -1;
        set_error("refinement: rasterisation plan overflow");
        return FEM_E_INVALID;
    }
    m->bm_clean = true;  // the round ran to the end: the next buffer is clear
    double mg = *(double*)(hs + 16);
    if (e) {
        reset_coop_state(m, s);
        set_error(e == FEM_E_TIMEOUT ? "refinement: a grid barrier wait ran out" : "refinement: closure did not settle");
        return (fem_status)e;
    }
    if (k > 0 && nn <= 0) {
        set_error("refinement: selected triangles produced no new vertex");
        return FEM_E_INVALID;
    }
    if (k_out) *k_out = k;
    if (margin_out) *margin_out = mg;
    if (k > 0) {
        std::swap(m->order, m->order_tmp);
        m->V = V + nn;
        m->T = T + nt;
        m->nK += nkm;
        m->nU = m->V - m->nK;
        m->mesh_version++;
        // the build ahead ran to the end when the refined mesh fit its
        // capacities: the system and the next solve's right-hand side and
        // start (from the vertex values k_bisect completed) are in place
        if (ahead && m->V <= Vcap && m->T <= Tcap) {
            m->sys_version = m->mesh_version;
            m->sys_full = false;  // the unknowns' rows only
            m->rhs_fresh = m->nU > 0;
            note_bytes(F_ASSEMBLY, build_bytes(m->T, m->V, m->nU, m->nU > 0, true));
        }
    }
    return FEM_OK;
}

}  // namespace fem

using namespace fem;

// keys summed over the channels -> composite selection keys (eligible
// triangles: the FP64 key bits under the top bit; the others 0)
__global__ void k_add_keys(int T, const double* __restrict__ add, double* __restrict__ keys) {
    pdl_wait();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T) keys[t] += add[t];
}

__global__ void k_keyc_from_keys(int T, const int4* __restrict__ tri, const int2* __restrict__ vxy, Dom D,
                                 const double* __restrict__ keys, unsigned long long* __restrict__ keyc) {
    pdl_wait();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int4 tr = tri[t];
    const int2 a = vxy[tr.x], b = vxy[tr.y], c = vxy[tr.z];
    keyc[t] = dom_eligible(a.x, a.y, b.x, b.y, c.x, c.y, D)
                  ? ((unsigned long long)__double_as_longlong(keys[t]) | (1ull << 63))
                  : 0ull;
}

// Channel c >= 1 of a colour image in the mesh's working arrays: its vertex
// values (with their float-float copies), its squared image and its padded
// image are swapped with channel 0's, so that the solver and the error pass
// run on it unchanged; a second call swaps them back.
static void swap_channel(fem_mesh* m, int c) {
    std::swap(m->uv, m->uvc[c - 1]);
    std::swap(m->uvf, m->uvfc[c - 1]);
    std::swap(m->fsq, m->fsqc[c - 1]);
    std::swap(m->fedge, m->fedgec[c - 1]);
    std::swap(m->fpad, m->fpadc[c - 1]);
}

// The spatial optimisation of Sec. 3 (adapted) on C channels of W x H
// images (plane c of f at c W H).  C = 1 is the grey case; with more
// channels (reading R10) each channel has its own mask values and Laplace
// solve, and a triangle's error is the sum of its channels' exact errors.
static fem_status spatial_refine(fem_mesh* m, const float* f_dev, int C, double density, const fem_params* p,
                                 cudaStream_t s) {
    // within the loop only Laplace solves read the system, so the systems
    // built ahead of the host hold the unknown vertices' rows only
    struct UnknownRowsScope {
        fem_mesh* m;
        explicit UnknownRowsScope(fem_mesh* mm) : m(mm) { m->unknown_rows_ok = true; }
        ~UnknownRowsScope() { m->unknown_rows_ok = false; }
    } rows_scope(m);
    m->last_stream = s;
    m->stats = fem_stats{};
    m->stats.min_margin = INFINITY;
    long long vstar = (long long)ceil(density * (double)m->PI);  // vertices per image pixel
    int round = 0;
    // solve results are accumulated on the device and read once at the end
    FEM_TRY(solve_totals_reset(m, s));
    FEM_CUDA(cudaMemsetAsync(m->dflag.p + 8, 0, sizeof(int), s));  // scan wait flag
    // a W x H image is padded to the domain (the values of mask vertices
    // outside it); only its own pixels are data.  The error passes read each
    // channel's image as squares, laid out once per call.
    const float* fc[kMaxChannels] = {};
    int valid[kMaxChannels] = {};  // vertices with a value, per extra channel
    for (int c = C - 1; c >= 0; --c) {
        if (c > 0) swap_channel(m, c);
        FEM_TRY(domain_image(m, f_dev + (size_t)c * m->PI, s, &fc[c]));
        FEM_TRY(sq_image(m, fc[c], s));
        if (c > 0) {
            FEM_TRY(ensure(m->uv, (size_t)m->V, s));
            FEM_TRY(ensure(m->uvf, (size_t)m->V, s));
            FEM_CUDA(cudaMemsetAsync(m->uv.p, 0, sizeof(double) * m->V, s));
            FEM_CUDA(cudaMemsetAsync(m->uvf.p, 0, sizeof(float2) * m->V, s));
            valid[c] = m->V;
            swap_channel(m, c);
        }
    }
    // channel 0's mask vertices take their image values once; vertices made
    // by the refinement get theirs when they are created (k_bisect)
    FEM_TRY(set_uv_from_f(m, fc[0], s));
    const bool fp64 = p->precision == FEM_PREC_FP64;
    while ((long long)m->V < vstar && (p->max_rounds <= 0 || round < p->max_rounds)) {
        Nvtx round_range("spatial round");
        FEM_TRY(check_cancel(m));
        // solve_laplace builds the system of the refined mesh (with its
        // right-hand side in the same kernel)
        fem_status st = solve_laplace(m, fp64, p->tol, p->maxit, s, nullptr, nullptr, true);
        if (st != FEM_OK) return st;
        FEM_TRY(ensure(m->keys, (size_t)m->T, s));
        FEM_TRY(ensure(m->keyc, (size_t)m->T, s));
        // in the spatial loop every vertex value was just written together with
        // its float-float copy (mask vertices from f, unknowns by the solve);
        // the fast keys serve one channel
        bool band = C == 1 && (p->fast_keys > 0 || (p->fast_keys < 0 && m->PI >= 2049LL * 2049));
        {
            Nvtx pass_range("error pass");
            if (band)
                FEM_TRY(raster_keys_fast(m, m->uv.p, m->uvf.p, p->topk_frac, vstar - m->V, s,
                                         round > 0 && p->fast_keys != 2));
            else
                FEM_TRY(raster_errors(m, m->uv.p, m->uvf.p, m->keys.p, s, C == 1 ? m->keyc.p : nullptr));
        }
        if (C > 1) {
            Nvtx ch_range("other channels");
            FEM_TRY(ensure(m->keys_acc, (size_t)m->T, s));
            const int tb = (m->T + 255) / 256;
            for (int c = 1; c < C; ++c) {
                swap_channel(m, c);
                fem_status cs = FEM_OK;
                do {
                    // vertices made since the channel's last solve start at 0
                    // (the solve warm-starts from the others)
                    cs = ensure(m->uv, (size_t)m->V, s, (size_t)valid[c]);
                    if (cs) break;
                    cs = ensure(m->uvf, (size_t)m->V, s, (size_t)valid[c]);
                    if (cs) break;
                    if (m->V > valid[c]) {
                        cudaMemsetAsync(m->uv.p + valid[c], 0, sizeof(double) * (m->V - valid[c]), s);
                        cudaMemsetAsync(m->uvf.p + valid[c], 0, sizeof(float2) * (m->V - valid[c]), s);
                        valid[c] = m->V;
                    }
                    cs = set_uv_from_f(m, fc[c], s);
                    if (cs) break;
                    cs = solve_laplace(m, fp64, p->tol, p->maxit, s, nullptr, nullptr, true);
                    if (cs) break;
                    cs = raster_errors(m, m->uv.p, m->uvf.p, m->keys_acc.p, s, nullptr);
                } while (0);
                swap_channel(m, c);
                FEM_TRY(cs);
                FEM_LAUNCH(F_RASTER, s, k_add_keys, tb, 256, 0, m->T, (const double*)m->keys_acc.p, m->keys.p);
            }
            FEM_LAUNCH(F_RASTER, s, k_keyc_from_keys, tb, 256, 0, m->T, m->tri.p, m->vxy.p, dom_of(m),
                       (const double*)m->keys.p, m->keyc.p);
        }
        double margin = 0.0;
        int k = 0;
        {
            Nvtx refine_range("top-k and refinement");
            FEM_TRY(refine_round(m, fc[0], p->topk_frac, vstar, s, &margin, &k, band));
        }
        if (k == 0) break;
        if (margin < m->stats.min_margin) m->stats.min_margin = margin;
        round++;
    }
    m->rhs_fresh = false;  // only the loop's next solve may take the right-hand side built ahead
    fem_status st = solve_totals_read(m, s);
    m->stats.rounds = round;
    return st;
}

extern "C" fem_status fem_spatial_refine(fem_mesh* m, const float* f_dev, double density, const fem_params* p,
                                         void* stream) {
    Nvtx range("fem_spatial_refine");
    if (!m || !f_dev || !(density > 0.0) || density > 1.0) {
        set_error("fem_spatial_refine: null argument or density outside (0, 1]");
        return FEM_E_INVALID;
    }
    fem_params d;
    fem_params_default(&d);
    return spatial_refine(m, f_dev, 1, density, p ? p : &d, (cudaStream_t)stream);
}

extern "C" fem_status fem_spatial_refine_channels(fem_mesh* m, const float* f_dev, int channels, double density,
                                                  const fem_params* p, void* stream) {
    Nvtx range("fem_spatial_refine_channels");
    if (!m || !f_dev || !(density > 0.0) || density > 1.0 || channels < 1 || channels > kMaxChannels) {
        set_error("fem_spatial_refine_channels: null argument, density outside (0, 1] or channels outside 1..4");
        return FEM_E_INVALID;
    }
    fem_params d;
    fem_params_default(&d);
    return spatial_refine(m, f_dev, channels, density, p ? p : &d, (cudaStream_t)stream);
}
