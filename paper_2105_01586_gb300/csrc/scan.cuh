// scan.cuh -- single-launch exclusive scans with fused producer and consumer.
//
// k_scan_fused<In, Out> runs a decoupled look-back scan: tiles take their
// index from an atomic counter in the order they start, so every tile's
// predecessors are running or finished; each tile publishes its aggregate,
// then its inclusive prefix, in a 64-bit status word (epoch | flag | value)
// with release semantics.  The epoch changes every call, so status words
// never need clearing.  The first warp of a tile looks back over 32
// predecessors at a time.  Waits are bounded: after kLookbackLimitNs the
// tile records FEM_E_TIMEOUT and stops waiting.
//
// The input of element i is in(i) (which may have side effects: it is
// evaluated exactly once), the consumer out(i, prefix, value) receives the
// exclusive prefix and the element's own value.  A count -> scan -> scatter
// sequence is therefore one launch: the count is the input and the scatter
// the output, as long as the scatter of element i needs only its own prefix.
#pragma once

#include "fem_internal.cuh"

namespace fem {

constexpr int SCAN_BT = 256;
constexpr int SCAN_IPT = 8;  // elements per thread of plain scans
constexpr int SCAN_TILE = SCAN_BT * SCAN_IPT;
constexpr unsigned long long kLookbackLimitNs = 1000000000ull;

// exclusive scan of v[] within the block; returns the block total
template <int IPT = SCAN_IPT>
__device__ __forceinline__ int block_exclusive_scan(int (&v)[IPT]) {
    __shared__ int s_warp[SCAN_BT / 32];
    __shared__ int s_total;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int sum = 0;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        int t = v[i];
        v[i] = sum;
        sum += t;
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = lane < SCAN_BT / 32 ? s_warp[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < SCAN_BT / 32) s_warp[lane] = wi - w;  // exclusive warp offsets
    }
    __syncthreads();
    int base = s_warp[wid] + incl - sum;
#pragma unroll
    for (int i = 0; i < IPT; ++i) v[i] += base;
    if (threadIdx.x == SCAN_BT - 1) s_total = base + sum;
    __syncthreads();
    int tot = s_total;
    __syncthreads();
    return tot;
}

__device__ __forceinline__ unsigned long long scan_ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void scan_st_release(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long scan_pack(unsigned epoch, unsigned flag, int value) {
    return ((unsigned long long)epoch << 34) | ((unsigned long long)flag << 32) | (unsigned)value;
}

// IPT elements per thread (contiguous per thread): 8 for plain loads, 1
// for inputs that do real work per element (one element per thread keeps
// the loads coalesced and spreads the work over more blocks)
template <class In, class Out, int IPT>
__global__ void __launch_bounds__(SCAN_BT) k_scan_fused(In in, Out out, int n, int* __restrict__ total,
                                                         unsigned long long* __restrict__ status,
                                                         unsigned long long* __restrict__ ctr,
                                                         unsigned long long base, unsigned epoch,
                                                         int* __restrict__ err) {
    pdl_wait();
    constexpr int TILE = SCAN_BT * IPT;
    __shared__ int s_tile, s_prefix;
    if (threadIdx.x == 0) s_tile = (int)(atomicAdd(ctr, 1ull) - base);
    __syncthreads();
    const int tile = s_tile;
    int v[IPT], own[IPT];
    const long long first = (long long)tile * TILE + (long long)threadIdx.x * IPT;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        own[i] = (first + i < n) ? in(first + i) : 0;
        v[i] = own[i];
    }
    const int agg = block_exclusive_scan<IPT>(v);
    // look-back by the first warp, 32 predecessors per step: lane i reads
    // the status of tile (p - i); the window is summed up to the nearest
    // tile that already holds its inclusive prefix
    if (threadIdx.x < 32) {
        const unsigned FULL = 0xffffffffu;
        const int lane = threadIdx.x;
        int prefix = 0;
        if (tile == 0) {
            if (lane == 0) scan_st_release(&status[0], scan_pack(epoch, 2, agg));
        } else {
            if (lane == 0) scan_st_release(&status[tile], scan_pack(epoch, 1, agg));
            int p = tile - 1;
            const unsigned long long t0 = globaltimer_ns();
            bool timed_out = false;
            while (p >= 0) {
                const int q = p - lane;
                const unsigned long long w = q >= 0 ? scan_ld_acquire(&status[q]) : scan_pack(epoch, 2, 0);
                const unsigned ep = (unsigned)(w >> 34), flag = (unsigned)(w >> 32) & 3u;
                const bool ready = ep == epoch && flag != 0;
                const unsigned incl = __ballot_sync(FULL, ready && flag == 2);
                const unsigned notready = __ballot_sync(FULL, !ready);
                const int stop = incl ? __ffs(incl) - 1 : 32;  // lanes 0..stop are summed
                const unsigned need = stop >= 31 ? FULL : ((2u << stop) - 1u);
                if (notready & need) {
                    // the decision to give up is taken by the whole warp
                    const bool late = globaltimer_ns() - t0 > kLookbackLimitNs;
                    if (__any_sync(FULL, late)) { timed_out = true; break; }
                    continue;
                }
                prefix += warp_sum(lane <= stop ? (int)(unsigned)w : 0);
                if (stop < 32) break;
                p -= 32;
            }
            if (timed_out && lane == 0) atomicCAS(err, 0, (int)FEM_E_TIMEOUT);
            if (lane == 0) scan_st_release(&status[tile], scan_pack(epoch, 2, prefix + agg));
        }
        if (lane == 0) {
            s_prefix = prefix;
            if ((long long)(tile + 1) * TILE >= n && total) *total = prefix + agg;
        }
    }
    __syncthreads();
    const int pre = s_prefix;
#pragma unroll
    for (int i = 0; i < IPT; ++i)
        if (first + i < n) out(first + i, v[i] + pre, own[i]);
}

// launch parameters of one scan over n elements (status words, tile
// counter, epoch); defined in mesh.cu
struct ScanPlan {
    int tiles;
    unsigned long long* status;
    unsigned long long* ctr;
    unsigned long long base;
    unsigned epoch;
    int* err;
};
fem_status scan_plan(fem_mesh* m, int n, int tile, cudaStream_t s, ScanPlan* plan);

template <int IPT, class In, class Out>
fem_status scan_fused_ipt(fem_mesh* m, In in, Out out, int n, cudaStream_t s, int* total_dev, int family) {
    ScanPlan sp;
    FEM_TRY(scan_plan(m, n, SCAN_BT * IPT, s, &sp));
    note_launch_begin(family, s);
    cudaError_t e = launch_pdl(k_scan_fused<In, Out, IPT>, dim3(sp.tiles), dim3(SCAN_BT), 0, s, in, out, n,
                               total_dev, sp.status, sp.ctr, sp.base, sp.epoch, sp.err);
    note_launch_end(family, s);
    if (e != cudaSuccess) return cuda_fail(e, "k_scan_fused");
    return FEM_OK;
}

// producer and consumer as separate element-parallel kernels (large inputs)
template <class In>
__global__ void k_scan_apply_in(In in, int* __restrict__ vals, int n) {
    pdl_wait();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) vals[i] = in(i);
}

template <class Out>
__global__ void k_scan_apply_out(Out out, const int* __restrict__ pre, const int* __restrict__ vals, int n) {
    pdl_wait();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out(i, pre[i], vals[i]);
}

struct ScanLoad {
    const int* src;
    __device__ __forceinline__ int operator()(long long i) const { return src[i]; }
};
struct ScanStoreTo {
    int* dst;
    __device__ __forceinline__ void operator()(long long i, int prefix, int) const { dst[i] = prefix; }
};

// two int scratch arrays of n elements for the unfused form; mesh.cu
fem_status scan_scratch(fem_mesh* m, int n, cudaStream_t s, int** vals, int** pre);

// Scan with producer in() and consumer out(): up to kScanSmallN elements
// one fused launch with one element per thread (per-element work spread
// over many blocks, no intermediate arrays); beyond, the producer, a plain
// scan and the consumer as three element-parallel launches, which keep
// every element's loads independent on large inputs.  *total_dev (if
// non-null) receives the sum of all inputs; n == 0 only writes the total.
constexpr int kScanSmallN = 1 << 17;

template <class In, class Out>
fem_status scan_fused(fem_mesh* m, In in, Out out, int n, cudaStream_t s, int* total_dev, int family) {
    if (n <= 0) {
        if (total_dev) FEM_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(int), s));
        return FEM_OK;
    }
    if (n <= kScanSmallN) return scan_fused_ipt<1>(m, in, out, n, s, total_dev, family);
    int *vals = nullptr, *pre = nullptr;
    FEM_TRY(scan_scratch(m, n, s, &vals, &pre));
    int blocks = (n + 255) / 256;
    note_launch_begin(family, s);
    cudaError_t e = launch_pdl(k_scan_apply_in<In>, dim3(blocks), dim3(256), 0, s, in, vals, n);
    note_launch_end(family, s);
    if (e != cudaSuccess) return cuda_fail(e, "k_scan_apply_in");
    FEM_TRY(scan_fused_ipt<SCAN_IPT>(m, ScanLoad{vals}, ScanStoreTo{pre}, n, s, total_dev, family));
    note_launch_begin(family, s);
    e = launch_pdl(k_scan_apply_out<Out>, dim3(blocks), dim3(256), 0, s, out, (const int*)pre, (const int*)vals, n);
    note_launch_end(family, s);
    if (e != cudaSuccess) return cuda_fail(e, "k_scan_apply_out");
    return FEM_OK;
}

// plain consumer: out[i] = prefix
struct ScanStore {
    int* dst;
    __device__ __forceinline__ void operator()(long long i, int prefix, int) const { dst[i] = prefix; }
};

}  // namespace fem
