// mesh.cu -- mesh handle, import/export, errors, launch accounting, scans.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "fem_internal.cuh"
#include "scan.cuh"

namespace fem {

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

fem_status cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return FEM_E_OOM;
    return FEM_E_CUDA;
}

// ------------------------------------------------------ launch accounting
static std::atomic<long long> g_launches{0};
static std::atomic<int> g_prof_on{0};
static std::mutex g_prof_mu;
struct ProfRec {
    cudaEvent_t a, b;
};
static std::vector<ProfRec> g_prof_open[F_COUNT];
static long long g_prof_launches[F_COUNT];
static double g_prof_bytes[F_COUNT];
static std::vector<cudaEvent_t> g_event_pool;
static thread_local cudaEvent_t t_begin_ev = nullptr;

static cudaEvent_t pool_get() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

bool profiling(int family) { return (g_prof_on.load(std::memory_order_relaxed) >> family) & 1; }

void note_bytes(int family, double bytes) {
    if (!profiling(family)) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_bytes[family] += bytes;
}

bool pdl_enabled() {
    // FEM_PDL=0 turns programmatic dependent launch off (plain stream order)
    static const bool on = [] {
        const char* v = getenv("FEM_PDL");
        return !(v && v[0] == '0');
    }();
    return on;
}

void note_launch_begin(int family, cudaStream_t s) {
    if (!profiling(family)) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    t_begin_ev = pool_get();
    cudaEventRecord(t_begin_ev, s);
}

void note_launch_end(int family, cudaStream_t s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!profiling(family) || !t_begin_ev) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t e = pool_get();
    cudaEventRecord(e, s);
    g_prof_open[family].push_back({t_begin_ev, e});
    g_prof_launches[family]++;
    t_begin_ev = nullptr;
}

// Cooperative launches also take the programmatic-launch attribute (the
// kernels start with pdl_wait); if the runtime refuses the combination, the
// attribute is dropped for the rest of the process.
static std::atomic<bool> g_coop_pdl_ok{true};

fem_status launch_coop(int family, const void* func, int grid, int block, size_t smem, cudaStream_t s,
                       void** args, const char* name) {
    note_launch_begin(family, s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    const bool pdl = pdl_enabled() && g_coop_pdl_ok.load(std::memory_order_relaxed);
    cfg.numAttrs = pdl ? 2 : 1;
    cudaError_t e = cudaLaunchKernelExC(&cfg, func, args);
    if (e != cudaSuccess && pdl && (e == cudaErrorInvalidValue || e == cudaErrorNotSupported)) {
        cudaGetLastError();
        g_coop_pdl_ok.store(false);
        cfg.numAttrs = 1;
        e = cudaLaunchKernelExC(&cfg, func, args);
    }
    note_launch_end(family, s);
    if (e != cudaSuccess) return cuda_fail(e, name);
    return FEM_OK;
}

// After a failed cooperative kernel: barrier words and the system build's
// error word back to zero (a completed kernel leaves both at zero).
void reset_coop_state(fem_mesh* m, cudaStream_t s) {
    cudaMemsetAsync(m->bar.p, 0, 2 * sizeof(unsigned), s);
    cudaMemsetAsync(m->dflag.p + 2, 0, sizeof(int), s);
}

// ------------------------------------------------------------ domain image
__global__ void k_pad_image(const float* __restrict__ f, int W, int H, int N, float* __restrict__ out) {
    pdl_wait();
    const long long n = (long long)N * N;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(p / N), x = (int)(p - (long long)y * N);
        out[p] = f[(long long)min(y, H - 1) * W + min(x, W - 1)];
    }
}

fem_status domain_image(fem_mesh* m, const float* f, cudaStream_t s, const float** out) {
    if (m->W == m->N && m->H == m->N) {
        *out = f;
        return FEM_OK;
    }
    FEM_TRY(ensure(m->fpad, (size_t)m->P, s));
    const int grid = (int)std::min<long long>((m->P + 255) / 256, (long long)m->num_sms * 16);
    note_bytes(F_OTHER, 4.0 * (double)m->PI + 4.0 * (double)m->P);
    FEM_LAUNCH(F_OTHER, s, k_pad_image, grid, 256, 0, f, m->W, m->H, m->N, m->fpad.p);
    *out = m->fpad.p;
    return FEM_OK;
}

// ------------------------------------------------------------------ memory
// Every device allocation of the library comes through dalloc_raw: from the
// caller's pool when one is set, else from the device's current pool.  The
// attempt counter and the armed failure index serve fem_debug_alloc_fault.
static std::atomic<long long> g_alloc_calls{0};
static std::atomic<long long> g_alloc_fail_at{-1};
static std::atomic<cudaMemPool_t> g_pool{nullptr};

// Device bytes held per stream (the stream an allocation was made on), live
// and at their peak since the last stream_alloc_peak_take: the serving loop
// runs each request on its own stream and admits by what they measured.
// Allocations happen only when arrays grow, so a mutex is cheap here.
// The tables are never destroyed, so a mesh released during process exit
// still finds them.
struct AllocAcct {
    std::mutex mu;
    std::unordered_map<void*, std::pair<size_t, cudaStream_t>> ptr;
    std::unordered_map<cudaStream_t, std::pair<size_t, size_t>> stream;  // live, peak
};
static AllocAcct& acct() {
    static AllocAcct* a = new AllocAcct;
    return *a;
}

static void acct_alloc(void* p, size_t bytes, cudaStream_t s) {
    AllocAcct& A = acct();
    std::lock_guard<std::mutex> lk(A.mu);
    A.ptr[p] = {bytes, s};
    auto& a = A.stream[s];
    a.first += bytes;
    if (a.first > a.second) a.second = a.first;
}

static void acct_free(void* p) {
    AllocAcct& A = acct();
    std::lock_guard<std::mutex> lk(A.mu);
    auto it = A.ptr.find(p);
    if (it == A.ptr.end()) return;
    auto& a = A.stream[it->second.second];
    a.first -= std::min(a.first, it->second.first);
    A.ptr.erase(it);
}

size_t stream_alloc_peak_take(cudaStream_t s) {
    AllocAcct& A = acct();
    std::lock_guard<std::mutex> lk(A.mu);
    auto it = A.stream.find(s);
    if (it == A.stream.end()) return 0;
    const size_t peak = it->second.second;
    it->second.second = it->second.first;  // the next peak starts from what is live now
    return peak;
}

fem_status dalloc_raw(void** p, size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    long long k = g_alloc_calls.fetch_add(1);
    if (k == g_alloc_fail_at.load()) {
        *p = nullptr;
        set_error("device allocation of " + std::to_string(bytes) + " bytes failed: injected by fem_debug_alloc_fault");
        return FEM_E_OOM;
    }
    cudaMemPool_t pool = g_pool.load();
    cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        set_error("device allocation of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
        return FEM_E_OOM;
    }
    acct_alloc(*p, bytes, s);
    return FEM_OK;
}

void dfree_raw(void* p, cudaStream_t s) {
    if (p) {
        acct_free(p);
        cudaFreeAsync(p, s);
    }
}

int sm_count() {
    static const int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return n;
}

// ------------------------------------------------------------------- scans
__global__ void k_scan_tiles(const int* __restrict__ in, int* __restrict__ out, int n, int* __restrict__ tile_sums) {
    pdl_wait();
    int v[SCAN_IPT];
    long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_IPT;
#pragma unroll
    for (int i = 0; i < SCAN_IPT; ++i) v[i] = (base + i < n) ? in[base + i] : 0;
    int tot = block_exclusive_scan(v);
#pragma unroll
    for (int i = 0; i < SCAN_IPT; ++i)
        if (base + i < n) out[base + i] = v[i];
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_add(int* __restrict__ out, int n, const int* __restrict__ tile_off) {
    pdl_wait();
    long long base = (long long)blockIdx.x * SCAN_TILE;
    int add = tile_off[blockIdx.x];
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_BT)
        if (base + i < n) out[base + i] += add;
}

__global__ void k_scan_total(const int* in, const int* out, int n, int* total) {
    pdl_wait();
    *total = n > 0 ? out[n - 1] + in[n - 1] : 0;
}

fem_status scan_scratch(fem_mesh* m, int n, cudaStream_t s, int** vals, int** pre) {
    FEM_TRY(ensure(m->scan_vals, (size_t)n, s));
    FEM_TRY(ensure(m->scan_pre, (size_t)n, s));
    *vals = m->scan_vals.p;
    *pre = m->scan_pre.p;
    return FEM_OK;
}

fem_status scan_plan(fem_mesh* m, int n, int tile, cudaStream_t s, ScanPlan* plan) {
    int tiles = (n + tile - 1) / tile;
    unsigned long long* before = m->scan_status.p;
    FEM_TRY(ensure(m->scan_status, (size_t)tiles, s));
    if (m->scan_status.p != before)  // fresh memory: no word may look like one of this call's epoch
        FEM_CUDA(cudaMemsetAsync(m->scan_status.p, 0, sizeof(unsigned long long) * m->scan_status.n, s));
    if (!m->scan_ctr.p) {
        FEM_TRY(ensure(m->scan_ctr, 1, s));
        FEM_CUDA(cudaMemsetAsync(m->scan_ctr.p, 0, sizeof(unsigned long long), s));
        m->scan_tiles_issued = 0;
    }
    plan->tiles = tiles;
    plan->status = m->scan_status.p;
    plan->ctr = m->scan_ctr.p;
    plan->base = m->scan_tiles_issued;
    m->scan_tiles_issued += (unsigned long long)tiles;
    unsigned epoch = (unsigned)(++m->scan_epoch & ((1u << 30) - 1));
    if (epoch == 0) epoch = (unsigned)(++m->scan_epoch & ((1u << 30) - 1));
    plan->epoch = epoch;
    plan->err = m->dflag.p + 8;
    return FEM_OK;
}

// out[i] = sum of in[0..i-1]; *total_dev (if non-null) = sum of all.  out may alias in? no.
fem_status exclusive_scan_i32(const int* in, int* out, int n, cudaStream_t s, int* total_dev) {
    if (n <= 0) {
        if (total_dev) FEM_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(int), s));
        return FEM_OK;
    }
    int tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    int* sums = nullptr;
    FEM_TRY(dalloc_raw((void**)&sums, sizeof(int) * (size_t)(2 * tiles + 2), s));
    int* sums_off = sums + tiles + 1;
    fem_status st = FEM_OK;
    do {
        note_launch_begin(F_OTHER, s);
        k_scan_tiles<<<tiles, SCAN_BT, 0, s>>>(in, out, n, sums);
        cudaError_t e = cudaGetLastError();
        note_launch_end(F_OTHER, s);
        if (e != cudaSuccess) { st = cuda_fail(e, "k_scan_tiles"); break; }
        if (tiles > 1) {
            st = exclusive_scan_i32(sums, sums_off, tiles, s, nullptr);
            if (st != FEM_OK) break;
            note_launch_begin(F_OTHER, s);
            k_scan_add<<<tiles, SCAN_BT, 0, s>>>(out, n, sums_off);
            e = cudaGetLastError();
            note_launch_end(F_OTHER, s);
            if (e != cudaSuccess) { st = cuda_fail(e, "k_scan_add"); break; }
        }
        if (total_dev) {
            note_launch_begin(F_OTHER, s);
            k_scan_total<<<1, 1, 0, s>>>(in, out, n, total_dev);
            e = cudaGetLastError();
            note_launch_end(F_OTHER, s);
            if (e != cudaSuccess) { st = cuda_fail(e, "k_scan_total"); break; }
        }
    } while (0);
    dfree_raw(sums, s);
    return st;
}

// The same scan with caller-provided temporary storage (no allocation):
// tmp must hold at least scan_tmp_ints(n) ints.
int scan_tmp_ints(int n) {
    if (n <= SCAN_TILE) return 0;
    int tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    return 2 * tiles + 2 + scan_tmp_ints(tiles);
}

fem_status exclusive_scan_i32_scratch(const int* in, int* out, int n, cudaStream_t s, int* total_dev, int* tmp,
                                      int tmp_n) {
    if (n <= 0) {
        if (total_dev) FEM_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(int), s));
        return FEM_OK;
    }
    if (tmp_n < scan_tmp_ints(n)) {
        set_error("scan: temporary storage too small");
        return FEM_E_INVALID;
    }
    int tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    int* sums = tmp;
    int* sums_off = tmp + tiles + 1;
    FEM_LAUNCH(F_OTHER, s, k_scan_tiles, tiles, SCAN_BT, 0, in, out, n, sums);
    if (tiles > 1) {
        FEM_TRY(exclusive_scan_i32_scratch(sums, sums_off, tiles, s, nullptr, tmp + 2 * tiles + 2,
                                           tmp_n - (2 * tiles + 2)));
        FEM_LAUNCH(F_OTHER, s, k_scan_add, tiles, SCAN_BT, 0, out, n, sums_off);
    }
    if (total_dev) FEM_LAUNCH(F_OTHER, s, k_scan_total, 1, 1, 0, in, out, n, total_dev);
    return FEM_OK;
}

// ------------------------------------------------------------- capacities
fem_status ensure_mesh_capacity(fem_mesh* m, int needV, int needT, cudaStream_t s) {
    long long maxV = m->P, maxT = 2LL * (m->N - 1) * (m->N - 1);
    size_t nv = (size_t)std::min<long long>(std::max(needV, 4), maxV);
    size_t nt = (size_t)std::min<long long>(std::max(needT, 2), maxT);
    if (needV > maxV) nv = (size_t)needV;
    if (needT > maxT) nt = (size_t)needT;
    FEM_TRY(ensure(m->vxy, nv, s, m->V));
    FEM_TRY(ensure(m->mask, nv, s, m->V));
    FEM_TRY(ensure(m->uv, nv, s, m->V));
    FEM_TRY(ensure(m->uvf, nv, s, m->V));
    FEM_TRY(ensure(m->tri, nt, s, m->T));
    FEM_TRY(ensure(m->order, nt, s, m->T));
    return FEM_OK;
}

fem_status sync_counts(fem_mesh* m, cudaStream_t s) {
    FEM_CUDA(cudaStreamSynchronize(s));
    return FEM_OK;
}

// Diagnostic for the bounded waits: block 0 enters the grid barrier, block 1
// returns without arriving, so the barrier's arrival count never completes
// and block 0 must give up after the barrier's time limit and record
// FEM_E_TIMEOUT instead of hanging.
__global__ void k_selftest_barrier(unsigned* bar, int* err) {
    pdl_wait();
    if (blockIdx.x != 0) return;
    grid_barrier(bar, err);
}

}  // namespace fem

using namespace fem;

static fem_status check_mesh(const fem_mesh* m) {
    if (!m) {
        set_error("null mesh handle");
        return FEM_E_INVALID;
    }
    return FEM_OK;
}

namespace fem {
// the triangles' (a, b, c) without the padding word of the int4 rows
__global__ void k_pack_tri(const int4* __restrict__ tri, int T, int* __restrict__ out) {
    pdl_wait();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const int4 v = tri[t];
        out[3 * (size_t)t] = v.x;
        out[3 * (size_t)t + 1] = v.y;
        out[3 * (size_t)t + 2] = v.z;
    }
}
}  // namespace fem

extern "C" {

void fem_params_default(fem_params* p) {
    if (!p) return;
    p->tol = 1e-12;
    p->maxit = 20000;
    p->precision = FEM_PREC_FP32_IR;
    p->topk_frac = 0.01;
    p->max_rounds = 0;
    p->tonal_tol = 1e-8;
    p->tonal_maxit = 2000;
    p->inner_tol = 1e-11;
    p->fast_keys = -1;
}

const char* fem_last_error(void) { return g_last_error.c_str(); }

long long fem_launch_count(void) { return g_launches.load(); }

fem_status fem_set_mem_pool(void* pool) {
    g_pool.store((cudaMemPool_t)pool);
    return FEM_OK;
}

fem_status fem_debug_alloc_fault(long long fail_after, long long* calls_out) {
    long long now = g_alloc_calls.load();
    if (calls_out) *calls_out = now;
    g_alloc_fail_at.store(fail_after >= 0 ? now + fail_after : -1);
    return FEM_OK;
}

void fem_profile_enable(int family_mask) { g_prof_on.store(family_mask); }

int fem_profile_read(int family, long long* launches, double* ms, double* bytes, const char** name) {
    static const char* names[F_COUNT] = {"raster", "cg", "assembly", "topk", "refine", "tonal", "other", "raster_pass"};
    if (family < 0 || family >= F_COUNT) return -1;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    double tot = 0.0;
    for (auto& r : g_prof_open[family]) {
        cudaEventSynchronize(r.b);
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) tot += t;
        g_event_pool.push_back(r.a);
        g_event_pool.push_back(r.b);
    }
    cudaGetLastError();
    g_prof_open[family].clear();
    if (launches) *launches = g_prof_launches[family];
    if (ms) *ms = tot;
    if (name) *name = names[family];
    if (family == F_SQPASS) g_prof_bytes[family] += sq_inc_bytes_take();
    if (bytes) *bytes = g_prof_bytes[family];
    g_prof_launches[family] = 0;
    g_prof_bytes[family] = 0.0;
    return 0;
}

fem_status fem_mesh_create(int width, int height, void* stream, fem_mesh** out) {
    if (!out) {
        set_error("fem_mesh_create: out is NULL");
        return FEM_E_INVALID;
    }
    *out = nullptr;
    if (width < 2 || height < 2 || width > 32769 || height > 32769) {
        set_error("fem_mesh_create: width and height must be 2..32769");
        return FEM_E_SHAPE;
    }
    // the smallest domain side 2^L + 1 that holds the image
    int n = 3;
    while (n < width || n < height) n = 2 * n - 1;
    cudaStream_t s = (cudaStream_t)stream;
    fem_mesh* m = new fem_mesh();
    m->N = n;
    m->P = (long long)n * n;
    m->W = width;
    m->H = height;
    m->PI = (long long)width * height;
    cudaGetDevice(&m->dev);
    m->num_sms = sm_count();
    m->last_stream = s;
    fem_status st = FEM_OK;
    do {
        st = ensure_mesh_capacity(m, 64, 64, s);
        if (st) break;
        st = ensure(m->red, (size_t)8 * 4096, s);
        if (st) break;
        st = ensure(m->bar, 64, s);
        if (st) break;
        st = ensure(m->dflag, 64, s);
        if (st) break;
        st = ensure(m->dscal, 256, s);
        if (st) break;
        st = ensure(m->dcount, 64, s);
        if (st) break;
        st = ensure(m->ccount, CC_COUNTERS, s);
        if (st) break;
        cudaError_t e = cudaMallocHost(&m->host_stage, 1 << 16);
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaMallocHost"); break; }
        // kernels may write small results straight into the staging area
        if (cudaHostGetDevicePointer(&m->host_stage_dev, m->host_stage, 0) != cudaSuccess) {
            m->host_stage_dev = nullptr;
            cudaGetLastError();
        }
        e = cudaMemsetAsync(m->bar.p, 0, 64 * sizeof(unsigned), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(m->dflag.p, 0, 64 * sizeof(int), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(m->dcount.p, 0, 64 * sizeof(int), s);
        if (e != cudaSuccess) { st = cuda_fail(e, "memset"); break; }
        int n1 = n - 1;
        int2 xy[4] = {{0, 0}, {n1, 0}, {0, n1}, {n1, n1}};
        unsigned char mk[4] = {1, 1, 1, 1};
        int4 tr[2] = {{0, 3, 2, 0}, {3, 0, 1, 0}};
        double uv0[4] = {0, 0, 0, 0};
        int ord0[2] = {0, 1};  // the curve enters (v0,v3,v2) at v0 and leaves (v3,v0,v1) at v0
        e = cudaMemcpyAsync(m->vxy.p, xy, sizeof(xy), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(m->mask.p, mk, sizeof(mk), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(m->tri.p, tr, sizeof(tr), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(m->uv.p, uv0, sizeof(uv0), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(m->order.p, ord0, sizeof(ord0), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { st = cuda_fail(e, "fem_mesh_create upload"); break; }
        m->V = 4;
        m->T = 2;
        m->nK = 4;
        m->nU = 0;
    } while (0);
    if (st != FEM_OK) {
        fem_mesh_destroy(m);
        return st;
    }
    *out = m;
    return FEM_OK;
}

fem_status fem_selftest_wait_timeout(void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* bar = nullptr;
    FEM_TRY(dalloc_raw((void**)&bar, 64, s));
    int* err = (int*)(bar + 8);
    fem_status st = FEM_OK;
    do {
        cudaError_t e = cudaMemsetAsync(bar, 0, 64, s);
        if (e != cudaSuccess) { st = cuda_fail(e, "memset"); break; }
        void* args[] = {&bar, &err};
        st = launch_coop(F_OTHER, (const void*)k_selftest_barrier, 2, 32, 0, s, args, "k_selftest_barrier");
        if (st != FEM_OK) break;
        int h = 0;
        e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { st = cuda_fail(e, "selftest read-back"); break; }
        st = (fem_status)h;
        if (st == FEM_E_TIMEOUT) set_error("bounded wait ran out as intended");
    } while (0);
    dfree_raw(bar, s);
    cudaStreamSynchronize(s);
    return st;
}

fem_status fem_mesh_destroy(fem_mesh* m) {
    if (!m) return FEM_OK;
    cudaStream_t s = m->last_stream;
    cudaStreamSynchronize(s);
    release(m->vxy, s); release(m->mask, s); release(m->tri, s); release(m->uv, s); release(m->uvf, s);
    release(m->order, s); release(m->order_tmp, s); release(m->ocnt, s); release(m->ooff, s);
    release(m->item_cnt, s); release(m->item_off, s); release(m->item_tri, s); release(m->partial, s);
    release(m->keys_lo, s); release(m->keys_hi, s); release(m->fast_hist, s);
    release(m->band, s);
    release(m->keys, s);
    release(m->keyc, s);
    release(m->bmM, s); release(m->bmS, s); release(m->wpre, s);
    release(m->flags, s); release(m->fscan, s); release(m->wcnt, s); release(m->topk_hist, s);
    release(m->uidx, s); release(m->kidx, s); release(m->nbr, s); release(m->coefA, s); release(m->diagA, s);
    release(m->ucol, s); release(m->uval32, s); release(m->uval64, s); release(m->udiag, s); release(m->ucnt, s); release(m->dinv32, s); release(m->dinv64, s);
    release(m->urow_vertex, s); release(m->kvert, s); release(m->ulist, s); release(m->gcnt, s);
    release(m->cc_parent, s); release(m->cc_root, s); release(m->cc_size, s); release(m->cc_fill, s);
    release(m->cc_cstart, s); release(m->rowcomp, s); release(m->blk_list, s); release(m->warp_list, s);
    release(m->ccount, s);
    release(m->comp_stats, s);
    release(m->x64, s); release(m->b64, s); release(m->r64, s); release(m->p64, s); release(m->q64, s); release(m->z64, s);
    release(m->r32, s); release(m->p32, s); release(m->q32, s); release(m->z32, s); release(m->d32, s);
    release(m->bvec, s); release(m->browptr, s); release(m->bent, s); release(m->bdg2, s);
    release(m->bxff, s); release(m->bbff, s);
    release(m->scan_status, s); release(m->scan_ctr, s); release(m->scan_vals, s); release(m->scan_pre, s);
    release(m->red, s); release(m->bar, s); release(m->dflag, s); release(m->dscal, s); release(m->dcount, s);
    release(m->inc, s); release(m->loc, s); release(m->Moff, s); release(m->Mdiag, s);
    release(m->tv, s); release(m->ty, s); release(m->tz, s); release(m->tg, s);
    release(m->tr, s); release(m->tp, s); release(m->tw, s); release(m->tc, s);
    release(m->lossk, s); release(m->lossred, s); release(m->tyr, s);
    release(m->fsq, s); release(m->fedge, s); release(m->fpad, s);
    for (int c = 0; c < 3; ++c) {
        release(m->uvc[c], s); release(m->uvfc[c], s); release(m->fsqc[c], s); release(m->fedgec[c], s);
        release(m->fpadc[c], s);
    }
    release(m->keys_acc, s); release(m->wimg, s); release(m->wfimg, s); release(m->sq_nodeof, s); release(m->sq_off, s);
    release(m->sq_cov, s); release(m->sq_slot, s); release(m->sq_seg, s); release(m->sq_part, s);
    release(m->sq_coarse, s); release(m->sq_long, s); release(m->sq_piece, s); release(m->sq_psum, s);
    release(m->sq_pdone, s); release(m->sq_ctr, s); release(m->sq_list, s); release(m->sq_rec, s);
    release(m->sq_pos, s); release(m->sq_bcoarse, s); release(m->sq_mark, s); release(m->bsel, s);
    release(m->uvk, s); release(m->uvfk, s); release(m->vchg, s); release(m->tchg, s); release(m->tdirty, s);
    release(m->sq_dmark, s); release(m->sq_dlist, s); release(m->hcnt, s);
    cudaStreamSynchronize(s);
    if (m->host_stage) cudaFreeHost(m->host_stage);
    if (m->round_ev) cudaEventDestroy(m->round_ev);
    cudaGetLastError();
    delete m;
    return FEM_OK;
}

fem_status fem_mesh_info(const fem_mesh* m, int* V, int* T, int* nmask) {
    FEM_TRY(check_mesh(m));
    if (V) *V = m->V;
    if (T) *T = m->T;
    if (nmask) *nmask = m->nK;
    return FEM_OK;
}

fem_status fem_mesh_size(const fem_mesh* m, int* width, int* height, int* domain) {
    FEM_TRY(check_mesh(m));
    if (width) *width = m->W;
    if (height) *height = m->H;
    if (domain) *domain = m->N;
    return FEM_OK;
}

fem_status fem_mesh_stats(const fem_mesh* m, fem_stats* out) {
    FEM_TRY(check_mesh(m));
    if (out) *out = m->stats;
    return FEM_OK;
}

fem_status fem_mesh_export(fem_mesh* m, int* xy, int* tri, unsigned char* is_mask) {
    FEM_TRY(check_mesh(m));
    cudaStream_t s = m->last_stream;
    if (tri && m->T > 0) {
        // (a, b, c) packed from the int4 rows on the device, then one copy
        // straight into the caller's array
        int* t3 = nullptr;
        FEM_TRY(dalloc_raw((void**)&t3, sizeof(int) * 3 * (size_t)m->T, s));
        const int grid = (int)std::min<long long>(((long long)m->T + 255) / 256, (long long)m->num_sms * 16);
        FEM_LAUNCH(F_OTHER, s, k_pack_tri, grid, 256, 0, (const int4*)m->tri.p, m->T, t3);
        cudaError_t e = cudaMemcpyAsync(tri, t3, sizeof(int) * 3 * (size_t)m->T, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        dfree_raw(t3, s);
        if (e != cudaSuccess) return cuda_fail(e, "fem_mesh_export: triangles");
    }
    FEM_CUDA(cudaStreamSynchronize(s));
    if (xy) FEM_CUDA(cudaMemcpy(xy, m->vxy.p, sizeof(int2) * m->V, cudaMemcpyDeviceToHost));
    if (is_mask) FEM_CUDA(cudaMemcpy(is_mask, m->mask.p, m->V, cudaMemcpyDeviceToHost));
    return FEM_OK;
}

fem_status fem_mesh_curve_order(fem_mesh* m, int* order, int* is_curve) {
    FEM_TRY(check_mesh(m));
    FEM_CUDA(cudaStreamSynchronize(m->last_stream));
    if (order) FEM_CUDA(cudaMemcpy(order, m->order.p, sizeof(int) * m->T, cudaMemcpyDeviceToHost));
    if (is_curve) *is_curve = m->order_is_curve ? 1 : 0;
    return FEM_OK;
}

}  // extern "C"

namespace {

struct P2 {
    long long x, y;
};

// strictly inside the positively oriented triangle (a, b, c); p has three
// times the coordinates, the vertices are scaled here
bool inside3_host(P2 p, P2 a, P2 b, P2 c) {
    a = {3 * a.x, 3 * a.y};
    b = {3 * b.x, 3 * b.y};
    c = {3 * c.x, 3 * c.y};
    const long long e0 = (b.x - a.x) * (p.y - a.y) - (b.y - a.y) * (p.x - a.x);
    const long long e1 = (c.x - b.x) * (p.y - b.y) - (c.y - b.y) * (p.x - b.x);
    const long long e2 = (a.x - c.x) * (p.y - c.y) - (a.y - c.y) * (p.x - c.x);
    return e0 > 0 && e1 > 0 && e2 > 0;
}

// Position of a triangle (a, b, c) on the space-filling curve of the
// bisection tree of the two-triangle mesh of an image of side D + 1: the
// path from the root (first bit: which initial triangle; then at every
// bisection whether the child holding the triangle comes first or second on
// the curve), left-aligned in 64 bits, so that sorting the keys gives the
// curve order.  The curve enters a triangle with legs along the axes at a
// and one with diagonal legs at b; (a, b, c) is bisected into (c, a, m) and
// (b, c, m), and the child holding the entry comes first.  False when the
// triangle is not a node of the tree.
bool curve_key(long long D, P2 a, P2 b, P2 c, unsigned long long* key) {
    const P2 g{a.x + b.x + c.x, a.y + b.y + c.y};
    P2 na{0, 0}, nb{D, D}, nc{0, D};
    unsigned long long bits = 0;
    int depth = 1;
    if (!inside3_host(g, na, nb, nc)) {
        na = {D, D};
        nb = {0, 0};
        nc = {D, 0};
        bits = 1;
        if (!inside3_host(g, na, nb, nc)) return false;
    }
    const long long l2 = (a.x - c.x) * (a.x - c.x) + (a.y - c.y) * (a.y - c.y);
    for (;;) {
        if (na.x == a.x && na.y == a.y && nb.x == b.x && nb.y == b.y && nc.x == c.x && nc.y == c.y) break;
        const long long nl2 = (na.x - nc.x) * (na.x - nc.x) + (na.y - nc.y) * (na.y - nc.y);
        if (nl2 <= l2 || ((na.x + nb.x) & 1) || ((na.y + nb.y) & 1) || depth >= 63) return false;
        const P2 m{(na.x + nb.x) / 2, (na.y + nb.y) / 2};
        const bool at_b = nc.x != na.x && nc.y != na.y;
        int bit;
        if (inside3_host(g, nc, na, m)) {  // (c, a, m)
            bit = at_b ? 1 : 0;
            const P2 o = na;
            na = nc;
            nb = o;
            nc = m;
        } else if (inside3_host(g, nb, nc, m)) {  // (b, c, m)
            bit = at_b ? 0 : 1;
            const P2 o = nb;
            na = o;
            nb = nc;
            nc = m;
        } else {
            return false;
        }
        bits = (bits << 1) | (unsigned long long)bit;
        ++depth;
    }
    *key = bits << (64 - depth);
    return true;
}

}  // namespace

extern "C" {

fem_status fem_mesh_import(fem_mesh* m, int V, const int* xy, int T, const int* tri, const unsigned char* is_mask) {
    FEM_TRY(check_mesh(m));
    if (V < 3 || T < 1 || !xy || !tri || !is_mask || (long long)V > m->P || (long long)T > 2LL * (m->N - 1) * (m->N - 1)) {
        set_error("fem_mesh_import: bad sizes or null arrays");
        return FEM_E_INVALID;
    }
    int N = m->N;
    for (int i = 0; i < V; ++i) {
        if (xy[2 * i] < 0 || xy[2 * i] >= N || xy[2 * i + 1] < 0 || xy[2 * i + 1] >= N) {
            set_error("fem_mesh_import: vertex off the pixel grid");
            return FEM_E_INVALID;
        }
    }
    long long area2 = 0;
    std::vector<int4> t4(T);
    for (int t = 0; t < T; ++t) {
        int a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
        if (a < 0 || b < 0 || c < 0 || a >= V || b >= V || c >= V) {
            set_error("fem_mesh_import: triangle index out of range");
            return FEM_E_INVALID;
        }
        long long ax = xy[2 * a], ay = xy[2 * a + 1], bx = xy[2 * b], by = xy[2 * b + 1], cx = xy[2 * c], cy = xy[2 * c + 1];
        long long cr = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
        long long d1x = ax - cx, d1y = ay - cy, d2x = bx - cx, d2y = by - cy;
        bool right = (d1x * d2x + d1y * d2y == 0) && (d1x * d1x + d1y * d1y == d2x * d2x + d2y * d2y);
        bool axial = (d1x == 0 || d1y == 0 || d1x == d1y || d1x == -d1y);
        if (cr <= 0 || !right || !axial) {
            set_error("fem_mesh_import: triangle " + std::to_string(t) + " is not a positively oriented right-isosceles lattice triangle with c at the right angle");
            return FEM_E_INVALID;
        }
        area2 += cr;
        t4[t] = make_int4(a, b, c, 0);
    }
    if (area2 != 2LL * (N - 1) * (N - 1)) {
        set_error("fem_mesh_import: triangle areas do not add up to the image");
        return FEM_E_INVALID;
    }
    // every triangle must be a node of the bisection tree of the
    // two-triangle mesh; the kernels visit them along the tree's curve
    std::vector<std::pair<unsigned long long, int>> keyed(T);
    for (int t = 0; t < T; ++t) {
        const int a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
        unsigned long long key = 0;
        if (!curve_key(N - 1, P2{xy[2 * a], xy[2 * a + 1]}, P2{xy[2 * b], xy[2 * b + 1]},
                       P2{xy[2 * c], xy[2 * c + 1]}, &key)) {
            set_error("fem_mesh_import: triangle " + std::to_string(t) +
                      " is not a newest-vertex-bisection triangle of the two-triangle mesh");
            return FEM_E_INVALID;
        }
        keyed[t] = {key, t};
    }
    std::sort(keyed.begin(), keyed.end());
    std::vector<int> ord(T);
    for (int i = 0; i < T; ++i) {
        if (i > 0 && keyed[i].first == keyed[i - 1].first) {
            set_error("fem_mesh_import: triangles " + std::to_string(keyed[i - 1].second) + " and " +
                      std::to_string(keyed[i].second) + " coincide");
            return FEM_E_INVALID;
        }
        ord[i] = keyed[i].second;
    }
    cudaStream_t s = m->last_stream;
    FEM_TRY(ensure_mesh_capacity(m, V, T, s));
    FEM_CUDA(cudaMemcpyAsync(m->vxy.p, xy, sizeof(int2) * V, cudaMemcpyHostToDevice, s));
    FEM_CUDA(cudaMemcpyAsync(m->mask.p, is_mask, V, cudaMemcpyHostToDevice, s));
    FEM_CUDA(cudaMemcpyAsync(m->tri.p, t4.data(), sizeof(int4) * T, cudaMemcpyHostToDevice, s));
    FEM_CUDA(cudaMemsetAsync(m->uv.p, 0, sizeof(double) * V, s));
    FEM_CUDA(cudaMemcpyAsync(m->order.p, ord.data(), sizeof(int) * T, cudaMemcpyHostToDevice, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    m->order_is_curve = true;
    FEM_CUDA(cudaStreamSynchronize(s));
    int nk = 0;
    for (int i = 0; i < V; ++i) nk += is_mask[i] ? 1 : 0;
    m->V = V;
    m->T = T;
    m->nK = nk;
    m->nU = V - nk;
    m->mesh_version++;
    return FEM_OK;
}

}  // extern "C"
