// noalloc.cu -- per-triangle squared errors for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: programs whose own caching allocator
// has reserved all device memory (a foreign allocation would fail or
// fragment it), and real-time or serving loops that must not allocate after
// start-up (cudaMalloc can synchronise the device and its latency is
// unbounded).  For them this file offers
// one entry point that computes the same per-triangle errors as
// fem_triangle_errors on mesh arrays the caller owns, using as scratch a
// file-scope device array of fixed size instead of any allocation.
//
// The array lives in every GPU that loads this library, for the life of the
// process.  In host code its name is only a host-side stand-in, so the host
// looks up the device address once per device with cudaGetSymbolAddress and
// passes that address to the kernels.
#include <mutex>

#include "fem_internal.cuh"

namespace fem {
namespace {

constexpr int kMaxT = 65536;       // triangles
constexpr int kMaxWidth = 2049;    // image side
constexpr int kMaxDevices = 64;
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
// rasterisation items of a valid mesh: at most 3T + P/128 + 1024
constexpr int kItemCap = 3 * kMaxT + (kMaxWidth * kMaxWidth) / 128 + 1024;
constexpr int kScanTmpInts = 1024;
constexpr size_t kOffCnt = 0;
constexpr size_t kOffOff = kOffCnt + align256(sizeof(int) * kMaxT);
constexpr size_t kOffTri = kOffOff + align256(sizeof(int) * (kMaxT + 1));
constexpr size_t kOffPart = kOffTri + align256(sizeof(int) * kItemCap);
constexpr size_t kOffCounters = kOffPart + align256(sizeof(double) * kItemCap);
constexpr size_t kOffScan = kOffCounters + 256;
constexpr size_t kScratchBytes = kOffScan + align256(sizeof(int) * kScanTmpInts);  // about 3.4 MB

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_dev_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
fem_status scratch_address(void** out) {
    int dev = 0;
    FEM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("fem_triangle_errors_noalloc: device ordinal out of range");
        return FEM_E_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
        g_dev_addr[dev] = p;
    }
    *out = g_dev_addr[dev];
    return FEM_OK;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace
}  // namespace fem

using namespace fem;

extern "C" fem_status fem_triangle_errors_noalloc(int width, int V, const int* xy_dev, int T, const int* tri_dev,
                                                  const double* uv_dev, const float* f_dev, double* err_dev,
                                                  void* stream) {
    int L = width - 1;
    if (width < 3 || width > kMaxWidth || (L & (L - 1)) != 0) {
        set_error("fem_triangle_errors_noalloc: width must be 2^L + 1 and at most 2049");
        return FEM_E_SHAPE;
    }
    if (T < 1 || T > kMaxT || V < 3 || (long long)V > (long long)width * width) {
        set_error("fem_triangle_errors_noalloc: need 1 <= T <= 65536 triangles and 3 <= V <= width^2 vertices "
                  "(the fixed scratch holds no more)");
        return FEM_E_INVALID;
    }
    if (!xy_dev || !tri_dev || !uv_dev || !f_dev || !err_dev) {
        set_error("fem_triangle_errors_noalloc: null argument");
        return FEM_E_INVALID;
    }
    if (!aligned(tri_dev, 16) || !aligned(xy_dev, 8) || !aligned(uv_dev, 8) || !aligned(err_dev, 8) ||
        !aligned(f_dev, 4)) {
        set_error("fem_triangle_errors_noalloc: tri must be 16-byte aligned, xy/uv/err 8-byte aligned");
        return FEM_E_INVALID;
    }
    void* base = nullptr;
    FEM_TRY(scratch_address(&base));
    unsigned char* b = (unsigned char*)base;
    cudaStream_t s = (cudaStream_t)stream;
    RasterScratch w;
    w.item_cnt = (int*)(b + kOffCnt);
    w.item_off = (int*)(b + kOffOff);
    w.item_tri = (int*)(b + kOffTri);
    w.partial = (double*)(b + kOffPart);
    w.item_cap = kItemCap;
    w.counters = (int*)(b + kOffCounters);
    w.scan_tmp = (int*)(b + kOffScan);
    w.scan_tmp_n = kScanTmpInts;
    w.grid = sm_count() * 8;
    // the array keeps the last call's contents: clear the item count and the overflow flag
    FEM_CUDA(cudaMemsetAsync(w.counters, 0, 2 * sizeof(int), s));
    FEM_TRY(raster_errors_scratch((const int4*)tri_dev, (const int2*)xy_dev, T, width, uv_dev, f_dev, err_dev, s, w));
    int overflow = 0;
    FEM_CUDA(cudaMemcpyAsync(&overflow, w.counters + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    if (overflow) {
        set_error("fem_triangle_errors_noalloc: the mesh needs more rasterisation items than the fixed scratch "
                  "holds (is it a valid mesh of this image?)");
        return FEM_E_INVALID;
    }
    return FEM_OK;
}
