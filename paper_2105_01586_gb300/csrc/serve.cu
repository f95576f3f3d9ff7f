// serve.cu -- continuous-batching request loop for data optimisation jobs.
//
// A server owns `slots` worker threads, each with its own CUDA stream.  A
// request (an image, a vertex density and parameters) waits in a FIFO queue
// until a slot is free and its device memory fits the budget next to the
// requests already running.  That memory is a static upper estimate scaled
// by the largest ratio of measured peak to estimate among the requests that
// have finished (each request's allocations are counted on its slot's
// stream).  It is then admitted and runs the whole
// path on its slot's stream: mesh creation, spatial optimisation (Sec. 3),
// g = f at the mask vertices and tonal optimisation (Sec. 4).  Requests on
// different slots overlap on the device: most kernels of one request occupy
// a few SMs (one-block solver, one-block top-k), so several requests fill
// the GPU.  Every request computes exactly what it would compute alone: the
// kernels are deterministic and share no state across meshes.  Results (the
// mesh, g and timings) stay in host memory until the caller releases them.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "fem_internal.cuh"

namespace fem {
// peak device bytes allocated on stream s since the last call (mesh.cu)
size_t stream_alloc_peak_take(cudaStream_t s);
}  // namespace fem

namespace fem {
namespace {

using clock_type = std::chrono::steady_clock;

double now_s() {
    return std::chrono::duration<double>(clock_type::now().time_since_epoch()).count();
}

struct Request {
    long long id = 0;
    int width = 0;
    double density = 0.0;
    fem_params params{};
    std::vector<float> f;  // host copy of the image
    size_t mem_estimate = 0;   // static upper estimate (estimate_bytes)
    size_t mem_reserved = 0;   // what admission reserved: the estimate scaled by the measured ratio
    size_t mem_measured = 0;   // peak device bytes the request's stream held (after it ran)
    double t_submit = 0, t_start = 0, t_end = 0;
    fem_status status = FEM_OK;
    std::string error;
    // results
    int V = 0, T = 0, nK = 0;
    std::vector<int> xy, tri;
    std::vector<unsigned char> mask;
    std::vector<float> g;
    fem_stats spatial{}, tonal{};
    bool done = false;
    bool running = false;
    std::atomic<int> cancel{0};  // fem_server_cancel: the mesh loops stop at their next check
};

}  // namespace
}  // namespace fem

struct fem_server {
    int slots = 0;
    size_t budget = 0;
    size_t in_use = 0;
    // largest measured peak / static estimate over the finished requests,
    // with a margin (1 until a request has finished): admission reserves
    // the estimate scaled by it
    double mem_scale = 1.0;
    bool measured_any = false;
    int dev = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<fem::Request>> queue;
    std::map<long long, std::shared_ptr<fem::Request>> all;
    long long next_id = 1;
    bool stopping = false;
    int running = 0;
    std::vector<std::thread> workers;
};

namespace fem {
namespace {

// Upper estimate of the device memory a request holds at its peak: the
// image, the per-pixel bitmaps, and per-vertex / per-triangle arrays (with
// the capacity doubling of the growing mesh) for V* = ceil(density * P)
// vertices and about 2 V* triangles.  The systems built ahead of the host
// size their per-unknown arrays for 1.25 times the vertices (140 B each).
size_t estimate_bytes(int width, double density) {
    double P = (double)width * width;
    double V = std::ceil(density * P) * 1.2 + 64;
    double T = 2.0 * V;
    return (size_t)(4.0 * P + 0.5 * P + 2.0 * (260.0 * V + 220.0 * T + 140.0 * V) + (64 << 20));
}

// Margin on the measured ratio: requests of other sizes and densities may
// hold a little more per estimated byte than those measured so far.
constexpr double kMeasuredMargin = 1.25;

fem_status run_request(Request& r, cudaStream_t s) {
    fem_mesh* m = nullptr;
    float* f_dev = nullptr;
    float* g_dev = nullptr;
    size_t P = (size_t)r.width * r.width;
    fem_status st = fem_mesh_create(r.width, r.width, s, &m);
    if (st != FEM_OK) return st;
    m->cancel = &r.cancel;
    do {
        st = check_cancel(m);
        if (st != FEM_OK) break;
        st = dalloc_raw((void**)&f_dev, sizeof(float) * P, s);
        if (st != FEM_OK) break;
        cudaError_t e = cudaMemcpyAsync(f_dev, r.f.data(), sizeof(float) * P, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) { st = cuda_fail(e, "request image upload"); break; }
        st = fem_spatial_refine(m, f_dev, r.density, &r.params, s);
        if (st != FEM_OK) break;
        r.spatial = m->stats;
        st = dalloc_raw((void**)&g_dev, sizeof(float) * (size_t)(m->nK > 0 ? m->nK : 1), s);
        if (st != FEM_OK) break;
        st = fem_gather_mask(m, f_dev, g_dev, s);
        if (st != FEM_OK) break;
        st = fem_tonal_opt(m, f_dev, g_dev, &r.params, s);
        r.tonal = m->stats;
        if (st != FEM_OK && st != FEM_E_NOT_CONVERGED) break;
        fem_status st_tonal = st;
        r.V = m->V;
        r.T = m->T;
        r.nK = m->nK;
        r.xy.resize(2 * (size_t)r.V);
        r.tri.resize(3 * (size_t)r.T);
        r.mask.resize(r.V);
        r.g.resize(r.nK);
        st = fem_mesh_export(m, r.xy.data(), r.tri.data(), r.mask.data());
        if (st != FEM_OK) break;
        e = cudaMemcpyAsync(r.g.data(), g_dev, sizeof(float) * r.nK, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { st = cuda_fail(e, "request result read-back"); break; }
        st = st_tonal;
    } while (0);
    if (g_dev) dfree_raw(g_dev, s);
    if (f_dev) dfree_raw(f_dev, s);
    fem_mesh_destroy(m);
    return st;
}

void worker_main(fem_server* sv) {
    cudaSetDevice(sv->dev);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (;;) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            // FIFO admission: the head request starts when its memory fits
            // next to the running ones (a request larger than the whole
            // budget runs alone)
            auto need_of = [&](const Request& q) {
                return (size_t)std::ceil(sv->mem_scale * (double)q.mem_estimate);
            };
            sv->cv_work.wait(lk, [&] {
                if (sv->stopping) return true;
                if (sv->queue.empty()) return false;
                size_t need = need_of(*sv->queue.front());
                return sv->in_use + need <= sv->budget || sv->running == 0;
            });
            if (sv->stopping && sv->queue.empty()) break;
            if (sv->stopping) break;
            r = sv->queue.front();
            sv->queue.pop_front();
            r->mem_reserved = need_of(*r);
            sv->in_use += r->mem_reserved;
            sv->running++;
            r->running = true;
            r->t_start = now_s();
        }
        stream_alloc_peak_take(s);  // the peak from here on is this request's
        fem_status st = run_request(*r, s);
        const size_t measured = stream_alloc_peak_take(s);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            r->mem_measured = measured;
            if (st == FEM_OK && r->mem_estimate > 0) {
                const double ratio = kMeasuredMargin * (double)measured / (double)r->mem_estimate;
                sv->mem_scale = sv->measured_any ? std::max(sv->mem_scale, ratio) : ratio;
                sv->measured_any = true;
            }
            r->status = st;
            if (st != FEM_OK) r->error = fem_last_error();
            r->t_end = now_s();
            r->done = true;
            r->running = false;
            r->f.clear();
            r->f.shrink_to_fit();
            sv->in_use -= r->mem_reserved;
            sv->running--;
        }
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
}

}  // namespace
}  // namespace fem

using namespace fem;

extern "C" {

fem_status fem_server_create(int slots, size_t mem_budget_bytes, fem_server** out) {
    if (!out || slots < 1 || slots > 256) {
        set_error("fem_server_create: need 1..256 slots and an output pointer");
        return FEM_E_INVALID;
    }
    fem_server* sv = new fem_server();
    sv->slots = slots;
    FEM_CUDA(cudaGetDevice(&sv->dev));
    if (mem_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        FEM_CUDA(cudaMemGetInfo(&fr, &tot));
        mem_budget_bytes = fr / 2;
    }
    sv->budget = mem_budget_bytes;
    for (int i = 0; i < slots; ++i) sv->workers.emplace_back(worker_main, sv);
    *out = sv;
    return FEM_OK;
}

fem_status fem_server_submit(fem_server* sv, int width, const float* f_host, double density, const fem_params* p,
                             long long* id_out) {
    int L = width - 1;
    if (!sv || !f_host || !id_out || width < 3 || (L & (L - 1)) != 0 || !(density > 0.0) || density > 1.0) {
        set_error("fem_server_submit: bad argument (width 2^L+1, density in (0, 1], non-null pointers)");
        return FEM_E_INVALID;
    }
    auto r = std::make_shared<Request>();
    r->width = width;
    r->density = density;
    if (p) r->params = *p; else fem_params_default(&r->params);
    r->f.assign(f_host, f_host + (size_t)width * width);
    r->mem_estimate = estimate_bytes(width, density);
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        r->id = sv->next_id++;
        r->t_submit = now_s();
        sv->queue.push_back(r);
        sv->all[r->id] = r;
    }
    sv->cv_work.notify_all();
    *id_out = r->id;
    return FEM_OK;
}

fem_status fem_server_wait(fem_server* sv, long long id, double timeout_s, int* done) {
    if (!sv || !done) {
        set_error("fem_server_wait: null argument");
        return FEM_E_INVALID;
    }
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(id);
    if (it == sv->all.end()) {
        set_error("fem_server_wait: unknown request id");
        return FEM_E_INVALID;
    }
    auto r = it->second;
    if (timeout_s < 0) sv->cv_done.wait(lk, [&] { return r->done; });
    else sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->done; });
    *done = r->done ? 1 : 0;
    return FEM_OK;
}

fem_status fem_server_result(fem_server* sv, long long id, int* sizes, int* xy, int* tri, unsigned char* is_mask,
                             float* g, double* times) {
    if (!sv) {
        set_error("fem_server_result: null server");
        return FEM_E_INVALID;
    }
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->all.find(id);
        if (it == sv->all.end()) {
            set_error("fem_server_result: unknown request id");
            return FEM_E_INVALID;
        }
        r = it->second;
        if (!r->done) {
            set_error("fem_server_result: request not finished");
            return FEM_E_INVALID;
        }
    }
    if (sizes) { sizes[0] = r->V; sizes[1] = r->T; sizes[2] = r->nK; sizes[3] = r->width; }
    if (xy) std::memcpy(xy, r->xy.data(), sizeof(int) * r->xy.size());
    if (tri) std::memcpy(tri, r->tri.data(), sizeof(int) * r->tri.size());
    if (is_mask) std::memcpy(is_mask, r->mask.data(), r->mask.size());
    if (g) std::memcpy(g, r->g.data(), sizeof(float) * r->g.size());
    if (times) {
        times[0] = r->t_submit;
        times[1] = r->t_start;
        times[2] = r->t_end;
        times[3] = r->spatial.rounds;
        times[4] = (double)r->spatial.cg_iters;
        times[5] = r->tonal.tonal_iters;
        times[6] = r->tonal.tonal_relres;
        times[7] = (double)r->mem_estimate;
        times[8] = (double)r->mem_measured;
    }
    if (r->status != FEM_OK && r->status != FEM_E_NOT_CONVERGED) set_error(r->error);
    return r->status;
}

fem_status fem_server_state(fem_server* sv, long long id, int* state) {
    if (!sv || !state) {
        set_error("fem_server_state: null argument");
        return FEM_E_INVALID;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(id);
    if (it == sv->all.end()) {
        set_error("fem_server_state: unknown request id");
        return FEM_E_INVALID;
    }
    *state = it->second->done ? 2 : (it->second->running ? 1 : 0);
    return FEM_OK;
}

fem_status fem_server_cancel(fem_server* sv, long long id) {
    if (!sv) {
        set_error("fem_server_cancel: null server");
        return FEM_E_INVALID;
    }
    bool dequeued = false;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->all.find(id);
        if (it == sv->all.end()) {
            set_error("fem_server_cancel: unknown request id");
            return FEM_E_INVALID;
        }
        auto r = it->second;
        if (r->done) return FEM_OK;
        r->cancel.store(1);
        for (auto q = sv->queue.begin(); q != sv->queue.end(); ++q) {
            if (*q != r) continue;
            sv->queue.erase(q);
            r->status = FEM_E_CANCELLED;
            r->error = "request cancelled";
            r->t_start = r->t_end = now_s();
            r->f.clear();
            r->f.shrink_to_fit();
            r->done = true;
            dequeued = true;
            break;
        }
    }
    // a running request finishes through its worker, which notifies as usual
    if (dequeued) {
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
    return FEM_OK;
}

fem_status fem_server_release(fem_server* sv, long long id) {
    if (!sv) return FEM_E_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(id);
    if (it == sv->all.end() || !it->second->done) {
        set_error("fem_server_release: unknown or unfinished request");
        return FEM_E_INVALID;
    }
    sv->all.erase(it);
    return FEM_OK;
}

fem_status fem_server_destroy(fem_server* sv) {
    if (!sv) return FEM_OK;
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        // let queued work finish before stopping the workers
        sv->cv_done.wait(lk, [&] { return sv->queue.empty() && sv->running == 0; });
        sv->stopping = true;
    }
    sv->cv_work.notify_all();
    for (auto& t : sv->workers) t.join();
    delete sv;
    return FEM_OK;
}

}  // extern "C"
