/*
 * feminpaint.h -- C ABI of the GB300 (sm_103a) library for FEM harmonic
 * inpainting with spatial and tonal data optimisation, after Chizhov &
 * Weickert, "Efficient Data Optimisation for Harmonic Inpainting with Finite
 * Elements" (arXiv 2105.01586).
 *
 * Conventions shared by every call
 *  - Images are width x height float32, row-major, y pointing down; pixel
 *    (x, y) is at offset y*width + x.  The mesh lives on the domain
 *    [0, N-1]^2 with N = 2^L + 1 the smallest such side >= max(width,
 *    height), so that every edge midpoint created by bisection is a pixel of
 *    the domain; the image lies at the domain's top-left.  Only image pixels
 *    are data: a triangle owns the pixels of the ownership rule that lie in
 *    the image, and the per-triangle errors and the tonal data term sum
 *    over image pixels.  A triangle can be selected when its bounding box
 *    meets the image.  Every vertex outside the image is a mask vertex and
 *    takes the value of the nearest image pixel.  For width == height ==
 *    2^L + 1 the domain is the image.
 *  - A mesh has V vertices (integer pixel positions) and T triangles.  A
 *    triangle is stored as (a, b, c): (a, b) is its refinement edge and c its
 *    newest vertex (the right-angle corner).  Vertices are either mask
 *    vertices (the Dirichlet set K of eqs. 1-3, "stored pixels") or unknown
 *    vertices (U), whose values the Laplace solve provides (Sec. 2.2).
 *  - g, the grey values at the mask vertices, is ordered by ascending vertex
 *    id among the mask vertices (nmask entries).
 *  - "_dev" pointers are device pointers on the current CUDA device; the
 *    caller owns them.  Host pointers are named "_host" or documented as host
 *    buffers.  The library owns the mesh and all its scratch memory, which it
 *    allocates with the stream-ordered allocator on the stream it is given,
 *    from the pool set with fem_set_mem_pool (default: the device's current
 *    pool).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call enqueues its work on that stream; calls that return
 *    sizes or convergence results synchronise that stream before returning.
 *  - Every call returns a fem_status and never aborts or traps; on failure
 *    fem_last_error() gives a message.  A solve that reaches its iteration
 *    cap returns FEM_E_NOT_CONVERGED with the last iterate written.  Waits
 *    inside persistent kernels are bounded; when one runs out the call
 *    returns FEM_E_TIMEOUT and the CUDA context stays usable.
 */
#ifndef FEMINPAINT_H
#define FEMINPAINT_H

#if defined(__GNUC__)
#define FEM_API __attribute__((visibility("default")))
#else
#define FEM_API
#endif

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fem_mesh fem_mesh;
typedef struct fem_server fem_server;

typedef enum {
    FEM_OK = 0,
    FEM_E_INVALID = 1,       /* bad argument or malformed mesh */
    FEM_E_SHAPE = 2,         /* image size out of range (see fem_mesh_create) */
    FEM_E_OOM = 3,           /* device allocation failed */
    FEM_E_NOT_CONVERGED = 4, /* iteration cap reached; last iterate written */
    FEM_E_TIMEOUT = 5,       /* a bounded device-side wait ran out */
    FEM_E_CUDA = 6,          /* a CUDA runtime error (message in fem_last_error) */
    FEM_E_CANCELLED = 7      /* a served request cancelled by fem_server_cancel */
} fem_status;

enum {
    FEM_PREC_FP32_IR = 0, /* FP32 preconditioned CG inside FP64 iterative refinement */
    FEM_PREC_FP64 = 1     /* plain FP64 preconditioned CG */
};

/* Solver and optimisation parameters.  fem_params_default() fills:
 * tol 1e-12, maxit 20000, precision FP32_IR, topk_frac 0.01, max_rounds 0,
 * tonal_tol 1e-8, tonal_maxit 2000, inner_tol 1e-11, fast_keys -1. */
typedef struct {
    double tol;         /* Laplace solve: stop at ||b - A x|| <= tol ||b|| (FP64 residual) */
    int maxit;          /* Laplace solve: cap on CG iterations summed over refinement steps */
    int precision;      /* FEM_PREC_FP32_IR or FEM_PREC_FP64 */
    double topk_frac;   /* spatial: k = max(1, ceil(topk_frac * T)) triangles per round */
    int max_rounds;     /* spatial: stop after this many rounds (0 = only the density rule) */
    double tonal_tol;   /* tonal: stop at ||B^T (f - B g)|| <= tonal_tol ||B^T f|| */
    int tonal_maxit;    /* tonal: cap on outer CG iterations */
    double inner_tol;   /* tonal and adjoint: relative tolerance of the inner Laplace solves */
    int fast_keys;      /* spatial: how the selection keys are computed (the selected set is
                           the same either way): 0 = float-float for every triangle; 1 = FP32
                           with a rigorous error bound for every triangle and float-float only
                           for the triangles whose bound straddles the k-th key; after a
                           call's first round the FP32 pass covers only the squares that
                           hold a triangle the last round bisected or whose vertex values
                           changed (the other bounds are kept: a full pass gives the same
                           bits); 2 = as 1 with a full FP32 pass every round; -1 = 1 from
                           2049 x 2049 pixels on, else 0 */
} fem_params;

/* Counters of the last call on a mesh (host copy). */
typedef struct {
    int rounds;            /* spatial: refinement rounds run */
    long long cg_iters;    /* CG iterations, all solves of the call */
    int solves;            /* Laplace solves run */
    double relres;         /* largest FP64 relative residual among the call's Laplace solves */
    int tonal_iters;       /* tonal: outer iterations */
    double tonal_relres;   /* tonal: ||B^T r|| / ||B^T f|| at exit */
    double min_margin;     /* spatial: smallest relative gap between the k-th and (k+1)-th key */
} fem_stats;

FEM_API void fem_params_default(fem_params *p);

/* Create the initial mesh for a width x height image (Sec. 2.2's mesh,
 * replaced by the two triangles of the domain square split along the
 * diagonal (0,0)-(N-1,N-1)): vertices 0..3 at the corners (0,0), (N-1,0),
 * (0,N-1), (N-1,N-1), all mask vertices, and triangles (v0,v3,v2),
 * (v3,v0,v1).  N is the smallest 2^L + 1 >= max(width, height) (and >= 3).
 * *out receives a library-owned handle.  FEM_E_SHAPE unless
 * 2 <= width, height <= 32769. */
FEM_API fem_status fem_mesh_create(int width, int height, void *stream, fem_mesh **out);

/* Free the mesh and its device memory (after the work on its streams ends). */
FEM_API fem_status fem_mesh_destroy(fem_mesh *m);

/* Sizes of the mesh: vertices, triangles, mask vertices (any pointer may be NULL). */
FEM_API fem_status fem_mesh_info(const fem_mesh *m, int *V, int *T, int *nmask);

/* The image width and height of the mesh and its domain side N (any
 * pointer may be NULL). */
FEM_API fem_status fem_mesh_size(const fem_mesh *m, int *width, int *height, int *domain);

/* Copy the mesh to host buffers: xy (2V ints: x0,y0,x1,y1,...), tri (3T ints:
 * a,b,c per triangle), is_mask (V bytes, 1 = mask vertex).  Any may be NULL.
 * Synchronises the mesh's last stream. */
FEM_API fem_status fem_mesh_export(fem_mesh *m, int *xy, int *tri, unsigned char *is_mask);

/* The order in which the kernels visit the triangles (host buffer, T ints):
 * the space-filling curve of the bisection tree (consecutive triangles share
 * the vertex where the curve leaves one and enters the next), for meshes
 * grown by fem_spatial_refine and for imported ones alike (*is_curve = 1).
 * Either pointer may be NULL. */
FEM_API fem_status fem_mesh_curve_order(fem_mesh *m, int *order, int *is_curve);

/* Replace the mesh by host arrays of the same layout (checkpoint/resume).
 * The arrays are checked: vertices on the grid, triangles positively
 * oriented and right-isosceles with c at the right angle, each a triangle of
 * the newest-vertex-bisection tree of the two-triangle mesh, none twice,
 * areas summing to the image.  Conformity is the caller's contract.
 * FEM_E_INVALID otherwise. */
FEM_API fem_status fem_mesh_import(fem_mesh *m, int V, const int *xy, int T, const int *tri,
                           const unsigned char *is_mask);

/* Harmonic inpainting on the mesh (Sec. 2.2, eqs. 1-3): the linear FEM
 * system A_UU x_U = -A_UK g is solved by preconditioned CG and the solution
 * is interpolated linearly inside each triangle (u = B g of Sec. 4).
 *   g_dev   in : nmask float32 mask-vertex values
 *   u_dev   out: width*height float32 image, or NULL
 *   uv_dev  out: V float64 vertex values (g at K, solution at U), or NULL
 * Each pixel takes its value from exactly one owning triangle. */
FEM_API fem_status fem_inpaint(fem_mesh *m, const float *g_dev, float *u_dev, double *uv_dev,
                       const fem_params *p, void *stream);

/* Dirichlet data taken from the image: g_dev[k] = f at the pixel of the k-th
 * mask vertex (the stored grey values before tonal optimisation, Sec. 3).
 *   f_dev in : width*height float32;  g_dev out: nmask float32 */
FEM_API fem_status fem_gather_mask(fem_mesh *m, const float *f_dev, float *g_dev, void *stream);

/* Per-triangle squared L2 error of Sec. 3: err[t] = sum over the pixels owned
 * by t of (u - f)^2, with u the linear interpolant of the vertex values.
 *   uv_dev  in : V float64 vertex values
 *   f_dev   in : width*height float32 image
 *   err_dev out: T float64 errors (interpolation and sums in FP64) */
FEM_API fem_status fem_triangle_errors(fem_mesh *m, const double *uv_dev, const float *f_dev, double *err_dev,
                               void *stream);

/* The per-triangle errors of fem_triangle_errors for callers that cannot
 * allocate device memory (no counterpart in the paper).  Some callers cannot
 * call cudaMalloc: programs whose own caching allocator has reserved all
 * device memory, and real-time or serving loops that must not allocate after
 * start-up (cudaMalloc can synchronise the device and takes unbounded
 * time).  This call allocates nothing: the
 * caller passes the mesh arrays, the vertex values, the image and the
 * output; the scratch it needs is a fixed 3.4 MB device array inside the
 * library, present on every GPU that loads the library until the process
 * exits.  The first call on a device looks up that array's address (once
 * per device, with the device current).  Every call synchronises `stream`
 * (it reads the item count back), so no call can be captured into a CUDA
 * graph.  The array is shared by all calls and keeps the last
 * call's contents (the call clears what must start at zero), so calls that
 * overlap on the GPU, on any stream, race: serialise them.
 *   width      image side, 2^L + 1, at most 2049
 *   V, xy_dev  vertices: 2V int32 (x, y) pairs, 8-byte aligned
 *   T, tri_dev triangles: 4T int32 (a, b, c, unused), 16-byte aligned;
 *              1 <= T <= 65536; the caller guarantees a valid mesh of the
 *              image (indices < V, as produced by fem_spatial_refine)
 *   uv_dev     V float64 vertex values; f_dev width*width float32
 *   err_dev    out: T float64
 * Sizes beyond the limits return FEM_E_SHAPE / FEM_E_INVALID with a message
 * before any work.  Synchronises `stream` before returning. */
FEM_API fem_status fem_triangle_errors_noalloc(int width, int V, const int *xy_dev, int T, const int *tri_dev,
                                               const double *uv_dev, const float *f_dev, double *err_dev,
                                               void *stream);

/* FP32 error bounds of the per-triangle squared errors (the fast keys of the
 * spatial optimisation, Sec. 3 error map): for every triangle t an interval
 * [lo_dev[t], hi_dev[t]] that contains the float-float key of
 * fem_triangle_errors (u linear on t from the vertex values uv_dev, f the
 * image).  The FP32 sum carries a rigorous bound from the number of
 * roundings of the plane evaluation, the difference and the summation,
 * widened by 1 %.  uv_dev: V doubles; f_dev: the width x height image; lo_dev, hi_dev: T
 * doubles (device, caller-owned).  FEM_E_INVALID on null pointers. */
FEM_API fem_status fem_triangle_error_bounds(fem_mesh *m, const double *uv_dev, const float *f_dev, double *lo_dev,
                                             double *hi_dev, void *stream);

/* Linear interpolation of vertex values to every pixel (end of Sec. 2.2).
 *   uv_dev    in : V float64 vertex values
 *   u_dev     out: width*height float32 image, or NULL
 *   owner_dev out: width*height int32 owning triangle per pixel, or NULL */
FEM_API fem_status fem_rasterize(fem_mesh *m, const double *uv_dev, float *u_dev, int *owner_dev, void *stream);

/* Spatial optimisation (Sec. 3, with bisection instead of insertion): until
 * V >= ceil(density * width*height) (or p->max_rounds rounds), each round
 * sets g = f at the mask vertices, solves (warm-started), computes the
 * per-triangle errors, selects the top k = max(1, ceil(topk_frac*T))
 * eligible triangles (error descending, id ascending; eligible = the
 * refinement-edge midpoint is a pixel and the triangle's bounding box meets
 * the image; k capped by the vertex target) and refines them by
 * newest-vertex bisection.  Midpoints of selected refinement edges become
 * mask vertices; midpoints created only to keep the mesh conforming become
 * unknown vertices.  New vertices are numbered by
 * ascending pixel index of the domain (y N + x), new
 * triangles by ascending (generation, parent id).
 *   f_dev in: width*height float32 image */
FEM_API fem_status fem_spatial_refine(fem_mesh *m, const float *f_dev, double density, const fem_params *p,
                              void *stream);

/* Spatial optimisation of a colour image (Sec. 5 notes that the extension
 * to colour is straightforward; this is its reading): f_dev holds
 * `channels` planes of width*height float32, plane c at offset
 * c*width*height.  The channels share the mesh and the mask vertices, each
 * has its own mask values and Laplace solve, and a triangle's error is the
 * sum over the channels of its squared errors.  channels = 1 is
 * fem_spatial_refine.  1 <= channels <= 4, else FEM_E_INVALID.  With more
 * than one channel every key is the exact (float-float) one; the fast keys
 * serve one channel.  After the call the mesh's vertex values are channel
 * 0's; for each channel, fem_gather_mask and fem_tonal_opt on its plane give
 * its mask values and tonally optimised values (B is the same for all). */
FEM_API fem_status fem_spatial_refine_channels(fem_mesh *m, const float *f_dev, int channels, double density,
                                               const fem_params *p, void *stream);

/* Tonal optimisation (Sec. 4, eqs. 4-5): g* = argmin ||B g - f||^2 by CG on
 * the normal equations B^T B g = B^T f, applying B and B^T through inner
 * Laplace solves; B is never formed.
 *   f_dev in : width*height float32 image
 *   g_dev in : nmask float32 start values; out: the optimised values */
FEM_API fem_status fem_tonal_opt(fem_mesh *m, const float *f_dev, float *g_dev, const fem_params *p, void *stream);

/* Tonal optimisation with the L1 data term (Sec. 5, after the cited work,
 * the L1 error instead of the L2 one): min_g sum over image pixels of
 * |(B g)_p - f_p| by iteratively reweighted least squares.  Each of the
 * `irls` steps sets the weights w_p = 1 / max(|(B g)_p - f_p|, eps) from the
 * current g and runs the tonal CG on the weighted problem
 * min_g sum_p w_p ((B g)_p - f_p)^2 from the current g, with p->tonal_tol and
 * p->tonal_maxit per step (B^T W B g = B^T W f, the pixel-mass matrix
 * P^T W P built by a weighted pixel pass).  The steps majorise the Huber
 * function with threshold eps, which therefore does not increase.
 *   f_dev    in : width*height float32 image
 *   g_dev    in : start (nmask float32); out: the result
 *   irls     steps (>= 0); eps > 0 (grey values in [0, 1]: 1e-3, say)
 * Returns FEM_E_NOT_CONVERGED when the last step hit tonal_maxit;
 * fem_mesh_stats' tonal_iters counts the CG iterations of all steps. */
FEM_API fem_status fem_tonal_opt_l1(fem_mesh *m, const float *f_dev, float *g_dev, int irls, double eps,
                                    const fem_params *p, void *stream);

/* Adjoint of u = B g (Sec. 4): gbar = B^T r = (P^T r)_K - A_KU A_UU^{-1} (P^T r)_U,
 * with P the pixel interpolation matrix.  This is the gradient of
 * <r, B g> with respect to g.
 *   r_dev    in : width*height float32 pixel co-vector
 *   gbar_dev out: nmask float32 */
FEM_API fem_status fem_adjoint(fem_mesh *m, const float *r_dev, float *gbar_dev, const fem_params *p, void *stream);

/* Tonal loss of Sec. 4 (eq. 4) and its gradient, whose zero is the normal
 * equations (eq. 5):  loss = 1/2 ||B g - f||^2,  grad = B^T (B g - f).
 * One inpainting solve gives the vertex values v = E g; the loss is half the
 * sum of the per-triangle squared errors of fem_triangle_errors (float-float
 * per pixel, FP64 per triangle and in the total); the gradient is
 * E^T (M v - P^T f) with the pixel-mass matrix M = P^T P, so no pixel
 * residual is formed, and takes one adjoint solve.
 *   g_dev    in : nmask float32 mask-vertex values
 *   f_dev    in : width*height float32 image
 *   loss_dev out: 1 float64 (device), or NULL
 *   grad_dev out: nmask float32, or NULL (at least one of the two is needed)
 * The solves use p->tol / p->inner_tol and p->precision.  Synchronises
 * `stream`. */
FEM_API fem_status fem_tonal_loss(fem_mesh *m, const float *g_dev, const float *f_dev, double *loss_dev,
                                  float *grad_dev, const fem_params *p, void *stream);

/* ---------------------------------------------------------------------
 * Serving: continuous batching of whole data-optimisation jobs (configuration
 * 5 of the benchmarks; the paper has no serving layer).  A server owns
 * `slots` worker threads, each with its own CUDA stream on the current
 * device.  Requests wait in a FIFO queue; the head request is admitted when a
 * slot is free and its device memory fits next to the running requests
 * within `mem_budget_bytes` (0 = half of the free device memory; a request
 * larger than the budget runs alone).  A request's memory is a static
 * estimate scaled by 1.25 times the largest ratio of measured peak to
 * estimate among the requests that have finished (the static estimate
 * alone before any has); the library counts every device allocation on the
 * stream it was made on.  An admitted request runs the
 * whole path on its slot's stream: fem_mesh_create, fem_spatial_refine,
 * fem_gather_mask, fem_tonal_opt and the result read-back.  Requests in
 * different slots overlap on the device; each computes exactly what it
 * computes alone (deterministic kernels, no shared state between meshes).
 * --------------------------------------------------------------------- */

/* Start the worker threads.  *out receives the handle. */
FEM_API fem_status fem_server_create(int slots, size_t mem_budget_bytes, fem_server **out);

/* Queue one job: the width x width float32 image at f_host (copied before
 * the call returns), the vertex density for fem_spatial_refine and the
 * parameters for both optimisations (NULL = defaults).  *id_out receives the
 * request id. */
FEM_API fem_status fem_server_submit(fem_server *sv, int width, const float *f_host, double density,
                                     const fem_params *p, long long *id_out);

/* Wait up to timeout_s seconds (< 0: no limit) for a request; *done = 1 when
 * it has finished (successfully or not). */
FEM_API fem_status fem_server_wait(fem_server *sv, long long id, double timeout_s, int *done);

/* Results of a finished request (host buffers, any may be NULL):
 * sizes[4] = V, T, nmask, width; xy (2V), tri (3T), is_mask (V) as in
 * fem_mesh_export; g (nmask float32, the tonally optimised values);
 * times[9] = submit, start and end time (seconds, steady clock), spatial
 * rounds, spatial CG iterations, tonal iterations, tonal relative residual,
 * the static estimate of its device bytes, the peak device bytes it held
 * (measured).  Query the sizes first with NULL arrays.  Returns
 * the request's own status (FEM_E_NOT_CONVERGED if the tonal cap was hit). */
FEM_API fem_status fem_server_result(fem_server *sv, long long id, int *sizes, int *xy, int *tri,
                                     unsigned char *is_mask, float *g, double *times);

/* State of a request: *state = 0 queued, 1 running, 2 finished. */
FEM_API fem_status fem_server_state(fem_server *sv, long long id, int *state);

/* Cancel a request.  A queued request is removed from the queue; a running
 * one stops at its next spatial round or tonal iteration (its kernels in
 * flight finish first, nothing is interrupted on the device) and frees its
 * memory.  Either way the request then counts as finished with status
 * FEM_E_CANCELLED (no results).  Cancelling a finished request does nothing
 * and returns FEM_OK; an unknown id returns FEM_E_INVALID. */
FEM_API fem_status fem_server_cancel(fem_server *sv, long long id);

/* Drop a finished request's results. */
FEM_API fem_status fem_server_release(fem_server *sv, long long id);

/* Finish the queued work, stop the workers and free the server. */
FEM_API fem_status fem_server_destroy(fem_server *sv);

/* Counters of the last inpaint / refine / tonal / adjoint call on m. */
FEM_API fem_status fem_mesh_stats(const fem_mesh *m, fem_stats *out);

/* Message of the last failure on the calling thread ("" if none). */
FEM_API const char *fem_last_error(void);

/* Instrumentation, off by default.  family_mask bit f turns on family f
 * (0 turns everything off).  For an enabled family the library records a
 * CUDA event pair around every launch on the launching stream and adds up
 * the algorithmic bytes of the work (bytes the operation must move at
 * least once: inputs read, outputs written; counted on the host from the
 * sizes and iteration counts).  fem_profile_read() synchronises, returns
 * per family the launches, summed device time in ms and algorithmic bytes,
 * and clears the records.  Families: 0 raster/error (plans, band, image
 * layout, tonal pixel sums), 1 CG, 2 assembly, 3 top-k, 4 refinement,
 * 5 tonal vector work, 6 other, 7 the square-tiled error pass over all
 * squares (that one kernel).  name receives a
 * static label.  Returns 0, or -1 for an unknown family. */
FEM_API void fem_profile_enable(int family_mask);
FEM_API int fem_profile_read(int family, long long *launches, double *ms, double *bytes, const char **name);

/* Check of the library's bounded device-side waits (no counterpart in the
 * paper): runs the grid barrier used by the persistent kernels with one of
 * its two blocks never arriving.  The waiting block must give up after the
 * barrier's limit (2 s) and report it; the call returns FEM_E_TIMEOUT when
 * that happened (the expected outcome) and the CUDA context stays usable. */
FEM_API fem_status fem_selftest_wait_timeout(void *stream);

/* Number of kernels this library has launched in the process so far. */
FEM_API long long fem_launch_count(void);

/* Memory pool for the library's device allocations (the mesh, its scratch,
 * the server's request buffers).  pool is a cudaMemPool_t passed as void*;
 * allocations from now on are made with cudaMallocFromPoolAsync on that
 * pool, on the stream of the call.  NULL returns to the current device's
 * current pool (cudaMallocAsync).  The setting is process-wide; memory
 * already allocated stays where it is and is freed in stream order as usual.
 * The caller keeps the pool alive until every mesh and server created while
 * it was set has been destroyed. */
FEM_API fem_status fem_set_mem_pool(void *pool);

/* Test hook for the library's handling of a full device (no counterpart in
 * the paper).  *calls_out (may be NULL) receives the number of device
 * allocations the library has attempted in this process so far.  With
 * fail_after >= 0 the allocation that comes fail_after attempts from now
 * (0: the next one) fails as if the device were full: it makes no CUDA call
 * and the operation that needed it returns FEM_E_OOM.  fail_after < 0
 * disarms the hook.  Host-side only: nothing runs on the device. */
FEM_API fem_status fem_debug_alloc_fault(long long fail_after, long long *calls_out);

#ifdef __cplusplus
}
#endif

#endif /* FEMINPAINT_H */
