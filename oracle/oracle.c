/*
 * oracle.c -- plain, slow, FP64 CPU oracle for FEM harmonic inpainting with
 * spatial and tonal data optimisation (Chizhov & Weickert, "Efficient Data
 * Optimisation for Harmonic Inpainting with Finite Elements", arXiv 2105.01586).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a test library that
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load.  The product path (the CUDA library and its Python binding) never
 * includes, links or calls it, and it shares no code with that path.
 *
 * Every routine is written for a reader checking it against the paper:
 * scalar loops, FP64 arithmetic, no blocking or fusion.  Where the paper is
 * silent the readings below are used (each also listed in the design notes):
 *
 *  R1  Mesh.  The image side is N = 2^L + 1.  The initial mesh has the four
 *      corners as vertices 0..3 = (0,0), (N-1,0), (0,N-1), (N-1,N-1) and the
 *      two triangles (v0,v3,v2) and (v3,v0,v1).  A triangle is stored as
 *      (a,b,c): (a,b) is its refinement edge, c its newest vertex.  This
 *      replaces the Delaunay triangulation of Sec. 2.2.
 *  R2  Newest-vertex bisection of (a,b,c) at m = (a+b)/2 gives (c,a,m), which
 *      keeps the parent's id, and (b,c,m), which gets a new id.
 *  R3  Refinement round: the refinement edges of the selected triangles are
 *      marked; closure marks the refinement edge of every triangle that has a
 *      marked edge, until nothing changes; then bisection runs in
 *      generations until no triangle has a marked refinement edge.
 *  R4  Numbering: new vertices get ids in ascending pixel index y*N + x; new
 *      triangles get ids in ascending (generation, parent id).
 *  R5  Mask (Dirichlet set K): the corners and the midpoints of the refinement
 *      edges of selected triangles.  Midpoints made only by closure are the
 *      unknown vertices U (Sec. 2.2 allows any subset of non-mask pixels).
 *  R6  Pixel ownership: pixel p belongs to the triangle whose interior holds
 *      p + eps*(sx, delta*sy) for 0 < delta << 1, eps -> 0+, where sx = +1
 *      (-1 on the last column) and sy = +1 (-1 on the last row).  Every pixel
 *      has exactly one owner, so the interpolation matrix P has one row per
 *      pixel and P^T is its exact adjoint.
 *  R7  Per-triangle error: key_t = sum over owned pixels of (u - f)^2, the
 *      squared L2 error of Sec. 3 (same order as the L2 norm).
 *  R8  Top-k: k = max(1, ceil(frac*T)), capped by the number of eligible
 *      triangles and by V* - V; order by key descending, then id ascending.
 *      A triangle is eligible when its refinement-edge midpoint is a pixel
 *      and its bounding box meets the image (R9).
 *  R9  Image sizes other than 2^L + 1 (the paper's 2^k images and its
 *      4896 x 3264 photograph, Sec. 5): a W x H image lies at the top-left
 *      of the domain [0, N-1]^2, N = 2^L + 1 >= max(W, H), which carries the
 *      mesh exactly as for a square image.  Only image pixels are data: a
 *      triangle owns the pixels of R6 that lie in the image, so P has one
 *      row per image pixel, the keys and the data term of the tonal
 *      optimisation run over image pixels, and V* = ceil(density W H).
 *      Triangles whose bounding box misses the image are not eligible; a
 *      selected midpoint may still lie outside the image (when the image is
 *      less than half the domain high, the two initial triangles bisect
 *      below it).  Every vertex outside the image is a mask vertex with the
 *      value of the nearest image pixel (f at the clamped position): the
 *      method runs on the image padded with its edge values, with the data
 *      term restricted to the image, and the padding holds no unknowns
 *      (with no data there, they would form large badly conditioned
 *      blocks).  With W = H = N everything reduces to the square case.
 *  R10 Colour (Sec. 5 says only that colour is straightforward): C <= 4
 *      channels share the mesh, the mask set and A_UU; each channel has its
 *      own mask values and solve, and a triangle's error is the sum of its
 *      channels' errors (channel 0 first).  C = 1 is the grey case.
 *  R11 The L1 data term of Sec. 5: min_g sum_p |(B g)_p - f_p| by
 *      iteratively reweighted least squares, weights 1 / max(|B g - f|, eps)
 *      from the current g, each step a weighted least-squares solve; with
 *      eps each step is a majorise-minimise step of the Huber function.
 *
 * Threads.  Compiled with -fopenmp (the multi-core CPU baseline), two loops
 * share their iterations among threads: the per-triangle raster loop and the
 * row loop of A_UU x.  In both each output element (a pixel, a key, a row) is
 * computed by one thread with the same operations in the same order, so the
 * results are bit-identical to the single-thread build.  Dot products, the
 * scatter P^T r, sorting and refinement stay serial.  Without -fopenmp the
 * pragmas are ignored.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define OM_OK 0
#define OM_E_INVALID 1
#define OM_E_OOM 3
#define OM_E_NOT_CONVERGED 4

typedef struct {
    int N;
    int W, H;  /* image size (R9); W = H = N for a square image */
    int V, T;
    int capV, capT;
    int *vx, *vy;
    unsigned char *mask;
    int *ta, *tb, *tc;
} om_mesh;

/* ------------------------------------------------------------------ */
/* mesh storage                                                        */
/* ------------------------------------------------------------------ */

static int grow_vertices(om_mesh *m, int need)
{
    if (need <= m->capV) return OM_OK;
    int cap = m->capV ? m->capV : 16;
    while (cap < need) cap *= 2;
    int *vx = realloc(m->vx, sizeof(int) * cap);
    if (!vx) return OM_E_OOM;
    m->vx = vx;
    int *vy = realloc(m->vy, sizeof(int) * cap);
    if (!vy) return OM_E_OOM;
    m->vy = vy;
    unsigned char *mk = realloc(m->mask, cap);
    if (!mk) return OM_E_OOM;
    m->mask = mk;
    m->capV = cap;
    return OM_OK;
}

static int grow_triangles(om_mesh *m, int need)
{
    if (need <= m->capT) return OM_OK;
    int cap = m->capT ? m->capT : 16;
    while (cap < need) cap *= 2;
    int *a = realloc(m->ta, sizeof(int) * cap);
    if (!a) return OM_E_OOM;
    m->ta = a;
    int *b = realloc(m->tb, sizeof(int) * cap);
    if (!b) return OM_E_OOM;
    m->tb = b;
    int *c = realloc(m->tc, sizeof(int) * cap);
    if (!c) return OM_E_OOM;
    m->tc = c;
    m->capT = cap;
    return OM_OK;
}

void om_mesh_free(om_mesh *m)
{
    if (!m) return;
    free(m->vx); free(m->vy); free(m->mask);
    free(m->ta); free(m->tb); free(m->tc);
    free(m);
}

static int add_vertex(om_mesh *m, int x, int y, int is_mask)
{
    if (grow_vertices(m, m->V + 1)) return -1;
    m->vx[m->V] = x; m->vy[m->V] = y; m->mask[m->V] = (unsigned char)is_mask;
    return m->V++;
}

static int add_triangle(om_mesh *m, int a, int b, int c)
{
    if (grow_triangles(m, m->T + 1)) return -1;
    m->ta[m->T] = a; m->tb[m->T] = b; m->tc[m->T] = c;
    return m->T++;
}

/* R1: four corner vertices (all in K) and two triangles split along the
 * diagonal (0,0)-(N-1,N-1). */
om_mesh *om_mesh_new(int N)
{
    if (N < 3) return NULL;
    int L = N - 1;
    if (L & (L - 1)) return NULL; /* N must be 2^L + 1 */
    om_mesh *m = calloc(1, sizeof(om_mesh));
    if (!m) return NULL;
    m->N = N;
    m->W = N;
    m->H = N;
    add_vertex(m, 0, 0, 1);
    add_vertex(m, N - 1, 0, 1);
    add_vertex(m, 0, N - 1, 1);
    add_vertex(m, N - 1, N - 1, 1);
    add_triangle(m, 0, 3, 2);
    add_triangle(m, 3, 0, 1);
    if (m->V != 4 || m->T != 2) { om_mesh_free(m); return NULL; }
    return m;
}

om_mesh *om_mesh_from(int N, int V, const int *vx, const int *vy, const unsigned char *mask,
                      int T, const int *ta, const int *tb, const int *tc)
{
    om_mesh *m = calloc(1, sizeof(om_mesh));
    if (!m) return NULL;
    m->N = N;
    m->W = N;
    m->H = N;
    if (grow_vertices(m, V > 0 ? V : 1) || grow_triangles(m, T > 0 ? T : 1)) { om_mesh_free(m); return NULL; }
    memcpy(m->vx, vx, sizeof(int) * V);
    memcpy(m->vy, vy, sizeof(int) * V);
    memcpy(m->mask, mask, V);
    memcpy(m->ta, ta, sizeof(int) * T);
    memcpy(m->tb, tb, sizeof(int) * T);
    memcpy(m->tc, tc, sizeof(int) * T);
    m->V = V; m->T = T;
    return m;
}

/* R9: the image W x H inside the domain of side N (2 <= W, H <= N). */
int om_mesh_set_image(om_mesh *m, int W, int H)
{
    if (W < 2 || H < 2 || W > m->N || H > m->N) return OM_E_INVALID;
    m->W = W;
    m->H = H;
    return OM_OK;
}

/* The initial mesh for a W x H image: the smallest domain N = 2^L + 1 that
 * holds it (R1, R9). */
om_mesh *om_mesh_new_image(int W, int H)
{
    if (W < 2 || H < 2) return NULL;
    int N = 3;
    while (N < W || N < H) N = 2 * N - 1;
    om_mesh *m = om_mesh_new(N);
    if (m && om_mesh_set_image(m, W, H)) { om_mesh_free(m); return NULL; }
    return m;
}

int om_mesh_W(const om_mesh *m) { return m->W; }
int om_mesh_H(const om_mesh *m) { return m->H; }
int om_mesh_V(const om_mesh *m) { return m->V; }
int om_mesh_T(const om_mesh *m) { return m->T; }
int om_mesh_N(const om_mesh *m) { return m->N; }

void om_mesh_get(const om_mesh *m, int *vx, int *vy, unsigned char *mask, int *ta, int *tb, int *tc)
{
    memcpy(vx, m->vx, sizeof(int) * m->V);
    memcpy(vy, m->vy, sizeof(int) * m->V);
    memcpy(mask, m->mask, m->V);
    memcpy(ta, m->ta, sizeof(int) * m->T);
    memcpy(tb, m->tb, sizeof(int) * m->T);
    memcpy(tc, m->tc, sizeof(int) * m->T);
}

void om_mesh_set_mask(om_mesh *m, const unsigned char *mask) { memcpy(m->mask, mask, m->V); }

/* ------------------------------------------------------------------ */
/* a set of undirected edges, keyed by their two vertex ids            */
/* ------------------------------------------------------------------ */

typedef struct {
    uint64_t *key;
    int *sel;  /* 1 if the edge is the refinement edge of a selected triangle */
    int *vid;  /* id of the midpoint vertex once numbered */
    size_t cap, n;
} edge_set;

#define EMPTY_KEY UINT64_MAX

static uint64_t edge_key(int i, int j)
{
    if (i > j) { int t = i; i = j; j = t; }
    return ((uint64_t)(uint32_t)i << 32) | (uint32_t)j;
}

static size_t edge_hash(uint64_t k, size_t cap)
{
    k ^= k >> 33; k *= 0xff51afd7ed558ccdULL; k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL; k ^= k >> 33;
    return (size_t)(k & (cap - 1));
}

static int eset_init(edge_set *s, size_t expected)
{
    size_t cap = 64;
    while (cap < 4 * expected) cap *= 2;
    s->key = malloc(sizeof(uint64_t) * cap);
    s->sel = calloc(cap, sizeof(int));
    s->vid = malloc(sizeof(int) * cap);
    if (!s->key || !s->sel || !s->vid) return OM_E_OOM;
    for (size_t i = 0; i < cap; ++i) { s->key[i] = EMPTY_KEY; s->vid[i] = -1; }
    s->cap = cap; s->n = 0;
    return OM_OK;
}

static void eset_free(edge_set *s) { free(s->key); free(s->sel); free(s->vid); }

static long eset_find(const edge_set *s, uint64_t k)
{
    size_t h = edge_hash(k, s->cap);
    for (;;) {
        if (s->key[h] == k) return (long)h;
        if (s->key[h] == EMPTY_KEY) return -1;
        h = (h + 1) & (s->cap - 1);
    }
}

/* insert; returns the slot; *fresh = 1 if it was not there before */
static long eset_insert(edge_set *s, uint64_t k, int *fresh)
{
    size_t h = edge_hash(k, s->cap);
    *fresh = 0;
    for (;;) {
        if (s->key[h] == k) return (long)h;
        if (s->key[h] == EMPTY_KEY) {
            if (2 * (s->n + 1) > s->cap) return -1; /* table full: caller sized it too small */
            s->key[h] = k; s->n++; *fresh = 1;
            return (long)h;
        }
        h = (h + 1) & (s->cap - 1);
    }
}

/* ------------------------------------------------------------------ */
/* R2-R5: one refinement round by newest-vertex bisection              */
/* ------------------------------------------------------------------ */

/* the refinement-edge midpoint is a lattice point (the edge can be bisected) */
static int lattice_mid(const om_mesh *m, int t)
{
    int a = m->ta[t], b = m->tb[t];
    return ((m->vx[a] + m->vx[b]) % 2 == 0) && ((m->vy[a] + m->vy[b]) % 2 == 0);
}

/* R8, R9: selectable when the edge can be bisected and the triangle's
 * bounding box meets the image (its smallest x and y lie in the image) */
int om_eligible(const om_mesh *m, int t)
{
    int a = m->ta[t], b = m->tb[t], c = m->tc[t];
    int xmin = m->vx[a] < m->vx[b] ? m->vx[a] : m->vx[b];
    int ymin = m->vy[a] < m->vy[b] ? m->vy[a] : m->vy[b];
    if (m->vx[c] < xmin) xmin = m->vx[c];
    if (m->vy[c] < ymin) ymin = m->vy[c];
    return lattice_mid(m, t) && xmin < m->W && ymin < m->H;
}

typedef struct { long pix; long slot; } pix_slot;

static int cmp_pix(const void *p, const void *q)
{
    const pix_slot *a = p, *b = q;
    return (a->pix > b->pix) - (a->pix < b->pix);
}

/* info[0] = new vertices, info[1] = new triangles, info[2] = generations,
 * info[3] = new mask vertices; par (optional, 2 per possible new vertex):
 * the ends of the edge each new vertex bisects, in new-vertex order */
static int refine_par(om_mesh *m, const int *sel, int nsel, int *info, int *par);

int om_refine(om_mesh *m, const int *sel, int nsel, int *info) { return refine_par(m, sel, nsel, info, NULL); }
int om_refine_par(om_mesh *m, const int *sel, int nsel, int *info, int *par)
{
    return refine_par(m, sel, nsel, info, par);
}

static int refine_par(om_mesh *m, const int *sel, int nsel, int *info, int *par)
{
    int rc = OM_OK;
    edge_set E;
    if (eset_init(&E, (size_t)m->T + (size_t)nsel + 16)) return OM_E_OOM;

    /* mark the refinement edges of the selected triangles (R3, R5) */
    for (int s = 0; s < nsel; ++s) {
        int t = sel[s];
        if (t < 0 || t >= m->T || !om_eligible(m, t)) { eset_free(&E); return OM_E_INVALID; }
        int fresh;
        long h = eset_insert(&E, edge_key(m->ta[t], m->tb[t]), &fresh);
        if (h < 0) { eset_free(&E); return OM_E_OOM; }
        E.sel[h] = 1;
    }

    /* closure: a triangle with any marked edge must bisect its refinement edge */
    int changed = 1;
    while (changed) {
        changed = 0;
        for (int t = 0; t < m->T; ++t) {
            int a = m->ta[t], b = m->tb[t], c = m->tc[t];
            uint64_t kref = edge_key(a, b);
            if (eset_find(&E, kref) >= 0) continue;
            if (eset_find(&E, edge_key(b, c)) >= 0 || eset_find(&E, edge_key(c, a)) >= 0) {
                if (!lattice_mid(m, t)) { eset_free(&E); return OM_E_INVALID; } /* never happens on valid meshes */
                int fresh;
                if (eset_insert(&E, kref, &fresh) < 0) { eset_free(&E); return OM_E_OOM; }
                changed = 1;
            }
        }
    }

    /* number the midpoints in ascending pixel index (R4) */
    pix_slot *order = malloc(sizeof(pix_slot) * (E.n ? E.n : 1));
    if (!order) { eset_free(&E); return OM_E_OOM; }
    size_t nn = 0;
    for (size_t h = 0; h < E.cap; ++h) {
        if (E.key[h] == EMPTY_KEY) continue;
        int i = (int)(E.key[h] >> 32), j = (int)(E.key[h] & 0xffffffffu);
        int sx = m->vx[i] + m->vx[j], sy = m->vy[i] + m->vy[j];
        if ((sx & 1) || (sy & 1)) { rc = OM_E_INVALID; break; }
        order[nn].pix = (long)(sy / 2) * m->N + (sx / 2);
        order[nn].slot = (long)h;
        nn++;
    }
    if (rc) { free(order); eset_free(&E); return rc; }
    qsort(order, nn, sizeof(pix_slot), cmp_pix);
    int V0 = m->V, nmask = 0;
    for (size_t r = 0; r < nn; ++r) {
        long h = order[r].slot;
        int x = (int)(order[r].pix % m->N), y = (int)(order[r].pix / m->N);
        /* R5, R9: selected midpoints, and every vertex outside the image */
        int is_mask = E.sel[h] || x >= m->W || y >= m->H;
        int id = add_vertex(m, x, y, is_mask);
        if (id < 0) { free(order); eset_free(&E); return OM_E_OOM; }
        E.vid[h] = id;
        if (par) {
            par[2 * (id - V0)] = (int)(E.key[h] >> 32);
            par[2 * (id - V0) + 1] = (int)(E.key[h] & 0xffffffffu);
        }
        nmask += is_mask;
    }
    free(order);

    /* bisection in generations (R2, R4) */
    int T0 = m->T, gens = 0;
    for (;;) {
        int Tg = m->T, nb = 0;
        for (int t = 0; t < Tg; ++t) {
            int a = m->ta[t], b = m->tb[t], c = m->tc[t];
            long h = eset_find(&E, edge_key(a, b));
            if (h < 0) continue;
            int mid = E.vid[h];
            m->ta[t] = c; m->tb[t] = a; m->tc[t] = mid;
            if (add_triangle(m, b, c, mid) < 0) { eset_free(&E); return OM_E_OOM; }
            nb++;
        }
        if (nb == 0) break;
        gens++;
        if (gens > 2) { eset_free(&E); return OM_E_INVALID; } /* NVB needs at most two */
        /* the bisected edges are gone from the mesh; drop them so that the
         * half-edges are not mistaken for them (they have other keys anyway) */
    }
    /* each marked edge was split by every triangle that contained it: no
     * remaining triangle may still have a marked edge */
    for (int t = 0; t < m->T; ++t) {
        if (eset_find(&E, edge_key(m->ta[t], m->tb[t])) >= 0 ||
            eset_find(&E, edge_key(m->tb[t], m->tc[t])) >= 0 ||
            eset_find(&E, edge_key(m->tc[t], m->ta[t])) >= 0) { rc = OM_E_INVALID; break; }
    }
    if (info) { info[0] = m->V - V0; info[1] = m->T - T0; info[2] = gens; info[3] = nmask; }
    eset_free(&E);
    return rc;
}

/* ------------------------------------------------------------------ */
/* P1 stiffness matrix A (Sec. 2.2), sparse rows                      */
/* ------------------------------------------------------------------ */

#define MAXNB 16

typedef struct {
    int V;
    int *deg;      /* number of off-diagonal entries per row */
    int *nb;       /* V*MAXNB neighbour ids */
    double *val;   /* V*MAXNB values */
    double *diag;  /* V */
} sp_rows;

static void sp_free(sp_rows *A) { free(A->deg); free(A->nb); free(A->val); free(A->diag); }

static int sp_add(sp_rows *A, int i, int j, double v)
{
    if (i == j) { A->diag[i] += v; return OM_OK; }
    for (int s = 0; s < A->deg[i]; ++s)
        if (A->nb[i * MAXNB + s] == j) { A->val[i * MAXNB + s] += v; return OM_OK; }
    if (A->deg[i] >= MAXNB) return OM_E_INVALID;
    A->nb[i * MAXNB + A->deg[i]] = j;
    A->val[i * MAXNB + A->deg[i]] = v;
    A->deg[i]++;
    return OM_OK;
}

/* Local P1 stiffness of a triangle from the gradients of its hat functions:
 * K_ij = |T| grad(phi_i).grad(phi_j) = (e_i . e_j) / (4|T|), e_i the edge
 * vector opposite vertex i.  Assembled over all triangles. */
static int assemble(const om_mesh *m, sp_rows *A)
{
    A->V = m->V;
    A->deg = calloc(m->V, sizeof(int));
    A->nb = malloc(sizeof(int) * (size_t)m->V * MAXNB);
    A->val = malloc(sizeof(double) * (size_t)m->V * MAXNB);
    A->diag = calloc(m->V, sizeof(double));
    if (!A->deg || !A->nb || !A->val || !A->diag) return OM_E_OOM;
    for (int t = 0; t < m->T; ++t) {
        int v[3] = {m->ta[t], m->tb[t], m->tc[t]};
        double px[3], py[3];
        for (int i = 0; i < 3; ++i) { px[i] = m->vx[v[i]]; py[i] = m->vy[v[i]]; }
        double twoA = (px[1] - px[0]) * (py[2] - py[0]) - (py[1] - py[0]) * (px[2] - px[0]);
        if (!(twoA > 0)) return OM_E_INVALID;
        double ex[3], ey[3];
        for (int i = 0; i < 3; ++i) {
            int j = (i + 1) % 3, k = (i + 2) % 3;
            ex[i] = px[k] - px[j]; ey[i] = py[k] - py[j];
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double kij = (ex[i] * ex[j] + ey[i] * ey[j]) / (2.0 * twoA);
                int rc = sp_add(A, v[i], v[j], kij);
                if (rc) return rc;
            }
    }
    return OM_OK;
}

/* Full stiffness matrix as CSR (diagonal first in each row) for the tests. */
int om_stiffness_csr(const om_mesh *m, int *rowptr, int *col, double *val, int cap)
{
    sp_rows A;
    memset(&A, 0, sizeof(A));
    int rc = assemble(m, &A);
    if (rc) { sp_free(&A); return rc; }
    int n = 0;
    for (int i = 0; i < m->V; ++i) {
        rowptr[i] = n;
        if (n + 1 + A.deg[i] > cap) { sp_free(&A); return OM_E_OOM; }
        col[n] = i; val[n] = A.diag[i]; n++;
        for (int s = 0; s < A.deg[i]; ++s) { col[n] = A.nb[i * MAXNB + s]; val[n] = A.val[i * MAXNB + s]; n++; }
    }
    rowptr[m->V] = n;
    sp_free(&A);
    return OM_OK;
}

/* ------------------------------------------------------------------ */
/* Laplace solve on the unknown vertices (Sec. 2.2): A_UU x_U = -A_UK g */
/* ------------------------------------------------------------------ */

/* y_U = A_UU x_U, using the vertex-indexed vector x (entries at K ignored) */
static void apply_AUU(const om_mesh *m, const sp_rows *A, const double *x, double *y)
{
    #pragma omp parallel for schedule(static) if (m->V > 4096)
    for (int i = 0; i < m->V; ++i) {
        if (m->mask[i]) continue;
        double s = A->diag[i] * x[i];
        for (int q = 0; q < A->deg[i]; ++q) {
            int j = A->nb[i * MAXNB + q];
            if (!m->mask[j]) s += A->val[i * MAXNB + q] * x[j];
        }
        y[i] = s;
    }
}

static double dot_U(const om_mesh *m, const double *x, const double *y)
{
    double s = 0.0;
    for (int i = 0; i < m->V; ++i) if (!m->mask[i]) s += x[i] * y[i];
    return s;
}

/* Jacobi-preconditioned CG on A_UU x_U = b_U.  x holds the start on entry and
 * the solution on exit (vertex-indexed; entries at K untouched).  Stops when
 * the recomputed residual satisfies ||b - A x|| <= tol ||b||. */
static int cg_UU(const om_mesh *m, const sp_rows *A, const double *b, double *x, double tol, int maxit,
                 int *iters_out, double *relres_out)
{
    int V = m->V;
    double *r = calloc(V, sizeof(double)), *z = calloc(V, sizeof(double));
    double *p = calloc(V, sizeof(double)), *q = calloc(V, sizeof(double));
    if (!r || !z || !p || !q) { free(r); free(z); free(p); free(q); return OM_E_OOM; }
    double bnorm = sqrt(dot_U(m, b, b));
    int it = 0;
    int status = OM_E_NOT_CONVERGED;
    double relres = 0.0;
    if (bnorm == 0.0) {
        for (int i = 0; i < V; ++i) if (!m->mask[i]) x[i] = 0.0;
        status = OM_OK;
        goto done;
    }
    for (int restart = 0; restart < 50 && it < maxit; ++restart) {
        apply_AUU(m, A, x, q);
        for (int i = 0; i < V; ++i) if (!m->mask[i]) r[i] = b[i] - q[i];
        relres = sqrt(dot_U(m, r, r)) / bnorm;
        if (relres <= tol) { status = OM_OK; goto done; }
        for (int i = 0; i < V; ++i) if (!m->mask[i]) { z[i] = r[i] / A->diag[i]; p[i] = z[i]; }
        double rz = dot_U(m, r, z);
        while (it < maxit) {
            apply_AUU(m, A, p, q);
            double alpha = rz / dot_U(m, p, q);
            for (int i = 0; i < V; ++i) if (!m->mask[i]) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
            it++;
            if (sqrt(dot_U(m, r, r)) <= tol * bnorm) break; /* verify with the true residual */
            for (int i = 0; i < V; ++i) if (!m->mask[i]) z[i] = r[i] / A->diag[i];
            double rz1 = dot_U(m, r, z);
            double beta = rz1 / rz;
            rz = rz1;
            for (int i = 0; i < V; ++i) if (!m->mask[i]) p[i] = z[i] + beta * p[i];
        }
    }
    apply_AUU(m, A, x, q);
    for (int i = 0; i < V; ++i) if (!m->mask[i]) r[i] = b[i] - q[i];
    relres = sqrt(dot_U(m, r, r)) / bnorm;
    if (relres <= tol) status = OM_OK;
done:
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = relres;
    free(r); free(z); free(p); free(q);
    return status;
}

/* b_U = -A_UK g_K for the vertex-indexed vector v (entries at K = g) */
static void rhs_U(const om_mesh *m, const sp_rows *A, const double *v, double *b)
{
    for (int i = 0; i < m->V; ++i) {
        if (m->mask[i]) continue;
        double s = 0.0;
        for (int q = 0; q < A->deg[i]; ++q) {
            int j = A->nb[i * MAXNB + q];
            if (m->mask[j]) s -= A->val[i * MAXNB + q] * v[j];
        }
        b[i] = s;
    }
}

/* uv: vertex values.  On entry the entries at K hold g and those at U the
 * starting guess; on exit the entries at U hold the FEM solution. */
int om_solve(const om_mesh *m, double *uv, double tol, int maxit, int *iters, double *relres)
{
    sp_rows A;
    memset(&A, 0, sizeof(A));
    int rc = assemble(m, &A);
    if (rc) { sp_free(&A); return rc; }
    double *b = calloc(m->V, sizeof(double));
    if (!b) { sp_free(&A); return OM_E_OOM; }
    rhs_U(m, &A, uv, b);
    rc = cg_UU(m, &A, b, uv, tol, maxit, iters, relres);
    free(b);
    sp_free(&A);
    return rc;
}

/* ------------------------------------------------------------------ */
/* rasterisation: pixel ownership (R6) and linear interpolation        */
/* ------------------------------------------------------------------ */

/* Does the perturbed pixel lie on the inner side of the directed edge P->Q?
 * w = cross(Q-P, X-P) at the pixel; (gx, gy) its gradient; the perturbation
 * is eps*(sx, delta*sy) with delta << 1, so the x part decides unless the
 * edge is horizontal. */
static int inner_side(long w, long gx, long gy, int sx, int sy)
{
    if (w > 0) return 1;
    if (w < 0) return 0;
    if (gx != 0) return gx * sx > 0;
    return gy * sy > 0;
}

/* Enumerate the pixels owned by triangle t with their barycentric
 * coordinates (lambda_a, lambda_b, lambda_c): those of R6 that lie in the
 * image (R9).  Returns the count. */
static long owned_pixels(const om_mesh *m, int t, int *px, int *py, double *la, double *lb, double *lc)
{
    int N = m->N;
    int a = m->ta[t], b = m->tb[t], c = m->tc[t];
    long ax = m->vx[a], ay = m->vy[a], bx = m->vx[b], by = m->vy[b], cx = m->vx[c], cy = m->vy[c];
    long twoA = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
    long x0 = ax < bx ? ax : bx; if (cx < x0) x0 = cx;
    long x1 = ax > bx ? ax : bx; if (cx > x1) x1 = cx;
    long y0 = ay < by ? ay : by; if (cy < y0) y0 = cy;
    long y1 = ay > by ? ay : by; if (cy > y1) y1 = cy;
    if (x1 > m->W - 1) x1 = m->W - 1;
    if (y1 > m->H - 1) y1 = m->H - 1;
    long n = 0;
    for (long y = y0; y <= y1; ++y) {
        int sy = (y < N - 1) ? 1 : -1;
        for (long x = x0; x <= x1; ++x) {
            int sx = (x < N - 1) ? 1 : -1;
            long w_ab = (bx - ax) * (y - ay) - (by - ay) * (x - ax);
            long w_bc = (cx - bx) * (y - by) - (cy - by) * (x - bx);
            long w_ca = (ax - cx) * (y - cy) - (ay - cy) * (x - cx);
            if (!inner_side(w_ab, -(by - ay), bx - ax, sx, sy)) continue;
            if (!inner_side(w_bc, -(cy - by), cx - bx, sx, sy)) continue;
            if (!inner_side(w_ca, -(ay - cy), ax - cx, sx, sy)) continue;
            px[n] = (int)x; py[n] = (int)y;
            la[n] = (double)w_bc / (double)twoA;
            lb[n] = (double)w_ca / (double)twoA;
            lc[n] = (double)w_ab / (double)twoA;
            n++;
        }
    }
    return n;
}

typedef struct { int *px, *py; double *la, *lb, *lc; long cap; } pix_buf;

static int pix_buf_fit(pix_buf *pb, const om_mesh *m, int t)
{
    int a = m->ta[t], b = m->tb[t], c = m->tc[t];
    int x0 = m->vx[a], x1 = m->vx[a], y0 = m->vy[a], y1 = m->vy[a];
    int xs[2] = {m->vx[b], m->vx[c]}, ys[2] = {m->vy[b], m->vy[c]};
    for (int i = 0; i < 2; ++i) {
        if (xs[i] < x0) x0 = xs[i];
        if (xs[i] > x1) x1 = xs[i];
        if (ys[i] < y0) y0 = ys[i];
        if (ys[i] > y1) y1 = ys[i];
    }
    long need = (long)(x1 - x0 + 1) * (long)(y1 - y0 + 1);
    if (need <= pb->cap) return OM_OK;
    free(pb->px); free(pb->py); free(pb->la); free(pb->lb); free(pb->lc);
    pb->px = malloc(sizeof(int) * need); pb->py = malloc(sizeof(int) * need);
    pb->la = malloc(sizeof(double) * need); pb->lb = malloc(sizeof(double) * need);
    pb->lc = malloc(sizeof(double) * need);
    if (!pb->px || !pb->py || !pb->la || !pb->lb || !pb->lc) {
        free(pb->px); free(pb->py); free(pb->la); free(pb->lb); free(pb->lc);
        memset(pb, 0, sizeof(*pb));
        return OM_E_OOM;
    }
    pb->cap = need;
    return OM_OK;
}

static void pix_buf_free(pix_buf *pb) { free(pb->px); free(pb->py); free(pb->la); free(pb->lb); free(pb->lc); }

/* u = P v: the piecewise-linear interpolant of the vertex values v at every
 * image pixel (Sec. 2.2, last step), and optionally the per-triangle squared
 * errors against f (Sec. 3) and the owner of each pixel.  Images are W x H,
 * row-major.  When owner is given, every image pixel must be owned exactly
 * once or OM_E_INVALID is returned. */
int om_raster(const om_mesh *m, const double *v, const float *f, double *u_img, double *keys, int *owner)
{
    long P = (long)m->W * m->H;
    int rc = OM_OK;
    if (owner) for (long p = 0; p < P; ++p) owner[p] = -1;
    /* The ownership check writes shared state, so it runs on one thread. */
    #pragma omp parallel if (!owner && m->T > 64)
    {
        pix_buf pb;
        memset(&pb, 0, sizeof(pb));
        #pragma omp for schedule(dynamic, 16)
        for (int t = 0; t < m->T; ++t) {
            if (pix_buf_fit(&pb, m, t)) {
                #pragma omp atomic write
                rc = OM_E_OOM;
                continue;
            }
            long n = owned_pixels(m, t, pb.px, pb.py, pb.la, pb.lb, pb.lc);
            double va = v[m->ta[t]], vb = v[m->tb[t]], vc = v[m->tc[t]];
            double err = 0.0;
            for (long q = 0; q < n; ++q) {
                long p = (long)pb.py[q] * m->W + pb.px[q];
                double u = pb.la[q] * va + pb.lb[q] * vb + pb.lc[q] * vc;
                if (u_img) u_img[p] = u;
                if (f) { double d = u - (double)f[p]; err += d * d; }
                if (owner) {
                    if (owner[p] != -1) rc = OM_E_INVALID;
                    owner[p] = t;
                }
            }
            if (keys) keys[t] = err;
        }
        pix_buf_free(&pb);
    }
    if (owner && !rc)
        for (long p = 0; p < P; ++p) if (owner[p] < 0) { rc = OM_E_INVALID; break; }
    return rc;
}

/* Threads the library computes with: 1 unless compiled with OpenMP. */
int om_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* s = P^T r: each pixel's value spread onto the three vertices of its owner
 * with its barycentric weights.  s has V entries. */
static int scatter_PT(const om_mesh *m, const double *r_img, double *s)
{
    pix_buf pb;
    memset(&pb, 0, sizeof(pb));
    for (int i = 0; i < m->V; ++i) s[i] = 0.0;
    for (int t = 0; t < m->T; ++t) {
        if (pix_buf_fit(&pb, m, t)) { pix_buf_free(&pb); return OM_E_OOM; }
        long n = owned_pixels(m, t, pb.px, pb.py, pb.la, pb.lb, pb.lc);
        for (long q = 0; q < n; ++q) {
            double r = r_img[(long)pb.py[q] * m->W + pb.px[q]];
            s[m->ta[t]] += pb.la[q] * r;
            s[m->tb[t]] += pb.lb[q] * r;
            s[m->tc[t]] += pb.lc[q] * r;
        }
    }
    pix_buf_free(&pb);
    return OM_OK;
}

int om_scatter(const om_mesh *m, const double *r_img, double *s) { return scatter_PT(m, r_img, s); }

/* ------------------------------------------------------------------ */
/* R8: top-k selection                                                 */
/* ------------------------------------------------------------------ */

typedef struct { double key; int id; } key_id;

static int cmp_key_desc_id_asc(const void *p, const void *q)
{
    const key_id *a = p, *b = q;
    if (a->key > b->key) return -1;
    if (a->key < b->key) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

int om_count_eligible(const om_mesh *m)
{
    int n = 0;
    for (int t = 0; t < m->T; ++t) n += om_eligible(m, t);
    return n;
}

/* k = max(1, ceil(frac*T)), capped by the eligible count and by vcap */
int om_topk_count(int T, double frac, int n_eligible, long vcap)
{
    long k = (long)ceil(frac * (double)T);
    if (k < 1) k = 1;
    if (k > n_eligible) k = n_eligible;
    if (k > vcap) k = vcap;
    if (k < 0) k = 0;
    return (int)k;
}

/* Writes the k selected ids (in selection order) to sel; *margin receives the
 * relative gap (key_k - key_{k+1}) / key_k, or +inf when nothing is left out. */
int om_select_topk(const om_mesh *m, const double *keys, int k, int *sel, double *margin)
{
    key_id *list = malloc(sizeof(key_id) * (m->T ? m->T : 1));
    if (!list) return -1;
    int ne = 0;
    for (int t = 0; t < m->T; ++t)
        if (om_eligible(m, t)) { list[ne].key = keys[t]; list[ne].id = t; ne++; }
    qsort(list, ne, sizeof(key_id), cmp_key_desc_id_asc);
    if (k > ne) k = ne;
    for (int i = 0; i < k; ++i) sel[i] = list[i].id;
    if (margin) {
        if (k < ne && k > 0) {
            double hi = list[k - 1].key, lo = list[k].key;
            *margin = hi > 0 ? (hi - lo) / hi : 0.0;
        } else {
            *margin = INFINITY;
        }
    }
    free(list);
    return k;
}

/* ------------------------------------------------------------------ */
/* spatial optimisation (Sec. 3, as adapted: top-k bisection)          */
/* ------------------------------------------------------------------ */

#define LOG_COLS 8

/* f at pixel (x, y) of the domain: the nearest image pixel (R9) */
static double f_at(const om_mesh *m, const float *f, int x, int y)
{
    if (x > m->W - 1) x = m->W - 1;
    if (y > m->H - 1) y = m->H - 1;
    return (double)f[(long)y * m->W + x];
}

/* Refines m until it has at least ceil(density*W*H) vertices (or max_rounds
 * rounds when > 0).  Each round: g = f at the mask vertices, Laplace solve
 * (warm-started), per-triangle squared errors, top-k, one refinement.
 * log rows: V, T, k, margin, CG iterations, relres, new vertices, new mask.
 *
 * R10 colour (Sec. 5: the extension to colour images is straightforward):
 * with C channels (f holds C planes of W x H, one after the other) the
 * channels share the mesh, the mask set and A_UU; each channel has its own
 * mask values and its own Laplace solve, and a triangle's error is the sum
 * over the channels of its squared errors (channel 0 first).  C = 1 is the
 * grey case.  CG iterations and relres in the log are channel 0's. */
int om_spatial_channels(om_mesh *m, const float *f, int C, double density, double frac, int max_rounds,
                        double tol, int maxit, double *log, int log_cap, int *rounds_out)
{
    if (C < 1) return OM_E_INVALID;
    long P = (long)m->W * m->H;
    long Vstar = (long)ceil(density * (double)P);
    int rc = OM_OK, round = 0;
    double *uv = NULL, *keys = NULL, *keys_c = NULL, *u_img = malloc(sizeof(double) * P);
    int *sel = NULL, *par = NULL;
    if (!u_img) return OM_E_OOM;
    int capV = 0;
    /* channel c's vertex values are uv[c * capV ...]; grow keeps them */
    #define GROW_UV()                                                                  \
        if (capV < m->V) {                                                             \
            int nc = m->capV;                                                          \
            double *nu = malloc(sizeof(double) * (size_t)nc * C);                      \
            if (!nu) { rc = OM_E_OOM; break; }                                         \
            for (int c_ = 0; c_ < C; ++c_)                                             \
                for (int i_ = 0; i_ < capV; ++i_) nu[(size_t)c_ * nc + i_] = uv[(size_t)c_ * capV + i_]; \
            free(uv); uv = nu; capV = nc;                                              \
        }
    while (m->V < Vstar && (max_rounds <= 0 || round < max_rounds)) {
        GROW_UV();
        int iters = 0; double relres = 0.0;
        double *nk = realloc(keys, sizeof(double) * m->T);
        double *nkc = realloc(keys_c, sizeof(double) * m->T);
        int *ns = realloc(sel, sizeof(int) * m->T);
        if (nk) keys = nk;
        if (nkc) keys_c = nkc;
        if (ns) sel = ns;
        if (!nk || !nkc || !ns) { rc = OM_E_OOM; break; }
        for (int c = 0; c < C && !rc; ++c) {
            double *v = uv + (size_t)c * capV;
            const float *fc = f + (size_t)c * P;
            if (round == 0) for (int i = 0; i < m->V; ++i) v[i] = 0.0;
            for (int i = 0; i < m->V; ++i)
                if (m->mask[i]) v[i] = f_at(m, fc, m->vx[i], m->vy[i]);
            int it_c = 0; double rr_c = 0.0;
            rc = om_solve(m, v, tol, maxit, &it_c, &rr_c);
            if (rc) break;
            if (c == 0) { iters = it_c; relres = rr_c; }
            rc = om_raster(m, v, fc, u_img, c == 0 ? keys : keys_c, NULL);
            if (rc) break;
            if (c > 0) for (int t = 0; t < m->T; ++t) keys[t] += keys_c[t];
        }
        if (rc) break;
        int ne = om_count_eligible(m);
        int k = om_topk_count(m->T, frac, ne, Vstar - m->V);
        if (k <= 0) break;
        double margin = 0.0;
        k = om_select_topk(m, keys, k, sel, &margin);
        int V0 = m->V, T0 = m->T, info[4];
        /* at most one new vertex per edge: V + T - 1 edges */
        int *np = realloc(par, sizeof(int) * 2 * (size_t)(m->V + m->T));
        if (!np) { rc = OM_E_OOM; break; }
        par = np;
        rc = refine_par(m, sel, k, info, par);
        if (rc) break;
        /* warm start: the previous interpolant at the new vertices, i.e. the
         * mean of the ends of the edge each one bisects */
        GROW_UV();
        for (int c = 0; c < C; ++c) {
            double *v = uv + (size_t)c * capV;
            for (int i = V0; i < m->V; ++i) v[i] = 0.5 * (v[par[2 * (i - V0)]] + v[par[2 * (i - V0) + 1]]);
        }
        if (log && round < log_cap) {
            double *row = log + (long)round * LOG_COLS;
            row[0] = V0; row[1] = T0; row[2] = k; row[3] = margin;
            row[4] = iters; row[5] = relres; row[6] = info[0]; row[7] = info[3];
        }
        round++;
    }
    #undef GROW_UV
    if (rounds_out) *rounds_out = round;
    free(uv); free(keys); free(keys_c); free(sel); free(u_img); free(par);
    return rc;
}

int om_spatial(om_mesh *m, const float *f, double density, double frac, int max_rounds,
               double tol, int maxit, double *log, int log_cap, int *rounds_out)
{
    return om_spatial_channels(m, f, 1, density, frac, max_rounds, tol, maxit, log, log_cap, rounds_out);
}

/* ------------------------------------------------------------------ */
/* tonal optimisation (Sec. 4): u = B g,  g* = argmin ||B g - f||^2      */
/* ------------------------------------------------------------------ */

typedef struct {
    const om_mesh *m;
    sp_rows A;
    double *v, *b, *s;  /* V-sized work */
    double tol;
    int maxit;
    long inner_iters;
    int nK;
} tonal_ctx;

static int ctx_init(tonal_ctx *c, const om_mesh *m, double tol, int maxit)
{
    memset(c, 0, sizeof(*c));
    c->m = m; c->tol = tol; c->maxit = maxit;
    int rc = assemble(m, &c->A);
    if (rc) return rc;
    c->v = calloc(m->V, sizeof(double));
    c->b = calloc(m->V, sizeof(double));
    c->s = calloc(m->V, sizeof(double));
    if (!c->v || !c->b || !c->s) return OM_E_OOM;
    for (int i = 0; i < m->V; ++i) c->nK += m->mask[i];
    return OM_OK;
}

static void ctx_free(tonal_ctx *c) { sp_free(&c->A); free(c->v); free(c->b); free(c->s); }

/* u = B g = P [g ; -A_UU^{-1} A_UK g] */
static int apply_B(tonal_ctx *c, const double *g, double *u_img)
{
    const om_mesh *m = c->m;
    int k = 0;
    for (int i = 0; i < m->V; ++i) c->v[i] = m->mask[i] ? g[k++] : 0.0;
    rhs_U(m, &c->A, c->v, c->b);
    int it = 0;
    int rc = cg_UU(m, &c->A, c->b, c->v, c->tol, c->maxit, &it, NULL);
    c->inner_iters += it;
    if (rc) return rc;
    return om_raster(m, c->v, NULL, u_img, NULL, NULL);
}

/* out = B^T r = (P^T r)_K - A_KU A_UU^{-1} (P^T r)_U */
static int apply_BT(tonal_ctx *c, const double *r_img, double *out)
{
    const om_mesh *m = c->m;
    int rc = scatter_PT(m, r_img, c->s);
    if (rc) return rc;
    for (int i = 0; i < m->V; ++i) c->v[i] = 0.0;
    int it = 0;
    rc = cg_UU(m, &c->A, c->s, c->v, c->tol, c->maxit, &it, NULL);
    c->inner_iters += it;
    if (rc) return rc;
    int k = 0;
    for (int i = 0; i < m->V; ++i) {
        if (!m->mask[i]) continue;
        double t = c->s[i];
        for (int q = 0; q < c->A.deg[i]; ++q) {
            int j = c->A.nb[i * MAXNB + q];
            if (!m->mask[j]) t -= c->A.val[i * MAXNB + q] * c->v[j];
        }
        out[k++] = t;
    }
    return OM_OK;
}

int om_apply_B(const om_mesh *m, const double *g, double *u_img, double tol, int maxit)
{
    tonal_ctx c;
    int rc = ctx_init(&c, m, tol, maxit);
    if (!rc) rc = apply_B(&c, g, u_img);
    ctx_free(&c);
    return rc;
}

int om_apply_BT(const om_mesh *m, const double *r_img, double *out, double tol, int maxit)
{
    tonal_ctx c;
    int rc = ctx_init(&c, m, tol, maxit);
    if (!rc) rc = apply_BT(&c, r_img, out);
    ctx_free(&c);
    return rc;
}

static double dotn(const double *x, const double *y, long n)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += x[i] * y[i];
    return s;
}

/* CG on the normal equations B^T B g = B^T f (eq. 5) in its least-squares
 * form (CGLS): the inner solves are the inpainting problems.  g holds the
 * start on entry and the result on exit.  Stops when
 * ||B^T (f - B g)|| <= tol ||B^T f|| or after maxit outer iterations.
 * stats: [0] outer iterations, [1] final relative normal residual,
 *        [2] inner CG iterations, [3] ||B g - f||^2 at the end. */
/* Weighted least squares min_g sum_p w_p ((B g)_p - f_p)^2 by CGLS on the
 * matrix W^(1/2) B (w = NULL: all weights 1, the tonal optimisation of
 * eq. 4).  The residual r = f - B g is kept unweighted and the weights enter
 * where W^(1/2) appears twice: s = B^T W r and |W^(1/2) q|^2.  Stops when
 * ||B^T W (f - B g)|| <= tol ||B^T W f|| or after maxit iterations. */
int om_tonal_weighted(const om_mesh *m, const float *f, const double *w, double *g, double tol, int maxit,
                      double inner_tol, int inner_maxit, double *stats)
{
    long P = (long)m->W * m->H;
    tonal_ctx c;
    int rc = ctx_init(&c, m, inner_tol, inner_maxit);
    int nK = c.nK;
    double *r = malloc(sizeof(double) * P), *q = malloc(sizeof(double) * P);
    double *s = malloc(sizeof(double) * nK), *p = malloc(sizeof(double) * nK);
    double *fd = malloc(sizeof(double) * P), *wr = malloc(sizeof(double) * P);
    if (rc || !r || !q || !s || !p || !fd || !wr) { rc = rc ? rc : OM_E_OOM; goto out; }
    for (long i = 0; i < P; ++i) fd[i] = f[i];
    for (long i = 0; i < P; ++i) wr[i] = w ? w[i] * fd[i] : fd[i];
    rc = apply_BT(&c, wr, s);                /* B^T W f, for the stopping test */
    if (rc) goto out;
    double cnorm = sqrt(dotn(s, s, nK));
    rc = apply_B(&c, g, q);
    if (rc) goto out;
    for (long i = 0; i < P; ++i) r[i] = fd[i] - q[i];
    for (long i = 0; i < P; ++i) wr[i] = w ? w[i] * r[i] : r[i];
    rc = apply_BT(&c, wr, s);
    if (rc) goto out;
    for (int i = 0; i < nK; ++i) p[i] = s[i];
    double gamma = dotn(s, s, nK);
    int it = 0;
    rc = OM_E_NOT_CONVERGED;
    for (;;) {
        if (sqrt(gamma) <= tol * cnorm) { rc = OM_OK; break; }
        if (it >= maxit) break;
        int e = apply_B(&c, p, q);
        if (e) { rc = e; break; }
        double qq = 0.0;
        if (w) { for (long i = 0; i < P; ++i) qq += w[i] * q[i] * q[i]; }
        else qq = dotn(q, q, P);
        if (qq == 0.0) { rc = OM_OK; break; }
        double alpha = gamma / qq;
        for (int i = 0; i < nK; ++i) g[i] += alpha * p[i];
        for (long i = 0; i < P; ++i) r[i] -= alpha * q[i];
        for (long i = 0; i < P; ++i) wr[i] = w ? w[i] * r[i] : r[i];
        e = apply_BT(&c, wr, s);
        if (e) { rc = e; break; }
        double gamma1 = dotn(s, s, nK);
        double beta = gamma1 / gamma;
        gamma = gamma1;
        for (int i = 0; i < nK; ++i) p[i] = s[i] + beta * p[i];
        it++;
    }
    if (stats) {
        stats[0] = it;
        stats[1] = cnorm > 0 ? sqrt(gamma) / cnorm : 0.0;
        stats[2] = (double)c.inner_iters;
        int e = apply_B(&c, g, q);
        double sse = 0.0;
        if (!e) for (long i = 0; i < P; ++i) { double d = q[i] - fd[i]; sse += d * d; }
        stats[3] = e ? NAN : sse;
    }
out:
    free(r); free(q); free(s); free(p); free(fd); free(wr);
    ctx_free(&c);
    return rc;
}

/* CG on the normal equations of eq. 4 in least-squares form (CGLS): the
 * inner solves are the inpainting problems.  g holds the start on entry and
 * the result on exit.  Stops when ||B^T (f - B g)|| <= tol ||B^T f|| or
 * after maxit outer iterations.  stats: [0] outer iterations, [1] final
 * relative normal residual, [2] inner CG iterations, [3] ||B g - f||^2. */
int om_tonal(const om_mesh *m, const float *f, double *g, double tol, int maxit,
             double inner_tol, int inner_maxit, double *stats)
{
    return om_tonal_weighted(m, f, NULL, g, tol, maxit, inner_tol, inner_maxit, stats);
}

/* R11, the L1 data term of Sec. 5 (after the cited work, the L1 error
 * instead of the L2 one): min_g sum_p |(B g)_p - f_p| by iteratively
 * reweighted least squares.  Each of the `irls` steps sets the weights
 * w_p = 1 / max(|(B g)_p - f_p|, eps) from the current g and solves the
 * weighted least-squares problem from the current g (om_tonal_weighted to
 * tol).  stats: [0] CG iterations over all steps, [1] the last step's
 * relative residual, [2] inner CG iterations, [3] sum_p |(B g)_p - f_p| at
 * the end, [4] the smoothed objective sum_p min(r^2 / (2 eps), |r| - eps/2)
 * at the end (Huber, which the iteration does not increase). */
int om_tonal_l1(const om_mesh *m, const float *f, double *g, int irls, double eps, double tol, int maxit,
                double inner_tol, int inner_maxit, double *stats)
{
    long P = (long)m->W * m->H;
    double *u = malloc(sizeof(double) * P), *w = malloc(sizeof(double) * P);
    int rc = (u && w && eps > 0.0 && irls >= 0) ? OM_OK : (eps > 0.0 && irls >= 0 ? OM_E_OOM : OM_E_INVALID);
    double its = 0.0, inner = 0.0, rel = 0.0;
    for (int k = 0; k < irls && !rc; ++k) {
        rc = om_apply_B(m, g, u, inner_tol, inner_maxit);
        if (rc) break;
        for (long i = 0; i < P; ++i) {
            double a = fabs(u[i] - (double)f[i]);
            w[i] = 1.0 / (a > eps ? a : eps);
        }
        double st[4];
        rc = om_tonal_weighted(m, f, w, g, tol, maxit, inner_tol, inner_maxit, st);
        its += st[0]; inner += st[2]; rel = st[1];
    }
    if (!rc && stats) {
        rc = om_apply_B(m, g, u, inner_tol, inner_maxit);
        double l1 = 0.0, hub = 0.0;
        for (long i = 0; i < P && !rc; ++i) {
            double a = fabs(u[i] - (double)f[i]);
            l1 += a;
            hub += a <= eps ? a * a / (2.0 * eps) : a - eps / 2.0;
        }
        stats[0] = its; stats[1] = rel; stats[2] = inner; stats[3] = l1; stats[4] = hub;
    }
    free(u); free(w);
    return rc;
}
