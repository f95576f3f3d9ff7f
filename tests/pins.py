"""Independent reference constructions used to pin the oracle.

Each helper states a fact the paper or plain mathematics fixes, written
without the oracle's code paths: a recursive textbook NVB, the 5-point finite
difference Laplacian with mirrored boundary, the P1 energy from per-triangle
gradients, and a closed-triangle membership test.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def triangle_set(mesh) -> set:
    """Triangles as labelled coordinate triples ((ax,ay),(bx,by),(cx,cy))."""
    out = set()
    for a, b, c in zip(mesh.ta, mesh.tb, mesh.tc):
        out.add(((int(mesh.vx[a]), int(mesh.vy[a])), (int(mesh.vx[b]), int(mesh.vy[b])),
                 (int(mesh.vx[c]), int(mesh.vy[c]))))
    return out


def nvb_recursive(tris: list, selected: list) -> tuple[set, set]:
    """Textbook recursive newest-vertex bisection.  `tris` is a list of
    labelled coordinate triples (a, b, c) with refinement edge (a, b);
    `selected` lists triples to bisect.  Before bisecting a triangle, its
    neighbour across the refinement edge is refined recursively until the
    two share that edge as refinement edge; then both are bisected.
    Returns (triangle set, set of midpoints of selected refinement edges)."""
    tris = list(tris)
    alive = set(tris)

    def mid(p, q):
        return ((p[0] + q[0]) // 2, (p[1] + q[1]) // 2)

    def neighbour(t, e):
        es = set(e)
        for s in alive:
            if s != t and es <= set(s):
                return s
        return None

    def bisect(t):
        a, b, c = t
        m = mid(a, b)
        alive.remove(t)
        alive.add((c, a, m))
        alive.add((b, c, m))

    def refine(t):
        a, b, c = t
        n = neighbour(t, (a, b))
        while n is not None and {n[0], n[1]} != {a, b}:
            refine(n)
            n = neighbour(t, (a, b))
        bisect(t)
        if n is not None:
            bisect(n)

    masks = set()
    for t in selected:
        masks.add(mid(t[0], t[1]))
    for t in selected:
        if t in alive:
            refine(t)
        else:
            # already split by an earlier refinement of this round: its
            # refinement edge was bisected then (its midpoint exists)
            pass
    return alive, masks


def fdm_matrix(N: int) -> sp.csr_matrix:
    """5-point Laplacian 4u_p - sum of the 4 neighbours on the N x N pixel grid,
    with the reflecting boundary realised by mirroring (ghost u_{-1} = u_1)."""
    idx = lambda x, y: y * N + x
    rows, cols, vals = [], [], []
    for y in range(N):
        for x in range(N):
            p = idx(x, y)
            rows.append(p); cols.append(p); vals.append(4.0)
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                qx, qy = x + dx, y + dy
                if qx < 0: qx = 1
                if qx > N - 1: qx = N - 2
                if qy < 0: qy = 1
                if qy > N - 1: qy = N - 2
                rows.append(p); cols.append(idx(qx, qy)); vals.append(-1.0)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N * N, N * N))


def p1_energy(mesh, x: np.ndarray) -> float:
    """sum over triangles of area * |grad u|^2 for the P1 interpolant of x,
    with the gradient from a 2x2 solve per triangle."""
    e = 0.0
    for a, b, c in zip(mesh.ta, mesh.tb, mesh.tc):
        P = np.array([[mesh.vx[b] - mesh.vx[a], mesh.vy[b] - mesh.vy[a]],
                      [mesh.vx[c] - mesh.vx[a], mesh.vy[c] - mesh.vy[a]]], dtype=np.float64)
        d = np.array([x[b] - x[a], x[c] - x[a]])
        grad = np.linalg.solve(P, d)
        area = 0.5 * abs(np.linalg.det(P))
        e += area * float(grad @ grad)
    return e


def in_closed_triangle(mesh, t: np.ndarray, px: np.ndarray, py: np.ndarray) -> np.ndarray:
    """Is pixel (px, py) inside or on triangle t (integer cross products)?"""
    ax, ay = mesh.vx[mesh.ta[t]].astype(np.int64), mesh.vy[mesh.ta[t]].astype(np.int64)
    bx, by = mesh.vx[mesh.tb[t]].astype(np.int64), mesh.vy[mesh.tb[t]].astype(np.int64)
    cx, cy = mesh.vx[mesh.tc[t]].astype(np.int64), mesh.vy[mesh.tc[t]].astype(np.int64)
    px = px.astype(np.int64); py = py.astype(np.int64)
    s = np.sign((bx - ax) * (cy - ay) - (by - ay) * (cx - ax))
    w1 = ((bx - ax) * (py - ay) - (by - ay) * (px - ax)) * s
    w2 = ((cx - bx) * (py - by) - (cy - by) * (px - bx)) * s
    w3 = ((ax - cx) * (py - cy) - (ay - cy) * (px - cx)) * s
    return (w1 >= 0) & (w2 >= 0) & (w3 >= 0)


def edges_of(mesh) -> dict:
    """Undirected edge -> number of triangles containing it."""
    cnt = {}
    for a, b, c in zip(mesh.ta, mesh.tb, mesh.tc):
        for i, j in ((a, b), (b, c), (c, a)):
            k = (min(i, j), max(i, j))
            cnt[k] = cnt.get(k, 0) + 1
    return cnt


def random_refined_mesh(oracle, N: int, rounds: int, seed: int, frac: float = 0.2):
    """A mesh from `rounds` NVB rounds with random selections."""
    rng = np.random.default_rng(seed)
    m = oracle.mesh_init(N)
    for _ in range(rounds):
        el = np.flatnonzero(oracle.eligible(m))
        if len(el) == 0:
            break
        k = max(1, int(frac * len(el)))
        sel = rng.choice(el, size=k, replace=False)
        m, _ = oracle.refine(m, np.sort(sel))
    return m


def fully_refined_mesh(oracle, N: int):
    """Refine every eligible triangle until none is left: every pixel is a vertex."""
    m = oracle.mesh_init(N)
    while True:
        el = np.flatnonzero(oracle.eligible(m))
        if len(el) == 0:
            return m
        m, _ = oracle.refine(m, el)
