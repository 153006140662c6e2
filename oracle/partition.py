"""Oracle for the chunked-evaluation planner (test infrastructure only).

Plain Python/NumPy restatements of Sect. 3.2 (Algorithm 1 and Algorithm 2), used to
check the library's host planner index for index. Shares no code with it.

Readings taken where the paper is silent (each is also listed in the design notes):

* Algorithm 1 with anisotropy alpha: in log variables u_k = log(h_k / B_k),
  v_k = log(eta_k / P_k) the objective is maximise sum(u) + sum(v) subject to
  u, v <= 0, every pairwise difference within log(alpha), and the memory budget.
  The isotropic point u_k = v_k = log t is always optimal and is the unique
  optimum at alpha = 1, so the box dimensions are h = t B, eta = t P.
* The memory budget is enforced on the padded grids that a full-size sub-problem
  actually allocates (spread grid n1 and FFT grid n2 per dimension, both complex),
  not on the unpadded volume product: t is the largest value in (0, 1] whose
  grids fit B bytes, found by bisection.
* Algorithm 2 fusion: occupied lattice cells are visited in lexicographic order of
  their integer index; an unassigned cell seeds a new chunk and then absorbs, in
  lexicographic order of the offset, each unassigned occupied cell of the 2x2x2
  window it opens at its minimum corner, as long as the bounding box of all the
  chunk's points stays within h in every dimension. (A box of size h overlaps at
  most two lattice cells per dimension, so no chunk can hold more than that window.)
  Chunks are numbered in seed order.
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------- grid sizing

def smooth_even(n: int) -> int:
    """Smallest even integer >= n whose prime factors are all in {2, 3, 5, 7}."""
    m = max(2, int(n))
    if m % 2:
        m += 1
    while True:
        r = m
        for f in (2, 3, 5, 7):
            while r % f == 0:
                r //= f
        if r == 1:
            return m
        m += 2


def grid_sizes(extent_pix: float, extent_vis: float, sigma: float, w: int):
    """(n1, n2) for one dimension of a sub-problem with full widths P (pixels) and B
    (wavelengths): n1 = even >= sigma*P*B + w + 2, n2 = smooth even >= max(sigma*n1, 2w)."""
    need = sigma * extent_pix * extent_vis + w + 2.0
    n1 = 2 * int(math.ceil(need / 2.0))
    n2 = smooth_even(max(int(math.ceil(sigma * n1)), 2 * w))
    return n1, n2


def grid_bytes(P, B, sigma, w, elem_bytes):
    n1p, n2p = 1, 1
    for d in range(3):
        n1, n2 = grid_sizes(P[d], B[d], sigma, w)
        n1p *= n1
        n2p *= n2
    return elem_bytes * (n1p + n2p)


# ---------------------------------------------------------------- Algorithm 1

def box_dims(P, B, budget_bytes: float, sigma: float, w: int, elem_bytes: int, iters: int = 64):
    """Maximum Heisenberg dimensions (eta, h, t) for a memory budget (Algorithm 1).

    P, B: full extents of the pixel and baseline point sets (per dimension).
    """
    P = [float(x) for x in P]
    B = [float(x) for x in B]
    if grid_bytes(P, B, sigma, w, elem_bytes) <= budget_bytes:
        t = 1.0
    else:
        lo, hi = 0.0, 1.0
        for _ in range(iters):
            mid = 0.5 * (lo + hi)
            Pm = [mid * x for x in P]
            Bm = [mid * x for x in B]
            if grid_bytes(Pm, Bm, sigma, w, elem_bytes) <= budget_bytes:
                lo = mid
            else:
                hi = mid
        t = lo
    return [t * x for x in P], [t * x for x in B], t


def box_dims_lp(P, B, log_budget: float, alpha: float = 1.0):
    """Algorithm 1 as the paper's LP in log variables (scipy.optimize.linprog), for the
    unpadded constraint sum(log eta_k h_k) <= log_budget. Returns (eta, h, objective)."""
    from scipy.optimize import linprog
    la = math.log(alpha)
    # variables x = [u0,u1,u2,v0,v1,v2]; maximise sum -> minimise -sum
    c = -np.ones(6)
    A, b = [], []
    const = sum(math.log(P[k] * B[k]) for k in range(3))
    A.append(np.ones(6))
    b.append(log_budget - const)
    for i in range(6):
        for j in range(6):
            if i != j:
                row = np.zeros(6)
                row[i], row[j] = 1.0, -1.0
                A.append(row)
                b.append(la)
    res = linprog(c, A_ub=np.array(A), b_ub=np.array(b), bounds=[(None, 0.0)] * 6, method="highs")
    if not res.success:
        raise RuntimeError(res.message)
    u, v = res.x[:3], res.x[3:]
    h = [B[k] * math.exp(u[k]) for k in range(3)]
    eta = [P[k] * math.exp(v[k]) for k in range(3)]
    return eta, h, float(-res.fun)


# ---------------------------------------------------------------- Algorithm 2

def lattice_cells(pts: np.ndarray, h) -> np.ndarray:
    """Integer lattice index (N, 3) of each point for h-sized cells anchored at the
    point set's minimum corner (steps 1-2). A dimension with h <= 0 has one cell."""
    pts = np.asarray(pts, dtype=np.float64)
    lo = pts.min(axis=0)
    idx = np.zeros(pts.shape, dtype=np.int64)
    for d in range(3):
        if h[d] > 0.0 and math.isfinite(h[d]):
            idx[:, d] = np.floor((pts[:, d] - lo[d]) / h[d]).astype(np.int64)
    return idx


def chunk(pts: np.ndarray, h):
    """Chunk label of every point (Algorithm 2, steps 1-4). Returns (labels, n_chunks)."""
    pts = np.asarray(pts, dtype=np.float64)
    n = len(pts)
    if n == 0:
        return np.zeros(0, dtype=np.int64), 0
    cell_idx = lattice_cells(pts, h)
    # Step 3: only occupied cells exist in this map.
    cells = {}
    for i in range(n):
        key = (int(cell_idx[i, 0]), int(cell_idx[i, 1]), int(cell_idx[i, 2]))
        if key in cells:
            lo, hi = cells[key]
            for d in range(3):
                lo[d] = min(lo[d], pts[i, d])
                hi[d] = max(hi[d], pts[i, d])
        else:
            cells[key] = ([pts[i, 0], pts[i, 1], pts[i, 2]], [pts[i, 0], pts[i, 1], pts[i, 2]])
    owner = {}
    n_chunks = 0
    offsets = [(dx, dy, dz) for dx in (0, 1) for dy in (0, 1) for dz in (0, 1)][1:]
    for key in sorted(cells):
        if key in owner:
            continue
        cid = n_chunks
        n_chunks += 1
        owner[key] = cid
        lo = list(cells[key][0])
        hi = list(cells[key][1])
        for off in offsets:
            nb = (key[0] + off[0], key[1] + off[1], key[2] + off[2])
            if nb not in cells or nb in owner:
                continue
            nlo, nhi = cells[nb]
            jlo = [min(lo[d], nlo[d]) for d in range(3)]
            jhi = [max(hi[d], nhi[d]) for d in range(3)]
            if all(jhi[d] - jlo[d] <= h[d] for d in range(3)):
                lo, hi = jlo, jhi
                owner[nb] = cid
    labels = np.empty(n, dtype=np.int64)
    for i in range(n):
        labels[i] = owner[(int(cell_idx[i, 0]), int(cell_idx[i, 1]), int(cell_idx[i, 2]))]
    return labels, n_chunks


def chunk_boxes(pts: np.ndarray, labels: np.ndarray, n_chunks: int):
    """(lo, hi) bounding boxes per chunk, (n_chunks, 3) each."""
    pts = np.asarray(pts, dtype=np.float64)
    lo = np.full((n_chunks, 3), np.inf)
    hi = np.full((n_chunks, 3), -np.inf)
    np.minimum.at(lo, labels, pts)
    np.maximum.at(hi, labels, pts)
    return lo, hi
