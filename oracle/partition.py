"""Geometric nested-dissection partitions (Sec. 5.1, Defs. 2.1-2.4).

Reading of the partition rule (the paper's cutting-plane coordinates are
garbled; this follows the "(d-1)^3 grid vertices per 3-cell" statement):
along an axis with N unknowns and cut spacing d = b * 2^(t-1) at level t, the
separator coordinates are S_t = { i <= N-2 : (i+1) mod d == 0 }, minus its
largest element when fewer than d/2 unknowns would follow it.  Each separator
is one grid layer; the runs of unknowns between them are the intervals.

A point's level-t cell is, per axis, either its separator coordinate or the
index of its interval.  Cells are encoded per axis as 2k for interval k and
2k+1 for separator k, so codes sort in spatial order.  The cell dimension is
the number of axes on which the cell spans an interval: cells of full
dimension are the interiors (3-cells in 3D, 2-cells in 2D), the others are
separators (2-, 1-, 0-cells: faces, edges, points).  Since S_{t+1} is a subset
of S_t, every level-t cell lies in one level-(t+1) cell (Def. 2.2).

The top level is the first one with no separator on any axis; it has one node.

General partitions (Sec. 5.2, the Gen-All-All scheme): every level-t cell is a
box of d = b * 2^(t-1) consecutive grid vertices per axis, [k d, (k+1) d - 1]
(the last one clipped to the grid), so the level-t cell holds (b 2^(t-1))^3
vertices; there are no separators and no interiors, every node is of full
dimension, and the 2 x 2 x 2 level-t cells of a level-(t+1) cell are its
children.  The top is the first level with a single cell.  Codes are 2k per
axis (the same encoding as intervals above).

Canonical node order within a level: interiors first, then separators, each
group sorted by the cell code tuple (z, y, x).  The active variables of a
level-1 node are its points' DOFs in natural order; those of a level-(t+1)
node are its children's surviving variables, children taken in their level-t
canonical order (interiors contribute nothing: they were eliminated).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def axis_separators(N: int, d: int) -> list:
    """Separator coordinates along one axis for cut spacing d."""
    s = [i for i in range(N - 1) if (i + 1) % d == 0]
    if s and (N - 1 - s[-1]) < d / 2.0:
        s.pop()
    return s


def axis_codes(N: int, seps: list) -> np.ndarray:
    """Per-coordinate cell code: 2k inside interval k, 2k+1 on separator k."""
    codes = np.empty(N, dtype=np.int64)
    k = 0
    sset = set(seps)
    for i in range(N):
        if i in sset:
            codes[i] = 2 * k + 1
            k += 1
        else:
            codes[i] = 2 * k
    return codes


def code_extent(N: int, seps: list, code: int):
    """Coordinate range [lo, hi] covered by a cell code along one axis."""
    k = code // 2
    if code % 2 == 1:
        return seps[k], seps[k]
    lo = seps[k - 1] + 1 if k > 0 else 0
    hi = seps[k] - 1 if k < len(seps) else N - 1
    return lo, hi


# Stencil point offsets (dx, dy, dz) of each operator.
def stencil_offsets(stencil: str):
    if stencil == "5pt_2d":
        return [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0)]
    if stencil in ("7pt_fv_3d", "7pt_3d"):
        return [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    if stencil == "q1_elastic_3d":
        return [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                if (dx, dy, dz) != (0, 0, 0)]
    raise KeyError(stencil)


@dataclass
class Level:
    t: int                      # 1-based level number
    d: int                      # cut spacing
    seps: list                  # separator coordinates per axis (x, y, z)
    codes: list                 # cell code tuple (cz, cy, cx) per node
    interior: np.ndarray        # bool per node
    cell_dim: np.ndarray        # int per node
    box: np.ndarray             # (nnodes, 2, 3): [lo, hi] x (x, y, z)
    children: list = field(default_factory=list)   # per node: previous-level node ids
    points: list = field(default_factory=list)     # level 1 only: natural point ids
    pattern: list = field(default_factory=list)    # pre-elimination pairs (i < j)
    post_pattern: list = field(default_factory=list)  # separator pairs after elimination
    top: bool = False

    @property
    def nnodes(self):
        return len(self.codes)

    def interiors(self):
        return [i for i in range(self.nnodes) if self.interior[i]]

    def separators(self):
        return [i for i in range(self.nnodes) if not self.interior[i]]


@dataclass
class Hierarchy:
    n: tuple        # (nx, ny, nz) point grid
    dim: int
    leaf: int
    dof: int
    stencil: str
    levels: list
    general: bool = False   # general partitions (no interiors)


def _sort_nodes(codes_list, interior_list):
    keyed = sorted(range(len(codes_list)),
                   key=lambda i: (0 if interior_list[i] else 1, codes_list[i]))
    return keyed


def build_hierarchy(n, dim: int, leaf: int, stencil: str, dof: int = 1, general: bool = False) -> Hierarchy:
    """Build P_1 < P_2 < ... < P_l with node orders, children and block patterns
    (nested dissection, or general partitions when `general`)."""
    nx, ny, nz = (list(n) + [1, 1, 1])[:3]
    if dim == 2:
        nz = 1
    N = (nx, ny, nz)
    npts = nx * ny * nz
    pid = np.arange(npts)
    px, py, pz = pid % nx, (pid // nx) % ny, pid // (nx * ny)
    levels = []
    t = 1
    prev = None
    prev_point_node = None
    while True:
        d = leaf * 2 ** (t - 1)
        if general:
            seps = [[], [], []]
            top = all(-(-N[a] // d) == 1 for a in range(3))
        else:
            seps = [axis_separators(N[a], d) if N[a] > 1 else [] for a in range(3)]
            top = all(len(s) == 0 for s in seps)
        if top:
            lev = Level(t=t, d=d, seps=seps, codes=[(0, 0, 0)], interior=np.array([False]),
                        cell_dim=np.array([dim]),
                        box=np.array([[[0, 0, 0], [nx - 1, ny - 1, nz - 1]]]), top=True)
            if prev is None:
                lev.points = [pid.copy()]
            else:
                lev.children = [[i for i in range(prev.nnodes) if not prev.interior[i]]]
            levels.append(lev)
            break
        if general:
            cx, cy, cz = (2 * (np.arange(N[a]) // d) for a in range(3))
        else:
            cx = axis_codes(nx, seps[0])
            cy = axis_codes(ny, seps[1])
            cz = axis_codes(nz, seps[2])
        # every cell is the product of per-axis codes
        all_codes = []
        ux, uy, uz = sorted(set(cx.tolist())), sorted(set(cy.tolist())), sorted(set(cz.tolist()))
        for czv in uz:
            for cyv in uy:
                for cxv in ux:
                    all_codes.append((czv, cyv, cxv))
        interior_flags = [(not general) and all(c % 2 == 0 for c in code) for code in all_codes]
        order = _sort_nodes(all_codes, interior_flags)
        codes = [all_codes[i] for i in order]
        interior = np.array([interior_flags[i] for i in order])
        cell_dim = np.array([sum(1 for a, c in enumerate(code[::-1]) if a < dim and c % 2 == 0)
                             for code in codes])   # = dim for every general cell
        index = {c: i for i, c in enumerate(codes)}
        box = np.zeros((len(codes), 2, 3), dtype=np.int64)
        for i, (czv, cyv, cxv) in enumerate(codes):
            for a, cv in enumerate((cxv, cyv, czv)):
                if general:
                    lo, hi = (cv // 2) * d, min((cv // 2 + 1) * d, N[a]) - 1
                else:
                    lo, hi = code_extent(N[a], seps[a], cv)
                box[i, 0, a], box[i, 1, a] = lo, hi
        lev = Level(t=t, d=d, seps=seps, codes=codes, interior=interior, cell_dim=cell_dim, box=box)
        # node of each point at this level
        key = (cz[pz] * (2 * ny + 2) + cy[py]) * (2 * nx + 2) + cx[px]
        code_key = {((c[0] * (2 * ny + 2) + c[1]) * (2 * nx + 2) + c[2]): i for c, i in index.items()}
        point_node = np.array([code_key[k] for k in key.tolist()], dtype=np.int64)
        if prev is None:
            lev.points = [np.nonzero(point_node == i)[0] for i in range(lev.nnodes)]
        else:
            # children: previous-level separators, mapped through a representative point
            kids = [[] for _ in range(lev.nnodes)]
            for c in range(prev.nnodes):
                if prev.interior[c]:
                    continue
                lo = prev.box[c, 0]
                p = lo[0] + nx * (lo[1] + ny * lo[2])
                kids[point_node[p]].append(c)
            lev.children = kids
        levels.append(lev)
        prev = lev
        prev_point_node = point_node
        t += 1
    H = Hierarchy(n=N, dim=dim, leaf=leaf, dof=dof, stencil=stencil, levels=levels, general=general)
    _patterns(H, px, py, pz)
    return H


def _patterns(H: Hierarchy, px, py, pz):
    """Block sparsity: stencil couplings at level 1, elimination fill, coarsening."""
    nx, ny, nz = H.n
    lev1 = H.levels[0]
    if lev1.top:
        return
    node_of = np.empty(nx * ny * nz, dtype=np.int64)
    for i, pts in enumerate(lev1.points):
        node_of[pts] = i
    pairs = set()
    for dx, dy, dz in stencil_offsets(H.stencil):
        qx, qy, qz = px + dx, py + dy, pz + dz
        ok = (qx >= 0) & (qx < nx) & (qy >= 0) & (qy < ny) & (qz >= 0) & (qz < nz)
        a = node_of[np.nonzero(ok)[0]]
        b = node_of[(qx + nx * (qy + ny * qz))[ok]]
        m = a != b
        for u, v in set(zip(np.minimum(a[m], b[m]).tolist(), np.maximum(a[m], b[m]).tolist())):
            pairs.add((u, v))
    for li, lev in enumerate(H.levels):
        if lev.top:
            break
        if li > 0:
            prev = H.levels[li - 1]
            parent = {}
            for D, kids in enumerate(lev.children):
                for c in kids:
                    parent[c] = D
            pairs = set()
            for (u, v) in prev.post_pattern:
                a, b = parent[u], parent[v]
                if a != b:
                    pairs.add((min(a, b), max(a, b)))
        lev.pattern = sorted(pairs)
        nbrs = {i: set() for i in range(lev.nnodes)}
        for u, v in lev.pattern:
            nbrs[u].add(v)
            nbrs[v].add(u)
        post = set((u, v) for (u, v) in lev.pattern
                   if not lev.interior[u] and not lev.interior[v])
        for I in lev.interiors():
            ss = sorted(nbrs[I])
            for a in range(len(ss)):
                for b in range(a + 1, len(ss)):
                    post.add((ss[a], ss[b]))
        lev.post_pattern = sorted(post)


def neighbours(pattern, i):
    """Sorted neighbours of node i in a list of (u < v) pairs."""
    out = [v for (u, v) in pattern if u == i] + [u for (u, v) in pattern if v == i]
    return sorted(out)
