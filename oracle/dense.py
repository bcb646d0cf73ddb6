"""Brute-force dense restatement of Algorithm 4.1 for tiny grids (pins `sgf`).

Everything lives in explicit n x n matrices with global index sets ("slots"):
the current matrix M and the accumulated factor F = G1 B1 G2 B2 ... so that
the approximation after k levels is A_k = F M F^T (Sec. 2.1, Sec. 6).

* Elimination of interior I with slots s (Eq. (elimination)): G = I_n with
  G[s, s] = L and G[rest, s] = M[rest, s] L^{-T}; M becomes identity on s and
  the Schur complement on the rest; F <- F G.
* Compression of B (Eq. (M')): with M_BB = L L^T, M^ = L^{-1} M[s, others],
  Phi_X for every node taken straight from its definition Eq. (PhiD),
  Phi_X = (F^T Pi_X)[active slots of X] with Pi_X the cell's basis on all of
  its unknowns (Eq. (def:PiB)) - no update or merge formula is used;
  N = [L^T Phi_B, M^_X Phi_X for every other node X] (zero blocks give zero
  columns), pivoted QR, rank r; if r < m: F <- F diag(L Q, I), M[s, s] = I,
  M[s[:r], others] = Q1^T M^, and the Q2 rows are decoupled (set to zero).
* Merge: a parent's slots are its children's surviving slots.

* Which nodes a scheme compresses (Sec. 5.1, Sec. 5.2) and the Nest-2-2
  rim are decided here from the cells' geometry, independently of `sgf`:
  the dimension of a cell is that of the affine hull of its points (the
  number of axes along which its box is more than one point wide), the
  interiors have full dimension; Nest-All-All compresses every separator of
  dimension >= 1, Nest-2-All and Nest-2-2 those of codimension 1, Gen-All-All
  every node; a lower-dimensional separator X lies on the rim of a
  codimension-1 separator B when some point of X is within one grid step of
  some point of B along every axis (brute force over the point pairs).

This is a second, independent implementation written against the same
equations; it shares no code with `sgf` beyond the partition, the basis
evaluation and the DOF numbering.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .basis import Basis
from .sgf import Options, dof_list, point_coords


def _cell_dofs(H, box):
    nx, ny, nz = H.n
    xs = np.arange(box[0][0], box[1][0] + 1)
    ys = np.arange(box[0][1], box[1][1] + 1)
    zs = np.arange(box[0][2], box[1][2] + 1)
    zz, yy, xx = np.meshgrid(zs, ys, xs, indexing="ij")
    pts = (xx + nx * (yy + ny * zz)).ravel()
    return np.sort(pts)


def _cell_dim(H, box):
    """Dimension of the affine hull of a cell's points."""
    lo, hi = np.asarray(box[0]), np.asarray(box[1])
    return int(np.sum(hi[:H.dim] > lo[:H.dim]))


def _compressed_by_scheme(H, lev, X, opts: Options) -> bool:
    """Sec. 5.1 / 5.2: is node X of this level selected for compression?"""
    if opts.scheme == "none" or lev.t < opts.compress_from_level:
        return False
    if opts.scheme == "gen_all_all":
        return True
    # nested dissection: intervals are at least two points wide for b >= 3,
    # so a cell's affine dimension is its number of interval axes
    assert H.leaf >= 3, "geometric cell dimension needs leaf >= 3"
    cd = _cell_dim(H, lev.box[X])
    if cd == H.dim:
        return False                 # an interior: eliminated, not compressed
    if opts.scheme == "nest_all_all":
        return cd >= 1               # 0-cells are not compressed (Sec. 5.1)
    if opts.scheme in ("nest_2_all", "nest_2_2"):
        return cd == H.dim - 1
    raise ValueError(opts.scheme)


def _on_rim(H, lev, B, X) -> bool:
    """Nest-2-2: X is a lower-dimensional separator touching separator B."""
    if _cell_dim(H, lev.box[X]) >= H.dim - 1:     # interiors and codimension-1 cells
        return False
    nx, ny, _ = H.n

    def coords(box):
        p = _cell_dofs(H, box)
        return np.stack([p % nx, (p // nx) % ny, p // (nx * ny)], 1)
    pb, px = coords(lev.box[B]), coords(lev.box[X])
    cheb = np.abs(pb[:, None, :] - px[None, :, :]).max(axis=2)
    return bool(cheb.min() <= 1)


def dense_sgf(A, H, opts: Options = Options()):
    """Return (A_l, [A_1, ..., A_l], ranks) built with explicit dense factors."""
    A = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    n = A.shape[0]
    basis = Basis(H.dim, opts.degree, opts.basis, H.dof)
    xyz = point_coords(H)
    M = A.copy()
    F = np.eye(n)
    lev1 = H.levels[0]
    slots = {i: list(dof_list(p, H.dof)) for i, p in enumerate(lev1.points)}
    approx = []
    ranks = {}

    def Pi_of(lev, X):
        pts = _cell_dofs(H, lev.box[X])
        P = np.zeros((n, basis.pi))
        P[dof_list(pts, H.dof)] = basis.evaluate(xyz[pts], lev.box[X])
        return P

    for li, lev in enumerate(H.levels):
        if lev.top:
            approx.append(F @ M @ F.T)
            break
        for I in lev.interiors():
            s = slots[I]
            if not s:
                continue
            rest = [q for X in slots if X != I for q in slots[X]]
            L = sla.cholesky(M[np.ix_(s, s)], lower=True)
            W = sla.solve_triangular(L, M[np.ix_(s, rest)], lower=True)
            G_cols = np.zeros((n, len(s)))
            G_cols[s] = L
            G_cols[rest] = W.T
            F[:, s] = F @ G_cols
            M[np.ix_(rest, rest)] -= W.T @ W
            M[np.ix_(s, s)] = np.eye(len(s))
            M[np.ix_(s, rest)] = 0.0
            M[np.ix_(rest, s)] = 0.0
            del slots[I]
        for B in [X for X in range(lev.nnodes) if not lev.interior[X] and _compressed_by_scheme(H, lev, X, opts)]:
            s = slots[B]
            others_nodes = [X for X in slots if X != B]
            others = [q for X in others_nodes for q in slots[X]]
            L = sla.cholesky(M[np.ix_(s, s)], lower=True)
            Mh = sla.solve_triangular(L, M[np.ix_(s, others)], lower=True)
            FT = F.T
            cols = [L.T @ (FT @ Pi_of(lev, B))[s]]
            o = 0
            adj = []
            for X in others_nodes:
                k = len(slots[X])
                cols.append(Mh[:, o:o + k] @ (FT @ Pi_of(lev, X))[slots[X]])
                if opts.scheme == "nest_2_2" and _on_rim(H, lev, B, X):
                    adj.append(Mh[:, o:o + k])   # kept exactly: whole block in span(Q1)
                o += k
            Nmat = np.hstack(cols + adj)
            Q, R, _ = sla.qr(Nmat, pivoting=True)
            d = np.abs(np.diag(R))
            r = int(np.sum(d > opts.tau * d[0]))
            m = len(s)
            ranks[(lev.t, B)] = (m, r, r < m)
            if r < m:
                F[:, s] = F[:, s] @ (L @ Q)
                Mp = Q.T @ Mh
                M[np.ix_(s, s)] = np.eye(m)
                M[np.ix_(s[:r], others)] = Mp[:r]
                M[np.ix_(others, s[:r])] = Mp[:r].T
                M[np.ix_(s[r:], others)] = 0.0
                M[np.ix_(others, s[r:])] = 0.0
                slots[B] = s[:r]
        approx.append(F @ M @ F.T)
        nxt = H.levels[li + 1]
        slots = {D: [q for C in kids for q in slots[C]] for D, kids in enumerate(nxt.children)}
    return approx[-1], approx, ranks
