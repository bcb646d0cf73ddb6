"""Near-kernel bases Pi (Sec. 3.1, Sec. 7.1.3, Sec. 7.2) in node-local coordinates.

Pi^j has the monomials of degree <= j as columns, in the order of Sec. 3.1:
  3D: 1, x, y, z | x^2, y^2, z^2, xy, yz, zx      (pi = 1, 4, 10)
  2D: 1, x, y    | x^2, y^2, xy                   (pi = 1, 3, 6)
Each node evaluates them at local coordinates u = (x - c) / h per axis, where
c and h are the midpoint and half-width of the node's cell box on that axis
(u = 0 on axes where the cell is flat).  Local and global monomials span the
same space on every cell, so the preserved space of Prop. 6.1 is unchanged;
the local form keeps the columns of the filtered interaction matrix well
scaled on small cells.  When nodes merge (Sec. 4.4) each child's Phi is
re-expressed in the parent's local monomials by the exact pi x pi matrix R of
the affine change of variables u_parent = a u_child + b, then stacked.

Vector problems (3 DOFs per point, interleaved): "poly" takes the block
diagonal diag(Pi^j, Pi^j, Pi^j) of Eq. (def:poly-linel); "rbm" takes the six
rigid-body modes (translations e_x, e_y, e_z; rotations about x, y, z), in
local coordinates with one isotropic scale per node so rotations stay rigid.
"""
from __future__ import annotations

from math import comb

import numpy as np


def exponents(dim: int, degree: int):
    """Monomial exponent tuples (ex, ey, ez) in the column order of Sec. 3.1."""
    if dim == 3:
        e = [(0, 0, 0)]
        if degree >= 1:
            e += [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
        if degree >= 2:
            e += [(2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (0, 1, 1), (1, 0, 1)]
        return e
    e = [(0, 0, 0)]
    if degree >= 1:
        e += [(1, 0, 0), (0, 1, 0)]
    if degree >= 2:
        e += [(2, 0, 0), (0, 2, 0), (1, 1, 0)]
    return e


def frame_poly(box):
    """Per-axis (centre, half-width) of a cell box [[lo], [hi]]."""
    lo = np.asarray(box[0], dtype=np.float64)
    hi = np.asarray(box[1], dtype=np.float64)
    return (lo + hi) / 2.0, (hi - lo) / 2.0


def local_coords_poly(xyz, frame):
    c, h = frame
    u = np.zeros_like(xyz, dtype=np.float64)
    for a in range(3):
        if h[a] > 0:
            u[:, a] = (xyz[:, a] - c[a]) / h[a]
    return u


def eval_monomials(u, exps):
    cols = [np.prod([u[:, a] ** e[a] for a in range(3)], axis=0) for e in exps]
    return np.stack(cols, axis=1)


def reexpansion_poly(child_frame, parent_frame, exps):
    """R with  Pi_parent(p) = Pi_child(p) @ R  for every point p of the child."""
    cc, hc = child_frame
    cp, hp = parent_frame
    a = np.zeros(3)
    b = np.zeros(3)
    for ax in range(3):
        if hp[ax] > 0:
            a[ax] = hc[ax] / hp[ax]
            b[ax] = (cc[ax] - cp[ax]) / hp[ax]
    col = {e: i for i, e in enumerate(exps)}
    R = np.zeros((len(exps), len(exps)))
    for j, e in enumerate(exps):
        # prod_ax (a u + b)^e_ax expanded by the binomial theorem
        terms = {(0, 0, 0): 1.0}
        for ax in range(3):
            new = {}
            for k in range(e[ax] + 1):
                coef = comb(e[ax], k) * a[ax] ** k * b[ax] ** (e[ax] - k)
                for ex, v in terms.items():
                    ex2 = list(ex)
                    ex2[ax] += k
                    ex2 = tuple(ex2)
                    new[ex2] = new.get(ex2, 0.0) + v * coef
            terms = new
        for ex, v in terms.items():
            R[col[ex], j] += v
    return R


def frame_rbm(box):
    c, h = frame_poly(box)
    s = float(np.max(h))
    return c, (s if s > 0 else 1.0)


def eval_rbm(xyz, frame):
    """(3 npts) x 6 rigid-body modes, DOF order 3*p + component."""
    c, s = frame
    u = (xyz - c[None, :]) / s
    npts = xyz.shape[0]
    P = np.zeros((npts, 3, 6))
    for k in range(3):
        P[:, k, k] = 1.0
    x, y, z = u[:, 0], u[:, 1], u[:, 2]
    # rotation about x: (0, -z, y); about y: (z, 0, -x); about z: (-y, x, 0)
    P[:, 1, 3], P[:, 2, 3] = -z, y
    P[:, 0, 4], P[:, 2, 4] = z, -x
    P[:, 0, 5], P[:, 1, 5] = -y, x
    return P.reshape(3 * npts, 6)


def reexpansion_rbm(child_frame, parent_frame):
    cc, sc = child_frame
    cp, sp = parent_frame
    a = sc / sp
    b = (cc - cp) / sp
    R = np.zeros((6, 6))
    R[:3, :3] = np.eye(3)
    for k in range(3):
        R[3 + k, 3 + k] = a
        w = np.zeros(3)
        w[k] = 1.0
        R[:3, 3 + k] = np.cross(w, b)
    return R


class Basis:
    """Node bases for one problem: kind in {"poly", "rbm"}, dof in {1, 3}."""

    def __init__(self, dim: int, degree: int, kind: str = "poly", dof: int = 1):
        self.dim, self.degree, self.kind, self.dof = dim, degree, kind, dof
        self.exps = exponents(dim, degree)
        if kind == "rbm":
            self.pi = 6
        else:
            self.pi = len(self.exps) * dof

    def frame(self, box):
        return frame_rbm(box) if self.kind == "rbm" else frame_poly(box)

    def evaluate(self, xyz, box):
        """Rows of Pi for the given points (DOF-interleaved for dof = 3)."""
        fr = self.frame(box)
        if self.kind == "rbm":
            return eval_rbm(np.asarray(xyz, dtype=np.float64), fr)
        P = eval_monomials(local_coords_poly(np.asarray(xyz, dtype=np.float64), fr), self.exps)
        if self.dof == 1:
            return P
        npts, q = P.shape
        out = np.zeros((npts, self.dof, self.dof * q))
        for c in range(self.dof):
            out[:, c, c * q:(c + 1) * q] = P
        return out.reshape(npts * self.dof, self.dof * q)

    def reexpansion(self, child_box, parent_box):
        if self.kind == "rbm":
            return reexpansion_rbm(self.frame(child_box), self.frame(parent_box))
        R = reexpansion_poly(self.frame(child_box), self.frame(parent_box), self.exps)
        if self.dof == 1:
            return R
        return np.kron(np.eye(self.dof), R)
