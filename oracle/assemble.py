"""Operator assembly for the test problems of Sec. 7.1 (FP64, CSR, natural order).

Unknown numbering: grid point (x, y, z) -> x + nx * (y + ny * z); for the
vector (elasticity) problem each point carries 3 interleaved DOFs
(3 * point + component).  Coefficient arrays are indexed [z, y, x] ([y, x] in
2D).

Scalar stencils (Sec. 7.1.1 Poisson, Sec. 7.1.2 Darcy flow with two-point flux):
  * the transmissibility of the face shared by cells a and b is the harmonic
    mean 2 k_a k_b / (k_a + k_b), computed in exactly that expression order;
  * a Dirichlet face contributes w * k_cell to the diagonal, with w = 1 for the
    finite-difference 5- and 7-point stencils (ghost node one spacing away)
    and w = 2 for the finite-volume 7-point stencil (boundary half a cell
    away);
  * Neumann faces contribute nothing;
  * the diagonal is the sum of the face terms in the order x-, x+, y-, y+,
    z-, z+; off-diagonals are minus the transmissibility.
With unit coefficients and all faces Dirichlet the 5-point stencil is the
classical (4, -1) Laplacian.  The grid spacing is taken as 1: it only scales A.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

FACE_BITS = (1, 2, 4, 8, 16, 32)  # x-, x+, y-, y+, z-, z+


def _dims(n, dim):
    nx, ny, nz = (list(n) + [1, 1, 1])[:3]
    if dim == 2:
        nz = 1
    return int(nx), int(ny), int(nz)


def assemble_scalar(n, dim: int, coeffs: np.ndarray, dirichlet: int, boundary_weight: float):
    """Assemble the scalar diffusion operator on an nx*ny(*nz) cell grid."""
    nx, ny, nz = _dims(n, dim)
    k = np.asarray(coeffs, dtype=np.float64).reshape(nz, ny, nx)
    N = nx * ny * nz
    idx = np.arange(N).reshape(nz, ny, nx)
    diag = np.zeros((nz, ny, nx))
    rows, cols, vals = [], [], []
    axes = [2, 1, 0] if dim == 3 else [2, 1]   # array axis of x, y, z
    for a_i, ax in enumerate(axes):
        # interior faces between index j and j+1 along this axis
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, k.shape[ax] - 1)
        hi[ax] = slice(1, k.shape[ax])
        ka, kb = k[tuple(lo)], k[tuple(hi)]
        t = 2.0 * ka * kb / (ka + kb)
        # minus side of the higher cell / plus side of the lower cell
        t_minus = np.zeros_like(k)
        t_plus = np.zeros_like(k)
        t_plus[tuple(lo)] = t
        t_minus[tuple(hi)] = t
        bm, bp = FACE_BITS[2 * a_i], FACE_BITS[2 * a_i + 1]
        first = [slice(None)] * 3
        last = [slice(None)] * 3
        first[ax] = slice(0, 1)
        last[ax] = slice(k.shape[ax] - 1, k.shape[ax])
        if dirichlet & bm:
            t_minus[tuple(first)] = boundary_weight * k[tuple(first)]
        if dirichlet & bp:
            t_plus[tuple(last)] = boundary_weight * k[tuple(last)]
        diag = diag + t_minus
        diag = diag + t_plus
        ia, ib = idx[tuple(lo)].ravel(), idx[tuple(hi)].ravel()
        rows += [ia, ib]
        cols += [ib, ia]
        vals += [-t.ravel(), -t.ravel()]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    A.sum_duplicates()
    A.sort_indices()
    return A


# ----------------------------------------------------------------------------
# Q1 hexahedral linear elasticity (Sec. 7.1.3 restated on a structured mesh)
# ----------------------------------------------------------------------------

def q1_element_stiffness(E: float, nu: float) -> np.ndarray:
    """24 x 24 stiffness of a unit-cube trilinear element, 2x2x2 Gauss rule.

    Node a of the element sits at corner (ax, ay, az) in {0,1}^3 with local
    number a = ax + 2 ay + 4 az; DOF 3a + c is displacement component c.
    Isotropic material: lam = E nu / ((1+nu)(1-2nu)), mu = E / (2(1+nu)).
    """
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    corners = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=float)
    K = np.zeros((24, 24))
    for gx in g:
        for gy in g:
            for gz in g:
                p = np.array([gx, gy, gz])
                # trilinear shape function derivatives on the unit cube
                dN = np.zeros((8, 3))
                for a in range(8):
                    f = [(p[d] if corners[a, d] else 1 - p[d]) for d in range(3)]
                    s = [(1.0 if corners[a, d] else -1.0) for d in range(3)]
                    dN[a, 0] = s[0] * f[1] * f[2]
                    dN[a, 1] = f[0] * s[1] * f[2]
                    dN[a, 2] = f[0] * f[1] * s[2]
                Bm = np.zeros((6, 24))
                for a in range(8):
                    bx, by, bz = dN[a]
                    c = 3 * a
                    Bm[0, c] = bx
                    Bm[1, c + 1] = by
                    Bm[2, c + 2] = bz
                    Bm[3, c] = by
                    Bm[3, c + 1] = bx
                    Bm[4, c + 1] = bz
                    Bm[4, c + 2] = by
                    Bm[5, c] = bz
                    Bm[5, c + 2] = bx
                K += Bm.T @ D @ Bm * 0.125   # Gauss weight (1/2)^3 on [0,1]^3
    return K


def assemble_elastic(elems, moduli: np.ndarray, nu: float = 0.3, clamp_xm: bool = True):
    """Assemble the Q1 stiffness on an ex*ey*ez element box (nodes (ex+1)...).

    With clamp_xm the nodes on the x = 0 face are removed (zero displacement);
    the free nodes then form an ex * (ey+1) * (ez+1) point grid whose x index
    is the node's x minus one.  Returns (K, point grid shape (nx, ny, nz)).
    """
    ex, ey, ez = (int(e) for e in elems)
    E = np.asarray(moduli, dtype=np.float64).reshape(ez, ey, ex)
    nxn, nyn, nzn = ex + 1, ey + 1, ez + 1
    x0 = 1 if clamp_xm else 0
    px = nxn - x0
    Kref = q1_element_stiffness(1.0, nu)
    rows, cols, vals = [], [], []
    ez_i, ey_i, ex_i = np.meshgrid(np.arange(ez), np.arange(ey), np.arange(ex), indexing="ij")
    ez_i, ey_i, ex_i = ez_i.ravel(), ey_i.ravel(), ex_i.ravel()
    Ev = E.ravel()
    gd = np.zeros((ez_i.size, 24), dtype=np.int64)
    for a in range(8):
        ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
        nx_ = ex_i + ax - x0
        point = nx_ + px * ((ey_i + ay) + nyn * (ez_i + az))
        point = np.where(nx_ < 0, -1, point)
        for c in range(3):
            gd[:, 3 * a + c] = np.where(point < 0, -1, 3 * point + c)
    for i in range(24):
        for j in range(24):
            ok = (gd[:, i] >= 0) & (gd[:, j] >= 0)
            rows.append(gd[ok, i])
            cols.append(gd[ok, j])
            vals.append(Ev[ok] * Kref[i, j])
    n = 3 * px * nyn * nzn
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    K.sum_duplicates()
    K.sort_indices()
    return K, (px, nyn, nzn)


def assemble(cfg: dict):
    """Assemble A for a workload dict from `sgf_inputs.config`."""
    st = cfg["stencil"]
    if st == "5pt_2d":
        return assemble_scalar(cfg["n"], 2, cfg["coeffs"], cfg["dirichlet"], 1.0)
    if st == "7pt_fv_3d":
        return assemble_scalar(cfg["n"], 3, cfg["coeffs"], cfg["dirichlet"], 2.0)
    if st == "7pt_3d":
        return assemble_scalar(cfg["n"], 3, cfg["coeffs"], cfg["dirichlet"], 1.0)
    if st == "q1_elastic_3d":
        K, pts = assemble_elastic(cfg["elems"], cfg["coeffs"], cfg.get("nu", 0.3), clamp_xm=True)
        assert tuple(pts) == tuple(cfg["n"])
        return K
    raise KeyError(st)
