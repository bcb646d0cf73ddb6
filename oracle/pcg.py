"""Preconditioned conjugate gradients (Sec. 7: CG with A_l^{-1} as preconditioner).

x0 = 0; the iteration stops when the recursive residual satisfies
||r_k||_2 <= rtol ||b||_2 (relative 2-norm residual below 1e-10 in the paper's
runs); the count is the number of products with A.  `flexible` switches the
beta of Hestenes-Stiefel, (r_{k+1}.z_{k+1}) / (r_k.z_k), to the Polak-Ribiere
form z_{k+1}.(r_{k+1} - r_k) / (r_k.z_k), which tolerates a preconditioner
applied in lower precision (not exactly symmetric).
"""
from __future__ import annotations

import numpy as np


def pcg(matvec, precond, b, rtol=1e-10, maxit=1000, flexible=False):
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return x, 0, 0.0
    r = b.copy()
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    while it < maxit:
        q = matvec(p)
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r_new = r - alpha * q
        it += 1
        if float(np.linalg.norm(r_new)) <= rtol * bnorm:
            r = r_new
            break
        z_new = precond(r_new)
        if flexible:
            beta = float(z_new @ (r_new - r)) / rz
        else:
            beta = float(r_new @ z_new) / rz
        rz = float(r_new @ z_new)
        p = z_new + beta * p
        r = r_new
    true_res = float(np.linalg.norm(b - matvec(x))) / bnorm
    return x, it, true_res
