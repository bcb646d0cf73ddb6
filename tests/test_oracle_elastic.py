"""Pins of the oracle's elasticity path (Sec. 7.1.3 on hexahedra, Sec. 7.2).

Q1 element: a homogeneous strain u = eps x is reproduced exactly by the
trilinear element and its strain energy density is constant, so the 2x2x2
Gauss rule integrates it exactly: u^T K u = vol (lam tr(eps)^2 + 2 mu eps:eps)
with lam = E nu / ((1+nu)(1-2nu)), mu = E / (2(1+nu)) (the isotropic Hooke
law).  A wrong Lame parameter, shear convention or quadrature weight changes
the energy of one of the strains below.  For any field of the trilinear span
the energy density has degree <= 2 per axis, so u^T K u is its exact integral
(which also pins the Gauss points and the shape-function derivatives).

Assembled operator: with a uniform modulus, a linear displacement field is in
equilibrium (the Q1 patch test), so K u vanishes at every node that is not on
the boundary; the forces of a free body sum to zero.

Factorization with the rigid-body basis, 3 DOFs per node:
P1  compression off => A_l = A (exact block Cholesky, one PCG iteration);
P2  A_l R = A R for the six global rigid-body modes R (Eq. (preserve-pi) with
    the user space of Sec. 7.2: the modes restricted to every node lie in
    that node's basis);
P4  positive pivots;
P5  the dense restatement reproduces A_l and the ranks.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import sgf_inputs as si
from oracle.assemble import assemble, assemble_elastic, q1_element_stiffness
from oracle.basis import eval_rbm
from oracle.dense import dense_sgf
from oracle.partition import build_hierarchy
from oracle.pcg import pcg
from oracle.sgf import Options, factorize

CORNERS = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=float)


def _hooke_energy(eps, E, nu):
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    return lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps)


@pytest.mark.parametrize("E,nu", [(1.0, 0.3), (2.5, 0.25), (1e3, 0.45)])
def test_q1_homogeneous_strain_energy_is_closed_form(E, nu):
    K = q1_element_stiffness(E, nu)
    rng = np.random.default_rng(7)
    strains = [np.diag([1.0, 0.0, 0.0]),                      # uniaxial: lam + 2 mu
               np.diag([1.0, 1.0, 1.0]),                      # dilatation: 9 lam + 6 mu
               np.array([[0, 1, 0], [1, 0, 0], [0, 0, 0.]]),  # pure shear: 4 mu
               np.array([[0, 0, 0], [0, 0, 1], [0, 1, 0.]]),
               np.array([[0, 0, 1], [0, 0, 0], [1, 0, 0.]])]
    G = rng.standard_normal((3, 3))
    strains.append(0.5 * (G + G.T))
    for eps in strains:
        u = (CORNERS @ eps.T).ravel()          # node a, component c -> 3 a + c
        assert abs(u @ K @ u - _hooke_energy(eps, E, nu)) <= 1e-12 * _hooke_energy(eps, E, nu)


def test_q1_trilinear_fields_energy_is_exact_integral():
    # every displacement in the trilinear span is reproduced by the element,
    # and its energy density is a polynomial of degree <= 2 per axis, which the
    # 2-point Gauss rule integrates exactly: u^T K u equals the exact integral
    # of lam tr(eps)^2 + 2 mu eps:eps over the unit cube (symbolic here)
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    E, nu = 1.7, 0.3
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    K = q1_element_stiffness(E, nu)
    mon = [1, x, y, z, x * y, y * z, z * x, x * y * z]
    rng = np.random.default_rng(11)
    X = (x, y, z)
    for _ in range(4):
        coef = rng.standard_normal((3, 8))
        u = [sum(float(coef[c, k]) * mon[k] for k in range(8)) for c in range(3)]
        eps = [[(sp.diff(u[i], X[j]) + sp.diff(u[j], X[i])) / 2 for j in range(3)] for i in range(3)]
        tr = eps[0][0] + eps[1][1] + eps[2][2]
        dens = lam * tr ** 2 + 2 * mu * sum(eps[i][j] ** 2 for i in range(3) for j in range(3))
        exact = float(sp.integrate(sp.expand(dens), (x, 0, 1), (y, 0, 1), (z, 0, 1)))
        un = np.array([[float(u[c].subs({x: p[0], y: p[1], z: p[2]})) if not isinstance(u[c], (int, float))
                        else u[c] for c in range(3)] for p in CORNERS]).ravel()
        assert abs(un @ K @ un - exact) <= 1e-12 * exact


def test_q1_element_scales_with_modulus_only():
    K1 = q1_element_stiffness(1.0, 0.3)
    assert np.allclose(q1_element_stiffness(3.0, 0.3), 3.0 * K1, rtol=1e-14, atol=0)


def test_q1_patch_test_linear_field_in_equilibrium():
    ex, ey, ez = 4, 3, 5
    K, (px, py, pz) = assemble_elastic((ex, ey, ez), np.full((ez, ey, ex), 2.0), 0.3, clamp_xm=False)
    p = np.arange(px * py * pz)
    xyz = np.stack([p % px, (p // px) % py, p // (px * py)], 1).astype(float)
    rng = np.random.default_rng(3)
    G = rng.standard_normal((3, 3))
    u = (xyz @ G.T + rng.standard_normal(3)).ravel()
    f = (K @ u).reshape(-1, 3)
    inner = ((xyz[:, 0] > 0) & (xyz[:, 0] < px - 1) & (xyz[:, 1] > 0) & (xyz[:, 1] < py - 1)
             & (xyz[:, 2] > 0) & (xyz[:, 2] < pz - 1))
    assert inner.sum() > 0
    scale = abs(K).max() * np.abs(u).max()
    assert np.abs(f[inner]).max() <= 1e-12 * scale
    assert np.abs(f[~inner]).max() > 1e-3 * scale          # tractions on the boundary
    assert np.abs(f.sum(axis=0)).max() <= 1e-11 * scale    # free body: forces balance


def _elastic(name):
    cfg = si.config(name)
    A = assemble(cfg)
    H = build_hierarchy(cfg["n"], 3, cfg["leaf"], cfg["stencil"], dof=3)
    return cfg, A, H


def _global_rbm(cfg):
    nx, ny, nz = cfg["n"]
    p = np.arange(nx * ny * nz)
    # point x index i is node x = i + 1 (the clamped x = 0 face is removed)
    xyz = np.stack([p % nx + 1, (p // nx) % ny, p // (nx * ny)], 1).astype(float)
    return eval_rbm(xyz, (np.array([nx / 2, ny / 2, nz / 2]), float(max(nx, ny, nz))))


def test_rbm_P1_no_compression_is_exact():
    cfg, A, H = _elastic("elastic_8")
    F = factorize(A, H, Options(scheme="none", basis="rbm", degree=1))
    assert F.pivots_min > 0
    rng = np.random.default_rng(2)
    b = rng.standard_normal(A.shape[0])
    x = sla.solve(A.toarray(), b, assume_a="pos")
    assert np.linalg.norm(F.solve(b) - x) <= 1e-12 * np.linalg.norm(x)
    assert np.linalg.norm(F.multiply(x) - b) <= 1e-12 * np.linalg.norm(b)
    _, it, res = pcg(lambda v: A @ v, F.solve, b)
    assert it == 1 and res < 1e-12


@pytest.mark.parametrize("name", ["elastic_8", "elastic_12"])
def test_rbm_P2_P4_preserves_rigid_body_modes(name):
    cfg, A, H = _elastic(name)
    F = factorize(A, H, Options(basis="rbm", degree=1))
    assert any(v[2] for v in F.ranks().values()), "some node must actually compress"
    assert F.pivots_min > 0
    R = _global_rbm(cfg)
    AR = A @ R
    AlR = np.stack([F.multiply(R[:, k]) for k in range(6)], 1)
    assert np.linalg.norm(AlR - AR) <= 1e-12 * np.linalg.norm(AR)
    # and A_l is a genuine approximation: it differs from A on a random vector
    v = np.random.default_rng(0).standard_normal(A.shape[0])
    assert np.linalg.norm(F.multiply(v) - A @ v) > 1e-8 * np.linalg.norm(A @ v)


def test_rbm_P5_dense_restatement_reproduces_block_oracle():
    cfg, A, H = _elastic("elastic_8")
    opts = Options(basis="rbm", degree=1)
    F = factorize(A, H, opts)
    Ad, _, ranks = dense_sgf(A, H, opts)
    assert ranks == F.ranks()
    assert any(v[2] for v in ranks.values())
    Al = F.dense_operator()
    assert np.abs(Al - Ad).max() <= 1e-12 * np.abs(Ad).max()
