"""Pins for oracle/assemble.py against closed forms (Sec. 7.1 operators)."""
import numpy as np
import pytest

from oracle.assemble import assemble_scalar, assemble_elastic, q1_element_stiffness
from oracle.basis import eval_rbm

pytestmark = pytest.mark.filterwarnings("ignore")


def test_5pt_unit_is_classical_laplacian_with_sine_eigenvectors():
    # FD Laplacian on an N x N grid with Dirichlet ghosts: eigenpairs are
    # sin(j pi x/(N+1)) sin(k pi y/(N+1)), 4 - 2cos(j pi/(N+1)) - 2cos(k pi/(N+1)).
    N = 13
    A = assemble_scalar((N, N, 1), 2, np.ones((N, N)), 15, 1.0).toarray()
    assert np.allclose(np.diag(A), 4.0)
    off = A - np.diag(np.diag(A))
    assert set(np.unique(off)) <= {0.0, -1.0}
    x = np.arange(1, N + 1)
    for j, k in [(1, 1), (2, 5), (13, 7)]:
        v = np.outer(np.sin(k * np.pi * x / (N + 1)), np.sin(j * np.pi * x / (N + 1))).ravel()
        lam = 4 - 2 * np.cos(j * np.pi / (N + 1)) - 2 * np.cos(k * np.pi / (N + 1))
        assert np.linalg.norm(A @ v - lam * v) <= 1e-13 * np.linalg.norm(v)


def test_7pt_fd_sine_eigenvector():
    N = 7
    A = assemble_scalar((N, N, N), 3, np.ones((N, N, N)), 63, 1.0)
    x = np.arange(1, N + 1)
    s = lambda j: np.sin(j * np.pi * x / (N + 1))
    v = np.einsum("i,j,k->ijk", s(1), s(2), s(3)).ravel()   # [z, y, x]
    lam = sum(2 - 2 * np.cos(j * np.pi / (N + 1)) for j in (1, 2, 3))
    assert np.linalg.norm(A @ v - lam * v) <= 1e-13 * np.linalg.norm(v)


def test_fv_harmonic_transmissibility_and_dirichlet_half_cell():
    # two cells along x with k = 1 and 3: T = 2*1*3/(1+3) = 1.5; Dirichlet on x-
    # gives the first cell 2*k = 2 extra on its diagonal (half-cell distance).
    k = np.array([[[1.0, 3.0]]])
    A = assemble_scalar((2, 1, 1), 3, k, 1, 2.0).toarray()
    assert np.array_equal(A, np.array([[1.5 + 2.0, -1.5], [-1.5, 1.5]]))


def test_fv_row_sums_vanish_away_from_dirichlet():
    rng = np.random.default_rng(0)
    k = np.exp(rng.standard_normal((5, 6, 7)))
    A = assemble_scalar((7, 6, 5), 3, k, 1, 2.0)
    rs = np.asarray(A.sum(axis=1)).ravel().reshape(5, 6, 7)
    assert np.allclose(rs[:, :, 1:], 0.0, atol=1e-12)
    assert np.allclose(rs[:, :, 0], 2 * k[:, :, 0], rtol=1e-14)
    assert abs(A - A.T).max() == 0
    ev = np.linalg.eigvalsh(A.toarray())
    assert ev[0] > 0


def test_q1_element_kernel_is_rigid_body_modes():
    K = q1_element_stiffness(1.0, 0.3)
    assert np.allclose(K, K.T, atol=1e-14)
    ev = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(ev) < 1e-12) == 6 and ev[6] > 1e-3
    xyz = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=float)
    R = eval_rbm(xyz, (np.array([0.3, -0.2, 0.7]), 1.7))
    assert np.abs(K @ R).max() < 1e-13


def test_q1_free_body_annihilates_rbm_and_clamped_is_spd():
    rng = np.random.default_rng(1)
    E = np.exp(rng.standard_normal((3, 3, 4)))
    K, (px, py, pz) = assemble_elastic((4, 3, 3), E, 0.3, clamp_xm=False)
    p = np.arange(px * py * pz)
    xyz = np.stack([p % px, (p // px) % py, p // (px * py)], 1).astype(float)
    R = eval_rbm(xyz, (np.zeros(3), 1.0))
    assert np.abs(K @ R).max() < 1e-12 * abs(K).max()
    Kc, _ = assemble_elastic((4, 3, 3), E, 0.3, clamp_xm=True)
    assert np.linalg.eigvalsh(Kc.toarray())[0] > 0
