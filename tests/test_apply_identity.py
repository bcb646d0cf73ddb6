"""The dense-block form of the apply of A_l^{-1} equals the triangular steps of
Sec. 4.7 (host check of the algebra the GPU programs use, plain numpy).

Sec. 4.7 applies an eliminated interior with its Cholesky factor,
forward y_I = L^{-1} b_I, b_S -= W^T y_I and backward x_I = L^{-T} (y_I -
W x_S) with W = L^{-1} A_IS, and a compressed separator with forward
c = L_B^{-1} b_B, k = Q1^T c and backward x_B = L_B^{-T} (c + Q1 (x_k - k)).
The GPU keeps instead Z = L^{-T} W = A_II^{-1} A_IS, A_II^{-1}, Qf = L_B^{-T}
Q1 and B^{-1} = L_B^{-T} L_B^{-1}, whose products give the same vectors:
b_S -= Z^T b_I, x_I = A_II^{-1} b_I - Z x_S, k = Qf^T b_B and
x_B = B^{-1} b_B + Qf (x_k - k).
"""
import numpy as np
import pytest


def _spd(rng, n):
    G = rng.standard_normal((n, n))
    return G @ G.T + n * np.eye(n)


@pytest.mark.parametrize("m,s", [(7, 5), (30, 12), (49, 70)])
def test_interior_steps(m, s):
    rng = np.random.default_rng(m + s)
    A = _spd(rng, m + s)
    Aii, Ais = A[:m, :m], A[:m, m:]
    L = np.linalg.cholesky(Aii)
    Li = np.linalg.inv(L)
    W = Li @ Ais
    Z = Li.T @ W
    Ai = Li.T @ Li
    assert np.allclose(Z, np.linalg.solve(Aii, Ais), rtol=1e-10, atol=1e-12)
    bI, bS, xS = rng.standard_normal(m), rng.standard_normal(s), rng.standard_normal(s)
    # forward: the separator update
    assert np.allclose(bS - W.T @ (Li @ bI), bS - Z.T @ bI, rtol=1e-12, atol=1e-12)
    # backward: the interior solution
    assert np.allclose(Li.T @ (Li @ bI - W @ xS), Ai @ bI - Z @ xS, rtol=1e-10, atol=1e-12)
    # A_II^{-1} is symmetric, so its rows are its columns (column dot products)
    assert np.allclose(Ai, Ai.T, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("m,k", [(9, 3), (49, 20), (64, 10)])
def test_compressed_separator_steps(m, k):
    rng = np.random.default_rng(100 + m + k)
    B = _spd(rng, m)
    LB = np.linalg.cholesky(B)
    LBi = np.linalg.inv(LB)
    Q1, _ = np.linalg.qr(rng.standard_normal((m, k)))
    Qf = LBi.T @ Q1
    Binv = LBi.T @ LBi
    bB, xk = rng.standard_normal(m), rng.standard_normal(k)
    c = LBi @ bB
    kept = Q1.T @ c
    # forward: the kept values sent to the next level
    assert np.allclose(kept, Qf.T @ bB, rtol=1e-10, atol=1e-12)
    # backward: the separator's solution from the next level's kept values
    tri = LBi.T @ (c + Q1 @ (xk - kept))
    dense = Binv @ bB + Qf @ (xk - Qf.T @ bB)
    assert np.allclose(tri, dense, rtol=1e-10, atol=1e-12)
    # with x_k equal to the forward value the block returns B^{-1} b_B
    assert np.allclose(Binv @ bB + Qf @ (kept - kept), np.linalg.solve(B, bB), rtol=1e-10, atol=1e-12)
