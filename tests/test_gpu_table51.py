"""Table 5.1 quantities of the GPU factor (Sec. 6, Table 5.1), through the C ABI.

For constant-coefficient 3D Poisson with Dirichlet faces the eigenvectors are
known in closed form (products of sines), so the error of A_l on the largest
eigenvector, E_1 = ||(A - A_l) v_1|| / lambda_1, and on the smallest,
E_n = ||(A - A_l) v_n|| / lambda_n, can be measured at any size.  On a grid
the oracle factors, the FP64 GPU values equal the oracle's (they are
functionals of A_l, which the GPU reproduces to 1e-10); at larger sizes the
paper's behaviour holds: E_1 small (the paper prints 4.5e-2 for Nest-All-All
with quadratics at 4M-16M unknowns) and E_n growing towards order one
(1.1-1.4 in the paper).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import sgf_inputs as si
from oracle.assemble import assemble
from oracle.partition import build_hierarchy
from oracle.sgf import Options, factorize

pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_03406_gb300 as sgf  # noqa: E402

DEV = torch.device("cuda:0")


def _eig(e, mode):
    # eigenvector sin(k pi (x_a + 1) / (e + 1)) on every axis, k = mode
    s = np.sin(mode * np.pi * (np.arange(e) + 1.0) / (e + 1.0))
    v = (s[None, None, :] * s[None, :, None] * s[:, None, None]).ravel()
    lam = 3.0 * (2.0 - 2.0 * np.cos(mode * np.pi / (e + 1.0)))
    return v / np.linalg.norm(v), lam


def _gpu_E(e, precision="fp64"):
    cfg = si.config(f"poisson3d_{e}")
    plan = sgf.Plan.from_config(cfg, precision=precision)
    F = sgf.Factor(plan, torch.tensor(cfg["coeffs"].ravel(), dtype=torch.float64, device=DEV))
    out = {}
    for key, mode in (("E_1", e), ("E_n", 1)):
        v, lam = _eig(e, mode)
        vt = torch.tensor(v, dtype=torch.float64, device=DEV)
        out[key] = torch.linalg.norm(F.spmv(vt) - F.apply_forward(vt)).item() / lam
    F.close()
    return out, cfg


def test_closed_form_eigenpairs_of_the_operator():
    cfg = si.config("poisson3d_12")
    A = assemble(cfg)
    for mode in (1, 5, 12):
        v, lam = _eig(12, mode)
        assert np.linalg.norm(A @ v - lam * v) <= 1e-12 * lam


@pytest.mark.parametrize("e", [16, 24])
def test_E1_En_match_the_oracle(e):
    got, cfg = _gpu_E(e)
    A = assemble(cfg)
    H = build_hierarchy(cfg["n"], 3, cfg["leaf"], cfg["stencil"])
    O = factorize(A, H, Options(degree=cfg["degree"], order="level"))
    for key, mode in (("E_1", e), ("E_n", 1)):
        v, lam = _eig(e, mode)
        want = np.linalg.norm(A @ v - O.multiply(v)) / lam
        assert abs(got[key] - want) <= 1e-7 * want, (key, got[key], want)


def test_E1_small_and_En_grows_to_order_one():
    # E_1 stays near the paper's 4.5e-2 (5.8e-2 on the oracle at 24^3 and
    # 32^3); E_n grows with n towards the paper's O(1) (0.03, 0.10, 0.14 on the
    # oracle at 16^3, 24^3, 32^3)
    E = {e: _gpu_E(e)[0] for e in (32, 64)}
    print({e: {k: f"{v:.3e}" for k, v in d.items()} for e, d in E.items()})
    for e in E:
        assert E[e]["E_1"] <= 0.1
        assert E[e]["E_n"] <= 10.0
    assert 0.1 <= E[32]["E_n"] <= E[64]["E_n"]
