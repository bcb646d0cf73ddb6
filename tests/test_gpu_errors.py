"""Failure detection through status codes (no GPU fault is ever provoked):
a non-SPD coefficient field gives SGF_ERR_NOT_SPD with the failing node, a
NaN coefficient SGF_ERR_NONFINITE, too few PCG iterations
SGF_ERR_NO_CONVERGENCE; the device keeps working afterwards."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_03406_gb300 as sgf  # noqa: E402
import sgf_inputs as si  # noqa: E402

DEV = torch.device("cuda:0")


def _coeffs(k):
    return torch.tensor(np.ascontiguousarray(k).ravel(), dtype=torch.float64, device=DEV)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_negative_coefficient_reports_failed_pivot(precision):
    cfg = si.config("grf3d_16")
    k = cfg["coeffs"].copy()
    k[3:5, 3:5, 3:5] = -1e6           # negative diagonal entries: not positive definite
    plan = sgf.Plan.from_config(cfg, precision=precision)
    with pytest.raises(sgf.SGFError) as e:
        sgf.Factor(plan, _coeffs(k))
    assert e.value.code in (-2, -3)   # SGF_ERR_NOT_SPD, or NONFINITE when a harmonic mean overflows
    # the context is still healthy: a valid factorization works
    F = sgf.Factor(plan, _coeffs(cfg["coeffs"]))
    x, info = F.pcg(torch.tensor(si.rhs(plan.n, 0), dtype=torch.float64, device=DEV))
    assert info["rel_residual"] <= 1e-10


def test_nan_coefficient_reports_nonfinite():
    cfg = si.config("grf3d_16")
    k = cfg["coeffs"].copy()
    k[2, 2, 2] = np.nan
    plan = sgf.Plan.from_config(cfg)
    with pytest.raises(sgf.SGFError) as e:
        sgf.Factor(plan, _coeffs(k))
    assert e.value.code in (-2, -3)


def test_maxit_reports_no_convergence():
    cfg = si.config("grf3d_16")
    plan = sgf.Plan.from_config(cfg)
    F = sgf.Factor(plan, _coeffs(cfg["coeffs"]))
    b = torch.tensor(si.rhs(plan.n, 0), dtype=torch.float64, device=DEV)
    x, info = F.pcg(b, rtol=1e-10, maxit=2, check=False)
    assert info["status"] == -5 and info["iterations"] == 2


def test_mixed_falls_back_to_fp64_when_an_fp32_pivot_fails():
    # an SPD field with a 1e39 inclusion: its diagonal entries (6e39) exceed
    # the single-precision range, so the FP32 factorization meets a
    # non-finite pivot while FP64 does not; the mixed request is refactored
    # in FP64 with the mixed plan's compression threshold (tau = 1e-6), so it
    # runs exactly as an FP64 plan with that threshold: the same PCG
    # iterations and residual (at this contrast neither reaches 1e-10: the
    # attainable residual is ~eps64 cond(A))
    cfg = si.config("grf3d_16")
    k = np.ones_like(cfg["coeffs"])
    k[2:6, 2:6, 2:6] = 1e39
    b = torch.tensor(si.rhs(int(np.prod(cfg["n"])), 0), dtype=torch.float64, device=DEV)
    plan64 = sgf.Plan.from_config(cfg, precision="fp64", tau=1e-6)
    F64 = sgf.Factor(plan64, _coeffs(k))
    assert F64.precision == "fp64"
    _, info64 = F64.pcg(b, rtol=1e-10, maxit=200, check=False)
    plan = sgf.Plan.from_config(cfg, precision="mixed")
    F = sgf.Factor(plan, _coeffs(k))
    assert F.precision == "fp64"          # the FP32 attempt failed, FP64 was used
    _, info = F.pcg(b, rtol=1e-10, maxit=200, check=False)
    assert info["iterations"] == info64["iterations"]
    assert info["rel_residual"] == info64["rel_residual"]
    F_ok = sgf.Factor(plan, _coeffs(cfg["coeffs"]))
    assert F_ok.precision == "mixed"      # an ordinary field stays in FP32


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sgf_sync_surfaces_a_nonfinite_apply(precision):
    # an apply is enqueued and returns before the device runs it; a NaN in the
    # host-made right-hand side reaches the output, and sgf_sync (through the
    # C ABI) reports it once, then the flag is clear again
    cfg = si.config("grf3d_16")
    plan = sgf.Plan.from_config(cfg, precision=precision)
    F = sgf.Factor(plan, _coeffs(cfg["coeffs"]))
    assert F.sync() == 0
    v = si.rhs(plan.n, 0)
    y = F.apply(torch.tensor(v, dtype=torch.float64, device=DEV))
    assert F.sync() == 0 and torch.isfinite(y).all()
    v[plan.n // 3] = np.nan
    y = F.apply(torch.tensor(v, dtype=torch.float64, device=DEV))
    assert F.sync() == -3                       # SGF_ERR_NONFINITE
    assert F.sync() == 0                        # read once, then cleared
    F.apply_forward(torch.tensor(v, dtype=torch.float64, device=DEV))
    assert F.sync() == -3                       # the multiply is checked too
    y = F.apply(torch.tensor(si.rhs(plan.n, 1), dtype=torch.float64, device=DEV))
    assert F.sync() == 0 and torch.isfinite(y).all()
