"""The allocation-free PCG entry point against the regular one (GPU).

sgf_pcg_solve_noalloc exists for callers that cannot let the library
allocate device memory during a solve; its scratch is a fixed device array
shared by all calls.  This file is collected last so that a run stopping at
the first failure has already run every other test.  It checks, through the
C ABI, that two calls in a row give the regular sgf_pcg_solve's answer, that
the scratch left by a previous call does not change the next result, and
that a factor larger than the array is rejected.  The first call is made on a
factor nothing has applied yet, and the library's allocation counter and the
device pool's used bytes must not move across the calls (sgf_memory_stats).
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_03406_gb300 as sgf  # noqa: E402
import sgf_inputs as si  # noqa: E402
from paper_1907_03406_gb300 import _lib  # noqa: E402

DEV = torch.device("cuda:0")


def _noalloc(F, b, rtol=1e-10, maxit=500, x=None):
    lib = _lib.load()
    if x is None:
        x = torch.full_like(b, float("nan"))
    info = _lib.sgf_solve_info()
    rc = lib.sgf_pcg_solve_noalloc(F.handle, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                   float(rtol), int(maxit),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(info))
    return rc, x, info


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_regular_pcg_two_calls(precision):
    cfg = si.config("grf3d_32")
    plan = sgf.Plan.from_config(cfg, precision=precision)
    coeffs = torch.tensor(cfg["coeffs"].ravel(), dtype=torch.float64, device=DEV)
    F = sgf.Factor(plan, coeffs)
    b1 = torch.tensor(si.rhs(plan.n, 0), dtype=torch.float64, device=DEV)
    b2 = torch.tensor(si.rhs(plan.n, 1), dtype=torch.float64, device=DEV)
    results = []
    xs = [torch.full_like(b1, float("nan")) for _ in range(2)]
    torch.cuda.synchronize()
    for b, x0 in zip((b1, b2), xs):   # two calls in a row on a fresh factor, nothing else in between
        before = sgf.memory_stats()
        rc, x, info = _noalloc(F, b, x=x0)
        after = sgf.memory_stats()
        assert rc == 0, sgf.SGFError(rc, "noalloc")
        assert after["alloc_events"] == before["alloc_events"]
        assert after["pool_used_bytes"] == before["pool_used_bytes"]
        results.append((x, info))
    for b, (x, info) in zip((b1, b2), results):   # the regular solve (which allocates) after
        x_ref, info_ref = F.pcg(b, rtol=1e-10, maxit=500)
        assert info.iterations == info_ref["iterations"]
        assert info.rel_residual <= 1e-10
        err = torch.linalg.norm(x - x_ref).item() / torch.linalg.norm(x_ref).item()
        assert err <= 1e-12, err


def test_noalloc_rejects_factor_beyond_scratch():
    cfg = si.config("grf3d_66")
    assert int(np.prod(cfg["n"])) > 262144
    plan = sgf.Plan.from_config(cfg, precision="mixed")
    F = sgf.Factor(plan, torch.tensor(cfg["coeffs"].ravel(), dtype=torch.float64, device=DEV))
    b = torch.tensor(si.rhs(plan.n, 0), dtype=torch.float64, device=DEV)
    rc, x, info = _noalloc(F, b)
    assert rc == -1   # SGF_ERR_INVALID_ARG
