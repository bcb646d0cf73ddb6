"""Device memory of factors: blocks come from the stream-ordered pool, go
back to it when a factor is destroyed (a second factorization of the same
plan reuses them instead of growing the device footprint) and are handed
back to the device by release_cached_memory.  A factor made from reused
blocks applies bit for bit like the first one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_03406_gb300 as sgf  # noqa: E402
import sgf_inputs as si  # noqa: E402


def _free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_factor_memory_is_pooled_and_released():
    dev = torch.device("cuda:0")
    cfg = si.config("grf3d_32")
    plan = sgf.Plan.from_config(cfg, precision="mixed")
    c = torch.tensor(cfg["coeffs"].ravel(), dtype=torch.float64, device=dev)
    v = torch.tensor(np.random.default_rng(5).standard_normal(plan.n), dtype=torch.float64, device=dev)
    sgf.release_cached_memory()
    free0 = _free()
    F = sgf.Factor(plan, c)
    y1 = F.apply(v).cpu().numpy()
    free1 = _free()
    used = free0 - free1
    assert used > 50e6   # a 32^3 factor holds well over 50 MB
    F.close()
    assert _free() <= free1 + 0.05 * used   # cached by the pool, not unmapped
    F2 = sgf.Factor(plan, c)
    y2 = F2.apply(v).cpu().numpy()
    assert _free() >= free1 - 0.05 * used   # served from the cache
    assert np.array_equal(y1, y2)
    F2.close()
    sgf.release_cached_memory()
    assert _free() >= free0 - 0.05 * used
