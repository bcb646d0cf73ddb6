"""The apply of A_l^{-1} (Sec. 4.7) replays a captured graph whose kernels
launch programmatically (each may start while the previous one drains and
waits for it before touching a vector).  The launch mode must not change a
single bit of the result, and the launch accounting must see every replay.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_03406_gb300 as sgf  # noqa: E402
import sgf_inputs as si  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SCRIPT = r"""
import sys
import numpy as np
import torch
import paper_1907_03406_gb300 as sgf
import sgf_inputs as si
name, precision, out = sys.argv[1], sys.argv[2], sys.argv[3]
cfg = si.config(name)
dev = torch.device("cuda:0")
plan = sgf.Plan.from_config(cfg, precision=precision)
F = sgf.Factor(plan, torch.tensor(cfg["coeffs"].ravel(), dtype=torch.float64, device=dev))
rng = np.random.default_rng(3)
X = torch.tensor(rng.standard_normal((3, plan.n)).ravel(), dtype=torch.float64, device=dev)
ys = [F.apply(X).cpu().numpy()]
for _ in range(4):   # repeated replays of the same graph
    ys.append(F.apply(X).cpu().numpy())
x, info = F.pcg(torch.tensor(si.rhs(plan.n, 0), dtype=torch.float64, device=dev), rtol=1e-10, maxit=500)
np.savez(out, y=np.stack(ys), x=x.cpu().numpy(), it=info["iterations"])
"""


def _run(tmp_path, name, precision, dependent):
    out = str(tmp_path / f"{name}_{precision}_{dependent}.npz")
    env = dict(os.environ, SGF_DEPENDENT_LAUNCH="1" if dependent else "0")
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    subprocess.run([sys.executable, "-c", _SCRIPT, name, precision, out], check=True, env=env, cwd=ROOT,
                   timeout=600)
    return np.load(out)


@pytest.mark.parametrize("name,precision", [("grf3d_32", "mixed"), ("grf3d_24", "fp64"),
                                            ("elastic_12", "mixed")])
def test_dependent_launch_is_bitwise_identical(tmp_path, name, precision):
    a = _run(tmp_path, name, precision, True)
    b = _run(tmp_path, name, precision, False)
    for k in range(1, a["y"].shape[0]):   # every replay gives the first one's bits
        assert np.array_equal(a["y"][k], a["y"][0])
    assert np.array_equal(a["y"], b["y"])
    assert np.array_equal(a["x"], b["x"]) and int(a["it"]) == int(b["it"])


def test_profile_counts_apply_replays_and_their_kernels():
    cfg = si.config("grf3d_16")
    dev = torch.device("cuda:0")
    plan = sgf.Plan.from_config(cfg, precision="mixed")
    F = sgf.Factor(plan, torch.tensor(cfg["coeffs"].ravel(), dtype=torch.float64, device=dev))
    b = torch.tensor(si.rhs(plan.n, 0), dtype=torch.float64, device=dev)
    F.apply(b)   # the first apply captures the graph
    sgf.profile_reset(timing="contractions")
    for _ in range(5):
        F.apply(b)
    p = sgf.profile_read()
    assert p["apply"]["launches"] == 5
    assert p["apply"]["ms"] > 0 and p["apply"]["bytes"] > 0
    # the replays' nodes are counted under their own kinds, untimed
    gemv = p["k_gemv_t"]["launches"] + p["k_gemv_n"]["launches"]
    assert gemv > 0 and gemv % 5 == 0
    assert p["k_gemv_t"]["ms"] == 0.0
    node_bytes = sum(p[k]["bytes"] for k in ("k_gemv_t", "k_gemv_n", "k_veccopy"))
    assert p["apply"]["bytes"] == pytest.approx(node_bytes, rel=1e-12)
    sgf.profile_reset(timing=False)
    F.close()


def test_wide_gemv_chunks_match_the_default_and_stay_rhs_independent():
    # gemv_cols = 64 only regroups the column dot products into wider tasks:
    # every column's sum runs over the same rows in the same lane order, so
    # the apply stays within rounding of the 32-wide one, and k right-hand
    # sides still give exactly the single-RHS answers
    cfg = si.config("grf3d_24")
    dev = torch.device("cuda:0")
    c = torch.tensor(cfg["coeffs"].ravel(), dtype=torch.float64, device=dev)
    rng = np.random.default_rng(11)
    plan = sgf.Plan.from_config(cfg, precision="mixed")
    X = rng.standard_normal((3, plan.n))
    F32 = sgf.Factor(plan, c)
    y32 = F32.apply(torch.tensor(X[0], device=dev)).cpu().numpy()
    F32.close()
    plan.tuning = {"gemv_cols": 64}
    F = sgf.Factor(plan, c)
    Y = F.apply(torch.tensor(X.ravel(), device=dev)).cpu().numpy().reshape(3, plan.n)
    for j in range(3):
        assert np.array_equal(Y[j], F.apply(torch.tensor(X[j], device=dev)).cpu().numpy())
    assert np.linalg.norm(Y[0] - y32) <= 1e-5 * np.linalg.norm(y32)
    x, info = F.pcg(torch.tensor(si.rhs(plan.n, 0), device=dev), rtol=1e-10, maxit=500)
    assert info["rel_residual"] <= 1e-10
    F.close()
