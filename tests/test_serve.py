"""Serving loop: admission logic on the host, and on the GPU that every
result of a concurrent mix equals the same solve run alone (continuous
batching must not change answers)."""
import numpy as np
import pytest

import sgf_inputs as si
from paper_1907_03406_gb300.serve import Admission


def test_admission_respects_slots_and_budget():
    a = Admission(slots=2, budget_bytes=100)
    assert a.fits(60)
    a.take(60)
    assert not a.fits(50)          # memory
    assert a.fits(40)
    a.take(40)
    assert not a.fits(0)           # slots
    a.release(60)
    assert a.fits(50) and not a.fits(61)
    a.resident = 30
    assert not a.fits(31) and a.fits(30)


def test_request_stream_is_seeded_and_mixed():
    r1 = si.request_stream(seed=1, count=256)
    r2 = si.request_stream(seed=1, count=256)
    assert r1 == r2
    kinds = [r["kind"] for r in r1]
    assert 0.3 < kinds.count("factor") / 256 < 0.5
    assert all(32 <= r["edge"] <= 96 and 1 <= r["nrhs"] <= 8 for r in r1)
    t = [r["arrival_s"] for r in r1]
    assert t == sorted(t)


@pytest.mark.gpu
def test_results_alone_equal_results_in_the_mix():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1907_03406_gb300 as sgf
    from paper_1907_03406_gb300.serve import Server
    reqs = si.request_stream(seed=3, count=16, rate_hz=400.0, edge_lo=16, edge_hi=30, max_rhs=3)
    srv = Server(slots=4, keep_results=True)
    summ = srv.run(reqs)
    assert summ["failed"] == 0, srv.records
    assert summ["max_rel_residual"] <= 1e-10
    byid = {r["id"]: r for r in reqs}
    # every request again, alone, on the factor it used in the mix
    dev = torch.device("cuda:0")
    for rec in srv.records:
        freq = byid[rec["factor_of"]]
        cfg = dict(n=(freq["edge"],) * 3)
        plan = sgf.Plan(cfg["n"], 3, "7pt_fv_3d", 1, 8, 2, precision="mixed")
        F = sgf.Factor(plan, torch.from_numpy(si.request_coeffs(freq).ravel()).to(dev))
        req = byid[rec["id"]]
        b = torch.from_numpy(si.rhs(plan.n, req["rhs_seed"], nrhs=req["nrhs"]).reshape(-1)).to(dev)
        x, info = F.pcg(b, rtol=1e-10, maxit=500)
        x = x.reshape(req["nrhs"], plan.n).cpu().numpy()
        mix = srv.results[rec["id"]]
        assert np.linalg.norm(x - mix) <= 1e-12 * np.linalg.norm(x), rec
        F.close()
    srv.close()
