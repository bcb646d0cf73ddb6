"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Tolerances: FP64 apply of A_l^{-1} (and of A_l) on random vectors within
max(1e-10, 4 s) relative of the oracle, where s is the oracle's own
sensitivity: how far its operator moves when every entry of the filtered
interaction matrix N is perturbed by 4 ulps before the pivoted QR.  A_l
depends on span(Q1), which a rank cut with a graded R diagonal (kept values
near tau) fixes only to ~eps / R_rr; where the cut is clean s ~ 1e-13 and the
bound is 1e-10.  Ranks of every node equal; PCG iteration counts within +-1;
true relative residual <= 1e-10.  The GPU computes all compressions of a
level from the post-elimination matrix, the oracle's "level" reading (equal
to the paper's sequential recursion when Q2^T N vanishes; the oracle tests
pin the two readings against each other).
Mixed precision: PCG still reaches 1e-10 (FP64 outer loop) within +-1
iteration of the FP64 oracle run with the mixed rank rule (tau = 1e-6); the
FP32 apply is within 2^-20 kappa_2(A) of that oracle (a first-order forward
error bound for a factorization backward stable in the product precision).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import sgf_inputs as si
from oracle.assemble import assemble, assemble_scalar
from oracle.basis import eval_monomials, exponents
from oracle.partition import build_hierarchy
from oracle.pcg import pcg
from oracle.sgf import Options, factorize

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_03406_gb300 as sgf  # noqa: E402

DEV = torch.device("cuda:0")
_ORACLE_CACHE = {}


def _problem(name, seed=0):
    if name.startswith("rand2d_"):
        _, nx, ny, b = name.split("_")
        nx, ny, b = int(nx), int(ny), int(b)
        rng = np.random.default_rng(seed)
        k = np.exp(rng.standard_normal((ny, nx)))
        return dict(name=name, dim=2, n=(nx, ny, 1), stencil="5pt_2d", dirichlet=15, coeffs=k,
                    leaf=b, degree=1, basis="poly", dof=1)
    if name.startswith("rand3d_"):
        _, nx, ny, nz, b = name.split("_")
        nx, ny, nz, b = int(nx), int(ny), int(nz), int(b)
        rng = np.random.default_rng(seed)
        k = np.exp(1.5 * rng.standard_normal((nz, ny, nx)))
        return dict(name=name, dim=3, n=(nx, ny, nz), stencil="7pt_fv_3d", dirichlet=1, coeffs=k,
                    leaf=b, degree=2, basis="poly", dof=1)
    return si.config(name, seed)


def _oracle(cfg, scheme=None):
    scheme = scheme or cfg.get("scheme", "nest_all_all")
    key = (cfg["name"], scheme)
    if key not in _ORACLE_CACHE:
        A = assemble(cfg)
        H = build_hierarchy(cfg["n"], cfg["dim"], cfg["leaf"], cfg["stencil"], dof=cfg.get("dof", 1),
                            general=scheme == "gen_all_all")
        F = factorize(A, H, Options(scheme=scheme, degree=cfg["degree"], order="level",
                                    basis=cfg.get("basis", "poly")))
        _ORACLE_CACHE[key] = (A, H, F)
    return _ORACLE_CACHE[key]


def _tolerance(cfg, v):
    """max(1e-10, 4 x the oracle's self-sensitivity) for apply and multiply."""
    A, H, O = _oracle(cfg)
    a, m = O.solve(v), O.multiply(v)
    sa = sm = 0.0
    for seed in range(3):
        P = factorize(A, H, Options(scheme=cfg.get("scheme", "nest_all_all"), degree=cfg["degree"],
                                    order="level", qr_noise=4 * 2.2e-16, qr_noise_seed=seed,
                                    basis=cfg.get("basis", "poly")))
        sa = max(sa, np.linalg.norm(P.solve(v) - a) / np.linalg.norm(a))
        sm = max(sm, np.linalg.norm(P.multiply(v) - m) / np.linalg.norm(m))
    return max(1e-10, 4 * sa), max(1e-10, 4 * sm)


def _log(record: dict):
    """Print a parity record; with SGF_PARITY_LOG=<path> also append it there
    as one JSON line (the per-case bounds and errors of a run)."""
    import json
    import os
    print(json.dumps(record))
    path = os.environ.get("SGF_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(record) + "\n")


def _gpu(cfg, precision="fp64", scheme=None):
    plan = sgf.Plan.from_config(cfg, precision=precision, scheme=scheme or cfg.get("scheme", "nest_all_all"))
    c = torch.tensor(np.ascontiguousarray(cfg["coeffs"]).ravel(), dtype=torch.float64, device=DEV)
    return plan, sgf.Factor(plan, c)


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


SMALL = ["poisson2d_64", "rand2d_29_23_4", "grf3d_16", "rand3d_21_18_13_4", "grf3d_24",
         "twophase3d_24", "grf3d_32", "elastic_8", "elastic_12", "gengrf3d_20", "gengrf3d_24"]


@pytest.mark.parametrize("name", SMALL)
def test_spmv_matches_oracle_operator(name):
    cfg = _problem(name)
    A, _, _ = _oracle(cfg)
    plan, F = _gpu(cfg)
    x = np.random.default_rng(1).standard_normal(plan.n)
    y = F.spmv(_t(x)).cpu().numpy()
    assert np.abs(y - A @ x).max() <= 1e-13 * np.abs(A @ x).max()


@pytest.mark.parametrize("name", SMALL)
def test_ranks_match_oracle(name):
    cfg = _problem(name)
    A, H, O = _oracle(cfg)
    plan, F = _gpu(cfg)
    want = {}
    for (t, node), v in O.comp_info.items():
        want[(t, node)] = (v["m"], v["r"])
    for li, lev in enumerate(H.levels[:-1]):
        m, r = F.ranks(li, lev.nnodes)
        for node in range(lev.nnodes):
            if (lev.t, node) in want:
                wm, wr = want[(lev.t, node)]
                assert (m[node], r[node]) == (wm, wr), (lev.t, node, m[node], r[node], wm, wr)


@pytest.mark.parametrize("name", SMALL)
def test_apply_and_forward_match_oracle(name):
    cfg = _problem(name)
    A, H, O = _oracle(cfg)
    plan, F = _gpu(cfg)
    rng = np.random.default_rng(7)
    for k in range(2):
        v = rng.standard_normal(plan.n)
        ta, tm = _tolerance(cfg, v)
        y = F.apply(_t(v)).cpu().numpy()
        yo = O.solve(v)
        z = F.apply_forward(_t(v)).cpu().numpy()
        zo = O.multiply(v)
        ea = np.linalg.norm(y - yo) / np.linalg.norm(yo)
        em = np.linalg.norm(z - zo) / np.linalg.norm(zo)
        _log({"test": "fp64_apply", "case": name, "vector": k, "apply_err": ea, "apply_bound": ta,
              "multiply_err": em, "multiply_bound": tm})
        assert ea <= ta
        assert em <= tm


@pytest.mark.parametrize("name", ["poisson2d_64", "grf3d_24", "twophase3d_24", "elastic_12"])
def test_pcg_iterations_match_oracle(name):
    cfg = _problem(name)
    A, H, O = _oracle(cfg)
    plan, F = _gpu(cfg)
    b = si.rhs(plan.n, 0)
    _, it_o, res_o = pcg(lambda v: A @ v, O.solve, b)
    x, info = F.pcg(_t(b), rtol=1e-10, maxit=500)
    assert abs(info["iterations"] - it_o) <= 1
    assert info["rel_residual"] <= 1e-10
    xs = x.cpu().numpy()
    assert np.linalg.norm(A @ xs - b) <= 1e-10 * np.linalg.norm(b) * 1.01


def test_no_compression_is_exact_solve():
    cfg = _problem("rand3d_21_18_13_4")
    A, H, O = _oracle(cfg, scheme="none")
    plan, F = _gpu(cfg, scheme="none")
    b = np.random.default_rng(3).standard_normal(plan.n)
    y = F.apply(_t(b)).cpu().numpy()
    assert np.linalg.norm(A @ y - b) <= 1e-12 * np.linalg.norm(b)
    x, info = F.pcg(_t(b))
    assert info["iterations"] == 1


@pytest.mark.parametrize("name", ["grf3d_32", "grf3d_64"])
def test_preservation_on_gpu(name):
    # A_l Pi = A Pi (Eq. (preserve-pi)) holds at any size
    cfg = _problem(name)
    plan, F = _gpu(cfg)
    e = cfg["n"][0]
    p = np.arange(plan.n)
    xyz = np.stack([p % e, (p // e) % e, p // (e * e)], 1).astype(float)
    Pi = eval_monomials(xyz, exponents(3, 2))
    for k in range(Pi.shape[1]):
        v = _t(Pi[:, k])
        a = F.apply_forward(v)
        b = F.spmv(v)
        assert torch.linalg.norm(a - b).item() <= 1e-11 * torch.linalg.norm(b).item()


@pytest.mark.parametrize("name", ["poisson2d_64", "grf3d_24", "twophase3d_24", "elastic_12", "gengrf3d_20"])
def test_mixed_precision_error_bound_and_iterations(name):
    # Reading of the mixed-precision policy: the FP32 factor compresses with
    # tau = 1e-6, so it is compared with the FP64 oracle run with the same
    # rank rule; what remains is rounding.  A factorization that is backward
    # stable in a working precision u_p perturbs A_l by ~c u_p ||A||, so the
    # relative forward error of A_l^{-1} v is at most ~kappa(A_l) c u_p, and
    # A_l is spectrally equivalent to A.  With u_p = 8 u32 (3xTF32 products,
    # relative error ~2^-21) and c = 2 the bound is 2^-20 kappa_2(A), kappa_2
    # computed here from A's extreme eigenvalues.  PCG is the same FP64 outer
    # loop, so the iteration count stays within +-1 of the oracle's.
    import scipy.sparse.linalg as spla
    cfg = _problem(name)
    A = assemble(cfg)
    H = build_hierarchy(cfg["n"], cfg["dim"], cfg["leaf"], cfg["stencil"], dof=cfg.get("dof", 1),
                        general=cfg.get("scheme") == "gen_all_all")
    O = factorize(A, H, Options(scheme=cfg.get("scheme", "nest_all_all"), degree=cfg["degree"], order="level",
                                basis=cfg.get("basis", "poly"), tau=1e-6))
    lmax = spla.eigsh(A, k=1, which="LA", return_eigenvectors=False)[0]
    lmin = spla.eigsh(A.tocsc(), k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
    kappa = lmax / lmin
    bound = 2.0 ** -20 * kappa
    plan, F = _gpu(cfg, precision="mixed")
    assert F.precision == "mixed"
    v = np.random.default_rng(5).standard_normal(plan.n)
    y = F.apply(_t(v)).cpu().numpy()
    yo = O.solve(v)
    err = np.linalg.norm(y - yo) / np.linalg.norm(yo)
    b = si.rhs(plan.n, 0)
    x, info = F.pcg(_t(b), rtol=1e-10, maxit=500)
    _, it_o, _ = pcg(lambda q: A @ q, O.solve, b)
    _log({"test": "mixed_apply", "case": name, "kappa2_A": kappa, "apply_err_vs_oracle_tau1e-6": err,
          "bound": bound, "pcg_it": info["iterations"], "oracle_it_tau1e-6": it_o,
          "rel_residual": info["rel_residual"]})
    assert err <= bound
    assert info["rel_residual"] <= 1e-10
    assert abs(info["iterations"] - it_o) <= 1


def test_host_buffer_path():
    cfg = _problem("grf3d_16")
    A, H, O = _oracle(cfg)
    plan = sgf.Plan.from_config(cfg)
    b = si.rhs(plan.n, 2, nrhs=2)
    x, info = sgf.solve_host(plan, cfg["coeffs"].ravel(), b.ravel())
    x = x.reshape(2, -1)
    for j in range(2):
        assert np.linalg.norm(A @ x[j] - b[j]) <= 1e-10 * np.linalg.norm(b[j]) * 1.01


@pytest.mark.slow
def test_full_size_64cube_apply_and_iterations():
    cfg = _problem("grf3d_64")
    A, H, O = _oracle(cfg)
    plan, F = _gpu(cfg)
    v = np.random.default_rng(11).standard_normal(plan.n)
    y = F.apply(_t(v)).cpu().numpy()
    yo = O.solve(v)
    assert np.linalg.norm(y - yo) <= 1e-10 * np.linalg.norm(yo)   # clean rank cuts at 64^3
    b = si.rhs(plan.n, 0)
    x, info = F.pcg(_t(b), rtol=1e-10, maxit=500)
    _, it_o, _ = pcg(lambda q: A @ q, O.solve, b)
    assert abs(info["iterations"] - it_o) <= 1
    assert info["rel_residual"] <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multi_rhs_apply_and_block_pcg_equal_single_rhs(precision):
    # several right-hand sides share one pass over the factor; each must get
    # exactly the single-RHS answer (same arithmetic per RHS)
    cfg = _problem("grf3d_24")
    plan, F = _gpu(cfg, precision=precision)
    rng = np.random.default_rng(9)
    for k in (3, 8, 11):
        X = rng.standard_normal((k, plan.n))
        Y = F.apply(_t(X.ravel())).cpu().numpy().reshape(k, plan.n)
        for j in range(k):
            y1 = F.apply(_t(X[j])).cpu().numpy()
            assert np.array_equal(Y[j], y1)
    B = si.rhs(plan.n, 4, nrhs=5)
    x, info = F.pcg(_t(B.ravel()), rtol=1e-10, maxit=500)
    x = x.cpu().numpy().reshape(5, plan.n)
    assert info["rel_residual"] <= 1e-10
    for j in range(5):
        x1, info1 = F.pcg(_t(B[j]), rtol=1e-10, maxit=500)
        assert np.array_equal(x[j], x1.cpu().numpy())


@pytest.mark.parametrize("name,precision", [("elastic_16", "fp64"), ("elastic_48", "mixed")])
def test_rigid_body_modes_preserved_on_gpu(name, precision):
    # Sec. 7.2: with the rigid-body basis A_l reproduces A on the six modes
    from oracle.basis import eval_rbm
    cfg = _problem(name)
    plan, F = _gpu(cfg, precision=precision)
    nx, ny, nz = cfg["n"]
    p = np.arange(nx * ny * nz)
    xyz = np.stack([p % nx + 1, (p // nx) % ny, p // (nx * ny)], 1).astype(float)
    R = eval_rbm(xyz, (np.array([nx / 2, ny / 2, nz / 2]), float(max(nx, ny, nz))))
    # mixed: tau = 1e-6 truncation, FP32 storage and 3xTF32 tensor-core products
    # (relative error ~2^-21 per product against FP32's 2^-24, so about 8x the
    # FP32-only preservation error of ~3e-5)
    tol = 1e-11 if precision == "fp64" else 1e-3
    worst = 0.0
    for k in range(6):
        v = _t(R[:, k])
        a = F.apply_forward(v)
        b = F.spmv(v)
        err = torch.linalg.norm(a - b).item() / torch.linalg.norm(b).item()
        worst = max(worst, err)
        assert err <= tol
    print(f"{name} {precision}: max relative |A_l r - A r| over the six rigid-body modes {worst:.2e}")
    bvec = _t(si.rhs(plan.n, 0))
    x, info = F.pcg(bvec, rtol=1e-10, maxit=1000)
    assert info["rel_residual"] <= 1e-10


@pytest.mark.gpu
def test_autotune_keeps_a_valid_tuning_and_the_solution():
    # the autotuner only changes launch shapes: the tuned plan solves to the
    # same tolerance in the same number of iterations (+-1)
    cfg = _problem("grf3d_16")
    plan, F = _gpu(cfg, precision="mixed")
    b = _t(si.rhs(plan.n, 0))
    _, info0 = F.pcg(b, rtol=1e-10, maxit=500)
    F.close()
    best, ms = plan.autotune(_t(cfg["coeffs"].ravel()), napply=3)
    assert ms > 0 and plan.tuning == best
    assert best["tensor_cores"] in (1, 2) and 64 <= best["front_small"] <= 512
    assert best["tc_min_dim"] in (32, 64, 128)
    F2 = sgf.Factor(plan, _t(cfg["coeffs"].ravel()))
    _, info1 = F2.pcg(b, rtol=1e-10, maxit=500)
    assert info1["rel_residual"] <= 1e-10
    assert abs(info1["iterations"] - info0["iterations"]) <= 1
    F2.close()


@pytest.mark.slow
def test_full_size_128cube_two_phase_properties():
    # 128^3 high-contrast workload at full size, in the configuration the
    # bench and the examples run: properties that hold at any size - the FP64
    # factor reproduces A on the quadratics (Eq. (preserve-pi)), both
    # precisions reach the 1e-10 residual, and the mixed-precision
    # preconditioner needs about as many iterations as the FP64 one
    cfg = _problem("twophase3d_128")
    e = cfg["n"][0]
    b = _t(si.rhs(e ** 3, 0))
    its = {}
    for precision in ("fp64", "mixed"):
        plan, F = _gpu(cfg, precision=precision)
        if precision == "fp64":
            p = np.arange(plan.n)
            xyz = np.stack([p % e, (p // e) % e, p // (e * e)], 1).astype(float)
            Pi = eval_monomials(xyz, exponents(3, 2))
            for k in range(Pi.shape[1]):
                v = _t(Pi[:, k])
                a, r = F.apply_forward(v), F.spmv(v)
                assert torch.linalg.norm(a - r).item() <= 1e-10 * torch.linalg.norm(r).item()
        x, info = F.pcg(b, rtol=1e-10, maxit=1000)
        assert info["rel_residual"] <= 1e-10
        its[precision] = info["iterations"]
        F.close()
    print(f"128^3 two-phase PCG iterations: {its}")
    assert its["mixed"] <= 1.3 * its["fp64"]


@pytest.mark.parametrize("name", ["rand2d_45_39_4", "rand3d_21_18_13_4", "grf3d_24"])
def test_nest_2_2_matches_oracle(name):
    # Nest-2-2 (Sec. 5.1): ranks equal, apply / multiply within the oracle's
    # own sensitivity, PCG iterations within +-1, and the mixed path converges
    cfg = dict(_problem(name), scheme="nest_2_2")
    A, H, O = _oracle(cfg)
    plan, F = _gpu(cfg)
    assert any(v["adj_cols"] > 0 and v["compressed"] for v in O.comp_info.values())
    for li, lev in enumerate(H.levels[:-1]):
        m, r = F.ranks(li, lev.nnodes)
        for node in range(lev.nnodes):
            if (lev.t, node) in O.comp_info:
                v = O.comp_info[(lev.t, node)]
                assert (m[node], r[node]) == (v["m"], v["r"]), (lev.t, node)
    v = np.random.default_rng(7).standard_normal(plan.n)
    ta, tm = _tolerance(cfg, v)
    yo, zo = O.solve(v), O.multiply(v)
    assert np.linalg.norm(F.apply(_t(v)).cpu().numpy() - yo) <= ta * np.linalg.norm(yo)
    assert np.linalg.norm(F.apply_forward(_t(v)).cpu().numpy() - zo) <= tm * np.linalg.norm(zo)
    b = si.rhs(plan.n, 0)
    _, it_o, _ = pcg(lambda u: A @ u, O.solve, b)
    _, info = F.pcg(_t(b), rtol=1e-10, maxit=500)
    assert abs(info["iterations"] - it_o) <= 1 and info["rel_residual"] <= 1e-10
    F.close()
    _, Fm = _gpu(cfg, precision="mixed")
    _, info = Fm.pcg(_t(b), rtol=1e-10, maxit=500)
    assert info["rel_residual"] <= 1e-10
