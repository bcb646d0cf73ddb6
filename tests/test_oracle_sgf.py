"""Pins for the SGF oracle (Algorithm 4.1) against what the paper fixes.

P1  compression off => exact block Cholesky (Sec. 2.1: without compression the
    factorization is an exact block Cholesky decomposition).
P2  A_l Pi = A Pi (Eq. (preserve-pi), Prop. 6.1) and, per level,
    E_i Pi_B = 0 for B in P_k, i <= k.
P3  Q2^T N = 0 up to the rank tolerance (Eq. (QR)).
P4  SPD: positive pivots, positive spectrum of A_l (Lemma 3.1).
P5  explicit dense G_i, B_i restatement reproduces A_l (Sec. 2.1, Eq. (M')).
P6  compressions inside a level commute (random order == canonical order).
P7  trends: near-flat CG counts in n; higher degree => fewer iterations;
    E_n = ||(A - A_l) v_n|| / lambda_n stays O(1) (Table 5.1).
Gen-All-All (Sec. 5.2): P1, P2/P4 and P5 on general partitions.
Nest-2-2 (Sec. 5.1): blocks to touching lower-dimensional separators kept
    exactly (Q2^T M^_BE = 0), P2/P4, level-1 ranks not below Nest-2-All's,
    the paper's accuracy order of the nested schemes, and P5.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import sgf_inputs as si
from oracle.assemble import assemble, assemble_scalar
from oracle.basis import eval_monomials, exponents
from oracle.dense import dense_sgf
from oracle.partition import build_hierarchy
from oracle.pcg import pcg
from oracle.sgf import Options, factorize, dof_list


def _grid_problem(n, dim, b, stencil, seed=0, weight=1.0, dmask=None, general=False):
    rng = np.random.default_rng(seed)
    shape = (n[1], n[0]) if dim == 2 else (n[2], n[1], n[0])
    k = np.exp(rng.standard_normal(shape))
    if dmask is None:
        dmask = 15 if dim == 2 else 1
    A = assemble_scalar(n, dim, k, dmask, weight)
    H = build_hierarchy(n, dim, b, stencil, general=general)
    return A, H


def _global_poly(H, degree):
    nx, ny, nz = H.n
    p = np.arange(nx * ny * nz)
    xyz = np.stack([p % nx, (p // nx) % ny, p // (nx * ny)], 1).astype(float)
    return eval_monomials(xyz, exponents(H.dim, degree))


def _elimination_order(F):
    """DOF ids in elimination order when nothing is compressed."""
    H = F.H
    vars_ = {i: list(v) for i, v in enumerate(F.vars1)}
    order = []
    for li, lev in enumerate(H.levels):
        if lev.top:
            order += vars_[0]
            break
        for I in lev.interiors():
            order += vars_[I]
        nxt = H.levels[li + 1]
        vars_ = {D: [q for C in kids for q in vars_[C]] for D, kids in enumerate(nxt.children)}
    return np.array(order)


@pytest.mark.parametrize("n,dim,b,st", [((29, 23, 1), 2, 4, "5pt_2d"), ((13, 11, 9), 3, 4, "7pt_fv_3d")])
def test_P1_no_compression_is_exact_block_cholesky(n, dim, b, st):
    A, H = _grid_problem(n, dim, b, st, weight=2.0 if dim == 3 else 1.0)
    F = factorize(A, H, Options(scheme="none", degree=1))
    perm = _elimination_order(F)
    assert np.array_equal(np.sort(perm), np.arange(A.shape[0]))
    Lfull = sla.cholesky(A.toarray()[np.ix_(perm, perm)], lower=True)
    pos = np.empty_like(perm)
    pos[perm] = np.arange(perm.size)
    # rebuild the DOF lists of every node to locate each factor block in Lfull
    vars_ = {i: list(v) for i, v in enumerate(F.vars1)}
    lev_i = 0
    scale = np.abs(Lfull).max()
    for op in F.ops:
        if op[0] == "elim":
            _, t, I, L, S_list, W = op
            pi = pos[vars_[I]]
            assert np.abs(Lfull[np.ix_(pi, pi)] - L).max() <= 1e-13 * scale
            for S, Ws in zip(S_list, W):
                ps = pos[vars_[S]]
                assert np.abs(Lfull[np.ix_(ps, pi)] - Ws.T).max() <= 1e-13 * scale
        elif op[0] == "merge":
            vars_ = {D: [q for C in kids for q in vars_[C]] for D, kids, _ in op[2]}
        elif op[0] == "top":
            pt = pos[vars_[0]]
            assert np.abs(Lfull[np.ix_(pt, pt)] - op[1]).max() <= 1e-13 * scale
    rng = np.random.default_rng(1)
    b_ = rng.standard_normal(A.shape[0])
    assert np.linalg.norm(F.solve(b_) - sla.solve(A.toarray(), b_)) <= 1e-12 * np.linalg.norm(sla.solve(A.toarray(), b_))
    x, it, res = pcg(lambda v: A @ v, F.solve, b_)
    assert it == 1 and res < 1e-12


@pytest.mark.parametrize("name,deg", [("poisson2d_64", 1), ("grf3d_24", 2), ("twophase3d_24", 2)])
def test_P2_preserves_action_on_polynomials(name, deg):
    cfg = si.config(name)
    A = assemble(cfg)
    H = build_hierarchy(cfg["n"], cfg["dim"], cfg["leaf"], cfg["stencil"])
    F = factorize(A, H, Options(degree=deg))
    assert any(v[2] for v in F.ranks().values()), "some node must actually compress"
    Pi = _global_poly(H, deg)
    AP = A @ Pi
    err = np.linalg.norm(np.stack([F.multiply(Pi[:, k]) for k in range(Pi.shape[1])], 1) - AP)
    assert err <= 1e-12 * np.linalg.norm(AP)


def test_P2_per_level_error_annihilates_level_polynomials():
    A, H = _grid_problem((23, 21, 1), 2, 4, "5pt_2d", seed=4)
    opts = Options(degree=0)
    Al, approx, ranks = dense_sgf(A, H, opts)
    assert any(v[2] for v in ranks.values())
    Ad = A.toarray()
    prev = Ad
    errs = []
    for k, Ak in enumerate(approx):
        errs.append(Ak - prev)
        prev = Ak
    Pi = _global_poly(H, 0)
    nx = H.n[0]
    for k, lev in enumerate(H.levels[:-1]):
        for B in range(lev.nnodes):
            lo, hi = lev.box[B]
            p = np.arange(Ad.shape[0])
            inside = (p % nx >= lo[0]) & (p % nx <= hi[0]) & (p // nx >= lo[1]) & (p // nx <= hi[1])
            PiB = Pi * inside[:, None]
            for i in range(k + 1):
                assert np.abs(errs[i] @ PiB).max() <= 1e-11 * np.abs(Ad).max() * np.abs(Pi).max()


def test_P3_Q2_annihilates_filtered_interaction_matrix():
    cfg = si.config("grf3d_24")
    A = assemble(cfg)
    H = build_hierarchy(cfg["n"], 3, 8, cfg["stencil"])
    F = factorize(A, H, Options(degree=2))
    for info in F.comp_info.values():
        assert info["q2n"] <= 10 * 1e-12 * info["nnorm"]


def test_P4_spd_pivots_and_spectrum():
    A, H = _grid_problem((19, 17, 1), 2, 4, "5pt_2d", seed=2)
    F = factorize(A, H, Options(degree=1))
    assert F.pivots_min > 0
    Al = F.dense_operator()
    assert np.abs(Al - Al.T).max() <= 1e-12 * np.abs(Al).max()
    assert np.linalg.eigvalsh(0.5 * (Al + Al.T))[0] > 0


@pytest.mark.parametrize("n,seed,deg", [((15, 15, 1), 0, 0), ((17, 13, 1), 3, 1), ((19, 17, 1), 0, 2)])
def test_P5_dense_brute_force_reproduces_block_oracle(n, seed, deg):
    A, H = _grid_problem(n, 2, 4, "5pt_2d", seed=seed)
    F = factorize(A, H, Options(degree=deg))
    Ad, _, ranks = dense_sgf(A, H, Options(degree=deg))
    assert ranks == F.ranks()
    assert any(v[2] for v in ranks.values())
    Al = F.dense_operator()
    assert np.abs(Al - Ad).max() <= 1e-12 * np.abs(Ad).max()
    Ainv = F.dense_inverse()
    assert np.abs(Ainv @ Ad - np.eye(Ad.shape[0])).max() <= 1e-10


def test_P6_compression_order_inside_a_level_does_not_matter():
    cfg = si.config("grf3d_24")
    A = assemble(cfg)
    H = build_hierarchy(cfg["n"], 3, 8, cfg["stencil"])
    F1 = factorize(A, H, Options(degree=2))
    F2 = factorize(A, H, Options(degree=2), order_seed=7)
    assert F1.ranks() == F2.ranks()
    rng = np.random.default_rng(0)
    for _ in range(2):
        v = rng.standard_normal(A.shape[0])
        a, b = F1.solve(v), F2.solve(v)
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)
        a, b = F1.multiply(v), F2.multiply(v)
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)


@pytest.mark.parametrize("name", ["grf3d_24", "twophase3d_24"])
def test_P6_level_reading_matches_sequential_recursion(name):
    # All compressions of a level from the post-elimination matrix (the form
    # the device path batches) against the paper's node-after-node recursion:
    # identical when Q2^T N vanishes, so they agree to rounding here.
    cfg = si.config(name)
    A = assemble(cfg)
    H = build_hierarchy(cfg["n"], 3, 8, cfg["stencil"])
    F1 = factorize(A, H, Options(degree=2))
    F2 = factorize(A, H, Options(degree=2, order="level"))
    assert F1.ranks() == F2.ranks()
    v = np.random.default_rng(2).standard_normal(A.shape[0])
    a, b = F1.solve(v), F2.solve(v)
    assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(a)
    Pi = _global_poly(H, 2)
    AP = A @ Pi
    err = np.linalg.norm(np.stack([F2.multiply(Pi[:, k]) for k in range(Pi.shape[1])], 1) - AP)
    assert err <= 1e-12 * np.linalg.norm(AP)


def test_P7_iteration_trends_and_smooth_eigenvector_accuracy():
    its = {}
    for e in (16, 32):
        cfg = si.config(f"poisson3d_{e}")
        A = assemble(cfg)
        H = build_hierarchy(cfg["n"], 3, 8, cfg["stencil"])
        for deg in (0, 2):
            F = factorize(A, H, Options(degree=deg))
            _, it, res = pcg(lambda v: A @ v, F.solve, si.rhs(A.shape[0], 0))
            assert res <= 1e-10
            its[(e, deg)] = it
            if deg == 2:
                x = np.arange(1, e + 1)
                s = np.sin(np.pi * x / (e + 1))
                vn = np.einsum("i,j,k->ijk", s, s, s).ravel()
                vn /= np.linalg.norm(vn)
                lam = 3 * (2 - 2 * np.cos(np.pi / (e + 1)))
                En = np.linalg.norm(A @ vn - F.multiply(vn)) / lam
                assert En < 2.0          # Table 5.1 reports O(1) values for pcw. quad.
    assert its[(32, 2)] <= its[(16, 2)] + 8
    assert its[(16, 2)] < its[(16, 0)] and its[(32, 2)] < its[(32, 0)]


def test_pcg_finite_termination_and_exact_preconditioner():
    # CG on an SPD matrix with k distinct eigenvalues ends in k steps (exactly,
    # up to rounding); with the exact inverse as preconditioner it ends in one.
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    ev = np.repeat([1.0, 3.0, 7.0, 20.0], 10)
    A = Q @ np.diag(ev) @ Q.T
    b = rng.standard_normal(40)
    _, it, res = pcg(lambda v: A @ v, lambda v: v, b, rtol=1e-10)
    assert it == 4 and res < 1e-10
    Ainv = np.linalg.inv(A)
    _, it, res = pcg(lambda v: A @ v, lambda v: Ainv @ v, b, rtol=1e-10)
    assert it == 1
    x1, it1, _ = pcg(lambda v: A @ v, lambda v: v / ev.mean(), b, flexible=True)
    x2, it2, _ = pcg(lambda v: A @ v, lambda v: v / ev.mean(), b, flexible=False)
    assert it1 == it2 and np.allclose(x1, x2, rtol=1e-8)


# ---- Gen-All-All (Sec. 5.2): general partitions, compression only --------

@pytest.mark.parametrize("n,dim,b", [((17, 15, 1), 2, 4), ((10, 9, 8), 3, 3)])
def test_gen_P1_no_compression_is_exact(n, dim, b):
    # without interiors and without compression nothing happens before the
    # top level, whose dense Cholesky is exact: A_l = A
    A, H = _grid_problem(n, dim, b, "5pt_2d" if dim == 2 else "7pt_fv_3d", seed=1, general=True)
    F = factorize(A, H, Options(scheme="none", degree=1))
    Al = F.dense_operator()
    Ad = A.toarray()
    assert np.abs(Al - Ad).max() <= 1e-12 * np.abs(Ad).max()


@pytest.mark.parametrize("n,dim,b,deg", [((24, 21, 1), 2, 4, 1), ((16, 15, 14), 3, 4, 1), ((20, 20, 20), 3, 5, 2)])
def test_gen_P2_P4_preserves_polynomials_and_stays_spd(n, dim, b, deg):
    A, H = _grid_problem(n, dim, b, "5pt_2d" if dim == 2 else "7pt_fv_3d", seed=2, general=True)
    F = factorize(A, H, Options(scheme="gen_all_all", degree=deg))
    assert F.pivots_min > 0
    assert any(v[2] for v in F.ranks().values()), "some node must actually compress"
    Pi = _global_poly(H, deg)
    AP = A @ Pi
    err = np.linalg.norm(np.stack([F.multiply(Pi[:, k]) for k in range(Pi.shape[1])], 1) - AP)
    assert err <= 1e-12 * np.linalg.norm(AP)


@pytest.mark.parametrize("n,seed,deg", [((20, 17, 1), 0, 0), ((23, 19, 1), 3, 1)])
def test_gen_P5_dense_brute_force_reproduces_block_oracle(n, seed, deg):
    A, H = _grid_problem(n, 2, 4, "5pt_2d", seed=seed, general=True)
    opts = Options(scheme="gen_all_all", degree=deg)
    F = factorize(A, H, opts)
    Ad, _, ranks = dense_sgf(A, H, opts)
    assert ranks == F.ranks()
    assert any(v[2] for v in ranks.values())
    Al = F.dense_operator()
    assert np.abs(Al - Ad).max() <= 1e-12 * np.abs(Ad).max()
    assert np.linalg.eigvalsh(0.5 * (Ad + Ad.T))[0] > 0


# --------------------------------------------------------------------------
# Nest-2-2 (Sec. 5.1): codimension-1 separators compressed with the span of
# their blocks to the touching lower-dimensional separators added to Q1, so
# only their interactions with non-adjacent cells are compressed; the paper
# ranks it the most accurate nested scheme.
# --------------------------------------------------------------------------
def _grf24(scheme):
    cfg = si.config("grf3d_24")
    A = assemble(cfg)
    H = build_hierarchy(cfg["n"], 3, 8, cfg["stencil"])
    return A, H, factorize(A, H, Options(degree=2, scheme=scheme))


def test_n22_adjacent_blocks_are_kept_exactly_and_polynomials_preserved():
    A, H, F = _grf24("nest_2_2")
    with_adj = [i for i in F.comp_info.values() if i["adj_cols"] > 0 and i["compressed"]]
    assert with_adj, "some compressed node must touch a lower-dimensional separator"
    for i in with_adj:   # Q2^T M^_BE = 0: the fine part does not see E
        assert i["adj_q2"] <= 1e-12 * i["adj_norm"]
    assert F.pivots_min > 0
    Pi = _global_poly(H, 2)
    AP = A @ Pi
    err = np.linalg.norm(np.stack([F.multiply(Pi[:, k]) for k in range(Pi.shape[1])], 1) - AP)
    assert err <= 1e-12 * np.linalg.norm(AP)


def test_n22_level_one_ranks_contain_nest_2_all_ranks():
    # at level 1 both schemes compress the same nodes of the same matrix and
    # Nest-2-2's N holds Nest-2-All's columns plus more: its rank is not lower
    _, H, F2 = _grf24("nest_2_all")
    _, _, F22 = _grf24("nest_2_2")
    r2, r22 = F2.ranks(), F22.ranks()
    lvl1 = [k for k in r2 if k[0] == 1]
    assert lvl1
    assert all(r22[k][1] >= r2[k][1] for k in lvl1)
    assert any(r22[k][1] > r2[k][1] for k in lvl1)


def test_n22_most_accurate_of_the_nested_schemes():
    # Sec. 5.1 orders the schemes Nest-All-All < Nest-2-All < Nest-2-2 in
    # accuracy: fewer PCG iterations, and a smaller condition number of
    # A_l^{-1} A on a grid small enough to form both densely
    A, H, _ = _grf24("nest_2_2")
    b = si.rhs(A.shape[0], 0)
    its = {}
    for sch in ("nest_all_all", "nest_2_all", "nest_2_2"):
        F = factorize(A, H, Options(degree=2, scheme=sch))
        _, its[sch], res = pcg(lambda v: A @ v, F.solve, b, rtol=1e-10)
        assert res <= 1e-10
    assert its["nest_2_2"] < its["nest_2_all"] <= its["nest_all_all"]
    A, H = _grid_problem((13, 11, 9), 3, 4, "7pt_fv_3d", seed=1)
    Ad = A.toarray()
    cond = {}
    for sch in ("nest_2_all", "nest_2_2"):
        ev = sla.eigvalsh(Ad, factorize(A, H, Options(degree=1, scheme=sch)).dense_operator())
        cond[sch] = ev.max() / ev.min()
    assert cond["nest_2_2"] < cond["nest_2_all"]


def test_n22_dense_brute_force_reproduces_block_oracle():
    A, H = _grid_problem((13, 11, 9), 3, 4, "7pt_fv_3d", seed=1)
    opts = Options(scheme="nest_2_2", degree=1)
    F = factorize(A, H, opts)
    Ad, _, ranks = dense_sgf(A, H, opts)
    assert ranks == F.ranks()
    assert ranks != factorize(A, H, Options(scheme="nest_2_all", degree=1)).ranks()
    Al = F.dense_operator()
    assert np.abs(Al - Ad).max() <= 1e-12 * np.abs(Ad).max()
    assert np.linalg.eigvalsh(0.5 * (Ad + Ad.T))[0] > 0


def test_P5_catches_a_scheme_selection_mistake(monkeypatch):
    # the dense restatement selects the compressed cells on its own (from the
    # cells' geometry); a wrong selection rule in the block oracle shows up
    import oracle.sgf as osgf
    A, H = _grid_problem((13, 11, 9), 3, 4, "7pt_fv_3d", seed=1)
    opts = Options(scheme="nest_2_all", degree=1)
    Ad, _, ranks = dense_sgf(A, H, opts)
    assert ranks == factorize(A, H, opts).ranks()
    good = osgf._eligible

    def wrong(lev, i, dim, o):   # Nest-2-All mistaken for Nest-All-All
        return good(lev, i, dim, Options(scheme="nest_all_all", tau=o.tau, degree=o.degree))
    monkeypatch.setattr(osgf, "_eligible", wrong)
    assert factorize(A, H, opts).ranks() != ranks

