"""Pins for oracle/partition.py (Sec. 5.1 nested-dissection partitions)."""
import json
import os

import numpy as np
import pytest

from oracle.partition import axis_separators, build_hierarchy
from oracle.basis import Basis, exponents, eval_monomials, local_coords_poly, frame_poly

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_axis_separator_rule():
    assert axis_separators(64, 8) == [7, 15, 23, 31, 39, 47, 55]
    assert axis_separators(64, 16) == [15, 31, 47]
    assert axis_separators(64, 64) == []
    # the last separator is dropped when fewer than d/2 unknowns follow it
    assert axis_separators(35, 8) == [7, 15, 23]
    assert axis_separators(36, 8) == [7, 15, 23, 31]
    assert axis_separators(7, 8) == []


def _closed_form_counts(N, d, dim):
    """Cell counts of a d-spaced cut of an N^dim box: k separators, k+1 intervals."""
    k = len(axis_separators(N, d))
    iv = k + 1
    from math import comb
    return {c: comb(dim, c) * iv ** c * k ** (dim - c) for c in range(dim + 1)}


@pytest.mark.parametrize("N,dim,b", [(64, 3, 8), (37, 3, 8), (64, 2, 16), (29, 2, 4)])
def test_level_cell_counts_match_closed_form(N, dim, b):
    n = (N, N, N) if dim == 3 else (N, N, 1)
    H = build_hierarchy(n, dim, b, "7pt_fv_3d" if dim == 3 else "5pt_2d")
    for lev in H.levels:
        if lev.top:
            assert lev.nnodes == 1
            continue
        counts = _closed_form_counts(N, lev.d, dim)
        got = np.bincount(lev.cell_dim, minlength=dim + 1)
        assert {c: int(got[c]) for c in range(dim + 1)} == counts


def test_golden_counts_64_cube():
    with open(os.path.join(GOLDEN, "nd_counts_64cube_b8.json")) as f:
        g = json.load(f)
    H = build_hierarchy((64, 64, 64), 3, 8, "7pt_fv_3d")
    for lev, want in zip(H.levels, g["levels"]):
        got = np.bincount(lev.cell_dim, minlength=4).tolist() if not lev.top else "top"
        assert got == want


def test_cells_partition_points_and_nest():
    H = build_hierarchy((23, 19, 17), 3, 4, "7pt_fv_3d")
    lev1 = H.levels[0]
    allp = np.concatenate(lev1.points)
    assert np.array_equal(np.sort(allp), np.arange(23 * 19 * 17))
    for li in range(1, len(H.levels)):
        lev, prev = H.levels[li], H.levels[li - 1]
        seen = []
        for D, kids in enumerate(lev.children):
            for C in kids:
                assert not prev.interior[C]
                assert np.all(prev.box[C, 0] >= lev.box[D, 0]) and np.all(prev.box[C, 1] <= lev.box[D, 1])
                seen.append(C)
        assert sorted(seen) == prev.separators()


def test_interiors_touch_only_separators_and_interior_size():
    H = build_hierarchy((32, 32, 32), 3, 8, "7pt_fv_3d")
    lev = H.levels[0]
    for u, v in lev.pattern:
        assert not (lev.interior[u] and lev.interior[v])
    # a full 3-cell holds (d-1)^3 grid vertices (Sec. 5.1)
    sizes = [len(lev.points[i]) for i in lev.interiors()]
    assert min(sizes) == 7 ** 3


def test_reexpansion_is_exact_change_of_polynomial_basis():
    rng = np.random.default_rng(0)
    for dim, deg, kind, dof in [(3, 2, "poly", 1), (2, 2, "poly", 1), (3, 1, "poly", 3), (3, 1, "rbm", 3)]:
        B = Basis(dim, deg, kind, dof)
        for _ in range(5):
            lo = rng.integers(0, 10, 3)
            hi = lo + rng.integers(0, 6, 3)
            if dim == 2:
                lo[2] = hi[2] = 0
            child = np.array([lo, hi])
            plo = lo - rng.integers(0, 5, 3)
            phi_ = hi + rng.integers(0, 5, 3)
            if dim == 2:
                plo[2] = phi_[2] = 0
            parent = np.array([plo, phi_])
            g = np.stack(np.meshgrid(*[np.arange(lo[a], hi[a] + 1) for a in range(3)], indexing="ij"), -1)
            xyz = g.reshape(-1, 3).astype(float)
            lhs = B.evaluate(xyz, parent)
            rhs = B.evaluate(xyz, child) @ B.reexpansion(child, parent)
            assert np.abs(lhs - rhs).max() < 1e-12


def test_local_basis_spans_global_monomials():
    # on any cell, local and global monomials of degree <= 2 span the same space
    xyz = np.stack(np.meshgrid(np.arange(3, 8), np.arange(10, 13), np.arange(4, 9), indexing="ij"), -1).reshape(-1, 3).astype(float)
    box = np.array([[3, 10, 4], [7, 12, 8]])
    loc = eval_monomials(local_coords_poly(xyz, frame_poly(box)), exponents(3, 2))
    glo = eval_monomials(xyz, exponents(3, 2))
    X, *_ = np.linalg.lstsq(loc, glo, rcond=None)
    assert np.abs(loc @ X - glo).max() < 1e-9 * np.abs(glo).max()


@pytest.mark.parametrize("n,dim,b", [((20, 18, 16), 3, 4), ((23, 19, 1), 2, 5), ((15, 15, 15), 3, 5)])
def test_general_partition_cells(n, dim, b):
    # Gen-All-All partitions (Sec. 5.2): level t has ceil(N / d) cells per axis
    # of d = b 2^(t-1) consecutive vertices, none interior, all of full
    # dimension; every point lies in one level-1 cell; a cell's children are
    # the level-(t-1) cells inside it; the top is the first single-cell level
    H = build_hierarchy(n, dim, b, "7pt_fv_3d" if dim == 3 else "5pt_2d", general=True)
    N = [n[0], n[1], n[2] if dim == 3 else 1]
    npts = N[0] * N[1] * N[2]
    assert sorted(np.concatenate(H.levels[0].points).tolist()) == list(range(npts))
    for li, lev in enumerate(H.levels):
        d = b * 2 ** li
        K = [-(-N[a] // d) if N[a] > 1 else 1 for a in range(3)]
        if lev.top:
            assert lev.nnodes == 1 and all(k == 1 for k in K)
            continue
        assert lev.nnodes == K[0] * K[1] * K[2]
        assert not lev.interior.any() and (lev.cell_dim == dim).all()
        sizes = [(lev.box[i, 1] - lev.box[i, 0] + 1) for i in range(lev.nnodes)]
        for sz in sizes:
            assert all(1 <= sz[a] <= d for a in range(3))
        if li == 0:
            assert [len(p) for p in lev.points] == [int(np.prod(sz)) for sz in sizes]
        else:
            prev = H.levels[li - 1]
            for D, kids in enumerate(lev.children):
                assert 1 <= len(kids) <= 2 ** dim
                for c in kids:   # child box inside the parent box
                    assert (prev.box[c, 0] >= lev.box[D, 0]).all() and (prev.box[c, 1] <= lev.box[D, 1]).all()
            assert sorted(c for k in lev.children for c in k) == list(range(prev.nnodes))
