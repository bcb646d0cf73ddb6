"""C-ABI library: exported symbols and bit-exact symbolic analysis vs the oracle.

sgf_analyze is host code (Sec. 5.1 partitions, Defs. 2.1-2.4), so the
comparison with oracle/partition.py runs without a GPU.
"""
import os
import re

import numpy as np
import pytest

import paper_1907_03406_gb300 as sgf
from paper_1907_03406_gb300 import _lib
from oracle.partition import build_hierarchy

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    txt = open(os.path.join(ROOT, "include", "sgf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sgf_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = _header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding misses {name}"


CASES = [
    ((64, 64, 1), 2, 16, "5pt_2d"),
    ((29, 23, 1), 2, 4, "5pt_2d"),
    ((16, 16, 16), 3, 8, "7pt_fv_3d"),
    ((37, 29, 23), 3, 8, "7pt_fv_3d"),
    ((64, 64, 64), 3, 8, "7pt_fv_3d"),
    ((7, 7, 7), 3, 8, "7pt_3d"),
    ((12, 13, 13), 3, 4, "q1_elastic_3d"),
    ((20, 20, 20), 3, 5, "gen"),
    ((24, 23, 17), 3, 5, "gen"),
    ((23, 19, 1), 2, 4, "gen"),
]


@pytest.mark.parametrize("n,dim,b,st", CASES)
def test_symbolic_analysis_bit_exact(n, dim, b, st):
    elastic = st == "q1_elastic_3d"
    general = st == "gen"   # general partitions (Gen-All-All)
    if general:
        st = "7pt_fv_3d" if dim == 3 else "5pt_2d"
    H = build_hierarchy(n, dim, b, st, dof=3 if elastic else 1, general=general)
    if elastic:
        P = sgf.Plan(n, dim, st, 1, b, 1, basis=1, dof=3)
    elif general:
        P = sgf.Plan(n, dim, st, 1, b, 2 if dim == 3 else 1, scheme="gen_all_all")
    else:
        P = sgf.Plan(n, dim, st, 1, b, 2 if dim == 3 else 1)
    assert P.nlevels == len(H.levels)
    for li, lev in enumerate(H.levels):
        ex = P.export_level(li)
        assert ex["nnodes"] == lev.nnodes
        if lev.top:
            if li > 0:
                assert ex["child_idx"].tolist() == lev.children[0]
            continue
        assert [tuple(c) for c in ex["codes"].tolist()] == [tuple(c) for c in lev.codes]
        assert ex["interior"].tolist() == lev.interior.tolist()
        assert ex["cell_dim"].tolist() == lev.cell_dim.tolist()
        assert [tuple(p) for p in ex["pairs"].tolist()] == list(lev.pattern)
        assert [tuple(p) for p in ex["post"].tolist()] == list(lev.post_pattern)
        if li > 0:
            kids = [ex["child_idx"][ex["child_ptr"][i]:ex["child_ptr"][i + 1]].tolist() for i in range(lev.nnodes)]
            assert kids == lev.children
        # Nest-All-All eligibility: separators of dimension >= 1; Gen-All-All: every node
        want = (~lev.interior) & (lev.cell_dim >= 1)
        assert ex["eligible"].tolist() == want.tolist()
        if general:
            assert not lev.interior.any()


@pytest.mark.parametrize("scheme", ["nest_all_all", "nest_2_all", "nest_2_2", "none"])
@pytest.mark.parametrize("n,dim,b,st", [((37, 29, 23), 3, 8, "7pt_fv_3d"), ((41, 37, 1), 2, 4, "5pt_2d")])
def test_eligibility_per_scheme_matches_oracle(scheme, n, dim, b, st):
    from oracle.sgf import Options, _eligible
    H = build_hierarchy(n, dim, b, st)
    P = sgf.Plan(n, dim, st, 1, b, 1, scheme=scheme)
    opts = Options(scheme=scheme)
    for li, lev in enumerate(H.levels):
        if lev.top:
            continue
        ex = P.export_level(li)
        want = [_eligible(lev, i, dim, opts) and not lev.interior[i] for i in range(lev.nnodes)]
        assert [bool(v) for v in ex["eligible"].tolist()] == want


def test_analyze_rejects_bad_arguments():
    with pytest.raises(sgf.SGFError):
        sgf.Plan((16, 16, 16), 3, "7pt_fv_3d", 1, 1, 2)      # leaf < 2
    with pytest.raises(sgf.SGFError):
        sgf.Plan((16, 16, 16), 3, "7pt_fv_3d", 1, 8, 3)      # degree 3
    with pytest.raises(sgf.SGFError):
        sgf.Plan((16, 16, 1), 2, "7pt_fv_3d", 1, 8, 1)       # stencil / dim mismatch


def test_footprint_is_positive_and_mixed_is_smaller():
    P = sgf.Plan((32, 32, 32), 3, "7pt_fv_3d", 1, 8, 2)
    a, b = P.footprint()
    assert a > b > 0


def test_tuning_round_trip_and_validation():
    P = sgf.Plan((16, 16, 16), 3, "7pt_fv_3d", 1, 8, 2, precision="mixed")
    assert P.tuning == {"gemv_min_elems": 4096, "gemv_max_elems": 32768, "front_small": 512, "tensor_cores": 1,
                        "gemv_cols": 32, "tc_min_dim": 64}
    P.tuning = {"gemv_min_elems": 1024, "front_small": 256, "tensor_cores": 0, "gemv_cols": 64, "tc_min_dim": 128}
    assert P.tuning == {"gemv_min_elems": 1024, "gemv_max_elems": 32768, "front_small": 256, "tensor_cores": 0,
                        "gemv_cols": 64, "tc_min_dim": 128}
    for bad in ({"gemv_min_elems": 100}, {"gemv_min_elems": 65536, "gemv_max_elems": 4096},
                {"front_small": 1024}, {"front_small": 32}, {"tensor_cores": 3}, {"tensor_cores": -1},
                {"gemv_cols": 48}, {"tc_min_dim": 0}, {"tc_min_dim": 5000}):
        with pytest.raises(sgf.SGFError):
            P.tuning = bad
    assert P.tuning["front_small"] == 256      # unchanged by the rejected calls
