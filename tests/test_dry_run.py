"""Host-only validation of every batched task the factor driver builds.

With SGF_DRY_RUN=1 the library makes no CUDA call: allocations are address
ranges, and each launch wrapper checks that every task reads and writes inside
one live allocation (see devmem.h).  This runs the whole level-by-level
driver (elimination fronts, Schur targets, compression, two-sided transforms,
merge, top) and both apply programs on grids with ragged tiles, empty
interiors and compressed / uncompressed separators.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import ctypes as C, json, sys
sys.path.insert(0, %r)
import paper_1907_03406_gb300 as sgf
from paper_1907_03406_gb300 import _lib
lib = _lib.load()
out = []
for case in json.loads(sys.argv[1]):
    (n, dim, st, dm, leaf, deg, prec, scheme) = case[:8]
    el = st == "q1_elastic_3d"
    P = sgf.Plan(tuple(n), dim, st, dm, leaf, deg, precision=prec, scheme=scheme,
                 basis=1 if el else 0, dof=3 if el else 1)
    if len(case) > 8:
        P.tuning = case[8]      # non-default launch shapes
    lib.sgf_dry_run_violations(1)
    h = C.c_void_p()
    rc = lib.sgf_factor(P.handle, C.c_void_p(4096), None, C.byref(h))
    rc2 = lib.sgf_apply(h, C.c_void_p(8192), C.c_void_p(16384), 1, None) if rc == 0 else -99
    rc3 = lib.sgf_apply_forward(h, C.c_void_p(8192), C.c_void_p(16384), 1, None) if rc == 0 else -99
    for nrhs in (2, 3, 8, 11):     # interleaved multi-RHS programs
        if rc == 0:
            rc2 = rc2 or lib.sgf_apply(h, C.c_void_p(8192), C.c_void_p(16384), nrhs, None)
    v = lib.sgf_dry_run_violations(0)
    rep = lib.sgf_dry_run_report().decode()
    if rc == 0:
        lib.sgf_factor_destroy(h)
    out.append(dict(case=[n, dim, st, prec, scheme], rc=[rc, rc2, rc3], violations=v, report=rep,
                    err=lib.sgf_last_error().decode()))
print("JSON" + json.dumps(out))
"""

CASES = [
    [[64, 64, 1], 2, "5pt_2d", 15, 16, 1, "fp64", "nest_all_all"],
    [[29, 23, 1], 2, "5pt_2d", 15, 4, 1, "fp64", "nest_all_all"],
    [[24, 24, 24], 3, "7pt_fv_3d", 1, 8, 2, "fp64", "nest_all_all"],
    [[37, 29, 23], 3, "7pt_fv_3d", 1, 8, 2, "mixed", "nest_all_all"],
    [[21, 18, 13], 3, "7pt_fv_3d", 1, 4, 2, "fp64", "nest_2_all"],
    [[21, 18, 13], 3, "7pt_fv_3d", 1, 4, 1, "fp64", "none"],
    [[7, 7, 7], 3, "7pt_3d", 63, 8, 2, "fp64", "nest_all_all"],
    [[130, 67, 1], 2, "5pt_2d", 15, 8, 2, "mixed", "nest_all_all"],
    [[12, 13, 13], 3, "q1_elastic_3d", 1, 4, 1, "fp64", "nest_all_all"],
    [[24, 25, 25], 3, "q1_elastic_3d", 1, 8, 1, "mixed", "nest_all_all"],
    [[20, 20, 20], 3, "7pt_fv_3d", 1, 5, 2, "fp64", "gen_all_all"],
    [[24, 23, 17], 3, "7pt_fv_3d", 1, 5, 2, "mixed", "gen_all_all"],
    [[23, 19, 1], 2, "5pt_2d", 15, 4, 1, "fp64", "gen_all_all"],
    [[37, 29, 23], 3, "7pt_fv_3d", 1, 8, 2, "mixed", "nest_2_2"],
    [[21, 18, 13], 3, "7pt_fv_3d", 1, 4, 1, "fp64", "nest_2_2"],
    [[41, 37, 1], 2, "5pt_2d", 15, 4, 1, "fp64", "nest_2_2"],
    [[37, 29, 23], 3, "7pt_fv_3d", 1, 8, 2, "mixed", "nest_all_all",
     {"gemv_min_elems": 256, "gemv_max_elems": 1024, "front_small": 64, "tensor_cores": 0, "gemv_cols": 64}],
    [[37, 29, 23], 3, "7pt_fv_3d", 1, 8, 2, "fp64", "nest_all_all",
     {"gemv_min_elems": 65536, "gemv_max_elems": 1 << 20, "front_small": 512, "tensor_cores": 1}],
    [[37, 29, 23], 3, "7pt_fv_3d", 1, 8, 2, "mixed", "nest_all_all", {"tensor_cores": 2, "tc_min_dim": 1}],
    # the bench's recipe at realistic sizes (many levels, thousands of
    # compressed separators, the padded apply blocks)
    [[64, 64, 64], 3, "7pt_fv_3d", 1, 8, 2, "mixed", "nest_all_all"],
    [[48, 48, 48], 3, "7pt_fv_3d", 1, 8, 2, "fp64", "nest_all_all"],
    [[24, 25, 25], 3, "q1_elastic_3d", 1, 8, 1, "mixed", "nest_all_all", {"tensor_cores": 1, "tc_min_dim": 200}],
]


def test_dry_run_has_no_out_of_range_task():
    env = dict(os.environ, SGF_DRY_RUN="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT % ROOT, json.dumps(CASES)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("JSON")][-1]
    res = json.loads(line[4:])
    for c in res:
        assert c["rc"] == [0, 0, 0], c
        assert c["violations"] == 0, c
