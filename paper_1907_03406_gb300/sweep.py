"""Size sweep of the solver on one GPU: by default 3D Poisson (7-point
stencil, unit coefficients, Dirichlet on every face) on e^3 grids,
Nest-All-All with piecewise quadratics, factor + PCG to a relative residual
of 1e-10; --family picks another synthetic workload family (grf3d: the
log-normal Gaussian-random-field diffusion, twophase3d: the 1 / 1e4
two-phase diffusion, elastic: Q1 elasticity with stiff inclusions and
rigid-body preservation, e^3 elements).

The paper's stated aim for its experiments is solve times that scale like
O(n) with near-flat iteration counts as the grid grows (Sec. 7, up to 16M
unknowns for Poisson).  This prints, per size, the factor time (a repeated factorization, its
memory already reserved in the pool, and the first one), the PCG time, the
iterations, the apply time, the factor's device memory (peak reservation of
the first factorization, work buffers included) and the time per unknown
(repeated factor + PCG).

    python -m paper_1907_03406_gb300.sweep --sizes 32 64 128 192 256 --precision mixed
    python -m paper_1907_03406_gb300.sweep --family grf3d --sizes 64
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def run(sizes, precision: str, rtol: float = 1e-10, maxit: int = 1000, family: str = "poisson3d",
        scheme: str | None = None):
    import torch

    import sgf_inputs as si

    from . import Factor, Plan, release_cached_memory

    dev = torch.device("cuda", torch.cuda.current_device())
    rows = []
    for e in sizes:
        cfg = si.config(f"{family}_{e}")
        kw = {"scheme": scheme} if scheme else {}
        plan = Plan.from_config(cfg, precision=precision, **kw)
        coeffs = torch.tensor(np.ascontiguousarray(cfg["coeffs"]).ravel(), dtype=torch.float64, device=dev)
        b = torch.tensor(si.rhs(plan.n, 0), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        release_cached_memory()   # the previous size's blocks, cached by the pool
        free0 = torch.cuda.mem_get_info()[0]
        # first factorization of this size: the pool reserves its memory
        # (measured here); the timed one below reuses it, as repeated
        # factorizations of a plan do
        t0 = time.perf_counter()
        F = Factor(plan, coeffs)
        torch.cuda.synchronize()
        first_ms = 1e3 * (time.perf_counter() - t0)
        free1 = torch.cuda.mem_get_info()[0]
        F.close()
        t0 = time.perf_counter()
        F = Factor(plan, coeffs)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        x, info = F.pcg(b, rtol=rtol, maxit=maxit, check=False)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            F.apply(b)
        e1.record()
        torch.cuda.synchronize()
        row = dict(family=family, scheme=scheme or cfg.get("scheme", "nest_all_all"), edge=e, n=plan.n,
                   precision=F.precision, factor_ms=round(1e3 * (t1 - t0), 1),
                   first_factor_ms=round(first_ms, 1), pcg_ms=round(1e3 * (t2 - t1), 1), iterations=info["iterations"],
                   rel_residual=info["rel_residual"], apply_ms=round(e0.elapsed_time(e1) / 3, 3),
                   factor_gb=round((free0 - free1) / 1e9, 2),
                   ns_per_unknown=round(1e9 * (t2 - t0) / plan.n, 1))
        rows.append(row)
        print(json.dumps(row), flush=True)
        F.close()
        del F, x, coeffs, b
        torch.cuda.empty_cache()
    return rows


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--sizes", type=int, nargs="+", default=[32, 64, 128])
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--family", choices=["poisson3d", "grf3d", "twophase3d", "elastic"], default="poisson3d")
    ap.add_argument("--scheme", choices=["nest_all_all", "nest_2_all", "nest_2_2"], default=None,
                    help="compression scheme (default: the workload's)")
    args = ap.parse_args()
    run(args.sizes, args.precision, family=args.family, scheme=args.scheme)


if __name__ == "__main__":
    main()
