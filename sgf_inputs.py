"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only draws random numbers and lays them out as grids: coefficient
fields, right-hand sides, the serving request stream and the named workload
configurations.  It holds none of the factorization's arithmetic (no stencil
assembly, no partition, no basis), so both sides can consume identical inputs
without sharing any of the method.

Stand-ins: the paper's SPE10 reservoir (Sec. 7.1.2) and MFEM cantilever beam
(Sec. 7.1.3) are not available here; the Gaussian random field and two-phase
block fields below reproduce the smooth and discontinuous coefficient regimes,
and the inclusion field the stiff/soft elasticity regime.
"""
from __future__ import annotations

import numpy as np

# Stencil names understood by both sides.
STENCIL_5PT_2D = "5pt_2d"          # finite-difference Laplacian, ghost Dirichlet
STENCIL_7PT_FV_3D = "7pt_fv_3d"    # two-point-flux finite volume, half-cell Dirichlet
STENCIL_7PT_3D = "7pt_3d"          # finite-difference Laplacian, ghost Dirichlet
STENCIL_Q1_ELASTIC_3D = "q1_elastic_3d"

# Dirichlet face bits (x-, x+, y-, y+, z-, z+).
FACE_XM, FACE_XP, FACE_YM, FACE_YP, FACE_ZM, FACE_ZP = 1, 2, 4, 8, 16, 32
ALL_FACES_2D = FACE_XM | FACE_XP | FACE_YM | FACE_YP
ALL_FACES_3D = ALL_FACES_2D | FACE_ZM | FACE_ZP


def rhs(n: int, seed: int, nrhs: int = 1) -> np.ndarray:
    """i.i.d. uniform[-1, 1] right-hand side(s), shape (n,) or (nrhs, n)."""
    rng = np.random.default_rng(seed)
    if nrhs == 1:
        return rng.uniform(-1.0, 1.0, size=n)
    return rng.uniform(-1.0, 1.0, size=(nrhs, n))


def unit_field(shape) -> np.ndarray:
    """Constant coefficient 1 on every cell (array indexed [z, y, x] / [y, x])."""
    return np.ones(tuple(shape), dtype=np.float64)


def gaussian_random_field(shape, corr_len: float, std: float, seed: int) -> np.ndarray:
    """Stationary Gaussian field with Gaussian covariance exp(-r^2 / (2 l^2)).

    Spectral synthesis on a periodic box padded by 4 correlation lengths per
    axis (so the periodic wrap does not correlate opposite faces), cropped, then
    shifted and scaled to sample mean 0 and sample standard deviation `std`.
    """
    shape = tuple(int(s) for s in shape)
    pad = int(np.ceil(4 * corr_len))
    big = tuple(s + pad for s in shape)
    rng = np.random.default_rng(seed)
    white = rng.standard_normal(big)
    freqs = np.meshgrid(*[np.fft.fftfreq(s) for s in big], indexing="ij")
    k2 = sum((2 * np.pi * f) ** 2 for f in freqs)
    amp = np.exp(-0.25 * k2 * corr_len ** 2)      # sqrt of exp(-k^2 l^2 / 2)
    field = np.real(np.fft.ifftn(np.fft.fftn(white) * amp))
    field = field[tuple(slice(0, s) for s in shape)]
    field = field - field.mean()
    field = field * (std / field.std())
    return np.ascontiguousarray(field)


def lognormal_field(shape, corr_len: float, std: float, seed: int) -> np.ndarray:
    """kappa = exp(g) with g a Gaussian random field (see above)."""
    return np.exp(gaussian_random_field(shape, corr_len, std, seed))


def two_phase_blocks(shape, block: int = 4, fill: float = 0.3, lo: float = 1.0,
                     hi: float = 1e4, seed: int = 0) -> np.ndarray:
    """Two-phase field: exactly round(fill * #blocks) of the block^d cubes get `hi`.

    The blocks tile the grid from the origin; ragged blocks at the far faces are
    truncated.  The chosen blocks come from a seeded permutation.
    """
    shape = tuple(int(s) for s in shape)
    nb = tuple((s + block - 1) // block for s in shape)
    total = int(np.prod(nb))
    rng = np.random.default_rng(seed)
    chosen = rng.permutation(total)[: int(round(fill * total))]
    mask = np.zeros(total, dtype=bool)
    mask[chosen] = True
    mask = mask.reshape(nb)
    for ax in range(len(shape)):
        mask = np.repeat(mask, block, axis=ax)
    mask = mask[tuple(slice(0, s) for s in shape)]
    out = np.full(shape, lo, dtype=np.float64)
    out[mask] = hi
    return out


def inclusion_moduli(elems, n_incl: int = 8, radius: float = 6.0, e0: float = 1.0,
                     e1: float = 1e3, seed: int = 0) -> np.ndarray:
    """Young's modulus per hexahedral element: e0 with `n_incl` spheres of e1.

    Sphere centres are uniform in the element box (seeded); an element belongs
    to an inclusion when its centroid lies within `radius` elements of a centre.
    Array indexed [ez, ey, ex].
    """
    ez, ey, ex = (int(s) for s in elems)
    rng = np.random.default_rng(seed)
    centres = rng.uniform([0, 0, 0], [ex, ey, ez], size=(n_incl, 3))
    zz, yy, xx = np.meshgrid(np.arange(ez) + 0.5, np.arange(ey) + 0.5,
                             np.arange(ex) + 0.5, indexing="ij")
    out = np.full((ez, ey, ex), e0, dtype=np.float64)
    for cx, cy, cz in centres:
        inside = (xx - cx) ** 2 + (yy - cy) ** 2 + (zz - cz) ** 2 <= radius ** 2
        out[inside] = e1
    return out


def request_stream(seed: int = 1, count: int = 256, rate_hz: float = 50.0,
                   edge_lo: int = 32, edge_hi: int = 96, p_factor: float = 0.4,
                   max_rhs: int = 8, field_std: float = 1.0, corr_len: float = 4.0):
    """Seeded serving workload: Poisson arrivals of 3D 7-point diffusion requests.

    Each request is a dict with arrival time (s), grid edge, kind ("factor" =
    new factor + solve, "solve" = solve on a resident factor), the number of
    right-hand sides, a coefficient seed and a right-hand-side seed.  The field
    itself is generated lazily by `request_coeffs` so the stream stays small.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=count)
    t = np.cumsum(gaps) - gaps[0]
    reqs = []
    for i in range(count):
        reqs.append({
            "id": i,
            "arrival_s": float(t[i]),
            "edge": int(rng.integers(edge_lo, edge_hi + 1)),
            "kind": "factor" if rng.uniform() < p_factor else "solve",
            "nrhs": int(rng.integers(1, max_rhs + 1)),
            "coeff_seed": int(rng.integers(0, 2 ** 31 - 1)),
            "rhs_seed": int(rng.integers(0, 2 ** 31 - 1)),
            "pick": float(rng.uniform()),
            "field_std": field_std,
            "corr_len": corr_len,
        })
    return reqs


def request_coeffs(req) -> np.ndarray:
    e = req["edge"]
    return lognormal_field((e, e, e), req["corr_len"], req["field_std"], req["coeff_seed"])


# Named workloads.  Grid arrays are indexed [z, y, x] (3D) or [y, x] (2D); the
# unknown with grid index (x, y, z) has natural number x + nx * (y + ny * z).
def config(name: str, seed: int = 0) -> dict:
    """Build one named workload: grid, stencil, coefficients and method options."""
    if name == "poisson2d_64":
        shape = (64, 64)
        return dict(name=name, dim=2, n=(64, 64, 1), stencil=STENCIL_5PT_2D,
                    dirichlet=ALL_FACES_2D, coeffs=unit_field(shape),
                    leaf=16, degree=1, basis="poly", dof=1)
    if name.startswith("grf3d_"):
        e = int(name.split("_")[1])
        shape = (e, e, e)
        return dict(name=name, dim=3, n=(e, e, e), stencil=STENCIL_7PT_FV_3D,
                    dirichlet=FACE_XM, coeffs=lognormal_field(shape, 8.0, 2.0, seed),
                    leaf=8, degree=2, basis="poly", dof=1)
    if name.startswith("gengrf3d_"):
        # the GRF workload on general partitions (Gen-All-All, Sec. 5.2), with
        # the paper's leaf size for piecewise-quadratic compression (b = 5)
        e = int(name.split("_")[1])
        shape = (e, e, e)
        return dict(name=name, dim=3, n=(e, e, e), stencil=STENCIL_7PT_FV_3D,
                    dirichlet=FACE_XM, coeffs=lognormal_field(shape, 8.0, 2.0, seed),
                    leaf=5, degree=2, basis="poly", dof=1, scheme="gen_all_all")
    if name.startswith("twophase3d_"):
        e = int(name.split("_")[1])
        shape = (e, e, e)
        return dict(name=name, dim=3, n=(e, e, e), stencil=STENCIL_7PT_FV_3D,
                    dirichlet=FACE_XM, coeffs=two_phase_blocks(shape, 4, 0.3, 1.0, 1e4, seed),
                    leaf=8, degree=2, basis="poly", dof=1)
    if name.startswith("poisson3d_"):
        e = int(name.split("_")[1])
        shape = (e, e, e)
        return dict(name=name, dim=3, n=(e, e, e), stencil=STENCIL_7PT_3D,
                    dirichlet=ALL_FACES_3D, coeffs=unit_field(shape),
                    leaf=8, degree=2, basis="poly", dof=1)
    if name.startswith("elastic_"):
        # Q1 hexahedra on an e^3 element cube, x = 0 face clamped: the free
        # nodes form an e x (e+1) x (e+1) point grid with 3 DOFs each;
        # E = 1 with 8 seeded spherical inclusions of E = 1e3 (radius e/8), nu = 0.3
        e = int(name.split("_")[1])
        return dict(name=name, dim=3, n=(e, e + 1, e + 1), elems=(e, e, e),
                    stencil=STENCIL_Q1_ELASTIC_3D, dirichlet=FACE_XM,
                    coeffs=inclusion_moduli((e, e, e), 8, e / 8.0, 1.0, 1e3, seed),
                    nu=0.3, leaf=8 if e >= 32 else 4, degree=1, basis="rbm", dof=3)
    raise KeyError(name)
