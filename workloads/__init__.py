"""Seeded synthetic SIMP elasticity problems shared by the oracle, the tests and the bench.

This module only *describes* problems: grid sizes, material constants, density fields,
fixed degrees of freedom and load vectors.  It contains none of the solver's arithmetic
(no element stiffness, no SIMP interpolation, no assembly), so both the CPU oracle and the
CUDA path can take their inputs from here without sharing any method code.

Numbering (the paper fixes none of it; this is the convention every part of the project uses):
  * nodes  n = i + (nx+1) * (j + (ny+1) * k), x fastest, i in [0, nx], j in [0, ny], k in [0, nz]
  * DOFs   dof = d * n + c, c = 0 (x), 1 (y), 2 (z); d = 2 in 2D and 3 in 3D
  * elements e = i + nx * (j + ny * k); unit square / cube elements, y is vertical ("down" = -y)

Density fields follow the recipe for "evolved topologies" without the paper's designs:
i.i.d. N(0, 1) numbers from ``numpy.random.default_rng(seed)`` blurred by a separable Gaussian
(sigma = length scale in elements, truncated at 4 sigma, reflect padding), then either
turned into thin connected 0/1 members (1e9 stiffness contrast) or min-max
mapped to [rho_lo, 1].
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

__all__ = [
    "Problem", "n_nodes", "n_dofs", "n_elems", "node_id", "smoothed_field",
    "mbb_beam", "cantilever_2d", "cantilever_3d", "batched_3d", "patch_tension",
    "random_problem", "serving_stream",
]


@dataclass
class Problem:
    """One SIMP elasticity solve: K(rho) u = f with u = 0 on ``fixed``.

    ``f`` has shape (nrhs, n): row r is right-hand side r (column r of the column-major
    n x nrhs array the C ABI takes).
    """
    name: str
    dim: int
    nx: int
    ny: int
    nz: int
    rho: np.ndarray
    fixed: np.ndarray
    f: np.ndarray
    E0: float = 1.0
    Emin: float = 1e-9
    penal: float = 3.0
    nu: float = 0.3
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return n_dofs(self.dim, self.nx, self.ny, self.nz)

    @property
    def nel(self) -> int:
        return n_elems(self.dim, self.nx, self.ny, self.nz)

    @property
    def nrhs(self) -> int:
        return int(self.f.shape[0])


def n_nodes(dim, nx, ny, nz=1):
    return (nx + 1) * (ny + 1) * ((nz + 1) if dim == 3 else 1)


def n_dofs(dim, nx, ny, nz=1):
    return dim * n_nodes(dim, nx, ny, nz)


def n_elems(dim, nx, ny, nz=1):
    return nx * ny * (nz if dim == 3 else 1)


def node_id(nx, ny, i, j, k=0):
    return np.asarray(i) + (nx + 1) * (np.asarray(j) + (ny + 1) * np.asarray(k))


def _blur(a: np.ndarray, sigma: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter1d
    out = a
    for ax in range(a.ndim):
        out = gaussian_filter1d(out, sigma, axis=ax, mode="reflect", truncate=4.0)
    return out


def smoothed_field(shape, sigma: float, seed: int) -> np.ndarray:
    """Gaussian-blurred white noise on an element grid of ``shape`` = (nz, ny, nx) or (ny, nx)."""
    rng = np.random.default_rng(seed)
    return _blur(rng.standard_normal(shape), sigma)


def _threshold(field_: np.ndarray, volfrac: float) -> np.ndarray:
    cut = np.percentile(field_, 100.0 * (1.0 - volfrac))
    return (field_ > cut).astype(np.float64)


def _members(field_: np.ndarray, volfrac: float, plate: int = 2) -> np.ndarray:
    """0/1 density of thin connected members: solid on the band |phi| < q around the zero
    level set of the smoothed field (q = the ``volfrac`` quantile of |phi|), plus solid plates
    ``plate`` elements wide along the clamped face x = 0 and the loaded face x = nx.  A plain
    percentile threshold at 40 % volume leaves disconnected islands (below percolation) and
    can put the load on void material; the band keeps members thin and connected."""
    a = np.abs(field_)
    rho = (a < np.percentile(a, 100.0 * volfrac)).astype(np.float64)
    if plate > 0:
        rho[..., :plate] = 1.0
        rho[..., -plate:] = 1.0
    return rho


def _minmax(field_: np.ndarray, lo: float) -> np.ndarray:
    a, b = field_.min(), field_.max()
    if b == a:  # single element: uniform solid
        return np.ones_like(field_)
    return lo + (1.0 - lo) * (field_ - a) / (b - a)


def _dofs_of_nodes(dim, nodes, comps=None):
    nodes = np.asarray(nodes, dtype=np.int64).ravel()
    comps = range(dim) if comps is None else comps
    return np.unique(np.concatenate([dim * nodes + c for c in comps]))


def mbb_beam(nx=96, ny=32, rho0=0.5, **mat) -> Problem:
    """Half MBB beam: u_x = 0 on the left edge (symmetry), u_y = 0 at the bottom-right node,
    unit downward point load at the top-left node; uniform density ``rho0``."""
    dim = 2
    left = node_id(nx, ny, 0, np.arange(ny + 1))
    fixed = np.unique(np.concatenate([
        _dofs_of_nodes(dim, left, comps=[0]),
        _dofs_of_nodes(dim, [node_id(nx, ny, nx, 0)], comps=[1]),
    ]))
    f = np.zeros((1, n_dofs(dim, nx, ny)))
    f[0, dim * node_id(nx, ny, 0, ny) + 1] = -1.0
    rho = np.full(nx * ny, float(rho0))
    return Problem("mbb_%dx%d" % (nx, ny), dim, nx, ny, 1, rho, fixed, f, **mat)


def cantilever_2d(nx=768, ny=384, seed=0, sigma=8.0, volfrac=0.4, **mat) -> Problem:
    """2D cantilever: left edge clamped, unit downward load at the right mid-edge node;
    density = thin connected members (:func:`_members`) of a smoothed random field, values
    {0, 1} (1e9 stiffness contrast with Emin = 1e-9), about ``volfrac`` solid."""
    dim = 2
    assert ny % 2 == 0
    left = node_id(nx, ny, 0, np.arange(ny + 1))
    fixed = _dofs_of_nodes(dim, left)
    f = np.zeros((1, n_dofs(dim, nx, ny)))
    f[0, dim * node_id(nx, ny, nx, ny // 2) + 1] = -1.0
    rho = _members(smoothed_field((ny, nx), sigma, seed), volfrac).ravel()
    return Problem("cantilever2d_%dx%d" % (nx, ny), dim, nx, ny, 1, rho, fixed, f,
                   meta={"seed": seed, "sigma": sigma, "volfrac": volfrac}, **mat)


def column_2d(nx=256, ny=1024, seed=None, sigma=8.0, rho_lo=0.1, **mat) -> Problem:
    """2D column (the stability example's geometry): bottom edge clamped, a total downward load
    of 1 spread over the top edge with consistent weights (end nodes half).  Density uniform 1,
    or with ``seed`` a smoothed random field min-max mapped to [rho_lo, 1]."""
    dim = 2
    bottom = node_id(nx, ny, np.arange(nx + 1), 0)
    fixed = _dofs_of_nodes(dim, bottom)
    f = np.zeros((1, n_dofs(dim, nx, ny)))
    w = np.full(nx + 1, 1.0 / nx)
    w[0] = w[-1] = 0.5 / nx
    f[0, dim * node_id(nx, ny, np.arange(nx + 1), ny) + 1] = -w
    if seed is None:
        rho = np.ones(nx * ny)
    else:
        rho = _minmax(smoothed_field((ny, nx), sigma, seed), rho_lo).ravel()
    return Problem("column2d_%dx%d" % (nx, ny), dim, nx, ny, 1, rho, fixed, f,
                   meta={"seed": seed}, **mat)


def _clamp_x0_3d(nx, ny, nz):
    jj, kk = np.meshgrid(np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    return _dofs_of_nodes(3, node_id(nx, ny, 0, jj, kk))


def cantilever_3d(nx=192, ny=96, nz=96, seed=0, sigma=8.0, rho_lo=1e-3, **mat) -> Problem:
    """3D cantilever: face x = 0 clamped; total downward load 1 spread along the bottom edge
    of the far face (nodes (nx, 0, k)) with consistent line-load weights (ends get half);
    density = smoothed random field min-max mapped to [rho_lo, 1]."""
    dim = 3
    fixed = _clamp_x0_3d(nx, ny, nz)
    f = np.zeros((1, n_dofs(dim, nx, ny, nz)))
    w = np.full(nz + 1, 1.0 / nz)
    w[0] *= 0.5
    w[-1] *= 0.5
    nodes = node_id(nx, ny, nx, 0, np.arange(nz + 1))
    f[0, dim * nodes + 1] = -w
    rho = _minmax(smoothed_field((nz, ny, nx), sigma, seed), rho_lo).ravel()
    return Problem("cantilever3d_%dx%dx%d" % (nx, ny, nz), dim, nx, ny, nz, rho, fixed, f,
                   meta={"seed": seed, "sigma": sigma, "rho_lo": rho_lo}, **mat)


def batched_3d(nx=128, ny=64, nz=64, field_seed=0, load_seed=1, rhs_seed=2,
               n_loads=8, n_adjoint=8, sigma=8.0, rho_lo=1e-3, **mat) -> Problem:
    """Many right-hand sides on one hex8 design: ``n_loads`` unit point loads (random free node,
    random unit direction) plus ``n_adjoint`` random unit-norm vectors supported on free DOFs
    (stand-ins for adjoint right-hand sides).  Face x = 0 clamped."""
    dim = 3
    fixed = _clamp_x0_3d(nx, ny, nz)
    n = n_dofs(dim, nx, ny, nz)
    free = np.ones(n, bool)
    free[fixed] = False
    free_nodes = np.flatnonzero(free.reshape(-1, dim).all(axis=1))
    rl = np.random.default_rng(load_seed)
    rr = np.random.default_rng(rhs_seed)
    f = np.zeros((n_loads + n_adjoint, n))
    for r in range(n_loads):
        node = free_nodes[rl.integers(len(free_nodes))]
        v = rl.standard_normal(dim)
        f[r, dim * node:dim * node + dim] = v / np.linalg.norm(v)
    for r in range(n_adjoint):
        v = rr.standard_normal(n) * free
        f[n_loads + r] = v / np.linalg.norm(v)
    rho = _minmax(smoothed_field((nz, ny, nx), sigma, field_seed), rho_lo).ravel()
    return Problem("batched3d_%dx%dx%d_x%d" % (nx, ny, nz, n_loads + n_adjoint), dim, nx, ny, nz,
                   rho, fixed, f, meta={"field_seed": field_seed}, **mat)


def patch_tension(dim=2, nx=6, ny=4, nz=3, sigma=1.0, E=1.0, nu=0.3) -> Problem:
    """Uniform-tension patch test on a uniform block: roller u_x = 0 on x = 0, u_y (and u_z)
    pinned at node (0,0,0), u_z pinned at (0, ny, 0) in 3D (removes the rotation about x);
    traction ``sigma`` on x = nx applied as consistent nodal loads.  The exact FE solution is
    u_x = sigma x / E, u_y = -nu sigma y / E (and u_z = -nu sigma z / E in 3D)."""
    if dim == 2:
        nzz = 1
        left = node_id(nx, ny, 0, np.arange(ny + 1))
        fixed = np.unique(np.concatenate([
            _dofs_of_nodes(2, left, comps=[0]), _dofs_of_nodes(2, [node_id(nx, ny, 0, 0)], [1])]))
        f = np.zeros((1, n_dofs(2, nx, ny)))
        w = np.full(ny + 1, sigma * 1.0)
        w[0] *= 0.5
        w[-1] *= 0.5
        f[0, 2 * node_id(nx, ny, nx, np.arange(ny + 1))] = w
    else:
        nzz = nz
        jj, kk = np.meshgrid(np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
        left = node_id(nx, ny, 0, jj, kk)
        fixed = np.unique(np.concatenate([
            _dofs_of_nodes(3, left, comps=[0]),
            _dofs_of_nodes(3, [node_id(nx, ny, 0, 0, 0)], [1, 2]),
            _dofs_of_nodes(3, [node_id(nx, ny, 0, ny, 0)], [2])]))
        f = np.zeros((1, n_dofs(3, nx, ny, nz)))
        wy = np.ones(ny + 1); wy[0] = wy[-1] = 0.5
        wz = np.ones(nz + 1); wz[0] = wz[-1] = 0.5
        W = sigma * np.outer(wy, wz)
        f[0, 3 * node_id(nx, ny, nx, jj, kk).ravel()] = W.ravel()
    rho = np.ones(nx * ny * nzz)
    return Problem("patch%d" % dim, dim, nx, ny, nzz, rho, fixed, f, E0=E, Emin=0.0, penal=1.0, nu=nu)


def random_problem(dim, nx, ny, nz=1, seed=0, sigma=2.0, contrast="threshold", nrhs=1,
                   bc="clamp", **mat) -> Problem:
    """Small seeded problems for parity tests: smoothed random density (0/1 members as in
    :func:`cantilever_2d`, or min-max mapped to [1e-3, 1] with ``contrast="minmax"``),
    x = 0 clamped, ``nrhs`` random unit-norm loads on free DOFs."""
    rng = np.random.default_rng(seed + 1000)
    shape = (ny, nx) if dim == 2 else (nz, ny, nx)
    fld = smoothed_field(shape, sigma, seed)
    rho = (_members(fld, 0.4) if contrast == "threshold" else _minmax(fld, 1e-3)).ravel()
    if dim == 2:
        fixed = _dofs_of_nodes(2, node_id(nx, ny, 0, np.arange(ny + 1)))
        n = n_dofs(2, nx, ny)
    else:
        fixed = _clamp_x0_3d(nx, ny, nz)
        n = n_dofs(3, nx, ny, nz)
    free = np.ones(n, bool)
    free[fixed] = False
    f = rng.standard_normal((nrhs, n)) * free
    f /= np.linalg.norm(f, axis=1, keepdims=True)
    return Problem("rand%d_%dx%dx%d_s%d" % (dim, nx, ny, nz, seed), dim, nx, ny,
                   nz if dim == 3 else 1, rho, fixed, f, **mat)


def serving_stream(n_requests=256, n_updates=10, arrival_seed=3, size_seed=4, field_seed0=5,
                   rate_per_s=50.0, noise=0.05, sizes_2d=None, sizes_3d=None):
    """Request stream for the serving loop: Poisson arrival times, a grid drawn uniformly from
    2D (64x32 .. 1024x512) and 3D (32x16x16 .. 192x96x96) sizes by doubling steps, and for each
    request ``n_updates`` successive designs rho_t = clip(rho_{t-1} (1 + noise xi), 1e-3, 1).

    Returns a list of dicts {t_arrive, dim, nx, ny, nz, field_seed}; densities are produced on
    demand by :func:`serving_density` so the stream itself stays small."""
    if sizes_2d is None:
        sizes_2d = [(64 << s, 32 << s, 1) for s in range(5)]
    if sizes_3d is None:
        sizes_3d = [(32, 16, 16), (64, 32, 32), (128, 64, 64), (192, 96, 96)]
    sizes = [(2,) + s for s in sizes_2d] + [(3,) + s for s in sizes_3d]
    ra = np.random.default_rng(arrival_seed)
    rs = np.random.default_rng(size_seed)
    t = np.cumsum(ra.exponential(1.0 / rate_per_s, n_requests))
    pick = rs.integers(len(sizes), size=n_requests)
    return [dict(t_arrive=float(t[i]), dim=sizes[pick[i]][0], nx=sizes[pick[i]][1],
                 ny=sizes[pick[i]][2], nz=sizes[pick[i]][3], field_seed=field_seed0 + i,
                 n_updates=n_updates, noise=noise) for i in range(n_requests)]


def serving_density(req, update: int) -> np.ndarray:
    """Density of design update ``update`` (0-based) for a request of :func:`serving_stream`."""
    dim, nx, ny, nz = req["dim"], req["nx"], req["ny"], req["nz"]
    shape = (ny, nx) if dim == 2 else (nz, ny, nx)
    rho = _minmax(smoothed_field(shape, 8.0, req["field_seed"]), 1e-3).ravel()
    rng = np.random.default_rng(req["field_seed"] + 100000)
    for _ in range(update):
        rho = np.clip(rho * (1.0 + req["noise"] * rng.standard_normal(rho.shape)), 1e-3, 1.0)
    return rho


def serving_problem(req, update: int) -> Problem:
    """Cantilever boundary conditions and load for a serving request at design ``update``."""
    dim, nx, ny, nz = req["dim"], req["nx"], req["ny"], req["nz"]
    if dim == 2:
        p = cantilever_2d(nx, ny, seed=req["field_seed"])
    else:
        p = cantilever_3d(nx, ny, nz, seed=req["field_seed"])
    p.rho = serving_density(req, update)
    p.name = "serve%d_%dx%dx%d" % (dim, nx, ny, nz)
    return p
