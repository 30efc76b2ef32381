"""Seeded synthetic inputs shared by the library's callers, its tests and the oracle.

This module draws random numbers and lays them out; it holds none of the
spectral-element arithmetic (no GLL points, no derivatives, no geometric
factors, no operator).  Both the CUDA path and the oracle build their own
discretisation from what is returned here.

Workload recipe (the paper's cubic meshes, Sec. "Experimental Setup", with the
random perturbation and fields used for every parity case and benchmark):

* ``box_vertices(n, seed)``: the unit cube split into n x n x n hexahedra;
  every vertex that is not on the boundary is moved by an independent
  uniform draw in [-0.1 h, 0.1 h] per coordinate (h = 1/n).  Elements stay
  trilinear, so no Jacobian can invert.
* ``uniform(shape, seed)``: fields such as u drawn uniform in [lo, hi].
* ``fourier_modes(seed)``: amplitudes, wave vectors and phases of the
  8-mode smooth coefficient used by the variable-h1 Poisson problem.
* ``batch_meshes(seed)``: the uneven multi-mesh batch (element counts
  log-uniform in [64, 8192], polynomial orders from {5, 6, 8, 10}).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "box_vertices",
    "uniform",
    "fourier_modes",
    "batch_meshes",
    "box_dims",
    "poisson_source",
]


def rng(seed: int) -> np.random.Generator:
    """The one generator every draw goes through (PCG64, seeded)."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def box_dims(nel: int) -> tuple[int, int, int]:
    """Split an element count into a box-like nx*ny*nz >= 1 (x fastest).

    Picks the factorisation of the largest count <= nel that is a product of
    three factors as close to each other as possible; returns (nx, ny, nz).
    """
    nel = max(int(nel), 1)
    best = (nel, 1, 1)
    best_score = None
    for target in range(nel, 0, -1):
        for nz in range(1, int(round(target ** (1 / 3))) + 2):
            if target % nz:
                continue
            rest = target // nz
            for ny in range(nz, int(rest ** 0.5) + 2):
                if rest % ny:
                    continue
                nx = rest // ny
                if nx < ny:
                    continue
                score = nx / nz
                if best_score is None or score < best_score:
                    best, best_score = (nx, ny, nz), score
        if best_score is not None and best_score <= 4.0:
            return best
    return best


def box_vertices(nx: int, ny: int | None = None, nz: int | None = None,
                 seed: int = 0, amp: float = 0.1) -> np.ndarray:
    """Vertices of the perturbed box mesh on [0,1]^3.

    Returns an array of shape (nz+1, ny+1, nx+1, 3) (x index fastest) holding
    the (x, y, z) position of each element vertex.  Interior vertices are
    displaced by amp*h*U(-1, 1) per coordinate, with h the element width in
    that direction; boundary vertices stay on the faces of the cube.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    g = rng(seed)
    xs = np.arange(nx + 1, dtype=np.float64) / nx
    ys = np.arange(ny + 1, dtype=np.float64) / ny
    zs = np.arange(nz + 1, dtype=np.float64) / nz
    v = np.empty((nz + 1, ny + 1, nx + 1, 3), dtype=np.float64)
    v[..., 0] = xs[None, None, :]
    v[..., 1] = ys[None, :, None]
    v[..., 2] = zs[:, None, None]
    d = g.uniform(-1.0, 1.0, size=v.shape)
    interior = np.zeros((nz + 1, ny + 1, nx + 1), dtype=bool)
    interior[1:-1, 1:-1, 1:-1] = True
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    v += np.where(interior[..., None], amp * h * d, 0.0)
    return v


def uniform(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """A float64 array of the given shape drawn uniform in [lo, hi]."""
    return rng(seed).uniform(lo, hi, size=shape)


def fourier_modes(seed: int, n_modes: int = 8, kmax: int = 3):
    """Random smooth-coefficient modes: (amplitudes, wave vectors, phases).

    amplitudes: (n_modes,) uniform in [0.5, 1]; wave vectors: (n_modes, 3)
    integer multiples of pi with entries in [1, kmax]; phases uniform in
    [0, 2 pi).  The coefficient is sum_m a_m sin(k_m . x + phi_m), rescaled
    affinely into [0.5, 2] by whoever evaluates it.
    """
    g = rng(seed)
    a = g.uniform(0.5, 1.0, size=n_modes)
    k = g.integers(1, kmax + 1, size=(n_modes, 3)).astype(np.float64) * np.pi
    phi = g.uniform(0.0, 2.0 * np.pi, size=n_modes)
    return a, k, phi


def poisson_source(x, y, z):
    """The benchmark's Poisson source f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z)
    (homogeneous Dirichlet data on the unit cube; exact solution
    sin(pi x) sin(pi y) sin(pi z))."""
    return 3.0 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def batch_meshes(seed: int, count: int = 64, emin: int = 64, emax: int = 8192,
                 orders=(5, 6, 8, 10)):
    """The uneven batch: a list of (nx, ny, nz, lx) for ``count`` meshes.

    Element counts are log-uniform in [emin, emax] and rounded down to a
    box-like nx*ny*nz; lx is drawn uniformly from ``orders``.
    """
    g = rng(seed)
    out = []
    for _ in range(count):
        ne = int(np.exp(g.uniform(np.log(emin), np.log(emax))))
        lx = int(orders[int(g.integers(0, len(orders)))])
        nx, ny, nz = box_dims(ne)
        out.append((nx, ny, nz, lx))
    return out
