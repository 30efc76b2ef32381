"""Oracle for the spectral-element Poisson operator and its solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It is plain,
slow and fp64 throughout; it shares no code with the CUDA library (neither
side imports the other; both read their inputs from ``synth``).

Contents, each with the passage it follows:

* ``gll(lx)`` - Gauss-Lobatto-Legendre nodes and weights on [-1, 1], the
  quadrature points of Sec. "The Spectral Element Method" (the nodes of the
  Lagrange basis of Eq. (2)).  Nodes: roots of (1 - x^2) L_N'(x) by Newton's
  method on L_{N-1}(x) - x L_N(x) from Chebyshev-Gauss-Lobatto starts;
  weights 2 / (N (N+1) L_N(x_i)^2).
* ``diff_matrix(lx)`` - D_{ij} = l_j'(xi_i) for the Lagrange basis of Eq. (2)
  read as l_i(x) = (x^2 - 1) L_N'(x) / (N (N+1) L_N(x_i) (x - x_i)).
* ``d_buffers(lx)`` - the (dx, dxt) buffers in the layout the kernel of
  Listing 2 indexes (dx[l, i] = D_{i l}, dxt[l, i] = D_{l i}).
* ``box_geometry(vertices, lx)`` - isoparametric trilinear hexahedra: node
  coordinates, Jacobian by D applied to the coordinates, G = jac * W *
  J^{-1} J^{-T} (the symmetric 3x3 factor G11..G33 that Listing 2 applies),
  mass B = jac * W.
* ``ax_helm(...)`` - the element-local operator of Listing 2 (C loop nest,
  ``ax_oracle.c``).
* ``gs_sum`` / ``multiplicity`` / ``numbering`` / ``boundary_mask`` -
  direct-stiffness summation over shared nodes (the gather-scatter named in
  Sec. "Neko and Small Tensor Kernel").
* ``jacobi_diagonal`` - exact diagonal of the assembled operator.
* ``pcg`` - textbook preconditioned conjugate gradients on the assembled,
  masked operator (the Poisson solve of Sec. "The Spectral Element Method";
  the paper itself prints no solver).

Parity pins live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


# ---------------------------------------------------------------------------
# build / load of the C part
# ---------------------------------------------------------------------------
def build(force: bool = False) -> str:
    """Compile ``ax_oracle.c`` into ``liboracle.so`` with gcc (OpenMP on)."""
    src = os.path.join(_HERE, "ax_oracle.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
           "-o", tmp, src]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_ax_helm.argtypes = [dp] * 15 + [ctypes.c_int, ctypes.c_int]
            lib.oracle_ax_helm.restype = ctypes.c_int
            lib.oracle_gs_sum.argtypes = [dp, ctypes.POINTER(ctypes.c_longlong),
                                          ctypes.c_longlong, ctypes.c_longlong]
            lib.oracle_gs_sum.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def set_threads(n: int = 0) -> int:
    """Sets the OpenMP threads of the C loops (n > 0) and returns the count
    in effect; timing only, results are independent of it."""
    return int(_load().oracle_set_threads(int(n)))


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------------------
# 1-D GLL basis
# ---------------------------------------------------------------------------
def legendre(n: int, x):
    """(L_n(x), L_{n-1}(x)) by the three-term recurrence
    (m+1) L_{m+1} = (2m+1) x L_m - m L_{m-1}."""
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.ones_like(x), np.zeros_like(x)
    p_prev, p = np.ones_like(x), x.copy()
    for m in range(1, n):
        p_prev, p = p, ((2 * m + 1) * x * p - m * p_prev) / (m + 1)
    return p, p_prev


def gll(lx: int):
    """GLL nodes (ascending) and weights for lx = N + 1 points."""
    if lx < 2:
        raise ValueError("lx must be >= 2")
    n = lx - 1
    x = -np.cos(np.pi * np.arange(lx) / n)
    for _ in range(100):
        ln, lm = legendre(n, x)
        dxn = (x * ln - lm) / (lx * ln)
        x = x - dxn
        if np.max(np.abs(dxn)) < 1e-16:
            break
    ln, _ = legendre(n, x)
    w = 2.0 / (n * (n + 1) * ln * ln)
    return x, w


def diff_matrix(lx: int) -> np.ndarray:
    """D[i, j] = derivative of the j-th Lagrange basis function at node i."""
    n = lx - 1
    x, _ = gll(lx)
    ln, _ = legendre(n, x)
    d = np.zeros((lx, lx))
    for i in range(lx):
        for j in range(lx):
            if i != j:
                d[i, j] = ln[i] / (ln[j] * (x[i] - x[j]))
    d[0, 0] = -n * (n + 1) / 4.0
    d[n, n] = n * (n + 1) / 4.0
    return d


def d_buffers(lx: int):
    """(dx, dxt) as the flat lx*lx buffers the operator reads:
    dx[l*lx + i] = D[i, l] and dxt[l*lx + i] = D[l, i]."""
    d = diff_matrix(lx)
    return np.ascontiguousarray(d.T).ravel(), np.ascontiguousarray(d).ravel()


# ---------------------------------------------------------------------------
# mesh, numbering, geometry
# ---------------------------------------------------------------------------
def element_corners(vertices: np.ndarray) -> np.ndarray:
    """(E, 2, 2, 2, 3) corner positions [e][c][b][a] of a structured box
    mesh whose vertices are laid out (nz+1, ny+1, nx+1, 3); elements are
    numbered e = ex + nx*(ey + ny*ez)."""
    nz, ny, nx = (s - 1 for s in vertices.shape[:3])
    out = np.empty((nz, ny, nx, 2, 2, 2, 3))
    for c in range(2):
        for b in range(2):
            for a in range(2):
                out[:, :, :, c, b, a, :] = vertices[c:c + nz, b:b + ny, a:a + nx, :]
    return out.reshape(nz * ny * nx, 2, 2, 2, 3)


def node_coordinates(vertices: np.ndarray, lx: int, elements=None) -> np.ndarray:
    """(E, lx, lx, lx, 3) positions of the GLL nodes [e][k][j][i] under the
    trilinear map of each element (all elements, or the listed ones)."""
    corners = element_corners(vertices)
    if elements is not None:
        corners = corners[np.asarray(elements)]
    return corners_to_nodes(corners, lx)


def corners_to_nodes(corners: np.ndarray, lx: int) -> np.ndarray:
    xi, _ = gll(lx)
    phi = np.stack([(1.0 - xi) / 2.0, (1.0 + xi) / 2.0])  # [a][i]
    # x[e,k,j,i,:] = sum_{c,b,a} corner[e,c,b,a,:] phi_c(xi_k) phi_b(xi_j) phi_a(xi_i)
    return np.einsum("ecbad,ck,bj,ai->ekjid", corners, phi, phi, phi, optimize=True)


def _ref_derivatives(f: np.ndarray, d: np.ndarray):
    """(df/dr, df/ds, df/dt) of element fields f[e,k,j,i] with the 1-D
    matrix d[i, l] applied along i, j and k respectively."""
    fr = np.einsum("il,ekjl->ekji", d, f, optimize=True)
    fs = np.einsum("jl,ekli->ekji", d, f, optimize=True)
    ft = np.einsum("kl,elji->ekji", d, f, optimize=True)
    return fr, fs, ft


def box_geometry(vertices: np.ndarray, lx: int, elements=None) -> dict:
    """Isoparametric geometry of a box mesh (all elements, or the listed ones).

    Returns a dict with xyz (E,lx,lx,lx,3), jac, B (mass = jac * W) and the
    six factors g11, g22, g33, g12, g13, g23 (each (E,lx,lx,lx)), where
    G = jac * W * J^{-1} J^{-T}, J[a][b] = d x_a / d r_b and
    W = w_i w_j w_k.
    """
    d = diff_matrix(lx)
    _, w = gll(lx)
    xyz = node_coordinates(vertices, lx, elements)
    jm = np.empty(xyz.shape[:4] + (3, 3))
    for a in range(3):
        fr, fs, ft = _ref_derivatives(xyz[..., a], d)
        jm[..., a, 0], jm[..., a, 1], jm[..., a, 2] = fr, fs, ft
    jac = np.linalg.det(jm)
    if np.any(jac <= 0):
        raise ValueError("inverted element")
    jinv = np.linalg.inv(jm)  # rows: grad r, grad s, grad t
    wq = w[:, None, None] * w[None, :, None] * w[None, None, :]  # [k][j][i]
    scale = jac * wq[None]
    gm = np.einsum("...ac,...bc->...ab", jinv, jinv) * scale[..., None, None]
    return {
        "xyz": xyz, "jac": jac, "B": jac * wq[None],
        "g11": gm[..., 0, 0].copy(), "g22": gm[..., 1, 1].copy(),
        "g33": gm[..., 2, 2].copy(), "g12": gm[..., 0, 1].copy(),
        "g13": gm[..., 0, 2].copy(), "g23": gm[..., 1, 2].copy(),
    }


def numbering(nx: int, ny: int, nz: int, lx: int) -> np.ndarray:
    """Global id of each local point [e][k][j][i] of the structured box:
    g = X + NX*(Y + NY*Z) with X = ex*(lx-1)+i, NX = nx*(lx-1)+1, etc."""
    n = lx - 1
    NX, NY = nx * n + 1, ny * n + 1
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kk, jj, ii = np.meshgrid(np.arange(lx), np.arange(lx), np.arange(lx), indexing="ij")
    X = ex.reshape(-1, 1, 1, 1) * n + ii[None]
    Y = ey.reshape(-1, 1, 1, 1) * n + jj[None]
    Z = ez.reshape(-1, 1, 1, 1) * n + kk[None]
    return (X + NX * (Y + NY * Z)).astype(np.int64)


def boundary_mask(nx: int, ny: int, nz: int, lx: int) -> np.ndarray:
    """1.0 at local points whose global node is interior, 0.0 on the
    boundary of the box (homogeneous Dirichlet)."""
    n = lx - 1
    NX, NY, NZ = nx * n + 1, ny * n + 1, nz * n + 1
    g = numbering(nx, ny, nz, lx)
    X = g % NX
    Y = (g // NX) % NY
    Z = g // (NX * NY)
    on = (X == 0) | (X == NX - 1) | (Y == 0) | (Y == NY - 1) | (Z == 0) | (Z == NZ - 1)
    return np.where(on, 0.0, 1.0)


# ---------------------------------------------------------------------------
# operator, gather-scatter, solver
# ---------------------------------------------------------------------------
def ax_helm(u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, lx,
            dy=None, dz=None, dyt=None, dzt=None) -> np.ndarray:
    """w = local stiffness apply of Listing 2 on element-major fp64 arrays."""
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    nel = u.size // (lx ** 3)
    assert u.size == nel * lx ** 3
    arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in
            (dx, dy if dy is not None else dx, dz if dz is not None else dx,
             dxt, dyt if dyt is not None else dxt, dzt if dzt is not None else dxt,
             h1, g11, g22, g33, g12, g13, g23)]
    for a in arrs[6:]:
        assert a.size == u.size
    w = np.empty_like(u)
    rc = lib.oracle_ax_helm(_dp(w), _dp(u.reshape(-1)), *[_dp(a) for a in arrs], lx, nel)
    if rc != 0:
        raise RuntimeError(f"oracle_ax_helm failed: {rc}")
    return w


def ax_helm_h2(u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, lx, h2, B) -> np.ndarray:
    """Helmholtz form w = A u + h2 B u: the stiffness apply of Listing 2 plus
    the mass term with coefficient h2 (B the diagonal mass, jac * W).  The
    paper's listing is h1-only; the h2 term is the other half of Neko's
    Helmholtz operator, added pointwise."""
    w = ax_helm(u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, lx)
    flat = lambda a: np.asarray(a, dtype=np.float64).reshape(-1)
    return w + (flat(h2) * flat(B) * flat(u)).reshape(w.shape)


def gs_sum(v: np.ndarray, glob: np.ndarray) -> np.ndarray:
    """Direct-stiffness summation: every copy of a global node gets the sum
    over all its local copies (C loop, dense scatter-add then gather)."""
    lib = _load()
    out = np.ascontiguousarray(v, dtype=np.float64).reshape(-1).copy()
    g = np.ascontiguousarray(glob, dtype=np.int64).reshape(-1)
    assert g.size == out.size
    nglob = int(g.max()) + 1 if g.size else 0
    rc = lib.oracle_gs_sum(_dp(out), g.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                           out.size, nglob)
    if rc != 0:
        raise RuntimeError("oracle_gs_sum failed")
    return out.reshape(np.shape(v))


def multiplicity(glob: np.ndarray) -> np.ndarray:
    """Number of local copies of each point's global node."""
    return gs_sum(np.ones(glob.shape), glob)


def jacobi_diagonal(dx, h1, g11, g22, g33, g12, g13, g23, lx) -> np.ndarray:
    """Diagonal of the element operator sum_ab D_a^T diag(h1 G_ab) D_b:
      sum_l D_li^2 (h1 G11)(k,j,l) + sum_l D_lj^2 (h1 G22)(k,l,i)
      + sum_l D_lk^2 (h1 G33)(l,j,i) + 2 h1 (D_ii D_jj G12 + D_ii D_kk G13
      + D_jj D_kk G23)(k,j,i),
    un-assembled (apply ``gs_sum`` for the assembled diagonal)."""
    d = np.asarray(dx).reshape(lx, lx).T  # d[i, l] = D_il
    shp = (-1, lx, lx, lx)
    a = lambda f: np.asarray(f).reshape(shp)
    hg11, hg22, hg33 = a(h1) * a(g11), a(h1) * a(g22), a(h1) * a(g33)
    d2 = d * d  # d2[l, i] = D_li^2
    out = (np.einsum("li,ekjl->ekji", d2, hg11)
           + np.einsum("lj,ekli->ekji", d2, hg22)
           + np.einsum("lk,elji->ekji", d2, hg33))
    dd = np.diag(d)
    di, dj, dk = dd[None, None, None, :], dd[None, None, :, None], dd[None, :, None, None]
    out += 2.0 * a(h1) * (di * dj * a(g12) + di * dk * a(g13) + dj * dk * a(g23))
    return out.reshape(np.shape(h1))


class Problem:
    """A Poisson problem on a perturbed box: operator data, numbering, mask,
    multiplicity, right-hand side.  ``apply(p)`` is mask(gs(Ax(p))); with h2
    the Helmholtz problem -div(h1 grad u) + h2 u = f, ``apply(p)`` then
    mask(gs(Ax(p) + h2 B p))."""

    def __init__(self, vertices: np.ndarray, lx: int, h1=None, f=None, h2=None):
        nz, ny, nx = (s - 1 for s in vertices.shape[:3])
        self.nx, self.ny, self.nz, self.lx = nx, ny, nz, lx
        self.geo = box_geometry(vertices, lx)
        self.dx, self.dxt = d_buffers(lx)
        shp = self.geo["jac"].shape
        self.h1 = np.ones(shp) if h1 is None else np.asarray(h1, dtype=np.float64).reshape(shp)
        self.glob = numbering(nx, ny, nz, lx)
        self.mask = boundary_mask(nx, ny, nz, lx)
        self.mult = multiplicity(self.glob)
        g = self.geo
        self.G = (g["g11"], g["g22"], g["g33"], g["g12"], g["g13"], g["g23"])
        self.h2 = None if h2 is None else np.broadcast_to(
            np.asarray(h2, dtype=np.float64), shp).copy()
        dloc = jacobi_diagonal(self.dx, self.h1, *self.G, lx)
        if self.h2 is not None:
            dloc = dloc + self.h2 * g["B"]
        self.diag = gs_sum(dloc, self.glob)
        if f is not None:
            x = g["xyz"]
            fv = f(x[..., 0], x[..., 1], x[..., 2])
            self.b = self.mask * gs_sum(g["B"] * fv, self.glob)
        else:
            self.b = None

    def ax_local(self, p):
        if self.h2 is not None:
            return ax_helm_h2(p, self.dx, self.dxt, self.h1, *self.G, self.lx, self.h2,
                              self.geo["B"]).reshape(p.shape)
        return ax_helm(p, self.dx, self.dxt, self.h1, *self.G, self.lx).reshape(p.shape)

    def apply(self, p):
        return self.mask * gs_sum(self.ax_local(p), self.glob)

    def dot(self, a, b):
        """Inner product over unique global nodes (local sum weighted by
        1/multiplicity)."""
        return float(np.sum(a * b / self.mult))


def pcg(prob: Problem, b: np.ndarray, tol: float = 1e-8, maxit: int = 10000,
        precond: str = "jacobi"):
    """Preconditioned CG from x0 = 0 until ||r|| / ||r0|| <= tol.

    Returns (x, iterations, relative residual history)."""
    x = np.zeros_like(b)
    r = b.copy()
    minv = prob.mask / np.where(prob.diag != 0, prob.diag, 1.0) if precond == "jacobi" \
        else prob.mask.copy()
    z = minv * r
    p = z.copy()
    rz = prob.dot(r, z)
    r0 = np.sqrt(prob.dot(r, r))
    hist = [1.0]
    if r0 == 0:
        return x, 0, hist
    it = 0
    while it < maxit:
        w = prob.apply(p)
        alpha = rz / prob.dot(p, w)
        x += alpha * p
        r -= alpha * w
        it += 1
        rel = np.sqrt(prob.dot(r, r)) / r0
        hist.append(rel)
        if rel <= tol:
            break
        z = minv * r
        rz_new = prob.dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, hist


def poisson_rhs_f(x, y, z):
    """f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z), whose Dirichlet solution on
    the unit cube is sin(pi x) sin(pi y) sin(pi z)."""
    return 3.0 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


if __name__ == "__main__":  # pragma: no cover - manual build helper
    print(build(force="--force" in sys.argv))
