"""GB300 (sm_103a) spectral-element Poisson operator library.

The matrix-free element stiffness apply ("Ax") studied in "Portable
High-Performance Kernel Generation for a CFD Code with DaCe" (Listing 2),
with its gather-scatter and a conjugate-gradient Poisson solve, as
hand-written CUDA behind the C ABI of ``include/axhelm.h``.  This package is
the thin Python binding: it checks tensors and passes their addresses and
the current CUDA stream to the library; every step of the computation runs
in the library's kernels.  PyTorch supplies device memory and streams only.
"""
from __future__ import annotations

import os

import numpy as np

from . import _lib
from ._lib import (AX_BATCH_F32, AX_BATCH_F64, AX_MLP_SYM, AX_MLP_TANH, AX_PREC_BF16,
                   AX_PREC_F32, AX_VARIANT_AUTO,
                   AX_VARIANT_F64_DF, AX_VARIANT_F64_DF_EO,
                   AX_VARIANT_F64_NATIVE, AxError,
                   check, lib)

__all__ = [
    "lib", "AxError", "gll", "dmat", "box_geometry", "box_numbering", "ax_helm",
    "ax_helm_f32", "ax_helm_bf16", "AX_VARIANT_AUTO", "AX_VARIANT_F64_DF",
    "AX_VARIANT_F64_NATIVE", "AX_VARIANT_F64_DF_EO", "df64_roundtrip", "build", "GatherScatter", "Poisson",
    "AX_PREC_F32", "AX_PREC_BF16", "Batch", "tune", "tune_set", "tune_get", "AX_BATCH_F64",
    "AX_BATCH_F32", "fourier_coefficient", "Mlp", "mlp_init_params", "training_pairs", "train_mlp", "axpby", "iterate_pairs",
    "train_energy", "AX_MLP_TANH", "AX_MLP_SYM", "Operator", "ax_helm_h2", "ax_helm_xyz", "ax_helm_trilinear_f32", "box_corners", "ax_helm_host", "tune_variant",
    "tune_variant_set", "tune_variant_get", "tune_save", "tune_load",
]


def build(**kw) -> str:
    """Compile libaxhelm.so in-tree (see make.py)."""
    from . import make
    return make.build(**kw)


# ---------------------------------------------------------------------------
# host set-up (numpy in, numpy out)
# ---------------------------------------------------------------------------
def _addr(a: np.ndarray) -> int:
    assert a.flags.c_contiguous
    return a.ctypes.data


def gll(lx: int):
    """GLL nodes and weights (ax_gll)."""
    x = np.empty(lx)
    w = np.empty(lx)
    check("ax_gll", lib().ax_gll(lx, _addr(x), _addr(w)))
    return x, w


def dmat(lx: int):
    """(dx, dxt) buffers, dx[l*lx+i] = D_il, dxt[l*lx+i] = D_li (ax_dmat)."""
    dx = np.empty(lx * lx)
    dxt = np.empty(lx * lx)
    check("ax_dmat", lib().ax_dmat(lx, _addr(dx), _addr(dxt)))
    return dx, dxt


def box_corners(vertices: np.ndarray) -> np.ndarray:
    """(E, 2, 2, 2, 3) corner vertices [e][c][b][a][coord] of a box mesh
    given its (nz+1, ny+1, nx+1, 3) vertex array (ax_box_corners)."""
    v = np.ascontiguousarray(vertices, dtype=np.float64)
    nz, ny, nx = (s - 1 for s in v.shape[:3])
    out = np.empty((nx * ny * nz, 2, 2, 2, 3))
    check("ax_box_corners", lib().ax_box_corners(nx, ny, nz, _addr(v), _addr(out)))
    return out


def box_geometry(vertices: np.ndarray, lx: int, want_xyz: bool = False) -> dict:
    """Geometric factors, mass and (optionally) node coordinates of a box
    mesh given its (nz+1, ny+1, nx+1, 3) vertex array (ax_box_geometry)."""
    v = np.ascontiguousarray(vertices, dtype=np.float64)
    nz, ny, nx = (s - 1 for s in v.shape[:3])
    shape = (nx * ny * nz, lx, lx, lx)
    out = {k: np.empty(shape) for k in ("g11", "g22", "g33", "g12", "g13", "g23", "mass")}
    xyz = np.empty(shape + (3,)) if want_xyz else None
    rc = lib().ax_box_geometry(nx, ny, nz, lx, _addr(v),
                               *[_addr(out[k]) for k in ("g11", "g22", "g33", "g12", "g13",
                                                         "g23", "mass")],
                               _addr(xyz) if xyz is not None else None)
    check("ax_box_geometry", rc)
    if xyz is not None:
        out["xyz"] = xyz
    return out


def box_numbering(nx: int, ny: int, nz: int, lx: int) -> np.ndarray:
    g = np.empty((nx * ny * nz, lx, lx, lx), dtype=np.int64)
    check("ax_box_numbering", lib().ax_box_numbering(nx, ny, nz, lx, _addr(g)))
    return g


def box_mask(nx: int, ny: int, nz: int, lx: int, dirichlet=(True,) * 6) -> np.ndarray:
    """Dirichlet mask of the box (ax_box_mask): 0 on the marked faces
    (x0, x1, y0, y1, z0, z1), 1 elsewhere."""
    d = np.asarray([1 if f else 0 for f in dirichlet], dtype=np.int32)
    m = np.empty((nx * ny * nz, lx, lx, lx))
    check("ax_box_mask", lib().ax_box_mask(nx, ny, nz, lx, _addr(d), _addr(m)))
    return m


def df64_roundtrip(x: np.ndarray):
    """Host twin of the device fp64 <-> fp32-pair conversion (diagnostic)."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    hi = np.empty(x.size, dtype=np.float32)
    lo = np.empty(x.size, dtype=np.float32)
    back = np.empty(x.size)
    check("ax_df64_roundtrip", lib().ax_df64_roundtrip(_addr(x), _addr(hi), _addr(lo),
                                                       _addr(back), x.size))
    return hi, lo, back


# ---------------------------------------------------------------------------
# device calls (torch CUDA tensors in and out)
# ---------------------------------------------------------------------------
def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _dev_args(lx, w, tensors, dtypes, d_tensors, d_dtype):
    import torch
    n = None
    for t, dt in zip([w] + list(tensors), dtypes):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("expected CUDA tensors")
        if t.dtype != dt:
            raise TypeError(f"expected {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")
        if n is None:
            n = t.numel()
        elif t.numel() != n:
            raise ValueError("all element fields must have the same size")
    for t in d_tensors:
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == d_dtype
                and t.is_contiguous() and t.numel() == lx * lx):
            raise ValueError(f"dx/dxt must be contiguous {d_dtype} CUDA tensors of lx*lx values")
    if n % (lx ** 3):
        raise ValueError("field size is not a multiple of lx^3")
    return n // (lx ** 3)


def ax_helm(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, lx: int,
            variant: int = AX_VARIANT_AUTO, elems_per_block: int = 0) -> None:
    """w <- element-local stiffness apply of u, fp64 (ax_helm_variant)."""
    import torch
    f = torch.float64
    nel = _dev_args(lx, w, [u, h1, g11, g22, g33, g12, g13, g23], [f] * 9, [dx, dxt], f)
    rc = lib().ax_helm_variant(variant, w.data_ptr(), u.data_ptr(), dx.data_ptr(),
                               dxt.data_ptr(), h1.data_ptr(), g11.data_ptr(), g22.data_ptr(),
                               g33.data_ptr(), g12.data_ptr(), g13.data_ptr(), g23.data_ptr(),
                               lx, nel, elems_per_block, _stream())
    check("ax_helm", rc)


def ax_helm_xyz(w, u, dx, dy, dz, dxt, dyt, dzt, h1, g11, g22, g33, g12, g13, g23,
                lx: int) -> None:
    """w <- element-local stiffness apply of u with one matrix per direction
    (the full argument list of Listings 1-2), fp64 (ax_helm_xyz)."""
    import torch
    f = torch.float64
    nel = _dev_args(lx, w, [u, h1, g11, g22, g33, g12, g13, g23], [f] * 9,
                    [dx, dy, dz, dxt, dyt, dzt], f)
    ts = [w, u, dx, dy, dz, dxt, dyt, dzt, h1, g11, g22, g33, g12, g13, g23]
    check("ax_helm_xyz", lib().ax_helm_xyz(*[t.data_ptr() for t in ts], lx, nel, _stream()))


def ax_helm_trilinear_f32(w, u, dx, dxt, h1, corners, xi, wq, lx: int) -> None:
    """fp32 operator with G computed from each element's corner vertices
    (ax_helm_trilinear_f32).  w, u, dx, dxt, h1: fp32 CUDA tensors (h1 may
    be None: h1 = 1); corners (E*24), xi, wq (lx): fp64 CUDA tensors."""
    import torch
    f = torch.float32
    fields = [u] if h1 is None else [u, h1]
    nel = _dev_args(lx, w, fields, [f] * (len(fields) + 1), [dx, dxt], f)
    for t, size in ((corners, nel * 24), (xi, lx), (wq, lx)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                and t.is_contiguous() and t.numel() == size):
            raise ValueError("corners, xi, wq must be contiguous fp64 CUDA tensors")
    check("ax_helm_trilinear_f32", lib().ax_helm_trilinear_f32(
        w.data_ptr(), u.data_ptr(), dx.data_ptr(), dxt.data_ptr(),
        None if h1 is None else h1.data_ptr(), corners.data_ptr(), xi.data_ptr(),
        wq.data_ptr(), lx, nel, _stream()))


def ax_helm_host(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, lx: int,
                 chunk: int = 0) -> None:
    """The fp64 operator on host (CPU, preferably pinned) tensors: chunks of
    elements stream through the device with copies and apply overlapped
    (ax_helm_host).  Synchronous."""
    ts = [w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23]
    for t in ts:
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("ax_helm_host needs contiguous host tensors")
    nelv = u.numel() // lx ** 3
    check("ax_helm_host", lib().ax_helm_host(*[t.data_ptr() for t in ts], lx, nelv, chunk,
                                             _stream()))


def ax_helm_h2(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, h2, B, lx: int) -> None:
    """Helmholtz form w = Ax(u) + h2 .* B .* u (fp64 CUDA tensors)."""
    ts = [w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, h2, B]
    nelv = u.numel() // lx ** 3
    check("ax_helm_h2", lib().ax_helm_h2(*[t.data_ptr() for t in ts], lx, nelv, _stream()))


def ax_helm_f32(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, lx: int) -> None:
    """fp32 storage and arithmetic (ax_helm_f32)."""
    import torch
    f = torch.float32
    nel = _dev_args(lx, w, [u, h1, g11, g22, g33, g12, g13, g23], [f] * 9, [dx, dxt], f)
    rc = lib().ax_helm_f32(w.data_ptr(), u.data_ptr(), dx.data_ptr(), dxt.data_ptr(),
                           h1.data_ptr(), g11.data_ptr(), g22.data_ptr(), g33.data_ptr(),
                           g12.data_ptr(), g13.data_ptr(), g23.data_ptr(), lx, nel, _stream())
    check("ax_helm_f32", rc)


def ax_helm_bf16(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, lx: int) -> None:
    """bf16 storage of u, h1, G; fp32 D, arithmetic and w (ax_helm_bf16)."""
    import torch
    b = torch.bfloat16
    nel = _dev_args(lx, w, [u, h1, g11, g22, g33, g12, g13, g23],
                    [torch.float32] + [b] * 8, [dx, dxt], torch.float32)
    rc = lib().ax_helm_bf16(w.data_ptr(), u.data_ptr(), dx.data_ptr(), dxt.data_ptr(),
                            h1.data_ptr(), g11.data_ptr(), g22.data_ptr(), g33.data_ptr(),
                            g12.data_ptr(), g13.data_ptr(), g23.data_ptr(), lx, nel, _stream())
    check("ax_helm_bf16", rc)


# ---------------------------------------------------------------------------
# gather-scatter and the Poisson solvers
# ---------------------------------------------------------------------------
class _DeviceArray:
    """A borrowed device array exposed through __cuda_array_interface__ so
    torch can view memory the library owns (no copy)."""

    def __init__(self, ptr: int, n: int, typestr: str, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


class Operator:
    """The element operator of one mesh for repeated applies (ax_op_*).
    Keeps references to the borrowed device arrays; for lx in {6, 8, 10, 12}
    the library holds the geometry in the persistent even-odd kernel's
    prepared order."""

    def __init__(self, lx: int, dx, dxt, h1, g11, g22, g33, g12, g13, g23):
        import ctypes
        self.lx, self.nelv = lx, h1.numel() // lx ** 3
        self._keep = [dx, dxt, h1, g11, g22, g33, g12, g13, g23]
        h = ctypes.c_void_p()
        check("ax_op_create", lib().ax_op_create(
            ctypes.addressof(h), lx, self.nelv, *[t.data_ptr() for t in self._keep],
            _stream()))
        self._h = h

    def apply(self, w, u) -> None:
        check("ax_op_apply", lib().ax_op_apply(self._h, w.data_ptr(), u.data_ptr(), _stream()))

    def set_h1(self, h1) -> None:
        check("ax_op_set_h1", lib().ax_op_set_h1(self._h, h1.data_ptr(), _stream()))
        self._keep[2] = h1

    def set_h2(self, h2, B) -> None:
        """Adds the Helmholtz mass term h2 .* B .* u (h2 None removes it)."""
        check("ax_op_set_h2", lib().ax_op_set_h2(
            self._h, None if h2 is None else h2.data_ptr(),
            None if B is None else B.data_ptr(), _stream()))

    def info(self):
        import ctypes
        p, b = ctypes.c_int(), ctypes.c_int64()
        check("ax_op_info", lib().ax_op_info(self._h, ctypes.addressof(p), ctypes.addressof(b)))
        return {"prepared": bool(p.value), "device_bytes": b.value}

    def error(self) -> int:
        """1 if a launch gave up waiting for a staged geometry copy (synchronises)."""
        import ctypes
        f = ctypes.c_int()
        check("ax_op_error", lib().ax_op_error(self._h, ctypes.addressof(f)))
        return f.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.ax_op_destroy(h)
            self._h = None


class GatherScatter:
    """Direct-stiffness summation over shared nodes (ax_gs_*)."""

    def __init__(self, glob: np.ndarray):
        import ctypes
        g = np.ascontiguousarray(glob, dtype=np.int64).ravel()
        h = ctypes.c_void_p()
        check("ax_gs_setup", lib().ax_gs_setup(ctypes.addressof(h), _addr(g), g.size, _stream()))
        self._h = h
        self.n_local = g.size

    @property
    def handle(self):
        return self._h

    def sum(self, v) -> None:
        import torch
        if v.dtype == torch.float64:
            check("ax_gs_sum", lib().ax_gs_sum(self._h, v.data_ptr(), _stream()))
        elif v.dtype == torch.float32:
            check("ax_gs_sum_f32", lib().ax_gs_sum_f32(self._h, v.data_ptr(), _stream()))
        else:
            raise TypeError("gs sum needs fp64 or fp32")

    def info(self):
        import ctypes
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check("ax_gs_info", lib().ax_gs_info(self._h, ctypes.addressof(a), ctypes.addressof(b),
                                             ctypes.addressof(c)))
        return {"n_local": a.value, "n_shared": b.value, "n_copies": c.value}

    def inverse_multiplicity(self):
        import torch
        ptr = lib().ax_gs_inverse_multiplicity(self._h)
        return torch.as_tensor(_DeviceArray(ptr, self.n_local, "<f8", self), device="cuda")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.ax_gs_free(h)
            self._h = None


def fourier_coefficient(seed: int, lo: float = 0.5, hi: float = 2.0):
    """Smooth variable coefficient: the sum of 8 random Fourier modes
    (synth.fourier_modes) rescaled affinely into [lo, hi] over the nodes it
    is evaluated on.  Returns a callable h1(x, y, z)."""
    from . import synth
    a, k, phi = synth.fourier_modes(seed)

    def h1(x, y, z):
        raw = sum(a[m] * np.sin(k[m, 0] * x + k[m, 1] * y + k[m, 2] * z + phi[m])
                  for m in range(len(a)))
        r0, r1 = raw.min(), raw.max()
        return lo + (hi - lo) * (raw - r0) / max(r1 - r0, 1e-300)
    return h1


class Poisson:
    """Poisson problem -div(h1 grad u) = f on a perturbed box with
    homogeneous Dirichlet boundaries, set up on the host by the library
    and solved on the GPU (ax_poisson_*, ax_cg_solve, ax_mpcg_solve)."""

    GKEYS = ("g11", "g22", "g33", "g12", "g13", "g23")

    def __init__(self, vertices: np.ndarray, lx: int, h1=None, device=None,
                 dirichlet=(True, True, True, True, True, True), h2=None):
        """dirichlet: which faces (x0, x1, y0, y1, z0, z1) carry the
        homogeneous Dirichlet condition; a face left open is an interface to
        another partition (see ``dist``).  h2 (callable, array or scalar)
        makes it the Helmholtz problem -div(h1 grad u) + h2 u = f."""
        import ctypes
        import torch
        self.device = torch.device("cuda") if device is None else torch.device(device)
        v = np.ascontiguousarray(vertices, dtype=np.float64)
        nz, ny, nx = (s - 1 for s in v.shape[:3])
        self.dims, self.lx = (nx, ny, nz), lx
        geo = box_geometry(v, lx, want_xyz=True)
        self.nelv = nx * ny * nz
        self.xyz = geo["xyz"]
        self.mass_host = geo["mass"]
        glob = box_numbering(nx, ny, nz, lx)
        self.glob = glob
        mask = box_mask(nx, ny, nz, lx, dirichlet)
        if callable(h1):
            h1 = h1(self.xyz[..., 0], self.xyz[..., 1], self.xyz[..., 2])
        if h1 is not None and np.size(h1) == mask.size:
            h1 = np.reshape(h1, mask.shape)
        h1v = np.ones_like(mask) if h1 is None else np.broadcast_to(
            np.asarray(h1, dtype=np.float64), mask.shape).copy()
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=self.device)
        dx, dxt = dmat(lx)
        self.d = {"dx": t(dx), "dxt": t(dxt), "h1": t(h1v), "mask": t(mask)}
        for k in self.GKEYS:
            self.d[k] = t(geo[k])
        self.mass = t(geo["mass"])
        with torch.cuda.device(self.device):
            self.gs = GatherScatter(glob)
            h = ctypes.c_void_p()
            d = self.d
            rc = lib().ax_poisson_create(
                ctypes.addressof(h), lx, self.nelv, d["dx"].data_ptr(), d["dxt"].data_ptr(),
                d["h1"].data_ptr(), *[d[k].data_ptr() for k in self.GKEYS],
                d["mask"].data_ptr(), self.gs.handle, _stream())
            check("ax_poisson_create", rc)
        self._h = h
        self.shape = mask.shape
        if h2 is not None:
            if callable(h2):
                h2 = h2(self.xyz[..., 0], self.xyz[..., 1], self.xyz[..., 2])
            h2v = np.broadcast_to(np.asarray(h2, dtype=np.float64).reshape(
                mask.shape) if np.size(h2) == mask.size else np.asarray(h2, dtype=np.float64),
                mask.shape).copy()
            self.d["h2"] = t(h2v)
            check("ax_poisson_set_h2", lib().ax_poisson_set_h2(
                self._h, self.d["h2"].data_ptr(), self.mass.data_ptr(), _stream()))

    def rhs(self, f) -> "torch.Tensor":
        """b = mask .* gs(B f) (ax_poisson_rhs) for a callable source f(x, y, z),
        sampled at the nodes on the host."""
        import torch
        x = self.xyz
        fv = f(x[..., 0], x[..., 1], x[..., 2])
        b = torch.as_tensor(np.ascontiguousarray(fv, dtype=np.float64), device=self.device)
        check("ax_poisson_rhs", lib().ax_poisson_rhs(self._h, self.mass.data_ptr(),
                                                     b.data_ptr(), b.data_ptr(), _stream()))
        return b

    def apply(self, w, u) -> None:
        check("ax_poisson_apply", lib().ax_poisson_apply(self._h, w.data_ptr(), u.data_ptr(),
                                                         _stream()))

    def jacobi(self):
        import ctypes
        import torch
        p = ctypes.c_void_p()
        check("ax_poisson_jacobi", lib().ax_poisson_jacobi(self._h, ctypes.addressof(p)))
        n = int(np.prod(self.shape))
        return torch.as_tensor(_DeviceArray(p.value, n, "<f8", self), device=self.device)

    def diag(self):
        """Assembled (over this handle's nodes), unmasked Jacobi diagonal."""
        import torch
        d = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        check("ax_poisson_diag", lib().ax_poisson_diag(self._h, d.data_ptr(), _stream()))
        return d

    def set_diag(self, d) -> None:
        """Use mask ./ d as the inverse Jacobi diagonal (d assembled by the caller)."""
        check("ax_poisson_set_diag", lib().ax_poisson_set_diag(self._h, d.data_ptr(), _stream()))

    def set_check_every(self, k: int) -> None:
        check("ax_poisson_set_check_every", lib().ax_poisson_set_check_every(self._h, k))

    def cg(self, b, tol=1e-8, maxit=10000, raise_on_error=True):
        """Jacobi-PCG in fp64; returns (x, iterations, relative residual, status)."""
        import ctypes
        import torch
        x = torch.empty_like(b)
        it, rel = ctypes.c_int(), ctypes.c_double()
        rc = lib().ax_cg_solve(self._h, x.data_ptr(), b.data_ptr(), tol, maxit,
                               ctypes.addressof(it), ctypes.addressof(rel), _stream())
        if raise_on_error and rc not in (0, _lib.AX_ENOTCONV):
            check("ax_cg_solve", rc)
        return x, it.value, rel.value, rc

    def mpcg(self, b, mode=_lib.AX_PREC_F32, tol=1e-8, inner_tol=1e-4, max_outer=50,
             max_inner=10000, raise_on_error=True):
        """fp64 iterative refinement around an fp32 (or bf16-data) inner PCG;
        returns (x, outer iterations, inner iterations, relres, status)."""
        import ctypes
        import torch
        x = torch.empty_like(b)
        no, ni, rel = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        rc = lib().ax_mpcg_solve(self._h, mode, x.data_ptr(), b.data_ptr(), tol, inner_tol,
                                 max_outer, max_inner, ctypes.addressof(no),
                                 ctypes.addressof(ni), ctypes.addressof(rel), _stream())
        if raise_on_error and rc not in (0, _lib.AX_ENOTCONV):
            check("ax_mpcg_solve", rc)
        return x, no.value, ni.value, rel.value, rc

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.ax_poisson_destroy(h)
            self._h = None


# ---------------------------------------------------------------------------
# batched multi-mesh launch and the elements-per-block autotuner
# ---------------------------------------------------------------------------
_FIELDS = ("w", "u", "dx", "dxt", "h1", "g11", "g22", "g33", "g12", "g13", "g23")


class Batch:
    """Many meshes (each a dict of CUDA tensors with keys w, u, dx, dxt, h1,
    g11..g23 and an int "lx") in one persistent launch (ax_batch_*)."""

    def __init__(self, meshes, dtype=_lib.AX_BATCH_F64, blocks_per_sm: int = 0):
        import ctypes
        import torch
        want = torch.float64 if dtype == _lib.AX_BATCH_F64 else torch.float32
        arr = (_lib.BatchMesh * max(1, len(meshes)))()
        for q, m in enumerate(meshes):
            lx = int(m["lx"])
            for k in _FIELDS:
                t = m[k]
                if t.dtype != want or not t.is_cuda or not t.is_contiguous():
                    raise TypeError(f"mesh {q}: {k} must be a contiguous CUDA {want} tensor")
            nel = m["u"].numel() // lx ** 3
            arr[q].lx, arr[q].nelv = lx, nel
            for k in _FIELDS:
                setattr(arr[q], k, m[k].data_ptr())
        self._meshes = meshes  # keep the tensors alive
        h = ctypes.c_void_p()
        check("ax_batch_create", lib().ax_batch_create(ctypes.addressof(h), dtype, len(meshes),
                                                       ctypes.addressof(arr), blocks_per_sm,
                                                       _stream()))
        self._h = h

    def launch(self, graph: bool = False) -> None:
        if graph:
            check("ax_batch_graph_launch", lib().ax_batch_graph_launch(self._h, _stream()))
        else:
            check("ax_batch_launch", lib().ax_batch_launch(self._h, _stream()))

    def info(self) -> dict:
        import ctypes
        a, b = ctypes.c_int(), ctypes.c_int()
        s, f, y = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        check("ax_batch_info", lib().ax_batch_info(self._h, *[ctypes.addressof(x) for x in
                                                              (a, b, s, f, y)]))
        return {"items": a.value, "blocks": b.value, "smem": s.value, "flops": f.value,
                "bytes": y.value}

    def error(self) -> int:
        """1 if a launch gave up waiting for a staged geometry copy (synchronises)."""
        import ctypes
        f = ctypes.c_int()
        check("ax_batch_error", lib().ax_batch_error(self._h, ctypes.addressof(f)))
        return f.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.ax_batch_destroy(h)
            self._h = None


def tune(dtype: int, lx: int, fields: dict, reps: int = 5):
    """Times every elements-per-block choice for (dtype, lx) on the given
    tensors (keys as in Batch; w is overwritten), records and returns
    (best_epb, best_ms)."""
    import ctypes
    nel = fields["u"].numel() // lx ** 3
    e, ms = ctypes.c_int(), ctypes.c_float()
    rc = lib().ax_tune_run(dtype, lx, nel, *[fields[k].data_ptr() for k in _FIELDS], reps,
                           ctypes.addressof(e), ctypes.addressof(ms), _stream())
    check("ax_tune_run", rc)
    return e.value, ms.value


def tune_set(dtype: int, lx: int, epb: int) -> None:
    check("ax_tune_set", lib().ax_tune_set(dtype, lx, epb))


def tune_get(dtype: int, lx: int) -> int:
    import ctypes
    e = ctypes.c_int()
    check("ax_tune_get", lib().ax_tune_get(dtype, lx, ctypes.addressof(e)))
    return e.value


def tune_save(path: str) -> None:
    """Writes the tuned elements-per-block and fp64-variant tables to a text
    file (ax_tune_save)."""
    check("ax_tune_save", lib().ax_tune_save(os.fsencode(path)))


def tune_load(path: str) -> None:
    """Reads tables written by tune_save and applies them, all or nothing
    (ax_tune_load)."""
    check("ax_tune_load", lib().ax_tune_load(os.fsencode(path)))


def tune_variant(lx: int, fields: dict, reps: int = 5):
    """Times the fp64 variants for lx on the given fp64 tensors (keys as in
    Batch; w is overwritten), records the fastest for AX_VARIANT_AUTO and
    returns (variant, ms)."""
    import ctypes
    nel = fields["u"].numel() // lx ** 3
    v, ms = ctypes.c_int(), ctypes.c_float()
    check("ax_tune_variant_run", lib().ax_tune_variant_run(
        lx, nel, *[fields[k].data_ptr() for k in _FIELDS], reps, ctypes.addressof(v),
        ctypes.addressof(ms), _stream()))
    return v.value, ms.value


def tune_variant_set(lx: int, variant: int) -> None:
    check("ax_tune_variant_set", lib().ax_tune_variant_set(lx, variant))


def tune_variant_get(lx: int) -> int:
    import ctypes
    v = ctypes.c_int()
    check("ax_tune_variant_get", lib().ax_tune_variant_get(lx, ctypes.addressof(v)))
    return v.value


# ---------------------------------------------------------------------------
# learned element preconditioner
# ---------------------------------------------------------------------------
def axpby(y, a: float, x, b: float) -> None:
    """y <- a x + b y (fp64 CUDA tensors, ax_axpby)."""
    check("ax_axpby", lib().ax_axpby(y.data_ptr(), a, x.data_ptr(), b, y.numel(), _stream()))


def mlp_init_params(n_in: int, n_hid: int, seed: int = 0, arch: int = AX_MLP_TANH,
                    scale: float = 0.05) -> np.ndarray:
    """Initial parameters.  Tanh form: W1 uniform in +-sqrt(6/(n_in+n_hid))
    (Glorot), b1 = 0 and a zero output layer, so the untrained preconditioner
    is exactly Jacobi.  Symmetric form: W = W1 = W2^T uniform in
    +-scale/sqrt(n_hid) (the gradient vanishes at W = 0, so W starts small but
    not zero).  Random numbers come from ``synth``."""
    from . import synth
    if arch == AX_MLP_SYM:
        lim = scale / np.sqrt(n_hid)
        W1 = synth.uniform((n_in, n_hid), seed, -lim, lim)
        return np.concatenate([W1.ravel(), np.zeros(n_hid), W1.T.ravel(),
                               np.zeros(n_in)]).astype(np.float32)
    lim = np.sqrt(6.0 / (n_in + n_hid))
    W1 = synth.uniform((n_in, n_hid), seed, -lim, lim)
    return np.concatenate([W1.ravel(), np.zeros(n_hid), np.zeros(n_hid * n_in),
                           np.zeros(n_in)]).astype(np.float32)


class Mlp:
    """The per-element network of the learned preconditioner (ax_mlp_*)."""

    def __init__(self, n_in: int, n_hid: int = 48, params=None, arch: int = AX_MLP_TANH):
        import ctypes
        h = ctypes.c_void_p()
        check("ax_mlp_create_ex", lib().ax_mlp_create_ex(ctypes.addressof(h), n_in, n_hid, arch))
        self._h, self.n_in, self.n_hid, self.arch = h, n_in, n_hid, arch
        n = ctypes.c_int64()
        check("ax_mlp_nparams", lib().ax_mlp_nparams(h, ctypes.addressof(n)))
        self.nparams = n.value
        if params is not None:
            self.set_params(params)

    @property
    def handle(self):
        return self._h

    def set_params(self, params) -> None:
        p = np.ascontiguousarray(params, dtype=np.float32).ravel()
        check("ax_mlp_set_params", lib().ax_mlp_set_params(self._h, _addr(p), p.size, _stream()))

    def get_params(self) -> np.ndarray:
        p = np.empty(self.nparams, dtype=np.float32)
        check("ax_mlp_get_params", lib().ax_mlp_get_params(self._h, _addr(p), p.size, _stream()))
        return p

    def loss_grad(self, X, T):
        import ctypes
        B = X.shape[0]
        loss = ctypes.c_double()
        g = np.empty(self.nparams, dtype=np.float32)
        check("ax_mlp_loss_grad", lib().ax_mlp_loss_grad(self._h, X.data_ptr(), T.data_ptr(), B,
                                                         ctypes.addressof(loss), _addr(g),
                                                         _stream()))
        return loss.value, g

    def adam(self, lr: float, beta1=0.9, beta2=0.999, eps=1e-8) -> None:
        check("ax_mlp_adam", lib().ax_mlp_adam(self._h, lr, beta1, beta2, eps, _stream()))

    def gather_pairs(self, r, err, minv, idx):
        """(X, T) fp32 CUDA tensors for the element ids idx (int32 tensor)."""
        import torch
        n = idx.numel()
        X = torch.empty((n, self.n_in), dtype=torch.float32, device=r.device)
        T = torch.empty_like(X)
        check("ax_mlp_gather_pairs", lib().ax_mlp_gather_pairs(
            self._h, r.data_ptr(), err.data_ptr(), minv.data_ptr(), idx.data_ptr(), n,
            X.data_ptr(), T.data_ptr(), _stream()))
        return X, T

    def train(self, X, T, perm, epochs: int, batch: int, lr: float) -> float:
        import ctypes
        loss = ctypes.c_double()
        check("ax_mlp_train", lib().ax_mlp_train(self._h, X.data_ptr(), T.data_ptr(),
                                                 X.shape[0], perm.data_ptr(), epochs, batch,
                                                 lr, ctypes.addressof(loss), _stream()))
        return loss.value

    def forward(self, corr, r, minv, mask, c, nelv: int) -> None:
        check("ax_mlp_forward", lib().ax_mlp_forward(self._h, r.data_ptr(), minv.data_ptr(),
                                                     mask.data_ptr(), c.data_ptr(),
                                                     corr.data_ptr(), nelv, _stream()))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.ax_mlp_destroy(h)
            self._h = None


def _poisson_fcg(self, b, mlp=None, tol=1e-8, maxit=10000, raise_on_error=True):
    """Flexible CG with the learned preconditioner (Jacobi if mlp is None);
    returns (x, iterations, relres, fallbacks, status)."""
    import ctypes
    import torch
    x = torch.empty_like(b)
    it, rel, fb = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
    rc = lib().ax_fcg_solve(self._h, mlp.handle if mlp is not None else None, x.data_ptr(),
                            b.data_ptr(), tol, maxit, ctypes.addressof(it),
                            ctypes.addressof(rel), ctypes.addressof(fb), _stream())
    if raise_on_error and rc not in (0, _lib.AX_ENOTCONV):
        check("ax_fcg_solve", rc)
    return x, it.value, rel.value, fb.value, rc


def _poisson_mpfcg(self, b, mlp=None, mode=_lib.AX_PREC_F32, tol=1e-8, inner_tol=1e-4,
                   max_outer=50, max_inner=10000, raise_on_error=True):
    """fp64 refinement around the fp32 flexible CG with the learned
    preconditioner; returns (x, outer, inner, relres, fallbacks, status)."""
    import ctypes
    import torch
    x = torch.empty_like(b)
    no, ni, rel, fb = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
    rc = lib().ax_mpfcg_solve(self._h, mlp.handle if mlp is not None else None, mode,
                              x.data_ptr(), b.data_ptr(), tol, inner_tol, max_outer, max_inner,
                              ctypes.addressof(no), ctypes.addressof(ni), ctypes.addressof(rel),
                              ctypes.addressof(fb), _stream())
    if raise_on_error and rc not in (0, _lib.AX_ENOTCONV):
        check("ax_mpfcg_solve", rc)
    return x, no.value, ni.value, rel.value, fb.value, rc


def _poisson_precondition(self, r, mlp=None):
    import torch
    z = torch.empty_like(r)
    check("ax_precondition", lib().ax_precondition(self._h, mlp.handle if mlp is not None
                                                   else None, z.data_ptr(), r.data_ptr(),
                                                   _stream()))
    return z


def _poisson_residual(self, b, x):
    """r = mask .* (b - A x) (fp64)."""
    import torch
    w = torch.empty_like(x)
    self.apply(w, x)
    r = b.clone()
    axpby(r, -1.0, w, 1.0)
    return r


Poisson.fcg = _poisson_fcg
Poisson.mpfcg = _poisson_mpfcg
Poisson.precondition = _poisson_precondition
Poisson.residual = _poisson_residual


def training_pairs(P: "Poisson", b, mlp: Mlp, n_pairs: int = 10240, iterates=(2, 4, 8, 16,
                   32, 64, 128), seed: int = 0, xstar=None):
    """Element training pairs from plain Jacobi-CG iterates x_k of P x = b:
    r_k = b - A x_k and err_k = x* - x_k with x* solved to 1e-12; n_pairs
    elements drawn uniformly (synth) across the iterates.  Returns fp32
    CUDA tensors (X, T)."""
    import torch
    from . import synth
    if xstar is None:
        xstar, _, _, _ = P.cg(b, tol=1e-12)
    minv = P.jacobi()
    per = -(-n_pairs // len(iterates))
    g = synth.rng(seed)
    Xs, Ts = [], []
    for k in iterates:
        xk, _, _, _ = P.cg(b, tol=0.0, maxit=k, raise_on_error=False)
        r = P.residual(b, xk)
        err = xstar.clone()
        axpby(err, -1.0, xk, 1.0)
        idx = torch.as_tensor(g.integers(0, P.nelv, size=per).astype(np.int32), device=b.device)
        X, T = mlp.gather_pairs(r, err, minv, idx)
        Xs.append(X)
        Ts.append(T)
    return torch.cat(Xs)[:n_pairs].contiguous(), torch.cat(Ts)[:n_pairs].contiguous()


def train_mlp(mlp: Mlp, X, T, epochs: int = 30, batch: int = 512, lr: float = 1e-3,
              seed: int = 0) -> float:
    """Adam over the sample set with per-epoch permutations from synth."""
    import torch
    from . import synth
    g = synth.rng(seed)
    n = X.shape[0]
    perm = np.concatenate([g.permutation(n) for _ in range(epochs)]).astype(np.int32)
    perm_t = torch.as_tensor(perm, device=X.device)
    return mlp.train(X, T, perm_t, epochs, batch, lr)


def iterate_pairs(P: "Poisson", b, iterates=(2, 4, 8, 16, 32, 64, 128, 256), xstar=None):
    """Residual/error pairs of plain Jacobi-CG on P x = b: for every k in
    iterates, r_k = mask .* (b - A x_k) and e_k = x* - x_k (x* solved to
    1e-12).  Returns two fp64 CUDA tensors of shape (K, n)."""
    import torch
    if xstar is None:
        xstar, _, _, _ = P.cg(b, tol=1e-12)
    R = torch.empty((len(iterates), b.numel()), dtype=torch.float64, device=b.device)
    E = torch.empty_like(R)
    for q, k in enumerate(iterates):
        xk, _, _, _ = P.cg(b, tol=0.0, maxit=k, raise_on_error=False)
        R[q] = P.residual(b, xk).reshape(-1)
        e = xstar.clone()
        axpby(e, -1.0, xk, 1.0)
        E[q] = e.reshape(-1)
    return R, E


def train_energy(P: "Poisson", mlp: Mlp, R, E, epochs: int = 50, lr: float = 1e-3) -> float:
    """Energy-norm training on the pairs (R[k], E[k]) (ax_mlp_train_energy);
    returns the mean relative energy error of the last pass."""
    import ctypes
    loss = ctypes.c_double()
    check("ax_mlp_train_energy", lib().ax_mlp_train_energy(
        P._h, mlp.handle, R.data_ptr(), E.data_ptr(), R.shape[0], epochs, lr,
        ctypes.addressof(loss), _stream()))
    return loss.value
