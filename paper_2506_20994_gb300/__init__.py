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

import numpy as np

from . import _lib
from ._lib import (AX_VARIANT_AUTO, AX_VARIANT_F64_DF, AX_VARIANT_F64_NATIVE, AxError,
                   check, lib)

__all__ = [
    "lib", "AxError", "gll", "dmat", "box_geometry", "box_numbering", "ax_helm",
    "ax_helm_f32", "ax_helm_bf16", "AX_VARIANT_AUTO", "AX_VARIANT_F64_DF",
    "AX_VARIANT_F64_NATIVE", "df64_roundtrip", "build",
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
