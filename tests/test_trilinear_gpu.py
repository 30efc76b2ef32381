"""GPU parity of the fp32 operator with on-the-fly trilinear geometry
(ax_helm_trilinear_f32) against the fp64 oracle.

The oracle's side is its stored-geometry operator with G from
``oracle.box_geometry`` (node coordinates differentiated by D, fp64); the
kernel forms G from the 8 corner vertices per point in fp32.  Tolerance:
relative L2 1e-6, the fp32-storage bar of ax_helm_f32.  Sizes: ragged E for
lx across the range, h1 variable or constant (NULL), strongly perturbed
vertices, and the full 32^3 box at lx = 8 on sampled elements.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2506_20994_gb300 as ax  # noqa: E402
from paper_2506_20994_gb300 import synth  # noqa: E402

from _cases import GKEYS, operator_case, rel_l2  # noqa: E402

TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ax.build()


def _f32(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float32)


def _f64(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


def _run(u, h1, vertices, lx):
    xi, wq = ax.gll(lx)
    dx, dxt = ax.dmat(lx)
    uu = _f32(u)
    w = torch.full_like(uu, float("nan"))
    ax.ax_helm_trilinear_f32(w, uu, _f32(dx), _f32(dxt), None if h1 is None else _f32(h1),
                             _f64(ax.box_corners(vertices)), _f64(xi), _f64(wq), lx)
    torch.cuda.synchronize()
    return w.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("lx", [2, 3, 4, 5, 6, 7, 8, 10, 12, 13, 16])
def test_trilinear_parity(lx):
    dims = (3, 2, 2) if lx <= 12 else (2, 1, 1)
    case = operator_case(dims, lx, seed=400 + lx)
    w = _run(case["u"], case["h1"], case["vertices"], lx)
    assert rel_l2(w, case["w"]) <= TOL


@pytest.mark.parametrize("lx", [5, 8])
def test_trilinear_constant_h1(lx):
    """h1 = NULL is h1 = 1 (the Poisson operator; 8 bytes per point)."""
    case = operator_case((5, 3, 1), lx, seed=11, h1_const=1.0)
    w = _run(case["u"], None, case["vertices"], lx)
    assert rel_l2(w, case["w"]) <= TOL


def test_trilinear_matches_stored_fp32():
    """Against ax_helm_f32 on the same mesh with G rounded to fp32: the two
    fp32 operators differ only in where G comes from."""
    lx = 8
    case = operator_case((4, 4, 4), lx, seed=13)
    w_tri = _run(case["u"], case["h1"], case["vertices"], lx)
    args = [_f32(case[k]) for k in ("u", "dx", "dxt", "h1") + GKEYS]
    w = torch.empty_like(args[0])
    ax.ax_helm_f32(w, *args, lx)
    torch.cuda.synchronize()
    assert rel_l2(w_tri, w.cpu().numpy()) <= TOL


def test_trilinear_strongly_perturbed():
    """Vertices moved by up to 0.3 h (far from affine, jac still > 0)."""
    lx = 6
    v = synth.box_vertices(3, 3, 2, seed=8, amp=0.3)
    geo = oracle.box_geometry(v, lx)
    u = synth.uniform(geo["jac"].shape, seed=9)
    h1 = synth.uniform(geo["jac"].shape, seed=10, lo=0.5, hi=2.0)
    dx, dxt = oracle.d_buffers(lx)
    ref = oracle.ax_helm(u, dx, dxt, h1, *[geo[k] for k in GKEYS], lx)
    assert rel_l2(_run(u, h1, v, lx), ref) <= TOL


def test_trilinear_full_size_sampled():
    """The 32^3 box at lx = 8 (E = 32768) in one launch; 24 elements
    (first, last, random) checked one by one against the oracle."""
    lx, n = 8, 32
    v = synth.box_vertices(n, seed=0)
    nel = n ** 3
    u = synth.uniform((nel, lx, lx, lx), seed=1)
    w = _run(u, None, v, lx)
    rng = np.random.default_rng(3)
    idx = np.unique(np.concatenate([[0, nel - 1], rng.integers(0, nel, 22)]))
    geo = oracle.box_geometry(v, lx, elements=idx)
    dx, dxt = oracle.d_buffers(lx)
    ref = oracle.ax_helm(u[idx], dx, dxt, np.ones((idx.size, lx, lx, lx)),
                         *[geo[k] for k in GKEYS], lx)
    assert rel_l2(w[idx], ref) <= TOL
    assert np.isfinite(w).all()
