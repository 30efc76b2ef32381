"""GPU parity of the fp64 entry points on inputs outside the comfortable
range of the double-float kernels, against the fp64 oracle.

The double-float kernels carry each fp64 value as two fp32 numbers, which
holds ~47 bits only inside the fp32 exponent range; the even-odd kernels also
read only half the rows of the 1-D matrices, which is exact only when they are
centro-antisymmetric (as the GLL matrix is).  Elements outside that window,
and every element when the matrices lack the symmetry, are recomputed with
fp64 units.  These cases check that every fp64 entry point (ax_helm in each
variant, the operator handle, the six-matrix form with equal matrices, the
batched launch) returns the oracle's result there:

* random, non-symmetric dx / dxt (Listing 2 takes them as free arguments) at
  lx 8, 10, 12 (the even-odd orders) and a k-loop order;
* u, G or h1 scaled by 1e-30 and 1e+30 (inside fp64, outside the double-float
  window), alone and combined, and values of 1e39 and 1e-300 in u;
* Inf and NaN in u and in G: the points the oracle returns as non-finite are
  non-finite, the other elements match.
Tolerance: relative L2 1e-12 over the finite outputs, as for every fp64 mode.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2506_20994_gb300 as ax  # noqa: E402
from paper_2506_20994_gb300 import synth  # noqa: E402

from _cases import GKEYS, operator_case, rel_l2  # noqa: E402

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ax.build()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


def _oracle(c):
    return oracle.ax_helm(c["u"], c["dx"], c["dxt"], c["h1"], *[c[k] for k in GKEYS], c["lx"])


def _run(c, how):
    """w from one fp64 entry point on the case's arrays."""
    lx = c["lx"]
    t = {k: _dev(c[k]) for k in ("u", "dx", "dxt", "h1") + GKEYS}
    w = torch.full_like(t["u"], 7.0)
    g = [t[k] for k in GKEYS]
    if how == "op":
        op = ax.Operator(lx, t["dx"], t["dxt"], t["h1"], *g)
        op.apply(w, t["u"])
    elif how == "xyz_same":
        ax.ax_helm_xyz(w, t["u"], t["dx"], t["dx"], t["dx"], t["dxt"], t["dxt"], t["dxt"],
                       t["h1"], *g, lx)
    else:
        ax.ax_helm(w, t["u"], t["dx"], t["dxt"], t["h1"], *g, lx, variant=how)
    torch.cuda.synchronize()
    return w.cpu().numpy()


def _check(got, ref):
    bad = ~np.isfinite(ref)
    assert np.all(~np.isfinite(got[bad])), "a non-finite oracle point came back finite"
    fin = np.isfinite(ref)
    assert np.all(np.isfinite(got[fin])), "a finite oracle point came back non-finite"
    scale = max(np.abs(ref[fin]).max(initial=0.0), 1e-300)  # norms of 1e250 values overflow
    assert rel_l2(got[fin] / scale, ref[fin] / scale) <= TOL


ENTRIES = [ax.AX_VARIANT_AUTO, ax.AX_VARIANT_F64_DF_EO, ax.AX_VARIANT_F64_DF, "op", "xyz_same"]
ENTRY_IDS = ["auto", "even_odd", "kloop", "op", "xyz_same"]


@pytest.mark.parametrize("lx", [8, 10, 12])
@pytest.mark.parametrize("how", ENTRIES, ids=ENTRY_IDS)
def test_general_matrices(lx, how):
    """Random dx and an unrelated random dxt (neither centro-antisymmetric)."""
    c = operator_case((3, 2, 2), lx, seed=900 + lx)
    g = synth.rng(901 + lx)
    c["dx"] = g.uniform(-1.0, 1.0, (lx, lx))
    c["dxt"] = g.uniform(-1.0, 1.0, (lx, lx))
    ref = _oracle(c)
    _check(_run(c, how), ref)


@pytest.mark.parametrize("lx", [8, 12])
def test_one_mirrored_entry_off(lx):
    """The GLL matrices with one entry moved by 1e-9 (relative): the
    symmetry check must catch a defect this small."""
    c = operator_case((2, 2, 1), lx, seed=910 + lx)
    dx = c["dx"].copy().reshape(lx, lx)
    dx[1, 2] *= 1.0 + 1e-9
    c["dx"] = dx.reshape(c["dx"].shape)
    ref = _oracle(c)
    _check(_run(c, ax.AX_VARIANT_AUTO), ref)
    _check(_run(c, "op"), ref)


SCALES = [(1e-30, 1, 1), (1e30, 1, 1), (1, 1e-30, 1), (1, 1e30, 1), (1, 1, 1e-30),
          (1e-30, 1e-30, 1), (1e30, 1e30, 1e-30), (1e-150, 1e-150, 1), (1e150, 1, 1e100)]


@pytest.mark.parametrize("lx", [5, 8])
@pytest.mark.parametrize("scale", SCALES, ids=lambda s: "u%.0e_g%.0e_h%.0e" % s)
@pytest.mark.parametrize("how", ENTRIES, ids=ENTRY_IDS)
def test_scaled_inputs(lx, scale, how):
    if how == ax.AX_VARIANT_F64_DF_EO and lx % 2:
        pytest.skip("the even-odd kernel takes even lx")
    su, sg, sh = scale
    c = operator_case((3, 2, 2), lx, seed=920 + lx)
    c["u"] = c["u"] * su
    for k in GKEYS:
        c[k] = c[k] * sg
    c["h1"] = c["h1"] * sh
    ref = _oracle(c)
    _check(_run(c, how), ref)


@pytest.mark.parametrize("lx", [6, 8, 9])
@pytest.mark.parametrize("how", [ax.AX_VARIANT_AUTO, ax.AX_VARIANT_F64_DF, "op"],
                         ids=["auto", "kloop", "op"])
def test_mixed_magnitudes_per_element(lx, how):
    """Elements of very different scale in one launch: some in the window,
    some beyond the fp32 range, one all zero, one with fp64 values near the
    bottom of the range (1e-300) and one with a single 1e39."""
    c = operator_case((4, 2, 1), lx, seed=930 + lx)
    u = c["u"].copy()
    u[1] *= 1e39
    u[2] *= 1e-300
    u[3] = 0.0
    u[4, 1, 1, 1] = 1e39
    u[5] *= 1e-45
    c["u"] = u
    c["g11"] = c["g11"].copy()
    c["g11"][6] *= 1e45
    ref = _oracle(c)
    _check(_run(c, how), ref)


@pytest.mark.parametrize("lx", [7, 8])
@pytest.mark.parametrize("bad", ["inf_u", "nan_u", "inf_g", "nan_h1"])
@pytest.mark.parametrize("how", [ax.AX_VARIANT_AUTO, ax.AX_VARIANT_F64_DF, "op"],
                         ids=["auto", "kloop", "op"])
def test_non_finite_inputs(lx, bad, how):
    c = operator_case((3, 1, 1), lx, seed=940 + lx)
    for k in ("u", "h1") + GKEYS:
        c[k] = c[k].copy()
    if bad == "inf_u":
        c["u"][1, 2, 3, 1] = np.inf
    elif bad == "nan_u":
        c["u"][0, 0, 0, 0] = np.nan
    elif bad == "inf_g":
        c["g22"][2, 1, 1, 1] = -np.inf
    else:
        c["h1"][1, 3, 2, 1] = np.nan
    ref = _oracle(c)
    got = _run(c, how)
    _check(got, ref)


def test_batched_launch_scaled_meshes():
    """The batched launch (one persistent kernel per order) on meshes whose
    scales leave the double-float window, next to ordinary ones."""
    meshes, refs, outs = [], [], []
    for m, (lx, s) in enumerate([(8, 1e-40), (8, 1.0), (5, 1e35), (10, 1e-60), (6, 1.0)]):
        c = operator_case((2, 2, 1), lx, seed=950 + m)
        c["u"] = c["u"] * s
        refs.append(_oracle(c))
        t = {k: _dev(c[k]) for k in ("u", "dx", "dxt", "h1") + GKEYS}
        t["w"] = torch.full_like(t["u"], 5.0)
        outs.append(t["w"])
        meshes.append(dict(lx=lx, **t))
    b = ax.Batch(meshes)
    b.launch()
    torch.cuda.synchronize()
    for w, ref in zip(outs, refs):
        _check(w.cpu().numpy(), ref)
