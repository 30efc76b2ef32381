"""Out-of-bounds write check for every operator entry point, in place of a
memory sanitizer: each output is a slice of a larger buffer whose
guard bands before and after hold a canary value; after the call the bands
must be untouched and every output value written (the slice starts as NaN).
Sizes are ragged against the kernels' elements per block.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_20994_gb300 as ax  # noqa: E402

from _cases import GKEYS, operator_case  # noqa: E402

CANARY = -1.2345e30
BAND = 4096


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ax.build()


def _guarded(n, dtype):
    """(slice of n values starting as NaN, the whole buffer)."""
    buf = torch.full((n + 2 * BAND,), CANARY, dtype=dtype, device="cuda")
    out = buf[BAND:BAND + n]
    out.fill_(float("nan"))
    return out, buf


def _check(out, buf):
    torch.cuda.synchronize()
    assert torch.all(buf[:BAND] == CANARY), "write before the output"
    assert torch.all(buf[BAND + out.numel():] == CANARY), "write after the output"
    assert torch.isfinite(out).all(), "output value not written"


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("lx", [3, 5, 8, 12, 13])
@pytest.mark.parametrize("dims", [(7, 1, 1), (3, 3, 1)], ids=["E7", "E9"])
def test_fp64_entry_points_stay_in_bounds(lx, dims):
    case = operator_case(dims, lx, seed=lx)
    f = {k: _dev(case[k]) for k in ("u", "dx", "dxt", "h1") + GKEYS}
    G = [f[k] for k in GKEYS]
    shape = f["u"].shape
    variants = [ax.AX_VARIANT_AUTO, ax.AX_VARIANT_F64_NATIVE]
    if lx <= 12:
        variants.append(ax.AX_VARIANT_F64_DF)
    if lx % 2 == 0 and lx <= 12:
        variants.append(ax.AX_VARIANT_F64_DF_EO)
    for v in variants:
        out, buf = _guarded(f["u"].numel(), torch.float64)
        ax.ax_helm(out.view(shape), f["u"], f["dx"], f["dxt"], f["h1"], *G, lx, variant=v)
        _check(out, buf)
    # operator handle (prepared geometry for even lx 6-12)
    op = ax.Operator(lx, f["dx"], f["dxt"], f["h1"], *G)
    out, buf = _guarded(f["u"].numel(), torch.float64)
    op.apply(out.view(shape), f["u"])
    _check(out, buf)
    # six separate matrices
    d = [f["dx"], f["dx"].clone(), f["dx"].clone(), f["dxt"], f["dxt"].clone(), f["dxt"].clone()]
    out, buf = _guarded(f["u"].numel(), torch.float64)
    ax.ax_helm_xyz(out.view(shape), f["u"], *d, f["h1"], *G, lx)
    _check(out, buf)


@pytest.mark.parametrize("lx", [3, 5, 8, 12, 16])
def test_reduced_precision_entry_points_stay_in_bounds(lx):
    dims = (7, 1, 1) if lx <= 12 else (3, 1, 1)
    case = operator_case(dims, lx, seed=2 * lx)
    f32 = {k: _dev(case[k], torch.float32) for k in ("u", "dx", "dxt", "h1") + GKEYS}
    shape = f32["u"].shape
    out, buf = _guarded(f32["u"].numel(), torch.float32)
    ax.ax_helm_f32(out.view(shape), f32["u"], f32["dx"], f32["dxt"], f32["h1"],
                   *[f32[k] for k in GKEYS], lx)
    _check(out, buf)
    b16 = {k: _dev(case[k], torch.bfloat16) for k in ("u", "h1") + GKEYS}
    out, buf = _guarded(f32["u"].numel(), torch.float32)
    ax.ax_helm_bf16(out.view(shape), b16["u"], f32["dx"], f32["dxt"], b16["h1"],
                    *[b16[k] for k in GKEYS], lx)
    _check(out, buf)
    xi, wq = (torch.as_tensor(a, device="cuda") for a in ax.gll(lx))
    cor = torch.as_tensor(ax.box_corners(case["vertices"]), device="cuda").reshape(-1)
    for h1 in (None, f32["h1"]):
        out, buf = _guarded(f32["u"].numel(), torch.float32)
        ax.ax_helm_trilinear_f32(out.view(shape), f32["u"], f32["dx"], f32["dxt"], h1, cor, xi,
                                 wq, lx)
        _check(out, buf)
