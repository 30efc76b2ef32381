"""GPU parity of the six-matrix element operator (the full argument list of
Listings 1-2: dx, dy, dz, dxt, dyt, dzt) against the fp64 oracle, through
the C ABI (ax_helm_xyz).

Tolerance: relative L2 1e-12 over the whole output, as for ax_helm.  The six
matrices are unrelated random ones, so a matrix used in the wrong direction
or a transposed index shows up at O(1).  Sizes: E = 7 and 12 (ragged against
the elements per block), lx over the double-float range (2-12) and the fp64
units above it (13-16).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2506_20994_gb300 as ax  # noqa: E402
from paper_2506_20994_gb300 import synth  # noqa: E402

from _cases import GKEYS, operator_case, rel_l2  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ax.build()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


def _mats(lx, seed):
    return [synth.uniform((lx * lx,), seed=seed + m) for m in range(6)]


def _run(case, mats):
    lx = case["lx"]
    d = [_dev(m) for m in mats]
    f = [_dev(case[k]) for k in ("u", "h1") + GKEYS]
    w = torch.full_like(f[0], float("nan"))
    ax.ax_helm_xyz(w, f[0], *d, *f[1:], lx)
    torch.cuda.synchronize()
    return w.cpu().numpy()


def _ref(case, mats):
    dx, dy, dz, dxt, dyt, dzt = mats
    return oracle.ax_helm(case["u"], dx, dxt, case["h1"], *[case[k] for k in GKEYS],
                          case["lx"], dy=dy, dz=dz, dyt=dyt, dzt=dzt)


@pytest.mark.parametrize("lx", list(range(2, 17)))
def test_xyz_parity(lx):
    dims = (7, 1, 1) if lx <= 12 else (3, 1, 1)
    case = operator_case(dims, lx, seed=200 + lx)
    mats = _mats(lx, seed=300 + lx)
    ref = _ref(case, mats)
    w = _run(case, mats)
    assert rel_l2(w, ref) <= 1e-12


@pytest.mark.parametrize("lx", [5, 8, 12])
def test_xyz_ragged_and_directions(lx):
    """E = 12 (a ragged last block for every elements-per-block choice);
    swapping dy and dz moves the result by O(1), and the kernel follows."""
    case = operator_case((3, 2, 2), lx, seed=17)
    mats = _mats(lx, seed=40)
    w = _run(case, mats)
    assert rel_l2(w, _ref(case, mats)) <= 1e-12
    swapped = [mats[0], mats[2], mats[1]] + mats[3:]
    w2 = _run(case, swapped)
    assert rel_l2(w2, _ref(case, swapped)) <= 1e-12
    assert rel_l2(w2, w) > 1e-3


@pytest.mark.parametrize("lx", [6, 8, 13])
def test_xyz_distinct_copies_of_d(lx):
    """The GLL matrices passed as six separate buffers (distinct pointers,
    equal contents) take the six-matrix kernel and agree with ax_helm."""
    case = operator_case((4, 2, 1), lx, seed=5)
    mats = [case["dx"], case["dx"].copy(), case["dx"].copy(),
            case["dxt"], case["dxt"].copy(), case["dxt"].copy()]
    w = _run(case, mats)
    assert rel_l2(w, case["w"]) <= 1e-12


def test_xyz_same_pointers_is_ax_helm():
    """dy == dz == dx and dyt == dzt == dxt as the same device pointers: the
    call is ax_helm itself, bit for bit."""
    lx = 8
    case = operator_case((4, 4, 2), lx, seed=9)
    dx, dxt = _dev(case["dx"]), _dev(case["dxt"])
    f = [_dev(case[k]) for k in ("u", "h1") + GKEYS]
    w1 = torch.empty_like(f[0])
    w2 = torch.empty_like(f[0])
    ax.ax_helm_xyz(w1, f[0], dx, dx, dx, dxt, dxt, dxt, *f[1:], lx)
    ax.ax_helm(w2, f[0], dx, dxt, *f[1:], lx)
    torch.cuda.synchronize()
    assert torch.equal(w1, w2)
    assert rel_l2(w1.cpu().numpy(), case["w"]) <= 1e-12


def test_xyz_errors_and_empty():
    lx = 4
    case = operator_case((1, 1, 1), lx, seed=1)
    mats = [_dev(m) for m in _mats(lx, seed=2)]
    f = [_dev(case[k]) for k in ("u", "h1") + GKEYS]
    w = torch.zeros_like(f[0])
    lib = ax._lib.lib()
    s = ax._stream()
    ptrs = [t.data_ptr() for t in [w, f[0]] + mats + f[1:]]
    assert lib.ax_helm_xyz(*ptrs, 17, 1, s) == ax._lib.AX_EINVAL      # lx out of range
    assert lib.ax_helm_xyz(*ptrs, lx, -1, s) == ax._lib.AX_EINVAL     # nelv < 0
    bad = list(ptrs)
    bad[3] = None                                                     # dy NULL
    assert lib.ax_helm_xyz(*bad, lx, 1, s) == ax._lib.AX_EINVAL
    assert lib.ax_helm_xyz(*bad, lx, 0, s) == ax._lib.AX_OK           # nelv == 0: no-op
    torch.cuda.synchronize()
    assert float(w.abs().max()) == 0.0
