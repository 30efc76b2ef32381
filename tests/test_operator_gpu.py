"""GPU parity of the operator handle (ax_op_*): the prepared-geometry
even-odd kernel against the fp64 oracle (relative L2 1e-12) and against the
on-the-fly even-odd kernel (same split; the packed pointwise step rounds
its tails in another order: both sit ~3e-14 from the oracle and within
1e-13 of each other, not bitwise); the
unprepared orders fall back to ax_helm bit for bit; h1 updates; the Poisson
solver applies through the handle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2506_20994_gb300 as ax  # noqa: E402
from paper_2506_20994_gb300 import synth  # noqa: E402

from _cases import GKEYS, operator_case, rel_l2  # noqa: E402

DIMS = [(1, 1, 1), (7, 1, 1), (4, 4, 4), (9, 9, 7)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ax.build()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


def _op(case):
    t = {k: _dev(case[k]) for k in ("u", "dx", "dxt", "h1") + GKEYS}
    op = ax.Operator(case["lx"], t["dx"], t["dxt"], t["h1"], *[t[k] for k in GKEYS])
    return op, t


@pytest.mark.parametrize("lx", [6, 8, 10, 12])
@pytest.mark.parametrize("dims", DIMS, ids=lambda d: "E%d" % (d[0] * d[1] * d[2]))
def test_prepared_parity_and_agreement_with_on_the_fly(lx, dims):
    case = operator_case(dims, lx, seed=70 + lx)
    op, t = _op(case)
    info = op.info()
    # geometry pairs and two exponent records per element, the coefficient block
    # (rows of lx/2 + 1 pairs, then lx/2 negated heads per row, for D and D^T),
    # the error word
    h = lx // 2
    assert info["prepared"] and info["device_bytes"] == (
        (56 * lx ** 3 + 8) * case["u"].shape[0] + 32 * h * (h + 1) + 16 * h * h + 4)
    w = torch.full_like(t["u"], float("nan"))
    op.apply(w, t["u"])
    w2 = torch.full_like(t["u"], float("nan"))
    ax.ax_helm(w2, t["u"], t["dx"], t["dxt"], t["h1"], *[t[k] for k in GKEYS], lx,
               variant=ax.AX_VARIANT_F64_DF_EO)
    torch.cuda.synchronize()
    got = w.cpu().numpy()
    assert rel_l2(got, case["w"]) <= 1e-12
    assert np.abs(got - case["w"]).max() <= 1e-11 * np.abs(case["w"]).max()
    assert rel_l2(got, w2.cpu().numpy()) <= 1e-13
    assert op.error() == 0


@pytest.mark.parametrize("lx", [2, 5, 7, 13])
def test_unprepared_orders_fall_back(lx):
    case = operator_case((3, 2, 2), lx, seed=80 + lx)
    op, t = _op(case)
    assert not op.info()["prepared"] and op.info()["device_bytes"] == 0
    w = torch.empty_like(t["u"])
    op.apply(w, t["u"])
    w2 = torch.empty_like(t["u"])
    ax.ax_helm(w2, t["u"], t["dx"], t["dxt"], t["h1"], *[t[k] for k in GKEYS], lx)
    assert torch.equal(w, w2)
    assert rel_l2(w.cpu().numpy(), case["w"]) <= 1e-12


def test_set_h1_refreshes_the_prepared_copy():
    lx = 8
    case = operator_case((4, 3, 2), lx, seed=90)
    op, t = _op(case)
    h1b = synth.uniform(case["h1"].shape, seed=91, lo=0.5, hi=2.0)
    th = _dev(h1b)
    op.set_h1(th)
    w = torch.empty_like(t["u"])
    op.apply(w, t["u"])
    ref = oracle.ax_helm(case["u"], case["dx"], case["dxt"], h1b, *[case[k] for k in GKEYS], lx)
    assert rel_l2(w.cpu().numpy(), ref) <= 1e-12


def test_adversarial_inputs_through_the_handle():
    lx = 8
    case = operator_case((3, 3, 3), lx, seed=95)
    op, t = _op(case)
    scale = 10.0 ** synth.uniform((case["u"].shape[0], 1, 1, 1), seed=96, lo=-6, hi=6)
    u = case["u"] * scale
    u[::4] = 0.0
    ref = oracle.ax_helm(u, case["dx"], case["dxt"], case["h1"], *[case[k] for k in GKEYS], lx)
    w = torch.empty_like(t["u"])
    op.apply(w, _dev(u))
    got = w.cpu().numpy()
    per_el = np.linalg.norm((got - ref).reshape(len(ref), -1), axis=1)
    per_ref = np.linalg.norm(ref.reshape(len(ref), -1), axis=1)
    nz = per_ref > 0
    assert np.all(per_el[nz] <= 1e-12 * per_ref[nz])
    assert np.all(got[::4] == 0.0)


def test_full_size_sampled_parity():
    """E = 32768, lx = 8 (the benchmark's mesh) through the handle; sampled
    elements against the oracle one by one."""
    lx, n = 8, 32
    v = synth.box_vertices(n, seed=0)
    g = ax.box_geometry(v, lx)
    sh = g["g11"].shape
    u = synth.uniform(sh, seed=1)
    dx, dxt = ax.dmat(lx)
    t = {"u": _dev(u), "h1": _dev(np.ones(sh)), "dx": _dev(dx), "dxt": _dev(dxt)}
    for k in GKEYS:
        t[k] = _dev(g[k])
    op = ax.Operator(lx, t["dx"], t["dxt"], t["h1"], *[t[k] for k in GKEYS])
    w = torch.empty_like(t["u"])
    op.apply(w, t["u"])
    idx = np.sort(synth.rng(7).choice(sh[0], 64, replace=False))
    idx[-1] = sh[0] - 1
    got = w.cpu().numpy()[idx]
    geo = oracle.box_geometry(v, lx, elements=idx)
    odx, odxt = oracle.d_buffers(lx)
    ref = oracle.ax_helm(u[idx], odx, odxt, np.ones((len(idx),) + sh[1:]),
                         *[geo[k] for k in GKEYS], lx)
    assert rel_l2(got, ref) <= 1e-12


def test_poisson_cg_unchanged_by_the_handle():
    """The solver's apply now runs through the handle: the CG solution still
    meets the oracle's fp64 residual bound."""
    lx = 8
    v = synth.box_vertices(4, seed=3)
    P = ax.Poisson(v, lx)
    b = P.rhs(oracle.poisson_rhs_f)
    x, it, rel, rc = P.cg(b, tol=1e-8)
    assert rc == 0 and rel <= 1e-8
    O = oracle.Problem(v, lx, f=oracle.poisson_rhs_f)
    r = O.b - O.apply(x.cpu().numpy().reshape(O.b.shape))
    assert np.sqrt(O.dot(r, r) / O.dot(O.b, O.b)) <= 1.5e-8


def test_small_config_through_the_handle():
    """E = 512 (8^3 perturbed hexahedra), lx = 8, h1 = 1, u uniform in
    [-1, 1]: the small workload, the whole output against the oracle."""
    lx = 8
    case = operator_case((8, 8, 8), lx, seed=0, h1_const=1.0)
    op, t = _op(case)
    w = torch.full_like(t["u"], float("nan"))
    op.apply(w, t["u"])
    got = w.cpu().numpy()
    assert rel_l2(got, case["w"]) <= 1e-12
    assert np.abs(got - case["w"]).max() <= 1e-11 * np.abs(case["w"]).max()
