"""GPU parity of the Helmholtz form w = Ax(u) + h2 B u (the mass term the
listing omits) through the C ABI, and the Helmholtz solves: fp64 CG (with
the fused p.Ap, which then includes the mass term's share), fp32 mixed
refinement and flexible CG, each checked against the oracle (relative L2
1e-12 for the operator; the fp64 residual of each solve recomputed by the
oracle)."""
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
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=torch.float64)


@pytest.mark.parametrize("lx", [5, 8])
def test_helm_h2_and_operator_parity(lx):
    dims = (4, 3, 2)
    case = operator_case(dims, lx, seed=30 + lx)
    geo = oracle.box_geometry(case["vertices"], lx)
    h2 = synth.uniform(case["u"].shape, seed=40 + lx, lo=0.1, hi=3.0)
    ref = oracle.ax_helm_h2(case["u"], case["dx"], case["dxt"], case["h1"],
                            *[case[k] for k in GKEYS], lx, h2, geo["B"])
    t = {k: _dev(case[k]) for k in ("u", "dx", "dxt", "h1") + GKEYS}
    th2, tB = _dev(h2), _dev(geo["B"])
    w = torch.full_like(t["u"], float("nan"))
    ax.ax_helm_h2(w, t["u"], t["dx"], t["dxt"], t["h1"], *[t[k] for k in GKEYS], th2, tB, lx)
    assert rel_l2(w.cpu().numpy(), ref) <= 1e-12
    op = ax.Operator(lx, t["dx"], t["dxt"], t["h1"], *[t[k] for k in GKEYS])
    op.set_h2(th2, tB)
    w2 = torch.full_like(t["u"], float("nan"))
    op.apply(w2, t["u"])
    assert rel_l2(w2.cpu().numpy(), ref) <= 1e-12
    op.set_h2(None, None)  # back to the stiffness part alone
    op.apply(w2, t["u"])
    assert rel_l2(w2.cpu().numpy(), case["w"]) <= 1e-12


def _problems(n, lx, seed):
    v = synth.box_vertices(n, seed=seed)
    xyz = ax.box_geometry(v, lx, want_xyz=True)["xyz"]
    h1 = ax.fourier_coefficient(seed + 1)(xyz[..., 0], xyz[..., 1], xyz[..., 2])
    h2 = ax.fourier_coefficient(seed + 2, lo=1.0, hi=50.0)(xyz[..., 0], xyz[..., 1],
                                                            xyz[..., 2])
    P = ax.Poisson(v, lx, h1=h1, h2=h2)
    O = oracle.Problem(v, lx, h1=h1, f=oracle.poisson_rhs_f, h2=h2)
    return P, O


def _oracle_relres(O, x):
    r = O.b - O.apply(x.cpu().numpy().reshape(O.b.shape))
    return np.sqrt(O.dot(r, r) / O.dot(O.b, O.b))


@pytest.mark.parametrize("n,lx", [(4, 6), (4, 8), (3, 5)])
def test_helmholtz_cg_matches_oracle(n, lx):
    P, O = _problems(n, lx, seed=12)
    b = P.rhs(oracle.poisson_rhs_f)
    np.testing.assert_allclose(b.cpu().numpy(), O.b, rtol=1e-12, atol=1e-14)
    x, its, rel, rc = P.cg(b, tol=1e-8)
    assert rc == 0 and rel <= 1e-8
    xo, its_o, _ = oracle.pcg(O, O.b, tol=1e-8)
    assert abs(its - its_o) <= 1
    assert rel_l2(x.cpu().numpy(), xo) <= 1e-7
    assert _oracle_relres(O, x) <= 1.5e-8
    # the Helmholtz system is better conditioned than the Poisson one
    Pp = ax.Poisson(synth.box_vertices(n, seed=12), lx, h1=O.h1)
    _, its_p, _, _ = Pp.cg(Pp.rhs(oracle.poisson_rhs_f), tol=1e-8)
    assert its <= its_p


def test_helmholtz_mixed_and_flexible_solves():
    P, O = _problems(4, 8, seed=21)
    b = P.rhs(oracle.poisson_rhs_f)
    x, no, ni, rel, rc = P.mpcg(b, mode=ax.AX_PREC_F32, tol=1e-8, inner_tol=1e-4)
    assert rc == 0 and rel <= 1e-8 and _oracle_relres(O, x) <= 1.5e-8
    x2, it2, rel2, fb2, rc2 = P.fcg(b, None, tol=1e-8)
    assert rc2 == 0 and rel2 <= 1e-8 and _oracle_relres(O, x2) <= 1.5e-8
    x3, no3, ni3, rel3, fb3, rc3 = P.mpfcg(b, None, tol=1e-8, inner_tol=1e-4)
    assert rc3 == 0 and rel3 <= 1e-8 and _oracle_relres(O, x3) <= 1.5e-8
