"""GPU parity of gather-scatter, the assembled operator and the solvers
against the oracle, through the C ABI.

  * gather-scatter: bit-exact (same summation order as the oracle);
  * assembled operator: relative L2 1e-12;
  * fp64 CG: the same iterates as the oracle's textbook PCG for the first
    iterations (relative 1e-9) and the same iteration count to 1e-8 (+-1);
  * iterative refinement (fp32 / bf16 inner data): the fp64 residual of
    the returned solution, recomputed by the oracle, is <= 1e-8.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2506_20994_gb300 as ax  # noqa: E402
from paper_2506_20994_gb300 import synth  # noqa: E402

from _cases import rel_l2  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ax.build()


def _problem(dims, lx, seed=0, h1=None):
    v = synth.box_vertices(*dims, seed=seed)
    P = ax.Poisson(v, lx, h1=h1)
    O = oracle.Problem(v, lx, h1=h1, f=oracle.poisson_rhs_f)
    return v, P, O


@pytest.mark.parametrize("dims,lx", [((3, 2, 4), 5), ((1, 1, 1), 2), ((4, 4, 4), 8),
                                     ((2, 3, 1), 12)])
def test_gs_bit_exact(dims, lx):
    glob = oracle.numbering(*dims, lx)
    gs = ax.GatherScatter(glob)
    v = synth.uniform(glob.shape, seed=3)
    t = torch.as_tensor(v, device="cuda")
    gs.sum(t)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(t.cpu().numpy(), oracle.gs_sum(v, glob))
    t32 = torch.as_tensor(v, device="cuda", dtype=torch.float32)
    gs.sum(t32)
    torch.cuda.synchronize()
    np.testing.assert_allclose(t32.cpu().numpy(), oracle.gs_sum(v, glob), rtol=1e-6, atol=1e-6)
    inv = gs.inverse_multiplicity().cpu().numpy()
    np.testing.assert_allclose(inv, 1.0 / oracle.multiplicity(glob).ravel())
    info = gs.info()
    assert info["n_local"] == glob.size
    assert info["n_shared"] == int(np.sum(np.bincount(glob.ravel()) > 1))


def test_gs_unstructured_ids():
    """Sparse, shuffled global ids (the non-dense set-up path)."""
    g = synth.rng(4)
    glob = g.integers(0, 10 ** 9, size=3000)
    glob[::7] = glob[3]  # a node with many copies
    gs = ax.GatherScatter(glob)
    v = synth.uniform(glob.shape, seed=5)
    t = torch.as_tensor(v, device="cuda")
    gs.sum(t)
    torch.cuda.synchronize()
    ref = oracle.gs_sum(v, np.unique(glob, return_inverse=True)[1])
    np.testing.assert_array_equal(t.cpu().numpy(), ref)


@pytest.mark.parametrize("dims,lx", [((3, 3, 2), 6), ((4, 4, 4), 8), ((2, 2, 2), 12)])
def test_assembled_apply(dims, lx):
    h1 = None
    _, P, O = _problem(dims, lx, seed=1, h1=h1)
    u = synth.uniform(O.mask.shape, seed=2)
    u = oracle.gs_sum(u, O.glob) / O.mult  # continuous field
    ut = torch.as_tensor(u, device="cuda")
    w = torch.empty_like(ut)
    P.apply(w, ut)
    torch.cuda.synchronize()
    assert rel_l2(w.cpu().numpy(), O.apply(u)) <= 1e-12
    # Jacobi diagonal
    minv = P.jacobi().cpu().numpy()
    ref = np.where(O.mask > 0, 1.0 / O.diag, 0.0)
    np.testing.assert_allclose(minv, ref.ravel(), rtol=1e-12)


@pytest.mark.parametrize("lx", [5, 6, 8])
def test_cg_iterates_match_oracle(lx):
    """lx = 6, 8: fp64 PCG with p . Ap fused into the prepared-geometry
    apply; lx = 5: the separate mask-and-dot pass."""
    _, P, O = _problem((3, 3, 3), lx, seed=4)
    b = P.rhs(oracle.poisson_rhs_f)
    np.testing.assert_allclose(b.cpu().numpy(), O.b, rtol=1e-12, atol=1e-14)
    for k in (1, 3, 8):
        x, its, rel, rc = P.cg(b, tol=0.0, maxit=k)
        assert its == k
        xo, _, hist = oracle.pcg(O, O.b, tol=0.0, maxit=k)
        assert rel_l2(x.cpu().numpy(), xo) <= 1e-9
        assert abs(rel - hist[-1]) <= 1e-8 * max(hist[-1], 1e-300) + 1e-12


@pytest.mark.parametrize("dims,lx", [((8, 8, 8), 8), ((4, 4, 4), 6)])
def test_cg_converges_like_oracle(dims, lx):
    _, P, O = _problem(dims, lx, seed=0)
    b = P.rhs(oracle.poisson_rhs_f)
    x, its, rel, rc = P.cg(b, tol=1e-8)
    assert rc == 0 and rel <= 1e-8
    xo, its_o, hist = oracle.pcg(O, O.b, tol=1e-8)
    assert abs(its - its_o) <= 1
    assert rel_l2(x.cpu().numpy(), xo) <= 1e-7
    # independent check of the residual in fp64 by the oracle
    r = O.b - O.apply(x.cpu().numpy())
    assert np.sqrt(O.dot(r, r) / O.dot(O.b, O.b)) <= 1.5e-8
    # discretisation error against the analytic solution
    xyz = P.xyz
    exact = np.sin(np.pi * xyz[..., 0]) * np.sin(np.pi * xyz[..., 1]) * np.sin(np.pi * xyz[..., 2])
    assert np.abs(x.cpu().numpy() - exact).max() < 1e-4


@pytest.mark.parametrize("mode", [ax.AX_PREC_F32, ax.AX_PREC_BF16])
def test_mixed_precision_refinement(mode):
    lx = 8
    _, P, O = _problem((6, 6, 6), lx, seed=2)
    b = P.rhs(oracle.poisson_rhs_f)
    inner = 1e-4 if mode == ax.AX_PREC_F32 else 2e-2
    x, outer, inner_its, rel, rc = P.mpcg(b, mode=mode, tol=1e-8, inner_tol=inner)
    assert rc == 0 and rel <= 1e-8
    r = O.b - O.apply(x.cpu().numpy())
    assert np.sqrt(O.dot(r, r) / O.dot(O.b, O.b)) <= 1.5e-8
    assert outer >= 2


def test_cg_breakdown_on_indefinite_operator():
    """Host-side fault injection: h1 < 0 makes A negative definite; the
    solver reports AX_EBREAKDOWN instead of iterating."""
    lx = 4
    v = synth.box_vertices(3, seed=6)
    P = ax.Poisson(v, lx, h1=-1.0)
    b = P.rhs(oracle.poisson_rhs_f)
    x, its, rel, rc = P.cg(b, tol=1e-8, maxit=50, raise_on_error=False)
    assert rc == ax._lib.AX_EBREAKDOWN


def test_cg_reports_maxit():
    _, P, O = _problem((4, 4, 4), 6, seed=3)
    b = P.rhs(oracle.poisson_rhs_f)
    x, its, rel, rc = P.cg(b, tol=1e-14, maxit=5, raise_on_error=False)
    assert rc == ax._lib.AX_ENOTCONV and its == 5 and rel > 1e-14


def test_cg_deterministic():
    _, P, _ = _problem((4, 4, 4), 6, seed=8)
    b = P.rhs(oracle.poisson_rhs_f)
    x1, i1, r1, _ = P.cg(b, tol=1e-8)
    x2, i2, r2, _ = P.cg(b, tol=1e-8)
    assert i1 == i2 and r1 == r2
    assert torch.equal(x1, x2)
