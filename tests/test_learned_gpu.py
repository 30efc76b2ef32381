"""GPU checks of the learned element preconditioner through the C ABI.

Tolerances: the bf16 tensor-core apply against the fp64 oracle network,
relative L2 2e-2; the fp32 loss and gradient against the oracle's backprop,
relative 1e-4; Adam against the oracle's update, relative 1e-5.  The
flexible CG with no network reproduces Jacobi-PCG; a zero network gives the
same bits as no network; a non-finite network falls back to Jacobi; and
the trained network is compared with Jacobi on iterations to 1e-8.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import mlp as omlp  # noqa: E402
import paper_2506_20994_gb300 as ax  # noqa: E402
from paper_2506_20994_gb300 import synth  # noqa: E402

from _cases import rel_l2  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ax.build()


def _random_params(n_in, n_hid, seed, scale=0.2):
    return (synth.rng(seed).normal(0, scale, size=omlp.nparams(n_in, n_hid))).astype(np.float32)


@pytest.mark.parametrize("lx,n_hid", [(4, 16), (6, 24), (8, 48)])
def test_apply_matches_oracle(lx, n_hid):
    v = synth.box_vertices(3, 2, 2, seed=lx)
    P = ax.Poisson(v, lx)
    O = oracle.Problem(v, lx)
    theta = _random_params(lx ** 3, n_hid, seed=lx)
    M = ax.Mlp(lx ** 3, n_hid, params=theta)
    r = O.mask * oracle.gs_sum(synth.uniform(O.mask.shape, seed=5), O.glob)
    minv = np.where(O.mask > 0, 1.0 / O.diag, 0.0)
    z_ref = omlp.precondition(theta.astype(np.float64), r, minv, O.mask, O.mult, O.glob, lx,
                              n_hid, oracle.gs_sum)
    z = P.precondition(torch.as_tensor(r.ravel(), device="cuda"), M).cpu().numpy()
    corr_ref = (z_ref - minv * r).ravel()
    corr = z - (minv * r).ravel()
    assert rel_l2(corr, corr_ref) <= 2e-2
    # fp32 local apply (no gs) through ax_mlp_forward
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a).ravel(), device="cuda",
                                  dtype=torch.float32)
    out = torch.empty(O.mask.size, dtype=torch.float32, device="cuda")
    M.forward(out, t(r), t(minv), t(O.mask), t(1.0 / O.mult), P.nelv)
    X, _, s = omlp.element_features(r, np.zeros_like(r), minv, lx)
    local_ref = (omlp.forward(theta.astype(np.float64), X, n_hid) * s[:, None]).ravel()
    local_ref = local_ref * O.mask.ravel() / O.mult.ravel()
    assert rel_l2(out.cpu().numpy(), local_ref) <= 2e-2


@pytest.mark.parametrize("n_in,n_hid,B", [(64, 16, 40), (512, 48, 300), (216, 24, 7)])
def test_loss_and_gradient_match_oracle(n_in, n_hid, B):
    g = synth.rng(n_in + B)
    theta = _random_params(n_in, n_hid, seed=B)
    X = g.normal(size=(B, n_in)).astype(np.float32)
    T = g.normal(size=(B, n_in)).astype(np.float32)
    M = ax.Mlp(n_in, n_hid, params=theta)
    L, grad = M.loss_grad(torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda"))
    L_ref, g_ref = omlp.loss_and_grad(theta.astype(np.float64), X, T, n_hid)
    assert abs(L - L_ref) <= 1e-5 * L_ref
    assert rel_l2(grad, g_ref) <= 1e-4
    # one Adam step
    M.adam(1e-3)
    new = M.get_params()
    ref, _, _ = omlp.adam_step(theta.astype(np.float64), grad.astype(np.float64),
                               np.zeros(theta.size), np.zeros(theta.size), 1, lr=1e-3)
    assert rel_l2(new, ref) <= 1e-5


def _var_problem(n, lx, seed=0):
    v = synth.box_vertices(n, seed=seed)
    return ax.Poisson(v, lx, h1=ax.fourier_coefficient(seed + 1))


def test_fcg_without_network_is_pcg():
    P = _var_problem(4, 6, seed=2)
    b = P.rhs(oracle.poisson_rhs_f)
    x1, i1, r1, rc1 = P.cg(b, tol=1e-8)
    x2, i2, r2, fb, rc2 = P.fcg(b, None, tol=1e-8)
    assert rc1 == rc2 == 0 and abs(i1 - i2) <= 1 and fb == 0
    assert rel_l2(x2.cpu().numpy(), x1.cpu().numpy()) <= 1e-7
    # a zero network is exactly Jacobi, bit for bit
    M0 = ax.Mlp(6 ** 3, 16)
    x3, i3, r3, fb3, _ = P.fcg(b, M0, tol=1e-8)
    assert i3 == i2 and r3 == r2 and fb3 == 0 and torch.equal(x3, x2)


def test_nonfinite_network_falls_back_to_jacobi():
    """Host-side fault injection: NaN weights make every learned step
    non-finite; each step falls back to Jacobi and the solve still
    converges like Jacobi."""
    lx = 6
    P = _var_problem(4, lx, seed=3)
    b = P.rhs(oracle.poisson_rhs_f)
    bad = np.full(omlp.nparams(lx ** 3, 16), np.nan, dtype=np.float32)
    M = ax.Mlp(lx ** 3, 16, params=bad)
    _, ij, _, _, _ = P.fcg(b, None, tol=1e-8)
    x, it, rel, fb, rc = P.fcg(b, M, tol=1e-8)
    assert rc == 0 and rel <= 1e-8
    assert it == ij and fb == it  # every application fell back


def test_training_reduces_loss_and_learned_fcg_converges():
    lx, n = 8, 6
    P = _var_problem(n, lx, seed=4)
    b = P.rhs(oracle.poisson_rhs_f)
    M = ax.Mlp(lx ** 3, 48, params=ax.mlp_init_params(lx ** 3, 48, seed=1))
    X, T = ax.training_pairs(P, b, M, n_pairs=4096, seed=2)
    L0, _ = M.loss_grad(X[:512], T[:512])
    L1 = ax.train_mlp(M, X, T, epochs=20, batch=256, lr=1e-3, seed=3)
    L_after, _ = M.loss_grad(X[:512], T[:512])
    assert L_after < 0.9 * L0
    x, it, rel, fb, rc = P.fcg(b, M, tol=1e-8)
    assert rc == 0 and rel <= 1e-8
    # fp64 residual recomputed by the oracle
    v = synth.box_vertices(n, seed=4)
    h1 = ax.fourier_coefficient(5)(P.xyz[..., 0], P.xyz[..., 1], P.xyz[..., 2])
    O = oracle.Problem(v, lx, h1=h1, f=oracle.poisson_rhs_f)
    r = O.b - O.apply(x.cpu().numpy().reshape(O.b.shape))
    assert np.sqrt(O.dot(r, r) / O.dot(O.b, O.b)) <= 1.5e-8
    # mixed precision with the learned inner preconditioner
    x2, no, ni, rel2, fb2, rc2 = P.mpfcg(b, M, tol=1e-8, inner_tol=1e-4)
    assert rc2 == 0 and rel2 <= 1e-8
    r2 = O.b - O.apply(x2.cpu().numpy().reshape(O.b.shape))
    assert np.sqrt(O.dot(r2, r2) / O.dot(O.b, O.b)) <= 1.5e-8


def _energy_rel_err(P, z, e):
    """||e - z||_A / ||e||_A with the assembled operator (inner product over
    unique nodes: weights 1/multiplicity)."""
    c = P.gs.inverse_multiplicity()
    d = e - z
    q = torch.empty_like(d)
    P.apply(q, d)
    qe = torch.empty_like(e)
    P.apply(qe, e)
    return float(torch.sqrt(torch.sum(c * d * q) / torch.sum(c * e * qe)))


def test_energy_training_gain_on_held_out_pairs():
    """What the trained network gains over Jacobi: the one-step
    approximation z(r) of the error of held-out CG iterates (a different
    right-hand side) is closer in the energy norm than the Jacobi step."""
    lx = 8
    P = _var_problem(5, lx, seed=6)
    b = P.rhs(oracle.poisson_rhs_f)
    R, E = ax.iterate_pairs(P, b, iterates=(2, 4, 8, 16, 32, 64))
    M = ax.Mlp(lx ** 3, 48, params=ax.mlp_init_params(lx ** 3, 48, seed=2))
    loss = ax.train_energy(P, M, R, E, epochs=100, lr=1e-3)
    assert loss < 0.95
    # held-out: right-hand side from a random smooth source
    f2 = ax.fourier_coefficient(9, lo=-1.0, hi=1.0)
    b2 = P.rhs(f2)
    R2, E2 = ax.iterate_pairs(P, b2, iterates=(3, 6, 12, 24))
    gains = []
    for k in range(R2.shape[0]):
        r, e = R2[k].contiguous(), E2[k].contiguous()
        ej = _energy_rel_err(P, P.precondition(r, None), e)
        el = _energy_rel_err(P, P.precondition(r, M), e)
        gains.append(ej - el)
    assert np.mean(gains) > 0.0


# ---------------------------------------------------------------------------
# Symmetric linear form (AX_MLP_SYM)
# ---------------------------------------------------------------------------
def _sym_params(n_in, n_hid, seed, scale=1.0):
    return ax.mlp_init_params(n_in, n_hid, seed=seed, arch=ax.AX_MLP_SYM, scale=scale)


@pytest.mark.parametrize("lx,n_hid", [(4, 16), (6, 24), (8, 48)])
def test_sym_apply_matches_oracle_and_is_symmetric(lx, n_hid):
    v = synth.box_vertices(3, 2, 2, seed=lx)
    P = ax.Poisson(v, lx)
    O = oracle.Problem(v, lx)
    theta = _sym_params(lx ** 3, n_hid, seed=lx)
    M = ax.Mlp(lx ** 3, n_hid, params=theta, arch=ax.AX_MLP_SYM)
    # set_params keeps the tie exactly
    W1, b1, W2, b2 = omlp.unpack(M.get_params(), lx ** 3, n_hid)
    assert np.array_equal(W2, W1.T) and not b1.any() and not b2.any()
    minv = np.where(O.mask > 0, 1.0 / O.diag, 0.0)
    cs = []
    for seed in (5, 6):
        r = O.mask * oracle.gs_sum(synth.uniform(O.mask.shape, seed=seed), O.glob)
        z_ref = omlp.precondition_sym(theta.astype(np.float64), r, minv, O.mask, O.glob, lx,
                                      n_hid, oracle.gs_sum)
        z = P.precondition(torch.as_tensor(r.ravel(), device="cuda"), M).cpu().numpy()
        corr_ref = (z_ref - minv * r).ravel()
        assert np.linalg.norm(corr_ref) > 0.1 * np.linalg.norm(minv * r)
        assert rel_l2(z - (minv * r).ravel(), corr_ref) <= 2e-2
        cs.append((r.ravel(), z))
    (a, Ba), (b, Bb) = cs
    w = 1.0 / O.mult.ravel()
    lhs, rhs = np.sum(w * Ba * b), np.sum(w * a * Bb)
    scale = np.sqrt(np.sum(w * Ba * Ba) * np.sum(w * b * b))
    assert abs(lhs - rhs) <= 1e-2 * scale
    assert np.sum(w * Ba * a) > 0
    # fp32 local apply (no gs): mask .* sqrt(minv) .* (x W) W^T * s_e
    t = lambda q: torch.as_tensor(np.ascontiguousarray(q).ravel(), device="cuda",
                                  dtype=torch.float32)
    out = torch.empty(O.mask.size, dtype=torch.float32, device="cuda")
    M.forward(out, t(a), t(minv), t(O.mask), t(1.0 / O.mult), P.nelv)
    S = np.sqrt(minv).ravel()
    local_ref = omlp.forward_sym(theta.astype(np.float64), (S * a).reshape(-1, lx ** 3),
                                 n_hid).ravel() * S * O.mask.ravel()
    assert rel_l2(out.cpu().numpy(), local_ref) <= 2e-2


@pytest.mark.parametrize("n_in,n_hid,B", [(64, 16, 40), (512, 48, 300)])
def test_sym_loss_and_tied_gradient_match_oracle(n_in, n_hid, B):
    g = synth.rng(n_in + B + 1)
    theta = _sym_params(n_in, n_hid, seed=B)
    X = g.normal(size=(B, n_in)).astype(np.float32)
    T = g.normal(size=(B, n_in)).astype(np.float32)
    M = ax.Mlp(n_in, n_hid, params=theta, arch=ax.AX_MLP_SYM)
    L, grad = M.loss_grad(torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda"))
    L_ref, g_ref = omlp.mse_loss_grad_sym(theta.astype(np.float64), X, T, n_hid)
    assert abs(L - L_ref) <= 1e-5 * L_ref
    assert rel_l2(grad, g_ref) <= 1e-4
    assert not grad[n_in * n_hid:].any()
    M.adam(1e-3)
    W1, b1, W2, b2 = omlp.unpack(M.get_params(), n_in, n_hid)
    assert np.array_equal(W2, W1.T) and not b1.any() and not b2.any()
    ref, _, _ = omlp.adam_step(theta.astype(np.float64), grad.astype(np.float64),
                               np.zeros(theta.size), np.zeros(theta.size), 1, lr=1e-3)
    nw = n_in * n_hid
    assert rel_l2(W1.ravel(), ref[:nw]) <= 1e-5


def test_sym_energy_loss_and_first_step_match_oracle():
    """One pair, one pass: the reported loss is the oracle's relative energy
    error at the initial W, and the first Adam step moves W by lr against
    the sign of the oracle's energy gradient (Adam's first-step closed form)."""
    lx, n_hid = 4, 8
    v = synth.box_vertices(3, 3, 2, seed=11)
    P = ax.Poisson(v, lx)
    O = oracle.Problem(v, lx)
    minv = np.where(O.mask > 0, 1.0 / O.diag, 0.0)
    r = O.mask * oracle.gs_sum(synth.uniform(O.mask.shape, seed=12), O.glob) / O.mult
    e = O.mask * oracle.gs_sum(synth.uniform(O.mask.shape, seed=13), O.glob) / O.mult
    theta = _sym_params(lx ** 3, n_hid, seed=3, scale=0.5)
    M = ax.Mlp(lx ** 3, n_hid, params=theta, arch=ax.AX_MLP_SYM)
    t = lambda q: torch.as_tensor(q.reshape(1, -1), device="cuda")
    lr = 1e-4
    loss = ax.train_energy(P, M, t(r), t(e), epochs=1, lr=lr)
    L_ref, g_ref = omlp.energy_loss_grad_sym(theta.astype(np.float64), [(r, e)], O.apply, O.dot,
                                             minv, O.mask, O.glob, lx, n_hid, oracle.gs_sum)
    assert abs(loss - L_ref) <= 1e-5 * L_ref
    nw = lx ** 3 * n_hid
    step = (theta[:nw].astype(np.float64) - M.get_params()[:nw].astype(np.float64)) / lr
    big = np.abs(g_ref[:nw]) > 1e-2 * np.abs(g_ref[:nw]).max()
    assert big.sum() > nw // 4
    assert np.array_equal(np.sign(step[big]), np.sign(g_ref[:nw][big]))
    np.testing.assert_allclose(np.abs(step[big]), 1.0, rtol=0, atol=2e-2)


def test_sym_trained_preconditioner_cuts_iterations():
    """Trained on CG iterates of one right-hand side, the symmetric form
    needs clearly fewer flexible-CG iterations than Jacobi on another
    right-hand side, in fp64 and inside fp32 refinement."""
    lx, n_hid = 6, 24
    P = _var_problem(4, lx, seed=6)
    b = P.rhs(oracle.poisson_rhs_f)
    R, E = ax.iterate_pairs(P, b, iterates=(2, 4, 8, 16, 32, 64))
    M = ax.Mlp(lx ** 3, n_hid, params=_sym_params(lx ** 3, n_hid, seed=1, scale=0.05),
               arch=ax.AX_MLP_SYM)
    loss = ax.train_energy(P, M, R, E, epochs=100, lr=5e-3)
    assert loss < 0.7
    b2 = P.rhs(ax.fourier_coefficient(9, lo=-1.0, hi=1.0))
    _, ij, _, _, rcj = P.fcg(b2, None, tol=1e-8)
    x, il, rel, fb, rc = P.fcg(b2, M, tol=1e-8)
    assert rcj == 0 and rc == 0 and rel <= 1e-8 and fb == 0
    assert il <= 0.8 * ij
    x2, no, ni, rel2, fb2, rc2 = P.mpfcg(b2, M, tol=1e-8, inner_tol=1e-4)
    assert rc2 == 0 and rel2 <= 1e-8
    r2, bf = P.residual(b2, x2).reshape(-1), b2.reshape(-1)
    c = P.gs.inverse_multiplicity()
    assert float(torch.sum(c * r2 * r2)) <= (1.5e-8) ** 2 * float(torch.sum(c * bf * bf))
