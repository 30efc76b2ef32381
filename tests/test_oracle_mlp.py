"""Pins for the oracle network: backprop gradient against central finite
differences in fp64, Adam against its closed form on a quadratic, and the
preconditioner's algebraic properties (zero network = Jacobi, positive
homogeneity in r)."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2506_20994_gb300 import synth


@pytest.mark.parametrize("n_in,n_hid,B", [(8, 3, 5), (27, 6, 4), (64, 10, 7)])
def test_gradient_matches_central_differences(n_in, n_hid, B):
    g = synth.rng(n_in)
    theta = g.normal(0, 0.3, size=mlp.nparams(n_in, n_hid))
    X = g.normal(size=(B, n_in))
    T = g.normal(size=(B, n_in))
    L, grad = mlp.loss_and_grad(theta, X, T, n_hid)
    h = 1e-6
    fd = np.empty_like(theta)
    for q in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[q] += h
        tm[q] -= h
        fd[q] = (mlp.loss_and_grad(tp, X, T, n_hid)[0] - mlp.loss_and_grad(tm, X, T, n_hid)[0]) / (2 * h)
    assert np.linalg.norm(grad - fd) <= 1e-6 * np.linalg.norm(fd)
    # the loss is the forward residual
    Y = mlp.forward(theta, X, n_hid)
    assert abs(L - np.mean((Y - T) ** 2)) < 1e-15


def test_adam_closed_form_first_step():
    """Step 1 of Adam moves every coordinate by lr * g/(|g| + eps') (the
    bias corrections cancel): the sign-descent closed form."""
    g = synth.rng(3)
    theta = g.normal(size=50)
    grad = g.normal(size=50)
    new, m, v = mlp.adam_step(theta, grad, np.zeros(50), np.zeros(50), 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(new, theta - 0.01 * np.sign(grad), rtol=0, atol=1e-15)
    # and it minimises a quadratic
    th = np.full(4, 3.0)
    m = v = np.zeros(4)
    for k in range(1, 3001):
        th, m, v = mlp.adam_step(th, 2 * th, m, v, k, lr=0.01)
    assert np.abs(th).max() < 1e-2


def test_zero_network_is_jacobi_and_homogeneous():
    lx = 4
    v = synth.box_vertices(2, seed=1)
    prob = oracle.Problem(v, lx)
    minv = np.where(prob.mask > 0, 1.0 / prob.diag, 0.0)
    r = prob.mask * oracle.gs_sum(synth.uniform(prob.mask.shape, seed=2), prob.glob)
    n_hid = 5
    theta0 = np.zeros(mlp.nparams(lx ** 3, n_hid))
    z = mlp.precondition(theta0, r, minv, prob.mask, prob.mult, prob.glob, lx, n_hid,
                         oracle.gs_sum)
    np.testing.assert_allclose(z, minv * r, rtol=0, atol=0)
    theta = synth.rng(4).normal(0, 0.2, size=theta0.size)
    z1 = mlp.precondition(theta, r, minv, prob.mask, prob.mult, prob.glob, lx, n_hid,
                          oracle.gs_sum)
    z3 = mlp.precondition(theta, 3.0 * r, minv, prob.mask, prob.mult, prob.glob, lx, n_hid,
                          oracle.gs_sum)
    np.testing.assert_allclose(z3, 3.0 * z1, rtol=1e-12, atol=1e-14)
    # continuous across shared nodes and zero on the boundary
    np.testing.assert_allclose(oracle.gs_sum(z1, prob.glob) / prob.mult, z1, rtol=1e-12, atol=1e-14)
    assert np.all(z1[prob.mask == 0] == 0)


# ---------------------------------------------------------------------------
# Symmetric linear form
# ---------------------------------------------------------------------------
def _sym_case(lx=3, n=2, n_hid=3, seed=5):
    v = synth.box_vertices(n, seed=seed)
    prob = oracle.Problem(v, lx)
    minv = np.where(prob.mask > 0, 1.0 / prob.diag, 0.0)
    theta = mlp.tie(synth.rng(seed + 1).normal(0, 0.3, size=mlp.nparams(lx ** 3, n_hid)),
                    lx ** 3, n_hid)
    return prob, minv, theta, n_hid


def _dense_sym(prob, minv, theta, n_hid):
    """B = diag(minv) + sum_e P_e^T S_e W W^T S_e P_e on global nodes, with
    P_e the 0/1 gather of element e's nodes (assembled entry by entry)."""
    lx = prob.lx
    n3 = lx ** 3
    glob = prob.glob.reshape(-1, n3)
    ng = int(glob.max()) + 1
    W = mlp.unpack(theta, n3, n_hid)[0]
    K = W @ W.T
    S = np.sqrt(minv).reshape(-1, n3)
    B = np.zeros((ng, ng))
    B[prob.glob.ravel(), prob.glob.ravel()] = minv.ravel()   # same value at every copy
    for e in range(glob.shape[0]):
        for a in range(n3):
            for b in range(n3):
                B[glob[e, a], glob[e, b]] += S[e, a] * K[a, b] * S[e, b]
    return B, glob


def test_sym_preconditioner_matches_dense_assembly():
    prob, minv, theta, n_hid = _sym_case()
    B, glob = _dense_sym(prob, minv, theta, n_hid)
    ng = B.shape[0]
    gmask = np.zeros(ng)
    gmask[prob.glob.ravel()] = prob.mask.ravel()
    a = synth.uniform(ng, seed=9) * gmask
    z = mlp.precondition_sym(theta, a[prob.glob], minv, prob.mask, prob.glob, prob.lx, n_hid,
                             oracle.gs_sum)
    ref = (B @ a)[prob.glob]
    np.testing.assert_allclose(z, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    # B restricted to the unconstrained nodes is symmetric positive definite
    idx = np.flatnonzero(gmask)
    Bi = B[np.ix_(idx, idx)]
    assert np.abs(Bi - Bi.T).max() <= 1e-15 * np.abs(Bi).max()
    assert np.linalg.eigvalsh(Bi).min() >= minv[prob.mask > 0].min() * (1 - 1e-12)


def test_sym_zero_basis_is_jacobi_and_tie_is_idempotent():
    prob, minv, theta, n_hid = _sym_case()
    r = prob.mask * oracle.gs_sum(synth.uniform(prob.mask.shape, seed=2), prob.glob)
    z0 = mlp.precondition_sym(np.zeros_like(theta), r, minv, prob.mask, prob.glob, prob.lx,
                              n_hid, oracle.gs_sum)
    np.testing.assert_array_equal(z0, minv * r)
    t2 = mlp.tie(theta, prob.lx ** 3, n_hid)
    np.testing.assert_array_equal(t2, theta)
    W1, b1, W2, b2 = mlp.unpack(t2, prob.lx ** 3, n_hid)
    np.testing.assert_array_equal(W2, W1.T)
    assert not b1.any() and not b2.any()


def _pairs(prob, k, seed):
    out = []
    for q in range(k):
        r = prob.mask * oracle.gs_sum(synth.uniform(prob.mask.shape, seed=seed + 2 * q),
                                      prob.glob) / prob.mult
        e = prob.mask * oracle.gs_sum(synth.uniform(prob.mask.shape, seed=seed + 2 * q + 1),
                                      prob.glob) / prob.mult
        out.append((r, e))
    return out


def test_sym_energy_loss_matches_dense_definition():
    prob, minv, theta, n_hid = _sym_case()
    B, glob = _dense_sym(prob, minv, theta, n_hid)
    ng = B.shape[0]
    # the assembled operator, column by column from unit global vectors
    A = np.zeros((ng, ng))
    for j in range(ng):
        ej = np.zeros(ng)
        ej[j] = 1.0
        col = prob.apply(ej[prob.glob])
        A[prob.glob.ravel(), j] = col.ravel()
    pairs = _pairs(prob, 3, seed=20)
    L, _ = mlp.energy_loss_grad_sym(theta, pairs, prob.apply, prob.dot, minv, prob.mask,
                                    prob.glob, prob.lx, n_hid, oracle.gs_sum)
    ref = 0.0
    for r, e in pairs:
        rg = np.zeros(ng)
        eg = np.zeros(ng)
        rg[prob.glob.ravel()] = r.ravel()
        eg[prob.glob.ravel()] = e.ravel()
        d = eg - B @ rg
        ref += (d @ A @ d) / (eg @ A @ eg)
    assert abs(L - ref / len(pairs)) <= 1e-12 * ref


def test_sym_energy_gradient_matches_central_differences():
    prob, minv, theta, n_hid = _sym_case()
    pairs = _pairs(prob, 2, seed=40)
    n_in = prob.lx ** 3
    args = (pairs, prob.apply, prob.dot, minv, prob.mask, prob.glob, prob.lx, n_hid,
            oracle.gs_sum)
    L, grad = mlp.energy_loss_grad_sym(theta, *args)
    nw = n_in * n_hid
    assert not grad[nw:].any()
    h = 1e-6
    W1 = theta[:nw]
    fd = np.empty(nw)
    for q in range(nw):
        # W enters both layers: perturb it through tie() so W2 follows W1
        tp, tm = theta.copy(), theta.copy()
        tp[q] += h
        tm[q] -= h
        tp, tm = mlp.tie(tp, n_in, n_hid), mlp.tie(tm, n_in, n_hid)
        fd[q] = (mlp.energy_loss_grad_sym(tp, *args)[0]
                 - mlp.energy_loss_grad_sym(tm, *args)[0]) / (2 * h)
    assert np.linalg.norm(grad[:nw] - fd) <= 1e-6 * np.linalg.norm(fd)
    assert np.linalg.norm(W1) > 0


def test_sym_mse_gradient_matches_central_differences():
    n_in, n_hid, B = 27, 4, 6
    g = synth.rng(77)
    theta = mlp.tie(g.normal(0, 0.3, size=mlp.nparams(n_in, n_hid)), n_in, n_hid)
    X = g.normal(size=(B, n_in))
    T = g.normal(size=(B, n_in))
    L, grad = mlp.mse_loss_grad_sym(theta, X, T, n_hid)
    assert abs(L - np.mean((mlp.forward_sym(theta, X, n_hid) - T) ** 2)) < 1e-15
    # the tied form is the general network with W2 = W1^T, b = 0
    assert abs(L - mlp.loss_and_grad(theta, X, T, n_hid)[0]) > 0  # tanh differs
    nw = n_in * n_hid
    fd = np.empty(nw)
    h = 1e-6
    for q in range(nw):
        tp, tm = theta.copy(), theta.copy()
        tp[q] += h
        tm[q] -= h
        fd[q] = (mlp.mse_loss_grad_sym(mlp.tie(tp, n_in, n_hid), X, T, n_hid)[0]
                 - mlp.mse_loss_grad_sym(mlp.tie(tm, n_in, n_hid), X, T, n_hid)[0]) / (2 * h)
    assert np.linalg.norm(grad[:nw] - fd) <= 1e-6 * np.linalg.norm(fd)
    assert not grad[nw:].any()
