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
