"""Pins for the oracle's 1-D GLL basis (nodes, weights, differentiation).

Each check compares the oracle with something other than itself: textbook
closed forms (tests/golden), numpy's independent Legendre module, exact
polynomial calculus, or a brute-force Vandermonde construction.
"""
import math
import os

import numpy as np
import numpy.polynomial.legendre as npleg
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.txt")


def _golden():
    env = {"sqrt": math.sqrt}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lx, xs, ws = (s.strip() for s in line.split("|"))
        x = [eval(t, env) for t in xs.split(";")]
        w = [eval(t, env) for t in ws.split(";")]
        yield int(lx), np.array(x), np.array(w)


@pytest.mark.parametrize("case", list(_golden()), ids=lambda c: f"lx{c[0]}")
def test_gll_closed_forms(case):
    lx, x_ref, w_ref = case
    x, w = oracle.gll(lx)
    np.testing.assert_allclose(x, x_ref, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, w_ref, rtol=1e-14, atol=0)


@pytest.mark.parametrize("lx", range(2, 17))
def test_gll_against_numpy_legendre(lx):
    """Interior nodes are the roots of L_N' (numpy's own Legendre module);
    weights are 2 / (N (N+1) L_N(x)^2) evaluated with numpy's series."""
    n = lx - 1
    x, w = oracle.gll(lx)
    cN = np.zeros(n + 1)
    cN[n] = 1.0
    interior = np.sort(npleg.legroots(npleg.legder(cN))) if n >= 2 else np.array([])
    np.testing.assert_allclose(x[1:-1], interior, atol=1e-13)
    assert x[0] == -1.0 and x[-1] == 1.0
    ln = npleg.legval(x, cN)
    np.testing.assert_allclose(w, 2.0 / (n * (n + 1) * ln ** 2), rtol=1e-12)


@pytest.mark.parametrize("lx", range(2, 17))
def test_gll_quadrature_degree(lx):
    """Exact for monomials of degree <= 2N-1, not for x^(2N)."""
    n = lx - 1
    x, w = oracle.gll(lx)
    assert abs(w.sum() - 2.0) < 1e-14
    for p in range(0, 2 * n):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.dot(w, x ** p) - exact) < 1e-13, p
    exact = 2.0 / (2 * n + 1)
    assert abs(np.dot(w, x ** (2 * n)) - exact) > 1e-10


@pytest.mark.parametrize("lx", range(2, 17))
def test_diff_matrix_exact_on_polynomials(lx):
    """D x^p = p x^(p-1) for p <= N; D 1 = 0 (rows sum to zero)."""
    n = lx - 1
    x, _ = oracle.gll(lx)
    d = oracle.diff_matrix(lx)
    np.testing.assert_allclose(d.sum(axis=1), 0.0, atol=1e-12 * lx * lx)
    for p in range(1, n + 1):
        np.testing.assert_allclose(d @ x ** p, p * x ** (p - 1), atol=5e-12 * lx ** 2)


@pytest.mark.parametrize("lx", range(2, 13))
def test_diff_matrix_vs_vandermonde(lx):
    """Brute force: l_j = sum_m c_mj x^m with V c = I; D_ij = l_j'(x_i)."""
    x, _ = oracle.gll(lx)
    V = np.vander(x, lx, increasing=True)
    Vd = np.zeros_like(V)
    for m in range(1, lx):
        Vd[:, m] = m * x ** (m - 1)
    D_bf = Vd @ np.linalg.inv(V)
    np.testing.assert_allclose(oracle.diff_matrix(lx), D_bf, atol=1e-9 * lx ** 3)


@pytest.mark.parametrize("lx", [3, 5, 8, 12])
def test_lagrange_basis_reading(lx):
    """The basis l_i(x) = (x^2-1) L_N'(x) / (N(N+1) L_N(x_i)(x - x_i)) is
    cardinal on the GLL nodes and its derivative at the nodes is D."""
    n = lx - 1
    x, _ = oracle.gll(lx)
    cN = np.zeros(n + 1)
    cN[n] = 1.0
    dcN = npleg.legder(cN)

    def basis(i, t):
        return (t * t - 1) * npleg.legval(t, dcN) / (
            n * (n + 1) * npleg.legval(x[i], cN) * (t - x[i]))

    for i in range(lx):
        for j in range(lx):
            if i != j:
                assert abs(basis(i, x[j])) < 1e-12
        eps = 1e-7
        assert abs(basis(i, x[i] + eps) - 1.0) < 1e-5
        # derivative of l_i at node j (j != i) by a central difference
        d = oracle.diff_matrix(lx)
        for j in range(lx):
            if j == i:
                continue
            h = 1e-6
            fd = (basis(i, x[j] + h) - basis(i, x[j] - h)) / (2 * h)
            assert abs(fd - d[j, i]) < 1e-5 * max(1.0, abs(d[j, i]))


@pytest.mark.parametrize("lx", [2, 4, 8, 12])
def test_d_buffers_reading(lx):
    """dx[l*lx+i] = D_il: with u = xi along i the r-derivative is one
    everywhere; the transposed reading of the buffer fails that."""
    x, _ = oracle.gll(lx)
    dx, dxt = oracle.d_buffers(lx)
    bx = dx.reshape(lx, lx)
    ur = np.array([sum(bx[l, i] * x[l] for l in range(lx)) for i in range(lx)])
    np.testing.assert_allclose(ur, 1.0, atol=1e-12)
    wrong = np.array([sum(bx[i, l] * x[l] for l in range(lx)) for i in range(lx)])
    assert np.max(np.abs(wrong - 1.0)) > 1e-3
    np.testing.assert_array_equal(dxt.reshape(lx, lx), bx.T)
