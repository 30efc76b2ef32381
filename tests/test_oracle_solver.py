"""Pins for the oracle's gather-scatter and conjugate-gradient solver.

gather-scatter is checked against a Boolean scatter matrix built with
scipy.sparse and the closed-form multiplicities of a structured box; the
solver against a dense numpy solve and the analytic Poisson solution.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2506_20994_gb300 import synth


@pytest.mark.parametrize("dims,lx", [((2, 2, 2), 3), ((3, 2, 1), 4), ((1, 1, 1), 5)])
def test_gs_against_boolean_matrix(dims, lx):
    nx, ny, nz = dims
    glob = oracle.numbering(nx, ny, nz, lx).ravel()
    n = glob.size
    Q = sp.csr_matrix((np.ones(n), (np.arange(n), glob)))  # local <- global
    v = synth.uniform(n, seed=1)
    ref = Q @ (Q.T @ v)
    np.testing.assert_allclose(oracle.gs_sum(v, glob), ref, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("lx", [2, 3, 6])
def test_multiplicity_closed_form(lx):
    """On a structured box, an element-interior node has multiplicity 1, a
    face node 2, an edge node 4 and a vertex node 8 (when fully surrounded)."""
    nx = ny = nz = 3
    glob = oracle.numbering(nx, ny, nz, lx)
    mult = oracle.multiplicity(glob)
    n = lx - 1
    NX = NY = nx * n + 1
    G = glob
    X, Y, Z = G % NX, (G // NX) % NY, G // (NX * NY)

    def count(c, N):
        # number of elements sharing coordinate index c along one axis
        on_el_face = (c % n == 0)
        inner = (c > 0) & (c < N - 1)
        return np.where(on_el_face & inner, 2, 1)

    expect = count(X, NX) * count(Y, NY) * count(Z, nz * n + 1)
    np.testing.assert_array_equal(mult, expect)
    # unique-node count
    assert len(np.unique(glob)) == (nx * n + 1) ** 3


def test_pcg_matches_dense_solve():
    lx = 4
    v = synth.box_vertices(2, seed=2)
    prob = oracle.Problem(v, lx, f=oracle.poisson_rhs_f)
    x, its, hist = oracle.pcg(prob, prob.b, tol=1e-12)
    assert hist[-1] <= 1e-12
    # dense assembled system on interior global nodes
    glob = prob.glob.ravel()
    nglob = glob.max() + 1
    Q = sp.csr_matrix((np.ones(glob.size), (np.arange(glob.size), glob))).toarray()
    n3 = lx ** 3
    AL = np.zeros((glob.size, glob.size))
    for p in range(glob.size):
        e = np.zeros(glob.size)
        e[p] = 1.0
        AL[:, p] = prob.ax_local(e.reshape(prob.h1.shape)).ravel()
    A = Q.T @ AL @ Q
    bg = (Q.T @ (prob.b.ravel() / prob.mult.ravel()))
    interior = np.zeros(nglob, dtype=bool)
    interior[glob[prob.mask.ravel() > 0]] = True
    xg = np.zeros(nglob)
    xg[interior] = np.linalg.solve(A[np.ix_(interior, interior)], bg[interior])
    np.testing.assert_allclose(x.ravel(), Q @ xg, rtol=0, atol=1e-10 * np.abs(xg).max())
    assert n3 > 0


def test_pcg_spectral_convergence_and_monotone_energy_error():
    """The nodal error against sin(pi x) sin(pi y) sin(pi z) falls
    spectrally with lx; the A-norm error of the CG iterates is monotone."""
    errs = []
    for lx in (3, 5, 7):
        v = synth.box_vertices(2, seed=0)
        prob = oracle.Problem(v, lx, f=oracle.poisson_rhs_f)
        x, its, hist = oracle.pcg(prob, prob.b, tol=1e-12)
        xyz = prob.geo["xyz"]
        exact = np.sin(np.pi * xyz[..., 0]) * np.sin(np.pi * xyz[..., 1]) * np.sin(np.pi * xyz[..., 2])
        errs.append(np.abs(x - exact).max())
    assert errs[0] > 10 * errs[1] > 100 * errs[2]
    # monotone A-norm error on a small case
    lx = 4
    v = synth.box_vertices(2, seed=9)
    prob = oracle.Problem(v, lx, f=oracle.poisson_rhs_f)
    xstar, _, _ = oracle.pcg(prob, prob.b, tol=1e-14)
    energies = []
    for k in range(1, 12):
        xk, _, _ = oracle.pcg(prob, prob.b, tol=0.0, maxit=k)
        e = xk - xstar
        energies.append(np.sum(e * prob.ax_local(e)))
    assert all(energies[i + 1] <= energies[i] * (1 + 1e-9) for i in range(len(energies) - 1))
