"""Pins for the oracle's geometry and element operator.

The operator is checked against dense matrices built a different way
(Kronecker products of the 1-D matrices, numpy only), the textbook tensor
form on affine elements, and exact properties of the weak Poisson form
(constants in the kernel, symmetry, semi-definiteness, the linear patch test).
"""
import numpy as np
import pytest

import oracle
from paper_2506_20994_gb300 import synth


def _dense_element(lx, d, h1, gs):
    """A_e = sum_ab D_a^T diag(h1 G_ab) D_b with D_r = I (x) I (x) D,
    D_s = I (x) D (x) I, D_t = D (x) I (x) I on the [k][j][i] ordering."""
    I = np.eye(lx)
    Dr = np.kron(I, np.kron(I, d))
    Ds = np.kron(I, np.kron(d, I))
    Dt = np.kron(d, np.kron(I, I))
    g11, g22, g33, g12, g13, g23 = (np.asarray(g).ravel() for g in gs)
    h = np.asarray(h1).ravel()
    Dm = [Dr, Ds, Dt]
    G = [[g11, g12, g13], [g12, g22, g23], [g13, g23, g33]]
    A = np.zeros((lx ** 3, lx ** 3))
    for a in range(3):
        for b in range(3):
            A += Dm[a].T @ np.diag(h * G[a][b]) @ Dm[b]
    return A


def _oracle_matrix(lx, dx, dxt, h1, gs):
    """The oracle operator of one element as a dense matrix (unit vectors)."""
    n3 = lx ** 3
    A = np.zeros((n3, n3))
    for p in range(n3):
        e = np.zeros(n3)
        e[p] = 1.0
        A[:, p] = oracle.ax_helm(e, dx, dxt, h1, *gs, lx)
    return A


@pytest.mark.parametrize("lx", [2, 3, 4, 6])
def test_affine_element_tensor_form(lx):
    """Undeformed cube of width h: A = K(x)M(x)M + M(x)K(x)M + M(x)M(x)K with
    M = (h/2) diag(w) and K = (2/h) D^T diag(w) D (textbook closed form)."""
    n = 3
    v = synth.box_vertices(n, seed=0, amp=0.0)
    geo = oracle.box_geometry(v, lx)
    h = 1.0 / n
    _, w = oracle.gll(lx)
    d = oracle.diff_matrix(lx)
    M = (h / 2) * np.diag(w)
    K = (2 / h) * d.T @ np.diag(w) @ d
    A_ref = np.kron(M, np.kron(M, K)) + np.kron(M, np.kron(K, M)) + np.kron(K, np.kron(M, M))
    dx, dxt = oracle.d_buffers(lx)
    e = 5  # any element
    gs = [geo[k][e] for k in ("g11", "g22", "g33", "g12", "g13", "g23")]
    A = _oracle_matrix(lx, dx, dxt, np.ones(lx ** 3), gs)
    np.testing.assert_allclose(A, A_ref, atol=1e-13 * np.abs(A_ref).max())


@pytest.mark.parametrize("lx", [3, 5, 7])
def test_deformed_elements_vs_kronecker(lx):
    """1-8 deformed elements with a random positive h1: oracle = dense
    Kronecker assembly, element by element."""
    v = synth.box_vertices(2, seed=3)
    geo = oracle.box_geometry(v, lx)
    h1 = synth.uniform(geo["jac"].shape, seed=4, lo=0.5, hi=2.0)
    d = oracle.diff_matrix(lx)
    dx, dxt = oracle.d_buffers(lx)
    for e in range(8):
        gs = [geo[k][e] for k in ("g11", "g22", "g33", "g12", "g13", "g23")]
        A = _oracle_matrix(lx, dx, dxt, h1[e], gs)
        A_ref = _dense_element(lx, d, h1[e], gs)
        np.testing.assert_allclose(A, A_ref, atol=1e-12 * np.abs(A_ref).max())
        # symmetric, PSD, exactly one zero eigenvalue (the constants)
        np.testing.assert_allclose(A, A.T, atol=1e-12 * np.abs(A).max())
        ev = np.linalg.eigvalsh(0.5 * (A + A.T))
        assert ev[0] > -1e-12 * ev[-1]
        assert ev[1] > 1e-8 * ev[-1]


def _kron_xyz(lx, mats, h1, gs):
    """Listing 2 with one matrix per direction as a dense matrix: buffer
    m[l*lx + i] is the (i, l) entry of the 1-D factor, so the forward
    gradient is (I(x)I(x)X, I(x)Y(x)I, Z(x)I(x)I) u and the transposed one
    sums (I(x)I(x)Xt) wr + (I(x)Yt(x)I) ws + (Zt(x)I(x)I) wt."""
    I = np.eye(lx)
    X, Y, Z, Xt, Yt, Zt = (np.asarray(m).reshape(lx, lx).T for m in mats)
    F = [np.kron(I, np.kron(I, X)), np.kron(I, np.kron(Y, I)), np.kron(Z, np.kron(I, I))]
    T = [np.kron(I, np.kron(I, Xt)), np.kron(I, np.kron(Yt, I)), np.kron(Zt, np.kron(I, I))]
    g11, g22, g33, g12, g13, g23 = (np.asarray(g).ravel() for g in gs)
    G = [[g11, g12, g13], [g12, g22, g23], [g13, g23, g33]]
    h = np.asarray(h1).ravel()
    A = np.zeros((lx ** 3, lx ** 3))
    for a in range(3):
        for b in range(3):
            A += T[a] @ np.diag(h * G[a][b]) @ F[b]
    return A


@pytest.mark.parametrize("lx", [2, 3, 5])
def test_separate_direction_matrices_vs_kronecker(lx):
    """The full signature of Listings 1-2 (dx, dy, dz, dxt, dyt, dzt): six
    unrelated random matrices on deformed elements against the dense
    Kronecker form; each matrix reaches its own direction (a swapped pair
    fails)."""
    v = synth.box_vertices(2, seed=5)
    geo = oracle.box_geometry(v, lx)
    h1 = synth.uniform(geo["jac"].shape, seed=6, lo=0.5, hi=2.0)
    mats = [synth.uniform((lx * lx,), seed=10 + m) for m in range(6)]
    dx, dy, dz, dxt, dyt, dzt = mats
    n3 = lx ** 3
    for e in (0, 5):
        gs = [geo[k][e] for k in ("g11", "g22", "g33", "g12", "g13", "g23")]
        A = np.zeros((n3, n3))
        for p in range(n3):
            u = np.zeros(n3)
            u[p] = 1.0
            A[:, p] = oracle.ax_helm(u, dx, dxt, h1[e], *gs, lx, dy=dy, dz=dz, dyt=dyt, dzt=dzt)
        A_ref = _kron_xyz(lx, mats, h1[e], gs)
        np.testing.assert_allclose(A, A_ref, atol=1e-12 * np.abs(A_ref).max())
        swapped = _kron_xyz(lx, [dy, dx, dz, dxt, dyt, dzt], h1[e], gs)
        assert np.abs(A - swapped).max() > 1e-3 * np.abs(A_ref).max()
    # with dy = dz = dx and dyt = dzt = dxt it is the one-matrix form, bit for bit
    u = synth.uniform(geo["jac"].shape, seed=7)
    gs = [geo[k] for k in ("g11", "g22", "g33", "g12", "g13", "g23")]
    a = oracle.ax_helm(u, dx, dxt, h1, *gs, lx)
    b = oracle.ax_helm(u, dx, dxt, h1, *gs, lx, dy=dx, dz=dx, dyt=dxt, dzt=dxt)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("lx", [2, 4, 8, 12])
def test_constants_in_kernel(lx):
    v = synth.box_vertices(3, seed=1)
    geo = oracle.box_geometry(v, lx)
    dx, dxt = oracle.d_buffers(lx)
    gs = [geo[k] for k in ("g11", "g22", "g33", "g12", "g13", "g23")]
    u = np.full(geo["jac"].shape, 3.7)
    w = oracle.ax_helm(u, dx, dxt, np.ones_like(u), *gs, lx)
    ref = oracle.ax_helm(synth.uniform(u.shape, seed=2), dx, dxt, np.ones_like(u), *gs, lx)
    assert np.abs(w).max() < 1e-13 * np.abs(ref).max() * 3.7 + 1e-14


@pytest.mark.parametrize("lx", [3, 4, 6, 8])
def test_symmetry_on_random_fields(lx):
    v = synth.box_vertices(3, seed=7)
    geo = oracle.box_geometry(v, lx)
    dx, dxt = oracle.d_buffers(lx)
    gs = [geo[k] for k in ("g11", "g22", "g33", "g12", "g13", "g23")]
    h1 = synth.uniform(geo["jac"].shape, seed=8, lo=0.5, hi=2.0)
    a = synth.uniform(geo["jac"].shape, seed=9)
    b = synth.uniform(geo["jac"].shape, seed=10)
    Aa = oracle.ax_helm(a, dx, dxt, h1, *gs, lx)
    Ab = oracle.ax_helm(b, dx, dxt, h1, *gs, lx)
    assert abs(np.sum(b * Aa) - np.sum(a * Ab)) < 1e-12 * np.sqrt(np.sum(Aa ** 2) * np.sum(b ** 2))
    assert np.sum(a * Aa) > 0


@pytest.mark.parametrize("lx", [3, 4, 6])
def test_linear_patch_test(lx):
    """u = a.x + c on a deformed trilinear mesh: the assembled residual is
    zero at interior nodes and u^T A u = |a|^2 |Omega| = |a|^2 (quadrature
    exact: the integrands have degree <= N+1 per variable)."""
    n = 3
    v = synth.box_vertices(n, seed=11)
    prob = oracle.Problem(v, lx)
    xyz = prob.geo["xyz"]
    a = np.array([0.3, -1.2, 0.7])
    u = xyz @ a + 0.25
    Au_local = prob.ax_local(u)
    Au = oracle.gs_sum(Au_local, prob.glob)
    interior = prob.mask > 0
    scale = np.abs(Au).max()
    assert np.abs(Au[interior]).max() < 1e-12 * scale
    energy = np.sum(u * Au_local)
    assert abs(energy - np.dot(a, a)) < 1e-12


@pytest.mark.parametrize("lx", [2, 3, 5, 8])
def test_geometry_volume_and_affine_factors(lx):
    """sum B = |Omega| = 1 on the perturbed cube (jac has degree <= 2 per
    variable); on the undeformed cube G = (h/2) W I."""
    v = synth.box_vertices(3, seed=5)
    geo = oracle.box_geometry(v, lx)
    if lx >= 3:
        assert abs(geo["B"].sum() - 1.0) < 1e-13
    h = 1.0 / 3
    geo0 = oracle.box_geometry(synth.box_vertices(3, seed=5, amp=0.0), lx)
    _, w = oracle.gll(lx)
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    for k in ("g11", "g22", "g33"):
        np.testing.assert_allclose(geo0[k], np.broadcast_to((h / 2) * W, geo0[k].shape), rtol=1e-12)
    for k in ("g12", "g13", "g23"):
        assert np.abs(geo0[k]).max() < 1e-15


@pytest.mark.parametrize("lx", [3, 4])
def test_jacobi_diagonal_vs_unit_vectors(lx):
    """The assembled diagonal equals e_g^T A e_g for every global node g."""
    v = synth.box_vertices(2, seed=6)
    h1 = None
    prob = oracle.Problem(v, lx, h1=h1)
    glob = prob.glob
    nglob = glob.max() + 1
    for g in range(0, nglob, max(1, nglob // 40)):
        e_loc = (glob == g).astype(np.float64)
        Ae = oracle.gs_sum(prob.ax_local(e_loc), glob)
        val = Ae[glob == g]
        np.testing.assert_allclose(prob.diag[glob == g], val, rtol=1e-12)


# ---------------------------------------------------------------------------
# Helmholtz mass term (h2 B)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("lx", [3, 5])
def test_helmholtz_affine_tensor_form(lx):
    """Affine cube of width h: A + h2 M(x)M(x)M with M = (h/2) diag(w), the
    textbook mass matrix, for a constant h2."""
    n, h2 = 3, 2.5
    v = synth.box_vertices(n, seed=0, amp=0.0)
    geo = oracle.box_geometry(v, lx)
    h = 1.0 / n
    _, wq = oracle.gll(lx)
    d = oracle.diff_matrix(lx)
    M = (h / 2) * np.diag(wq)
    K = (2 / h) * d.T @ np.diag(wq) @ d
    A_ref = (np.kron(M, np.kron(M, K)) + np.kron(M, np.kron(K, M)) + np.kron(K, np.kron(M, M))
             + h2 * np.kron(M, np.kron(M, M)))
    dx, dxt = oracle.d_buffers(lx)
    e = 4
    gs = [geo[k][e] for k in ("g11", "g22", "g33", "g12", "g13", "g23")]
    n3 = lx ** 3
    A = np.zeros((n3, n3))
    for p in range(n3):
        u = np.zeros(n3)
        u[p] = 1.0
        A[:, p] = oracle.ax_helm_h2(u, dx, dxt, np.ones(n3), *gs, lx, np.full(n3, h2),
                                    geo["B"][e])
    np.testing.assert_allclose(A, A_ref, atol=1e-13 * np.abs(A_ref).max())


def test_helmholtz_constant_and_solve():
    """A 1 = 0 leaves w = h2 B on constants (deformed mesh, variable h2), and
    the assembled Helmholtz system solved by PCG matches a dense solve; its
    Jacobi diagonal is the assembled unit-vector diagonal."""
    lx = 4
    v = synth.box_vertices(2, 2, 2, seed=7)
    geo = oracle.box_geometry(v, lx)
    sh = geo["jac"].shape
    h1 = synth.uniform(sh, seed=8, lo=0.5, hi=2.0)
    h2 = synth.uniform(sh, seed=9, lo=0.1, hi=3.0)
    dx, dxt = oracle.d_buffers(lx)
    G = [geo[k] for k in ("g11", "g22", "g33", "g12", "g13", "g23")]
    w = oracle.ax_helm_h2(np.ones(sh), dx, dxt, h1, *G, lx, h2, geo["B"])
    ref = h2 * geo["B"]
    np.testing.assert_allclose(w, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    P = oracle.Problem(v, lx, h1=h1, f=oracle.poisson_rhs_f, h2=h2)
    ng = int(P.glob.max()) + 1
    A = np.zeros((ng, ng))
    for j in range(ng):
        ej = np.zeros(ng)
        ej[j] = 1.0
        A[P.glob.ravel(), j] = P.apply(ej[P.glob]).ravel()
    gmask = np.zeros(ng)
    gmask[P.glob.ravel()] = P.mask.ravel()
    idx = np.flatnonzero(gmask)
    Ai = A[np.ix_(idx, idx)]
    assert np.abs(Ai - Ai.T).max() <= 1e-13 * np.abs(Ai).max()
    gdiag = np.zeros(ng)
    gdiag[P.glob.ravel()] = P.diag.ravel()
    np.testing.assert_allclose(gdiag[idx], np.diag(Ai), rtol=1e-12)
    bg = np.zeros(ng)
    bg[P.glob.ravel()] = P.b.ravel()
    xs = np.zeros(ng)
    xs[idx] = np.linalg.solve(Ai, bg[idx])
    x, it, _ = oracle.pcg(P, P.b, tol=1e-12)
    np.testing.assert_allclose(x, xs[P.glob], rtol=0, atol=1e-9 * np.abs(xs).max())
