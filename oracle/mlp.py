"""Oracle for the learned element preconditioner's network.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain numpy, fp64.

The paper has no learned component; the network follows the project's
reading of the learned-preconditioner workload: a per-element two-layer
perceptron acting on one element's normalised, Jacobi-scaled residual

    x = (D^-1 r)_e / s_e,   s_e = ||(D^-1 r)_e||_2,
    h = tanh(x W1 + b1),    y = h W2 + b2,

trained to predict t = (e_e - (D^-1 r)_e) / s_e (the part of the element
error that Jacobi misses) with the mean-squared loss

    L = sum_b sum_o (y_bo - t_bo)^2 / (B * n_out),

and updated by Adam (Kingma & Ba 2015, Algorithm 1).  Parameters are one
flat vector [W1 (n_in x n_hid, row-major), b1, W2 (n_hid x n_out), b2].
"""
from __future__ import annotations

import numpy as np


def nparams(n_in: int, n_hid: int, n_out: int | None = None) -> int:
    n_out = n_in if n_out is None else n_out
    return n_in * n_hid + n_hid + n_hid * n_out + n_out


def unpack(theta: np.ndarray, n_in: int, n_hid: int, n_out: int | None = None):
    n_out = n_in if n_out is None else n_out
    o = 0
    W1 = theta[o:o + n_in * n_hid].reshape(n_in, n_hid)
    o += n_in * n_hid
    b1 = theta[o:o + n_hid]
    o += n_hid
    W2 = theta[o:o + n_hid * n_out].reshape(n_hid, n_out)
    o += n_hid * n_out
    b2 = theta[o:o + n_out]
    return W1, b1, W2, b2


def forward(theta, X, n_hid):
    """Y = tanh(X W1 + b1) W2 + b2 for a batch X (B, n_in)."""
    X = np.asarray(X, dtype=np.float64)
    W1, b1, W2, b2 = unpack(np.asarray(theta, dtype=np.float64), X.shape[1], n_hid)
    H = np.tanh(X @ W1 + b1)
    return H @ W2 + b2


def loss_and_grad(theta, X, T, n_hid):
    """Mean-squared loss and its gradient by the chain rule (backprop)."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B, n_in = X.shape
    W1, b1, W2, b2 = unpack(np.asarray(theta, dtype=np.float64), n_in, n_hid)
    pre = X @ W1 + b1
    H = np.tanh(pre)
    Y = H @ W2 + b2
    R = Y - T
    n_out = Y.shape[1]
    L = float(np.sum(R * R) / (B * n_out))
    dY = 2.0 * R / (B * n_out)
    gW2 = H.T @ dY
    gb2 = dY.sum(axis=0)
    dH = dY @ W2.T
    dpre = dH * (1.0 - H * H)
    gW1 = X.T @ dpre
    gb1 = dpre.sum(axis=0)
    return L, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2])


def adam_step(theta, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (returns new theta, m, v); step counts from 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def element_features(r, e, minv, lx):
    """(X, T, s) of every element from local residual r, error e and the
    inverse Jacobi diagonal minv (all element-major arrays)."""
    n3 = lx ** 3
    zr = (np.asarray(minv) * np.asarray(r)).reshape(-1, n3)
    s = np.sqrt(np.sum(zr * zr, axis=1))
    safe = np.where(s > 0, s, 1.0)
    X = zr / safe[:, None]
    T = (np.asarray(e).reshape(-1, n3) - zr) / safe[:, None]
    return X, T, s


def precondition(theta, r, minv, mask, mult, glob, lx, n_hid, gs_sum):
    """z = D^-1 r + gs(mask * s_e * MLP(x_e) / multiplicity)."""
    n3 = lx ** 3
    zr = np.asarray(minv) * np.asarray(r)
    X, _, s = element_features(r, np.zeros_like(r), minv, lx)
    Y = forward(theta, X, n_hid) * s[:, None]
    corr = (Y.reshape(np.shape(r)) * mask) / mult
    return zr + gs_sum(corr, glob)


# ---------------------------------------------------------------------------
# Symmetric linear form: one shared basis W (n_in x n_hid) per element,
#   z = D^-1 r + gs(mask * S * W W^T * S * r_e),   S = sqrt(D^-1),
# a sum over elements of positive semi-definite terms, so z = B r with B
# symmetric positive definite (usable in plain CG).  Parameters use the same
# flat layout as above with W1 = W, b1 = 0, W2 = W^T, b2 = 0.
# ---------------------------------------------------------------------------
def tie(theta, n_in, n_hid):
    """Parameters with W2 = W1^T and zero biases (the symmetric form)."""
    t = np.array(theta, dtype=np.float64)
    W1, b1, W2, b2 = unpack(t, n_in, n_hid)
    W2[...] = W1.T
    b1[...] = 0.0
    b2[...] = 0.0
    return t


def forward_sym(theta, X, n_hid):
    """Y = (X W) W^T."""
    X = np.asarray(X, dtype=np.float64)
    W1 = unpack(np.asarray(theta, dtype=np.float64), X.shape[1], n_hid)[0]
    return (X @ W1) @ W1.T


def mse_loss_grad_sym(theta, X, T, n_hid):
    """Mean-squared loss of Y = (X W) W^T against T and its gradient with
    respect to the tied W (flat layout; zero in b1, W2, b2)."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B, n_in = X.shape
    W = unpack(np.asarray(theta, dtype=np.float64), n_in, n_hid)[0]
    H = X @ W
    R = H @ W.T - T
    L = float(np.sum(R * R) / (B * n_in))
    dY = 2.0 * R / (B * n_in)
    gW = X.T @ (dY @ W) + dY.T @ H      # W appears in both layers
    grad = np.zeros(nparams(n_in, n_hid))
    grad[:n_in * n_hid] = gW.ravel()
    return L, grad


def precondition_sym(theta, r, minv, mask, glob, lx, n_hid, gs_sum):
    """z = D^-1 r + gs(mask * S * (W W^T) (S r)_e), S = sqrt(D^-1)."""
    n3 = lx ** 3
    S = np.sqrt(np.asarray(minv))
    X = (S * np.asarray(r)).reshape(-1, n3)
    Y = forward_sym(theta, X, n_hid).reshape(np.shape(r))
    return np.asarray(minv) * np.asarray(r) + gs_sum(mask * S * Y, glob)


def energy_loss_grad_sym(theta, pairs, apply_A, dot, minv, mask, glob, lx, n_hid, gs_sum):
    """Mean relative energy error of the symmetric form over (r, e) pairs,
    L = mean_k ||e_k - z(r_k)||_A^2 / ||e_k||_A^2, and its gradient with
    respect to W (returned in the flat layout, zero in b1, W2, b2)."""
    n3 = lx ** 3
    n_in = n3
    W = unpack(np.asarray(theta, dtype=np.float64), n_in, n_hid)[0]
    S = np.sqrt(np.asarray(minv))
    L = 0.0
    gW = np.zeros_like(W)
    for r, e in pairs:
        z = precondition_sym(theta, r, minv, mask, glob, lx, n_hid, gs_sum)
        d = e - z
        q = apply_A(d)                 # assembled, masked A d
        eA = dot(e, apply_A(e))
        L += dot(d, q) / eA
        X = (S * r).reshape(-1, n3)    # rows: elements
        G = (-2.0 / eA) * (mask * S * q).reshape(-1, n3)   # dL/dY
        H = X @ W
        gW += X.T @ (G @ W) + G.T @ H
    k = len(pairs)
    grad = np.zeros(nparams(n_in, n_hid))
    grad[:n_in * n_hid] = (gW / k).ravel()
    return L / k, grad
