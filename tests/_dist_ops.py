"""Oracle-backed per-rank vector work for the partitioned-solve tests: the
same interface as ``dist.LibSlabOps`` (which runs on the GPU), computed by
the oracle on torch CPU tensors so that gloo ranks can exchange them."""
import numpy as np
import torch

import oracle


class OracleSlabOps:
    def __init__(self, plan, vertices, h1=None):
        lx = plan.lx
        self.plan, self.lx = plan, lx
        nx, ny, _ = plan.dims
        v = plan.vertices(vertices)
        g = oracle.box_geometry(v, lx)
        self.G = tuple(g[k] for k in ("g11", "g22", "g33", "g12", "g13", "g23"))
        self.dx, self.dxt = oracle.d_buffers(lx)
        shp = g["jac"].shape
        self.shape = shp
        self.h1 = np.ones(shp) if h1 is None else plan.elements(h1).reshape(shp)
        self.glob = oracle.numbering(nx, ny, plan.nzl, lx)
        assert np.array_equal(self.glob.ravel(), plan.glob)
        # Dirichlet on the faces of the whole box only
        n = lx - 1
        NX, NY = nx * n + 1, ny * n + 1
        NZ = plan.dims[2] * n + 1
        X, Y = self.glob % NX, (self.glob // NX) % NY
        Z = self.glob // (NX * NY) + plan.z0 * n
        on = (X == 0) | (X == NX - 1) | (Y == 0) | (Y == NY - 1) | (Z == 0) | (Z == NZ - 1)
        self.mask = np.where(on, 0.0, 1.0)
        self.B = g["B"]
        self.xyz = g["xyz"]
        self.wgt = None
        self.minv = None

    def _t(self, a):
        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(self.shape))

    def vector(self, a):
        return self._t(a).clone()

    def zeros(self):
        return torch.zeros(self.shape, dtype=torch.float64)

    def clone(self, v):
        return v.clone()

    def set_weights(self, mult):
        self.wgt = 1.0 / mult.numpy()

    def diag(self):
        d = oracle.jacobi_diagonal(self.dx, self.h1, *self.G, self.lx)
        return self._t(oracle.gs_sum(d, self.glob))

    def set_diag(self, d):
        d = d.numpy()
        self.minv = np.where((self.mask > 0) & (d != 0), 1.0 / np.where(d != 0, d, 1.0), 0.0)

    def rhs_partial(self, f):
        x = self.xyz
        fv = f(x[..., 0], x[..., 1], x[..., 2])
        return self._t(self.mask * oracle.gs_sum(self.B * fv, self.glob))

    def apply(self, w, p):
        a = oracle.ax_helm(p.numpy(), self.dx, self.dxt, self.h1, *self.G, self.lx)
        w.copy_(self._t(self.mask * oracle.gs_sum(a.reshape(self.shape), self.glob)))

    def precond(self, z, r):
        z.copy_(self._t(self.minv * r.numpy()))

    def axpby(self, y, a, x, b):
        y.copy_(self._t(a * x.numpy() + b * y.numpy()))

    def dot(self, a, b):
        return float(np.sum(self.wgt * a.numpy() * b.numpy()))

    def gather(self, v, nb):
        return torch.as_tensor(v.numpy().ravel()[self.plan.send_idx[nb]].copy())

    def scatter_add(self, v, nb, vals):
        flat = v.view(-1)
        idx = torch.as_tensor(self.plan.recv_idx[nb])
        pos = torch.as_tensor(self.plan.recv_pos[nb])
        flat[idx] += vals[pos]
