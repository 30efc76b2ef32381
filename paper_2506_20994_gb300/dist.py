"""The Poisson solve split across ranks (one GPU per rank).

The element apply needs nothing from other elements; what couples the ranks
is the gather-scatter sum at nodes that elements of two ranks share (the
direct-stiffness summation Neko runs after Ax, Sec. "Neko and Small Tensor
Kernel") and the global dot products of CG.  This module holds the host
logic of that split:

* ``SlabPlan``: the box's element layers along z are cut into ``world``
  contiguous slabs.  With the element-major layout (x fastest, then y, z) a
  slab is one contiguous element range, so a rank applies the operator to its
  own arrays without any reordering.  Neighbouring slabs share one plane of
  GLL nodes; the plan lists, per neighbour, one representative local copy of
  every plane node (what is sent) and every local copy with its plane
  position (where the received partial sums are added).
* ``halo_sum``: after the rank-local gather-scatter every copy of a plane node
  holds this rank's partial sum; one exchange per neighbour adds the other
  side's.  Both sides compute own + other with IEEE addition, which is
  commutative, so the two copies agree bit for bit.
* ``pcg``: Jacobi-PCG from x0 = 0 in SPMD form, run by the library's driver
  (``ax_cg_solve_part``: the scalar recurrences, stopping at
  ||r|| <= tol ||r0||, dots over unique global nodes with weights
  1/global multiplicity).  This module only hands the driver its callback
  tables: the halo exchange and the scalar all-sum (moving bytes between
  ranks) and, for rank-local work other than the library's own, the ops.

The vector work is done by an ``ops`` object (``LibSlabOps``: the library's
kernels on this rank's GPU, which the driver then calls directly) and the
communication by a ``comm`` object (``TorchComm``: torch.distributed;
``ThreadComm``: ranks as threads of one process, which lets several
partitions share one GPU without any kernel waiting on another).
"""
from __future__ import annotations

import threading

import numpy as np

from . import _lib


# ---------------------------------------------------------------------------
class SlabPlan:
    """Partition of an nx x ny x nz box of lx-order elements into ``world``
    z-slabs; the part of rank ``rank``."""

    def __init__(self, nx: int, ny: int, nz: int, lx: int, world: int, rank: int):
        if not (1 <= world <= nz) or not (0 <= rank < world):
            raise ValueError("need 1 <= world <= nz and 0 <= rank < world")
        from . import box_numbering
        self.dims, self.lx, self.world, self.rank = (nx, ny, nz), lx, world, rank
        self.z0 = rank * nz // world
        self.z1 = (rank + 1) * nz // world
        self.nzl = self.z1 - self.z0
        self.e0, self.e1 = self.z0 * nx * ny, self.z1 * nx * ny
        self.nelv = self.e1 - self.e0
        n = lx - 1
        NX, NY = nx * n + 1, ny * n + 1
        self.plane = NX * NY
        self.glob = np.asarray(box_numbering(nx, ny, self.nzl, lx), dtype=np.int64).ravel()
        # slab node id + offset = node id of the whole box
        self.offset = self.z0 * n * self.plane
        nodes = self.nzl * n * self.plane + self.plane
        ids, first = np.unique(self.glob, return_index=True)   # first local copy per node
        if ids.size != nodes:
            raise RuntimeError("slab numbering does not cover its nodes")
        self.neighbours = []                          # (rank, base id of the shared plane)
        if rank > 0:
            self.neighbours.append((rank - 1, 0))
        if rank < world - 1:
            self.neighbours.append((rank + 1, self.nzl * n * self.plane))
        self.send_idx, self.recv_idx, self.recv_pos = {}, {}, {}
        for nb, base in self.neighbours:
            self.send_idx[nb] = first[base:base + self.plane].copy()
            sel = np.flatnonzero((self.glob >= base) & (self.glob < base + self.plane))
            self.recv_idx[nb] = sel.astype(np.int64)
            self.recv_pos[nb] = (self.glob[sel] - base).astype(np.int64)
        # Dirichlet faces: the box's boundary only (interfaces stay open)
        self.dirichlet = (True, True, True, True, rank == 0, rank == world - 1)
        self.local_mult = np.bincount(self.glob, minlength=nodes)[self.glob].astype(np.float64)

    def vertices(self, v: np.ndarray) -> np.ndarray:
        """This slab's vertices out of the whole box's (nz+1, ny+1, nx+1, 3)."""
        return np.ascontiguousarray(v[self.z0:self.z1 + 1])

    def elements(self, a: np.ndarray) -> np.ndarray:
        """This slab's rows of an element-major array of the whole box."""
        return np.ascontiguousarray(np.asarray(a).reshape(-1, self.lx ** 3)[self.e0:self.e1])


# ---------------------------------------------------------------------------
class TorchComm:
    """Exchange and sums through torch.distributed (gloo on CPU tensors,
    NCCL on CUDA tensors; ``device`` is where the message buffers live)."""

    def __init__(self, device="cpu"):
        import torch.distributed as dist
        self.dist, self.device = dist, device
        self.rank, self.world = dist.get_rank(), dist.get_world_size()

    def allsum(self, x: float) -> float:
        return self.allsum_many([x])[0]

    def allsum_many(self, xs) -> list:
        import torch
        t = torch.tensor(list(xs), dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t)
        return [float(v) for v in t.cpu()]

    def exchange(self, sends: dict) -> dict:
        """sends: {neighbour rank: 1-D float64 tensor}; returns the tensors
        the neighbours sent, of the same lengths."""
        import torch
        reqs, recvs = [], {}
        for nb, t in sends.items():
            buf = torch.empty_like(t)
            recvs[nb] = buf
            reqs.append(self.dist.irecv(buf, src=nb))
        for nb, t in sends.items():
            reqs.append(self.dist.isend(t.contiguous(), dst=nb))
        for r in reqs:
            r.wait()
        return recvs


class ThreadComm:
    """Ranks as threads of one process (host-side barrier and mailboxes).
    ``ThreadComm.group(world)`` returns one endpoint per rank."""

    class _Shared:
        def __init__(self, world):
            self.world = world
            self.barrier = threading.Barrier(world)
            self.box = {}
            self.vals = [0.0] * world

    def __init__(self, shared, rank):
        self.s, self.rank, self.world = shared, rank, shared.world

    @classmethod
    def group(cls, world: int):
        sh = cls._Shared(world)
        return [cls(sh, r) for r in range(world)]

    def allsum(self, x: float) -> float:
        return self.allsum_many([x])[0]

    def allsum_many(self, xs) -> list:
        self.s.vals[self.rank] = [float(x) for x in xs]
        self.s.barrier.wait()
        out = []
        for q in range(len(xs)):
            total = 0.0
            for v in self.s.vals:             # rank order: the same bits everywhere
                total += v[q]
            out.append(total)
        self.s.barrier.wait()
        return out

    def exchange(self, sends: dict) -> dict:
        # messages go through host memory: .cpu() waits for the sender's
        # stream, .to() runs on the receiver's, so no device buffer is shared
        # between the threads' streams
        for nb, t in sends.items():
            self.s.box[(self.rank, nb)] = t.cpu()
        self.s.barrier.wait()
        out = {nb: self.s.box[(nb, self.rank)].to(sends[nb].device) for nb in sends}
        self.s.barrier.wait()
        for nb in sends:
            del self.s.box[(self.rank, nb)]
        return out


# ---------------------------------------------------------------------------
def halo_sum(ops, plan: SlabPlan, comm, v) -> None:
    """Adds the neighbours' partial sums to this rank's copies of the shared
    plane nodes (v is a locally gather-scattered vector)."""
    if not plan.neighbours:
        return
    sends = {nb: ops.gather(v, nb) for nb, _ in plan.neighbours}
    recv = comm.exchange(sends)
    for nb, _ in plan.neighbours:
        ops.scatter_add(v, nb, recv[nb])


def setup(ops, plan: SlabPlan, comm) -> None:
    """Global multiplicity weights and the assembled Jacobi diagonal."""
    m = ops.vector(plan.local_mult)
    halo_sum(ops, plan, comm, m)
    ops.set_weights(m)
    d = ops.diag()
    halo_sum(ops, plan, comm, d)
    ops.set_diag(d)


def pcg(ops, plan: SlabPlan, comm, b, tol: float = 1e-8, maxit: int = 10000):
    """Jacobi-PCG on the partitioned problem by the library's driver
    (ax_cg_solve_part_poisson for ``LibSlabOps``, ax_cg_solve_part with
    ``ops``' methods as callbacks otherwise).  b: this rank's part of the
    assembled, masked right-hand side.  Returns (x, iterations, relres)."""
    import ctypes
    x = ops.zeros()
    vecs = {}            # address -> vector, for the callbacks
    errors = []

    def reg(t):
        vecs[t.data_ptr()] = t
        return t.data_ptr()

    def at(addr):
        t = vecs.get(addr)
        return t if t is not None else ops.wrap(addr)

    def guarded(fn):
        def run(*a):
            try:
                fn(*a)
                return 0
            except Exception as exc:  # reported after the driver returns
                errors.append(exc)
                return 1
        return run

    def allsum(ctx, vals, n):
        out = comm.allsum_many([vals[q] for q in range(n)])
        for q in range(n):
            vals[q] = out[q]

    ctab = _lib.PartComm(None,
                         _lib.HALO_FN(guarded(lambda c, v, st: halo_sum(ops, plan, comm, at(v)))),
                         _lib.ALLSUM_FN(guarded(allsum)))
    it, rel = ctypes.c_int(), ctypes.c_double()
    reg(x)
    reg(b)
    if isinstance(ops, LibSlabOps):
        rc = _lib.lib().ax_cg_solve_part_poisson(
            ops.P._h, ops.wgt.data_ptr(), ctypes.addressof(ctab), x.data_ptr(), b.data_ptr(),
            float(tol), int(maxit), ctypes.addressof(it), ctypes.addressof(rel), ops._s())
    else:
        work = [ops.zeros() for _ in range(4)]
        for t in work:
            reg(t)

        def dot(c, a, bb, out, st):
            out[0] = ops.dot(at(a), at(bb))

        otab = _lib.PartOps(
            None,
            _lib.APPLY_FN(guarded(lambda c, w, p, st: ops.apply(at(w), at(p)))),
            _lib.APPLY_FN(guarded(lambda c, z, r, st: ops.precond(at(z), at(r)))),
            _lib.DOT_FN(guarded(dot)),
            _lib.AXPBY_FN(guarded(lambda c, y, a, xx, bb, st: ops.axpby(at(y), a, at(xx), bb))),
            _lib.APPLY_FN(guarded(lambda c, d, s_, st: at(d).copy_(at(s_)))),
            _lib.ZERO_FN(guarded(lambda c, v, st: at(v).zero_())))
        rc = _lib.lib().ax_cg_solve_part(
            ctypes.addressof(otab), ctypes.addressof(ctab), x.data_ptr(), b.data_ptr(),
            *[t.data_ptr() for t in work], float(tol), int(maxit), ctypes.addressof(it),
            ctypes.addressof(rel), None)
    if errors:
        raise errors[0]
    if rc not in (_lib.AX_OK, _lib.AX_ENOTCONV):
        _lib.check("ax_cg_solve_part", rc)
    return x, it.value, rel.value


# ---------------------------------------------------------------------------
class LibSlabOps:
    """This rank's vector work on its GPU through the library's kernels:
    operator apply + local gather-scatter + mask (ax_poisson_apply), the
    assembled Jacobi diagonal (ax_poisson_diag / ax_poisson_set_diag), the
    preconditioner (ax_precondition), axpby, weighted dots, and the pack /
    unpack of shared-plane values (ax_gather, ax_scatter_add)."""

    def __init__(self, plan: SlabPlan, vertices: np.ndarray, h1=None, device=None):
        import torch
        from . import Poisson
        self.plan = plan
        h = None if h1 is None else plan.elements(h1)
        self.P = Poisson(plan.vertices(vertices), plan.lx, h1=h, device=device,
                         dirichlet=plan.dirichlet)
        self.device = self.P.device
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=self.device)
        self.idx = {nb: (t(plan.send_idx[nb]), t(plan.recv_idx[nb]), t(plan.recv_pos[nb]))
                    for nb, _ in plan.neighbours}
        self.work = torch.empty(_lib.AX_DOT_WORK + 1, dtype=torch.float64, device=self.device)
        self.wgt = None
        self.shape = self.P.shape

    def _s(self):
        from . import _stream
        return _stream()

    def vector(self, a):
        import torch
        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(self.shape),
                               device=self.device).clone()

    def wrap(self, addr):
        """A view of a local vector the library owns (the solver's work)."""
        import torch
        from . import _DeviceArray
        n = int(np.prod(self.shape))
        return torch.as_tensor(_DeviceArray(addr, n, "<f8", self), device=self.device)

    def zeros(self):
        import torch
        return torch.zeros(self.shape, dtype=torch.float64, device=self.device)

    def clone(self, v):
        return v.clone()

    def set_weights(self, mult):
        self.wgt = 1.0 / mult          # set-up only

    def diag(self):
        return self.P.diag()

    def set_diag(self, d):
        self.P.set_diag(d)

    def rhs(self, f):
        return self.P.rhs(f)

    def apply(self, w, p):
        self.P.apply(w, p)

    def precond(self, z, r):
        _lib.check("ax_precondition", _lib.lib().ax_precondition(
            self.P._h, None, z.data_ptr(), r.data_ptr(), self._s()))

    def axpby(self, y, a, x, b):
        _lib.check("ax_axpby", _lib.lib().ax_axpby(y.data_ptr(), float(a), x.data_ptr(),
                                                   float(b), y.numel(), self._s()))

    def dot(self, a, b) -> float:
        out = self.work[_lib.AX_DOT_WORK:]
        _lib.check("ax_dot_weighted", _lib.lib().ax_dot_weighted(
            a.data_ptr(), b.data_ptr(), self.wgt.data_ptr(), a.numel(), self.work.data_ptr(),
            out.data_ptr(), self._s()))
        return float(out.item())

    def gather(self, v, nb):
        import torch
        idx = self.idx[nb][0]
        out = torch.empty(idx.numel(), dtype=torch.float64, device=self.device)
        _lib.check("ax_gather", _lib.lib().ax_gather(out.data_ptr(), v.data_ptr(),
                                                     idx.data_ptr(), idx.numel(), self._s()))
        return out

    def scatter_add(self, v, nb, vals):
        _, idx, pos = self.idx[nb]
        vals = vals.to(self.device)
        _lib.check("ax_scatter_add", _lib.lib().ax_scatter_add(
            v.data_ptr(), vals.data_ptr(), idx.data_ptr(), pos.data_ptr(), idx.numel(),
            self._s()))
