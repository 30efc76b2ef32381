"""GPU checks of the partitioned solve's pieces through the C ABI, and the
partitioned Jacobi-PCG with 2 and 3 partitions on one GPU (ranks as threads
exchanging through host memory; no kernel waits on another) against the
single-domain solver."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2506_20994_gb300 as ax  # noqa: E402
from paper_2506_20994_gb300 import _lib, dist as adist, synth  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ax.build()


def _s():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("n", [0, 1, 1000, 777_777])
def test_weighted_dot_gather_scatter(n):
    g = synth.rng(n + 1)
    a, b, w = (g.normal(size=n) for _ in range(3))
    t = lambda x: torch.as_tensor(x, device="cuda")
    work = torch.empty(_lib.AX_DOT_WORK + 1, dtype=torch.float64, device="cuda")
    ta, tb, tw = t(a), t(b), t(w)
    rc = _lib.lib().ax_dot_weighted(ta.data_ptr(), tb.data_ptr(), tw.data_ptr(), n,
                                    work.data_ptr(), work[_lib.AX_DOT_WORK:].data_ptr(), _s())
    assert rc == 0
    got = float(work[_lib.AX_DOT_WORK].item())
    ref = float(np.sum(w * a * b))
    assert abs(got - ref) <= 1e-13 * max(1.0, float(np.sum(np.abs(w * a * b))))
    if n == 0:
        return
    idx = g.permutation(n)[: max(1, n // 3)].astype(np.int64)
    out = torch.empty(idx.size, dtype=torch.float64, device="cuda")
    assert _lib.lib().ax_gather(out.data_ptr(), ta.data_ptr(), t(idx).data_ptr(), idx.size,
                                _s()) == 0
    assert np.array_equal(out.cpu().numpy(), a[idx])
    vals = g.normal(size=idx.size)
    pos = g.permutation(idx.size).astype(np.int64)
    v = ta.clone()
    assert _lib.lib().ax_scatter_add(v.data_ptr(), t(vals).data_ptr(), t(idx).data_ptr(),
                                     t(pos).data_ptr(), idx.size, _s()) == 0
    ref_v = a.copy()
    ref_v[idx] += vals[pos]
    assert np.array_equal(v.cpu().numpy(), ref_v)


def test_diag_and_set_diag():
    lx = 5
    v = synth.box_vertices(3, 2, 2, seed=8)
    P = ax.Poisson(v, lx)
    O = oracle.Problem(v, lx)
    d = P.diag()
    np.testing.assert_allclose(d.cpu().numpy(), O.diag, rtol=1e-13, atol=0)
    minv0 = P.jacobi().clone()
    P.set_diag(d)
    assert torch.equal(P.jacobi(), minv0)
    P.set_diag(2.0 * d)
    assert torch.equal(P.jacobi(), 0.5 * minv0)


@pytest.mark.parametrize("world,dims,lx", [(2, (4, 3, 4), 6), (3, (3, 3, 6), 8)])
def test_partitioned_pcg_on_one_gpu(world, dims, lx):
    nx, ny, nz = dims
    v = synth.box_vertices(nx, ny, nz, seed=5)
    xyz = ax.box_geometry(v, lx, want_xyz=True)["xyz"]
    h1 = ax.fourier_coefficient(2)(xyz[..., 0], xyz[..., 1], xyz[..., 2])
    whole = ax.Poisson(v, lx, h1=h1)
    b = whole.rhs(oracle.poisson_rhs_f)
    x_ref, it_ref, _, rc = whole.cg(b, tol=1e-8)
    assert rc == 0
    comms = adist.ThreadComm.group(world)
    out, errors = [None] * world, []

    def rank(r):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                plan = adist.SlabPlan(nx, ny, nz, lx, world, r)
                ops = adist.LibSlabOps(plan, v, h1=h1)
                adist.setup(ops, plan, comms[r])
                br = ops.rhs(oracle.poisson_rhs_f)
                adist.halo_sum(ops, plan, comms[r], br)
                x, it, rel = adist.pcg(ops, plan, comms[r], br, tol=1e-8)
                s.synchronize()
                out[r] = (x.cpu().numpy(), it, rel, br.cpu().numpy())
        except Exception as exc:  # surfaced below
            errors.append(exc)
            comms[r].s.barrier.abort()

    th = [threading.Thread(target=rank, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert not errors, errors
    n3 = lx ** 3
    x = np.concatenate([o[0].reshape(-1, n3) for o in out])
    bb = np.concatenate([o[3].reshape(-1, n3) for o in out])
    bref = b.cpu().numpy().reshape(-1, n3)
    np.testing.assert_allclose(bb, bref, rtol=0, atol=1e-13 * np.abs(bref).max())
    its = {o[1] for o in out}
    assert len(its) == 1 and abs(its.pop() - it_ref) <= 1
    xr = x_ref.cpu().numpy().reshape(-1, n3)
    assert np.linalg.norm(x - xr) <= 1e-9 * np.linalg.norm(xr)
