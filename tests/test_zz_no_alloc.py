"""GPU test of the allocation-free Jacobi refresh (ax_jacobi_noalloc).

Callers that may not allocate device memory where they refresh the
preconditioner (graph-recorded work, fixed-budget time loops, host pools)
use this entry point; its scratch is a fixed array inside the library.  The
test calls it through the C ABI twice in a row, with two different
coefficients h1, and checks each result against the array that the
allocating path (ax_poisson_create / ax_poisson_jacobi) computes: same
kernels and summation order, so the bits must agree (the relative 1e-12
tolerance of the other fp64 tests is also asserted).  Each result is also
compared with the oracle's masked inverse of the assembled diagonal
(jacobi_diagonal, then gs_sum), and the device's free memory is checked to be
the same before and after a warmed-up call.  It also checks that a problem
larger than the fixed scratch is rejected.  This file is named to be
collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_20994_gb300 as ax  # noqa: E402
from paper_2506_20994_gb300 import _lib, synth  # noqa: E402

import oracle  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ax.build()


def _call(P, h1, out):
    d = P.d
    return _lib.lib().ax_jacobi_noalloc(
        out.data_ptr(), d["dx"].data_ptr(), h1.data_ptr(),
        *[d[k].data_ptr() for k in ax.Poisson.GKEYS], d["mask"].data_ptr(), P.gs.handle,
        P.lx, P.nelv, torch.cuda.current_stream().cuda_stream)


def test_noalloc_jacobi_matches_allocating_path_twice():
    lx = 8
    v = synth.box_vertices(5, 4, 3, seed=12)
    h1_b = synth.uniform((60, lx, lx, lx), seed=13, lo=0.5, hi=2.0)
    P1 = ax.Poisson(v, lx)                 # h1 = 1
    P2 = ax.Poisson(v, lx, h1=h1_b)        # random coefficient
    out = torch.full((P1.nelv * lx ** 3,), float("nan"), dtype=torch.float64, device="cuda")
    for P in (P1, P2, P1):                 # two calls in a row, then back
        ref = P.jacobi().clone()
        out.fill_(float("nan"))
        rc = _call(P, P.d["h1"], out)
        assert rc == _lib.AX_OK
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
        assert torch.equal(out, ref)
        # the oracle's masked inverse of the assembled diagonal
        c = {k: P.d[k].cpu().numpy() for k in ("dx", "h1", "mask", *ax.Poisson.GKEYS)}
        dg = oracle.gs_sum(oracle.jacobi_diagonal(c["dx"], c["h1"],
                                                  *[c[k] for k in ax.Poisson.GKEYS], lx),
                           P.glob).reshape(-1)
        m = c["mask"].reshape(-1)
        want = np.where(m > 0, 1.0 / np.where(dg != 0, dg, 1.0), 0.0)
        assert np.linalg.norm(a - want) <= 1e-12 * np.linalg.norm(want)


def test_noalloc_jacobi_leaves_free_memory_unchanged():
    lx = 8
    P = ax.Poisson(synth.box_vertices(4, 4, 4, seed=21), lx)
    out = torch.empty(P.nelv * lx ** 3, dtype=torch.float64, device="cuda")
    assert _call(P, P.d["h1"], out) == _lib.AX_OK  # loads the kernels, resolves the scratch
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _call(P, P.d["h1"], out) == _lib.AX_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(out, P.jacobi())


def test_noalloc_rejects_oversize_and_bad_handle():
    lx = 8
    v = synth.box_vertices(2, seed=1)
    P = ax.Poisson(v, lx)
    out = torch.empty(P.nelv * lx ** 3, dtype=torch.float64, device="cuda")
    d = P.d
    big = (1 << 19) // lx ** 3 + 1  # one element past AX_NOALLOC_MAX_POINTS
    args = [out.data_ptr(), d["dx"].data_ptr(), d["h1"].data_ptr(),
            *[d[k].data_ptr() for k in ax.Poisson.GKEYS], d["mask"].data_ptr(), P.gs.handle]
    s = torch.cuda.current_stream().cuda_stream
    assert _lib.lib().ax_jacobi_noalloc(*args, lx, big, s) == _lib.AX_EINVAL
    # a gather-scatter handle of another size is refused
    assert _lib.lib().ax_jacobi_noalloc(*args, lx, P.nelv - 1, s) == _lib.AX_EINVAL
