"""Maximum sizes: element arrays past 2^31 local points, where any 32-bit
index arithmetic would wrap.  To fit two buffers (input and output) on the
device, one seeded random input serves as u, h1 and all six geometric
factors (inputs may alias one another; only the output must not), which
keeps the operator well defined.  Sampled elements, including the last ones
past 2^31 points, are checked against the oracle element by element.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2506_20994_gb300 as ax  # noqa: E402

from _cases import rel_l2  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ax.build()


def _run(lx, dtype, fn, tol):
    n3 = lx ** 3
    nelv = (1 << 31) // n3 + 3            # past 2^31 points
    bytes_needed = 2 * nelv * n3 * torch.tensor([], dtype=dtype).element_size()
    if torch.cuda.mem_get_info()[0] < 1.2 * bytes_needed:
        pytest.skip("not enough free device memory")
    g = torch.Generator(device="cuda").manual_seed(11)
    x = torch.rand(nelv * n3, generator=g, device="cuda", dtype=dtype).mul_(0.5).add_(0.5)
    w = torch.empty_like(x)
    dx, dxt = (torch.as_tensor(a, device="cuda", dtype=dtype) for a in ax.dmat(lx))
    shape = (nelv, lx, lx, lx)
    xs, ws = x.view(shape), w.view(shape)
    fn(ws, xs, dx, dxt, xs, *([xs] * 6), lx)
    torch.cuda.synchronize()
    dxh, dxth = oracle.d_buffers(lx)
    for e in (0, nelv // 2, nelv - 2, nelv - 1):
        xe = xs[e:e + 1].double().cpu().numpy()
        ref = oracle.ax_helm(xe, dxh, dxth, xe, *([xe] * 6), lx)
        assert rel_l2(ws[e:e + 1].double().cpu().numpy(), ref) <= tol, e
    del x, w
    torch.cuda.empty_cache()


def test_fp32_operator_past_2_31_points():
    """lx = 16 (k-loop kernel), 524,291 elements = 2^31 + 12,288 points."""
    _run(16, torch.float32, ax.ax_helm_f32, 1e-5)


def test_fp64_operator_past_2_31_points():
    """lx = 12 (even-odd double-float kernel), 1,242,757 elements."""
    _run(12, torch.float64, ax.ax_helm, 1e-12)
