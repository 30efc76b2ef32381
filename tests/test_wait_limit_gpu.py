"""The bounded waits of the persistent fp64 kernel, on the GPU, without a
fault: the operator handle is told not to issue the geometry copy of one
element (ax_op_inject_copy_loss), so the wait for it runs out after about
2 s.  The launch must then end by itself, the handle's error word must read
1, the elements that CTA had left must be NaN, every other element must
still match the oracle, and the handle must work normally once the testing
aid is switched off (the context stays usable)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_20994_gb300 as ax  # noqa: E402
from paper_2506_20994_gb300 import _lib  # noqa: E402

from _cases import GKEYS, operator_case, rel_l2  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ax.build()


def test_lost_copy_ends_launch_with_error_and_nan():
    lx = 8
    case = operator_case((4, 4, 4), lx, seed=77)  # 64 elements: one per CTA
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    op = ax.Operator(lx, t(case["dx"]), t(case["dxt"]), t(case["h1"]),
                     *[t(case[k]) for k in GKEYS])
    assert op.info()["prepared"]
    u = t(case["u"])
    w = torch.zeros_like(u)
    lost = 5
    assert _lib.lib().ax_op_inject_copy_loss(op._h, lost) == _lib.AX_OK
    t0 = time.perf_counter()
    op.apply(w, u)
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    assert elapsed < 60.0
    assert op.error() == 1
    got = w.cpu().numpy()
    assert np.all(np.isnan(got[lost]))
    others = np.ones(got.shape[0], dtype=bool)
    others[lost] = False
    assert np.all(np.isfinite(got[others]))
    assert rel_l2(got[others], case["w"][others]) <= 1e-12
    # switched off: the same handle applies correctly again
    assert _lib.lib().ax_op_inject_copy_loss(op._h, -1) == _lib.AX_OK
    w2 = torch.full_like(u, float("nan"))
    op.apply(w2, u)
    torch.cuda.synchronize()
    assert rel_l2(w2.cpu().numpy(), case["w"]) <= 1e-12


def test_inject_rejects_out_of_range():
    lx = 8
    case = operator_case((2, 1, 1), lx, seed=78)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    op = ax.Operator(lx, t(case["dx"]), t(case["dxt"]), t(case["h1"]),
                     *[t(case[k]) for k in GKEYS])
    assert _lib.lib().ax_op_inject_copy_loss(op._h, 2) == _lib.AX_EINVAL
    assert _lib.lib().ax_op_inject_copy_loss(op._h, -2) == _lib.AX_EINVAL
