"""The benchmark's throughput probe (bench_probe.cu, built apart from the
library by bench_extras.py) reports plausible per-SM, per-clock
multiply-add rates: positive and below the issue limit of four 32-lane
schedulers (two multiply-adds per lane for the packed form)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import bench_extras  # noqa: E402


def test_probe_rates_are_plausible():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = bench_extras.probe_rates()
    for k in ("fp64_fma", "fp32_fma", "fp32x2_fma"):
        assert 0.0 < r[k] <= 4 * 32 * 2 * 1.05, (k, r[k])
