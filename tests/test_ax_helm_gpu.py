"""GPU parity of the element operator (Listing 2) against the fp64 oracle,
through the C ABI.

Tolerances (relative L2 over the whole output, written per mode):
  * fp64 (both the double-float and the fp64-unit kernel): 1e-12;
  * fp32 storage + fp32 arithmetic: 1e-6;
  * bf16 storage of u, h1, G with fp32 D and arithmetic: 2e-2.
Sizes span several blocks and ragged tails (E = 1, 7, 64, 567); the full
benchmark size (E = 32768, lx = 8) is checked on sampled elements that the
oracle evaluates one by one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2506_20994_gb300 as ax  # noqa: E402
from paper_2506_20994_gb300 import synth  # noqa: E402

from _cases import GKEYS, operator_case, rel_l2  # noqa: E402

TOL = {"f64": 1e-12, "f32": 1e-6, "bf16": 2e-2}
DIMS = [(1, 1, 1), (7, 1, 1), (4, 4, 4), (9, 9, 7)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ax.build()


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _run_f64(case, variant, epb=0):
    lx = case["lx"]
    args = [_dev(case[k]) for k in ("u", "dx", "dxt", "h1") + GKEYS]
    w = torch.full_like(args[0], float("nan"))
    ax.ax_helm(w, *args, lx, variant=variant, elems_per_block=epb)
    torch.cuda.synchronize()
    return w.cpu().numpy()


@pytest.mark.parametrize("lx", range(2, 13))
@pytest.mark.parametrize("dims", DIMS, ids=lambda d: "E%d" % (d[0] * d[1] * d[2]))
def test_f64_df_parity(lx, dims):
    case = operator_case(dims, lx, seed=lx)
    w = _run_f64(case, ax.AX_VARIANT_F64_DF)
    assert rel_l2(w, case["w"]) <= TOL["f64"]
    assert np.abs(w - case["w"]).max() <= 1e-11 * np.abs(case["w"]).max()


@pytest.mark.parametrize("lx", list(range(2, 17)))
def test_f64_native_parity(lx):
    case = operator_case((3, 2, 2) if lx <= 12 else (2, 1, 1), lx, seed=100 + lx)
    w = _run_f64(case, ax.AX_VARIANT_F64_NATIVE)
    assert rel_l2(w, case["w"]) <= TOL["f64"]


@pytest.mark.parametrize("lx", [13, 14, 15, 16])
@pytest.mark.parametrize("dims", [(7, 1, 1), (3, 2, 2)], ids=["E7", "E12"])
def test_f64_df_parity_high_order(lx, dims):
    """The double-float k-loop kernel at lx 13-16 (one element, lx^2 threads,
    per block; ragged against nothing but the element count)."""
    case = operator_case(dims, lx, seed=50 + lx)
    w = _run_f64(case, ax.AX_VARIANT_F64_DF)
    assert rel_l2(w, case["w"]) <= TOL["f64"]


@pytest.mark.parametrize("lx", [13, 16])
def test_auto_variant_high_order(lx):
    case = operator_case((2, 1, 1), lx, seed=7)
    w = _run_f64(case, ax.AX_VARIANT_AUTO)
    assert rel_l2(w, case["w"]) <= TOL["f64"]


@pytest.mark.parametrize("epb", [1, 2, 3, 4])
def test_f64_df_elements_per_block(epb):
    case = operator_case((5, 3, 1), 8, seed=31)
    w = _run_f64(case, ax.AX_VARIANT_F64_DF, epb=epb)
    assert rel_l2(w, case["w"]) <= TOL["f64"]


def test_f64_df_adversarial_inputs():
    """Constant fields (w ~ 0 by cancellation), wide magnitude range, zeros."""
    lx = 8
    case = operator_case((3, 3, 3), lx, seed=41)
    # constant u: the oracle gives ~1e-16 noise; the kernel must too
    const = dict(case)
    const["u"] = np.full_like(case["u"], 2.5)
    w = _run_f64(const, ax.AX_VARIANT_F64_DF)
    ref_scale = np.abs(case["w"]).max() * 2.5
    assert np.abs(w).max() <= 1e-13 * ref_scale
    # per-element magnitudes spread over 1e-6 .. 1e6, some zero elements
    wide = dict(case)
    scale = 10.0 ** synth.uniform((case["u"].shape[0], 1, 1, 1), seed=42, lo=-6, hi=6)
    wide["u"] = case["u"] * scale
    wide["u"][::5] = 0.0
    ref = oracle.ax_helm(wide["u"], case["dx"], case["dxt"], case["h1"],
                         *[case[k] for k in GKEYS], lx)
    w = _run_f64(wide, ax.AX_VARIANT_F64_DF)
    per_el = np.linalg.norm((w - ref).reshape(len(ref), -1), axis=1)
    per_ref = np.linalg.norm(ref.reshape(len(ref), -1), axis=1)
    nz = per_ref > 0
    assert np.all(per_el[nz] <= 1e-12 * per_ref[nz])
    assert np.all(w[::5] == 0.0)


def test_f64_deterministic():
    case = operator_case((4, 4, 2), 6, seed=3)
    a = _run_f64(case, ax.AX_VARIANT_F64_DF)
    b = _run_f64(case, ax.AX_VARIANT_F64_DF)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("lx", [2, 4, 5, 6, 8, 10, 12, 16])
def test_f32_parity(lx):
    case = operator_case((4, 3, 2) if lx <= 12 else (2, 1, 1), lx, seed=200 + lx)
    f = torch.float32
    args = [_dev(case[k], f) for k in ("u", "dx", "dxt", "h1") + GKEYS]
    w = torch.empty_like(args[0])
    ax.ax_helm_f32(w, *args, lx)
    torch.cuda.synchronize()
    assert rel_l2(w.cpu().numpy(), case["w"]) <= TOL["f32"]


@pytest.mark.parametrize("lx", [2, 4, 5, 6, 8, 10, 12])
def test_bf16_parity(lx):
    case = operator_case((4, 3, 2), lx, seed=300 + lx)
    b = torch.bfloat16
    u = _dev(case["u"], b)
    fields = [_dev(case[k], b) for k in ("h1",) + GKEYS]
    dx, dxt = _dev(case["dx"], torch.float32), _dev(case["dxt"], torch.float32)
    w = torch.empty(u.shape, dtype=torch.float32, device="cuda")
    ax.ax_helm_bf16(w, u, dx, dxt, *fields, lx)
    torch.cuda.synchronize()
    assert rel_l2(w.cpu().numpy(), case["w"]) <= TOL["bf16"]


def _run_lowp(case, mode, off=0, dxm=None):
    """ax_helm_f32 / ax_helm_bf16 on the case; off > 0 shifts every array by
    `off` values inside a larger buffer (breaks 16-byte alignment)."""
    lx = case["lx"]
    st = torch.float32 if mode == "f32" else torch.bfloat16

    def put(a, dt):
        flat = np.ascontiguousarray(a).reshape(-1)
        buf = torch.zeros(flat.size + off, dtype=dt, device="cuda")
        buf[off:] = torch.as_tensor(flat).to(dtype=dt, device="cuda")
        return buf[off:].view(np.shape(a))

    u = put(case["u"], st)
    fields = [put(case[k], st) for k in ("h1",) + GKEYS]
    dx = put(case["dx"] if dxm is None else dxm[0], torch.float32)
    dxt = put(case["dxt"] if dxm is None else dxm[1], torch.float32)
    w = put(np.full(np.shape(case["u"]), np.nan), torch.float32)
    fn = ax.ax_helm_f32 if mode == "f32" else ax.ax_helm_bf16
    fn(w, u, dx, dxt, *fields, lx)
    torch.cuda.synchronize()
    return w.cpu().numpy()


@pytest.mark.parametrize("mode", ["f32", "bf16"])
@pytest.mark.parametrize("lx", [4, 8, 10, 12])
def test_lowp_general_matrices(mode, lx):
    """Random dx and an unrelated random dxt (not centro-antisymmetric): the
    even-odd fp32 kernel must take its general rows."""
    case = operator_case((3, 2, 2), lx, seed=400 + lx)
    g = synth.rng(401 + lx)
    dx = g.uniform(-1.0, 1.0, (lx, lx))
    dxt = g.uniform(-1.0, 1.0, (lx, lx))
    G = [case[k] for k in GKEYS]
    ref = oracle.ax_helm(case["u"], dx.reshape(-1), dxt.reshape(-1), case["h1"], *G, lx)
    w = _run_lowp(case, mode, dxm=(dx, dxt))
    assert rel_l2(w, ref) <= TOL[mode]


@pytest.mark.parametrize("lx", [6, 8, 10, 12])
@pytest.mark.parametrize("nel", [1, 3, 5, 611, 1237])
@pytest.mark.parametrize("general", [False, True])
def test_bf16_matches_f32_on_bf16_values(lx, nel, general):
    """bf16 storage only changes what is read: on values that bf16 holds
    exactly, ax_helm_bf16 and ax_helm_f32 do the same fp32 operations in the
    same order (even-odd chains, pointwise h1 G, w = (r + s) + t), whatever
    the layout of threads over the element (one warp per element at lx = 8
    for bf16, mirror octants for fp32), so w agrees bit for bit; element
    counts below, at and above one CTA's share, with ragged tails."""
    g = synth.rng(700 + lx + nel)
    shape = (nel, lx, lx, lx)
    b = torch.bfloat16
    q = lambda a: torch.as_tensor(a).to(device="cuda", dtype=b)
    u = q(g.uniform(-1.0, 1.0, shape))
    fields = [q(g.uniform(0.5, 2.0, shape))] + [q(g.uniform(-1.0, 1.0, shape)) for _ in GKEYS]
    if general:
        dx, dxt = g.uniform(-1.0, 1.0, (lx, lx)), g.uniform(-1.0, 1.0, (lx, lx))
    else:
        dx, dxt = ax.dmat(lx)
    dx, dxt = _dev(dx, torch.float32), _dev(dxt, torch.float32)
    wb = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    wf = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    ax.ax_helm_bf16(wb, u, dx, dxt, *fields, lx)
    ax.ax_helm_f32(wf, u.float(), dx, dxt, *[f.float() for f in fields], lx)
    torch.cuda.synchronize()
    a, c = wb.cpu().numpy(), wf.cpu().numpy()
    assert np.isfinite(a).all()
    np.testing.assert_array_equal(a.view(np.uint32), c.view(np.uint32))


@pytest.mark.parametrize("mode", ["f32", "bf16"])
@pytest.mark.parametrize("lx", [6, 8])
def test_lowp_unaligned_arrays(mode, lx):
    """Arrays that start 4 (fp32) or 2 (bf16) bytes past a 16-byte boundary
    cannot be bulk-copied; the entry point must still return the operator."""
    case = operator_case((3, 3, 2), lx, seed=420 + lx)
    w0 = _run_lowp(case, mode)
    w1 = _run_lowp(case, mode, off=1)
    assert rel_l2(w0, case["w"]) <= TOL[mode]
    assert rel_l2(w1, case["w"]) <= TOL[mode]


@pytest.mark.parametrize("mode", ["f32", "bf16"])
def test_lowp_full_size_sampled(mode):
    """E = 32768 (32^3), lx = 8 in the benchmark's launch configuration;
    the oracle evaluates 64 sampled elements, the first and last included."""
    lx, n = 8, 32
    v = synth.box_vertices(n, seed=0)
    g = ax.box_geometry(v, lx)
    shape = g["g11"].shape
    u = synth.uniform(shape, seed=1)
    h1 = synth.uniform(shape, seed=2, lo=0.5, hi=2.0)
    dx, dxt = ax.dmat(lx)
    st = torch.float32 if mode == "f32" else torch.bfloat16
    t = lambda a: torch.as_tensor(a).to(device="cuda", dtype=st)
    w = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    fn = ax.ax_helm_f32 if mode == "f32" else ax.ax_helm_bf16
    fn(w, t(u), _dev(dx, torch.float32), _dev(dxt, torch.float32), t(h1),
       *[t(g[k]) for k in GKEYS], lx)
    torch.cuda.synchronize()
    w = w.cpu().numpy()
    pick = np.unique(np.concatenate([[0, shape[0] - 1], synth.rng(19).integers(0, shape[0], 62)]))
    go = oracle.box_geometry(v, lx, elements=pick)
    dxo, dxto = oracle.d_buffers(lx)
    ref = oracle.ax_helm(u[pick], dxo, dxto, h1[pick], *[go[k] for k in GKEYS], lx)
    assert rel_l2(w[pick], ref) <= TOL[mode]


def test_full_size_sampled_parity():
    """E = 32768 (32^3), lx = 8, fp64, in the benchmark's launch
    configuration; the oracle evaluates 96 sampled elements."""
    lx, n = 8, 32
    v = synth.box_vertices(n, seed=0)
    g = ax.box_geometry(v, lx)
    shape = g["g11"].shape
    u = synth.uniform(shape, seed=1)
    h1 = np.ones(shape)
    dx, dxt = ax.dmat(lx)
    args = [_dev(a) for a in (u, dx, dxt, h1)] + [_dev(g[k]) for k in GKEYS]
    w = torch.empty_like(args[0])
    ax.ax_helm(w, *args, lx)
    torch.cuda.synchronize()
    w = w.cpu().numpy()
    pick = np.unique(np.concatenate([[0, shape[0] - 1], synth.rng(9).integers(0, shape[0], 94)]))
    go = oracle.box_geometry(v, lx, elements=pick)
    dxo, dxto = oracle.d_buffers(lx)
    ref = oracle.ax_helm(u[pick], dxo, dxto, h1[pick], *[go[k] for k in GKEYS], lx)
    assert rel_l2(w[pick], ref) <= TOL["f64"]


def test_zero_elements_is_noop():
    w = torch.full((8,), 7.0, dtype=torch.float64, device="cuda")
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    ax.ax_helm(e, e, d, d, e, e, e, e, e, e, e, 2)
    torch.cuda.synchronize()
    assert torch.all(w == 7.0)


def test_bad_elements_per_block_rejected():
    case = operator_case((1, 1, 1), 8, seed=1)
    with pytest.raises(ax.AxError):
        _run_f64(case, ax.AX_VARIANT_F64_DF, epb=5)


@pytest.mark.parametrize("lx", [4, 6, 8, 10, 12])
@pytest.mark.parametrize("dims", DIMS, ids=lambda d: "E%d" % (d[0] * d[1] * d[2]))
def test_f64_even_odd_parity(lx, dims):
    """The even-odd split of D (even lx) against the oracle."""
    case = operator_case(dims, lx, seed=50 + lx)
    w = _run_f64(case, ax.AX_VARIANT_F64_DF_EO)
    assert rel_l2(w, case["w"]) <= TOL["f64"]
    assert np.abs(w - case["w"]).max() <= 1e-11 * np.abs(case["w"]).max()


@pytest.mark.parametrize("lx", [6, 8, 10, 12])
@pytest.mark.parametrize("form", ["persistent", "per_block", "unaligned"])
def test_f64_even_odd_forms(lx, form):
    """Both forms of the even-odd variant on fp64 arrays: the persistent one
    (bulk-copied geometry; elements_per_block = 0, aligned arrays), the
    per-block one (an explicit elements-per-block count), and the fallback
    when the geometry arrays start 8 bytes past a 16-byte boundary."""
    case = operator_case((5, 3, 2), lx, seed=60 + lx)
    off = 1 if form == "unaligned" else 0

    def put(a):
        flat = np.ascontiguousarray(a).reshape(-1)
        buf = torch.zeros(flat.size + off, dtype=torch.float64, device="cuda")
        buf[off:] = torch.as_tensor(flat, device="cuda")
        return buf[off:].view(np.shape(a))

    args = [put(case[k]) for k in ("u", "dx", "dxt", "h1") + GKEYS]
    w = torch.full_like(args[0], float("nan"))
    ax.ax_helm(w, *args, lx, variant=ax.AX_VARIANT_F64_DF_EO,
               elems_per_block=(1 if form == "per_block" else 0))
    torch.cuda.synchronize()
    w = w.cpu().numpy()
    assert rel_l2(w, case["w"]) <= TOL["f64"]
    assert np.abs(w - case["w"]).max() <= 1e-11 * np.abs(case["w"]).max()


def test_f64_even_odd_rejects_odd_lx():
    case = operator_case((1, 1, 1), 5, seed=1)
    with pytest.raises(ax.AxError):
        _run_f64(case, ax.AX_VARIANT_F64_DF_EO)


def test_f64_even_odd_adversarial():
    lx = 8
    case = operator_case((3, 3, 3), lx, seed=61)
    const = dict(case)
    const["u"] = np.full_like(case["u"], -1.5)
    w = _run_f64(const, ax.AX_VARIANT_F64_DF_EO)
    assert np.abs(w).max() <= 1e-13 * np.abs(case["w"]).max() * 1.5
    wide = dict(case)
    scale = 10.0 ** synth.uniform((case["u"].shape[0], 1, 1, 1), seed=62, lo=-6, hi=6)
    wide["u"] = case["u"] * scale
    wide["u"][::4] = 0.0
    ref = oracle.ax_helm(wide["u"], case["dx"], case["dxt"], case["h1"],
                         *[case[k] for k in GKEYS], lx)
    w = _run_f64(wide, ax.AX_VARIANT_F64_DF_EO)
    per_el = np.linalg.norm((w - ref).reshape(len(ref), -1), axis=1)
    per_ref = np.linalg.norm(ref.reshape(len(ref), -1), axis=1)
    nz = per_ref > 0
    assert np.all(per_el[nz] <= 1e-12 * per_ref[nz])
    assert np.all(w[::4] == 0.0)


@pytest.mark.parametrize("chunk", [0, 1, 100, 567, 100000])
def test_host_buffers_streamed_in_chunks(chunk):
    """ax_helm_host on host tensors (pinned and pageable), chunks with a
    ragged tail (one element per chunk cycles both device buffer sets 567
    times; a chunk above the element count is clamped), against the oracle
    and bit for bit against ax_helm on the device (the same kernel runs on
    every chunk)."""
    lx = 8
    case = operator_case((9, 9, 7), lx, seed=90)
    keys = ("u", "dx", "dxt", "h1") + GKEYS
    pinned = {k: torch.as_tensor(np.ascontiguousarray(case[k])).pin_memory() for k in keys}
    w = torch.full(case["u"].shape, float("nan"), dtype=torch.float64).pin_memory()
    ax.ax_helm_host(w, *[pinned[k] for k in keys], lx, chunk=chunk)
    assert rel_l2(w.numpy(), case["w"]) <= TOL["f64"]
    wd = torch.empty(case["u"].shape, dtype=torch.float64, device="cuda")
    ax.ax_helm(wd, *[pinned[k].cuda() for k in keys], lx)
    assert torch.equal(wd.cpu(), w)
    pageable = {k: torch.as_tensor(np.ascontiguousarray(case[k])) for k in keys}
    w2 = torch.empty(case["u"].shape, dtype=torch.float64)
    ax.ax_helm_host(w2, *[pageable[k] for k in keys], lx, chunk=chunk)
    assert torch.equal(w2, w)
