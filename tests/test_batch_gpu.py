"""GPU checks of the batched multi-mesh launch and the autotuner.

Uneven meshes of mixed lx in one persistent launch (and its CUDA-graph
replay) must give, for every mesh, exactly the bits of the single-mesh
entry point with the same thread layout (the operator handle for fp64 lx 6,
8, 10; ax_helm / ax_helm_f32 otherwise; fp32 lx 12, which the batch runs in
the k-loop layout and ax_helm_f32 in the even-odd one, within 1e-6 of it),
and match the oracle within the
fp64 (1e-12) or fp32 (1e-6) relative L2 tolerance; at the benchmark's size
(64 meshes, E log-uniform in [64, 8192], lx in {5, 6, 8, 10}) sampled
elements of every mesh are checked against the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2506_20994_gb300 as ax  # noqa: E402
from paper_2506_20994_gb300 import synth  # noqa: E402

from _cases import GKEYS, rel_l2  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ax.build()


def _meshes(dtype, count=10, seed=0):
    """Small uneven batch: element counts log-uniform in [1, 150], lx from
    {5, 6, 8, 10} plus two extra orders; oracle w per mesh."""
    tdt = torch.float64 if dtype == ax.AX_BATCH_F64 else torch.float32
    g = synth.rng(seed)
    out = []
    lxs = [5, 6, 8, 10, 3, 12]
    for q in range(count):
        ne = int(np.exp(g.uniform(0, np.log(150))))
        lx = lxs[q % len(lxs)]
        dims = synth.box_dims(ne)
        v = synth.box_vertices(*dims, seed=seed + q)
        geo = oracle.box_geometry(v, lx)
        u = synth.uniform(geo["jac"].shape, seed=seed + 100 + q)
        h1 = synth.uniform(geo["jac"].shape, seed=seed + 200 + q, lo=0.5, hi=2.0)
        dx, dxt = oracle.d_buffers(lx)
        ref = oracle.ax_helm(u, dx, dxt, h1, *[geo[k] for k in GKEYS], lx)
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=tdt)
        m = {"lx": lx, "u": t(u), "dx": t(dx), "dxt": t(dxt), "h1": t(h1), "ref": ref}
        for k in GKEYS:
            m[k] = t(geo[k])
        m["w"] = torch.full_like(m["u"], float("nan"))
        out.append(m)
    return out


@pytest.mark.parametrize("dtype", [ax.AX_BATCH_F64, ax.AX_BATCH_F32])
@pytest.mark.parametrize("graph", [False, True])
def test_batch_matches_oracle_and_single_launch(dtype, graph):
    meshes = _meshes(dtype, seed=3 if graph else 1)
    B = ax.Batch(meshes, dtype=dtype)
    info = B.info()
    assert info["items"] > 0 and info["blocks"] > 0
    B.launch(graph=graph)
    if graph:  # replay twice more: same bits
        B.launch(graph=True)
    torch.cuda.synchronize()
    assert B.error() == 0
    tol = 1e-12 if dtype == ax.AX_BATCH_F64 else 1e-6
    for m in meshes:
        w = m["w"].double().cpu().numpy()
        assert rel_l2(w, m["ref"]) <= tol, m["lx"]
        # the single-mesh entry point of the same layout (fp64 even-odd orders:
        # the operator handle on prepared geometry): same bits
        w1 = torch.empty_like(m["u"])
        if dtype == ax.AX_BATCH_F64 and m["lx"] in (6, 8, 10):
            op = ax.Operator(m["lx"], m["dx"], m["dxt"], m["h1"], *[m[k] for k in GKEYS])
            op.apply(w1, m["u"])
        elif dtype == ax.AX_BATCH_F64:  # the double-float k-loop layout
            ax.ax_helm(w1, m["u"], m["dx"], m["dxt"], m["h1"], *[m[k] for k in GKEYS], m["lx"],
                       variant=ax.AX_VARIANT_F64_DF)
        else:
            ax.ax_helm_f32(w1, m["u"], m["dx"], m["dxt"], m["h1"], *[m[k] for k in GKEYS],
                           m["lx"])
        torch.cuda.synchronize()
        if dtype == ax.AX_BATCH_F32 and m["lx"] == 12:  # another layout: fp32 rounding
            assert rel_l2(w1.double().cpu().numpy(), w) <= 1e-6
        else:
            assert torch.equal(w1, m["w"])


def test_batch_empty_and_bad_meshes():
    B = ax.Batch([], dtype=ax.AX_BATCH_F64)
    B.launch()
    torch.cuda.synchronize()
    m = _meshes(ax.AX_BATCH_F64, count=1)[0]
    m["lx"] = 13  # outside the batched range
    with pytest.raises(ax.AxError):
        ax.Batch([m], dtype=ax.AX_BATCH_F64)


@pytest.mark.parametrize("dtype", [ax.AX_BATCH_F64, ax.AX_BATCH_F32])
def test_tuner_records_choice_and_parity_holds(dtype):
    lx = 6
    m = _meshes(dtype, count=1, seed=9)[0]
    m["lx"] = lx
    # a larger synthetic mesh so timings mean something
    tdt = m["u"].dtype
    nel = 2048
    f = {k: torch.rand(nel * lx ** 3, device="cuda", dtype=tdt) for k in
         ("w", "u", "h1") + GKEYS}
    dx, dxt = oracle.d_buffers(lx)
    f["dx"] = torch.as_tensor(dx, device="cuda", dtype=tdt)
    f["dxt"] = torch.as_tensor(dxt, device="cuda", dtype=tdt)
    epb, ms = ax.tune(dtype, lx, f, reps=3)
    assert 1 <= epb <= 256 // lx ** 2 and ms > 0
    assert ax.tune_get(dtype, lx) == epb
    try:
        meshes = _meshes(dtype, count=6, seed=11)
        B = ax.Batch(meshes, dtype=dtype)
        B.launch()
        torch.cuda.synchronize()
        tol = 1e-12 if dtype == ax.AX_BATCH_F64 else 1e-6
        for mm in meshes:
            assert rel_l2(mm["w"].double().cpu().numpy(), mm["ref"]) <= tol
    finally:
        ax.tune_set(dtype, lx, 0)


@pytest.mark.parametrize("lx", [5, 8])
def test_variant_tuner_drives_auto(lx):
    """The variant tuner times the admissible fp64 variants, records the
    fastest, and ax_helm's automatic choice then runs exactly that variant
    (same bits); parity holds; the table resets to the built-in choice."""
    from _cases import operator_case
    case = operator_case((6, 5, 4), lx, seed=70 + lx)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    f = {k: t(case[k]) for k in ("u", "dx", "dxt", "h1") + GKEYS}
    f["w"] = torch.empty_like(f["u"])
    try:
        v, ms = ax.tune_variant(lx, f, reps=2)
        assert v in (ax.AX_VARIANT_F64_NATIVE, ax.AX_VARIANT_F64_DF, ax.AX_VARIANT_F64_DF_EO)
        assert ms > 0 and ax.tune_variant_get(lx) == v
        if lx % 2:
            assert v != ax.AX_VARIANT_F64_DF_EO
        args = [f[k] for k in ("u", "dx", "dxt", "h1") + GKEYS]
        w_auto, w_v = torch.empty_like(f["u"]), torch.empty_like(f["u"])
        ax.ax_helm(w_auto, *args, lx)
        ax.ax_helm(w_v, *args, lx, variant=v)
        torch.cuda.synchronize()
        assert torch.equal(w_auto, w_v)
        assert rel_l2(w_auto.cpu().numpy(), case["w"]) <= 1e-12
        with pytest.raises(ax.AxError):
            ax.tune_variant_set(lx, 7)
    finally:
        ax.tune_variant_set(lx, 0)
    assert ax.tune_variant_get(lx) == 0


def test_batch_follows_the_tuned_thread_layout():
    """With the variant table set, the plan switches thread layout per lx:
    lx = 8 on the k-loop body (bitwise equal to ax_helm's double-float
    k-loop variant) and lx = 6 on the even-odd body on prepared geometry
    (bitwise equal to the operator handle)."""
    meshes = [m for m in _meshes(ax.AX_BATCH_F64, count=8, seed=5) if m["lx"] in (6, 8)]
    assert {m["lx"] for m in meshes} == {6, 8}
    try:
        ax.tune_variant_set(8, ax.AX_VARIANT_F64_DF)
        ax.tune_variant_set(6, ax.AX_VARIANT_F64_DF_EO)
        B = ax.Batch(meshes, dtype=ax.AX_BATCH_F64)
        B.launch()
        torch.cuda.synchronize()
        for m in meshes:
            assert rel_l2(m["w"].cpu().numpy(), m["ref"]) <= 1e-12
            w1 = torch.empty_like(m["u"])
            args = [m["u"], m["dx"], m["dxt"], m["h1"]] + [m[k] for k in GKEYS]
            if m["lx"] == 8:
                ax.ax_helm(w1, *args, 8, variant=ax.AX_VARIANT_F64_DF)
            else:
                ax.Operator(6, m["dx"], m["dxt"], m["h1"], *[m[k] for k in GKEYS]).apply(w1, m["u"])
            torch.cuda.synchronize()
            assert torch.equal(w1, m["w"]), m["lx"]
    finally:
        ax.tune_variant_set(8, 0)
        ax.tune_variant_set(6, 0)


@pytest.mark.parametrize("dtype", [ax.AX_BATCH_F64, ax.AX_BATCH_F32])
def test_benchmark_size_batch_sampled(dtype):
    """The benchmark's batch: 64 meshes from synth.batch_meshes (E log-uniform
    in [64, 8192], lx in {5, 6, 8, 10}; ~1e5 elements), one launch through the
    graph.  Inputs are seeded device-random fields (the operator is defined
    for any G; positive G and h1 keep it an SPD-like form); for every mesh
    four elements, its first and last among them, are checked against the
    oracle one by one."""
    tdt = torch.float64 if dtype == ax.AX_BATCH_F64 else torch.float32
    tol = 1e-12 if dtype == ax.AX_BATCH_F64 else 1e-6
    specs = synth.batch_meshes(seed=0)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1234)
    meshes = []
    for nx, ny, nz, lx in specs:
        ne = nx * ny * nz
        f = lambda lo, hi: (lo + (hi - lo) * torch.rand(ne * lx ** 3, device="cuda",
                                                        generator=gen, dtype=torch.float64)).to(tdt)
        dx, dxt = oracle.d_buffers(lx)
        m = {"lx": lx, "u": f(-1.0, 1.0), "h1": f(0.5, 2.0),
             "dx": torch.as_tensor(dx, device="cuda", dtype=tdt),
             "dxt": torch.as_tensor(dxt, device="cuda", dtype=tdt)}
        for k in GKEYS:
            m[k] = f(0.5, 1.0) if k in ("g11", "g22", "g33") else f(-0.1, 0.1)
        m["w"] = torch.full_like(m["u"], float("nan"))
        meshes.append(m)
    B = ax.Batch(meshes, dtype=dtype)
    B.launch(graph=True)
    torch.cuda.synchronize()
    assert B.error() == 0
    g = synth.rng(77)
    for m in meshes:
        lx, n3 = m["lx"], m["lx"] ** 3
        ne = m["u"].numel() // n3
        pick = sorted({0, ne - 1, int(g.integers(0, ne)), int(g.integers(0, ne))})
        sl = lambda t: t.view(ne, lx, lx, lx)[pick].double().cpu().numpy()
        ref = oracle.ax_helm(sl(m["u"]), m["dx"].double().cpu().numpy(),
                             m["dxt"].double().cpu().numpy(), sl(m["h1"]),
                             *[sl(m[k]) for k in GKEYS], lx)
        assert rel_l2(sl(m["w"]), ref) <= tol, (lx, ne)
