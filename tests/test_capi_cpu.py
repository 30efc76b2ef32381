"""CPU checks of the C-ABI library: it loads, exports every symbol the header
declares, its host set-up agrees with the oracle, the integer fp64 <-> fp32
pair conversions used by the fp64 kernels are correct bit for bit, and the
argument checks reject bad calls before touching the GPU."""
import glob
import os
import re

import numpy as np
import pytest

import oracle
import paper_2506_20994_gb300 as ax
from paper_2506_20994_gb300 import _lib, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    ax.build()


def _header_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"^[A-Za-z_][\w \*]*?\b(ax_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


def test_every_header_symbol_is_exported_and_bound():
    names = _header_functions()
    assert "ax_helm" in names and len(names) >= 10
    lib = _lib.lib()
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.PROTOTYPES, f"{n} has no ctypes prototype"
    assert lib.ax_version().decode().startswith("axhelm")


@pytest.mark.parametrize("lx", range(2, 17))
def test_host_gll_and_dmat_match_oracle(lx):
    x, w = ax.gll(lx)
    xo, wo = oracle.gll(lx)
    np.testing.assert_allclose(x, xo, atol=2e-16 * lx)
    np.testing.assert_allclose(w, wo, rtol=1e-14)
    dx, dxt = ax.dmat(lx)
    dxo, dxto = oracle.d_buffers(lx)
    scale = np.abs(dxo).max()
    np.testing.assert_allclose(dx, dxo, atol=1e-13 * scale)
    np.testing.assert_allclose(dxt, dxto, atol=1e-13 * scale)


@pytest.mark.parametrize("lx", [2, 3, 5, 8, 12])
def test_host_geometry_matches_oracle(lx):
    v = synth.box_vertices(3, 2, 4, seed=21)
    g = ax.box_geometry(v, lx, want_xyz=True)
    go = oracle.box_geometry(v, lx)
    for k in ("g11", "g22", "g33", "g12", "g13", "g23"):
        scale = np.abs(go["g11"]).max()
        np.testing.assert_allclose(g[k], go[k], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(g["mass"], go["B"], rtol=1e-12)
    np.testing.assert_allclose(g["xyz"], go["xyz"], atol=1e-15)


def test_host_corners_match_oracle():
    for dims, seed in (((3, 2, 4), 21), ((1, 1, 1), 2)):
        v = synth.box_vertices(*dims, seed=seed)
        np.testing.assert_array_equal(ax.box_corners(v), oracle.element_corners(v))


def test_host_numbering_matches_oracle():
    for dims, lx in (((3, 2, 4), 5), ((1, 1, 1), 2), ((2, 5, 3), 8)):
        np.testing.assert_array_equal(ax.box_numbering(*dims, lx), oracle.numbering(*dims, lx))


def _ulp64(x):
    return np.spacing(np.abs(x))


def test_host_mask_matches_oracle():
    """ax_box_mask with every face Dirichlet is the oracle's boundary mask;
    with faces left open (partition interfaces) exactly the marked faces
    are zero."""
    nx, ny, nz, lx = 3, 2, 4, 4
    np.testing.assert_array_equal(ax.box_mask(nx, ny, nz, lx),
                                  oracle.boundary_mask(nx, ny, nz, lx))
    n = lx - 1
    g = oracle.numbering(nx, ny, nz, lx)
    NX, NY = nx * n + 1, ny * n + 1
    Z = g // (NX * NY)
    X = g % NX
    m = ax.box_mask(nx, ny, nz, lx, (True, False, False, False, False, True))
    np.testing.assert_array_equal(m, np.where((X == 0) | (Z == nz * n), 0.0, 1.0))


def test_df64_split_is_exact_truncation():
    g = synth.rng(5)
    mags = 10.0 ** g.uniform(-20, 30, size=20000)
    x = mags * np.where(g.uniform(size=mags.size) < 0.5, -1.0, 1.0)
    x = np.concatenate([x, [1.0, -1.0, 2.0 ** -40, np.nextafter(1.0, 0), np.nextafter(1.0, 2),
                            3.0, 1.0 / 3.0, -2.0 ** 100, 123456789.123456789]])
    hi, lo, back = ax.df64_roundtrip(x)
    hi64 = hi.astype(np.float64)
    # hi is x truncated toward zero to fp32: |hi| <= |x| < |hi| + ulp32(hi)
    assert np.all(np.abs(hi64) <= np.abs(x))
    assert np.all(np.abs(x) - np.abs(hi64) < np.spacing(np.abs(hi)).astype(np.float64))
    assert np.all(np.sign(hi64) == np.sign(x))
    # hi + lo carries 47 bits
    err = np.abs(x - (hi64 + lo.astype(np.float64)))
    assert np.all(err <= 2.0 ** -46 * np.abs(x))
    # and the join brings it back to within one fp64 ulp
    assert np.all(np.abs(back - x) <= 2.0 ** -46 * np.abs(x))


def test_df64_small_and_special_values():
    x = np.array([0.0, -0.0, 1e-30, -1e-35, 2.0 ** -126, 2.0 ** -130, 1e-40])
    hi, lo, back = ax.df64_roundtrip(x)
    # absolute error stays below 2^-100 where relative accuracy is not promised
    assert np.all(np.abs(back - x) <= np.maximum(2.0 ** -46 * np.abs(x), 2.0 ** -100))
    assert back[0] == 0.0 and back[1] == 0.0


def test_df64_join_rounds_pairs():
    """join(hi, lo) of a normalised pair is within one fp64 ulp of hi + lo,
    including pairs that cross a power of two downwards."""
    g = synth.rng(6)
    hi = (g.uniform(0.5, 2.0, size=5000) * 2.0 ** g.integers(-40, 40, size=5000)).astype(np.float32)
    hi[:200] = (2.0 ** g.integers(-30, 30, size=200)).astype(np.float32)  # powers of two
    hi[::2] *= -1
    ulp32 = np.spacing(np.abs(hi)).astype(np.float64)
    lo = (g.uniform(-0.5, 0.5, size=hi.size) * ulp32).astype(np.float32)
    exact = hi.astype(np.float64) + lo.astype(np.float64)
    # join via the roundtrip entry: split(exact) -> norm -> join
    _, _, back = ax.df64_roundtrip(exact)
    assert np.all(np.abs(back - exact) <= 2.0 ** -46 * np.abs(exact))


def test_argument_checks_need_no_gpu():
    lib = _lib.lib()
    nul = [None] * 11
    # nelv == 0 is a no-op that succeeds
    assert lib.ax_helm(*nul, 8, 0, None) == _lib.AX_OK
    assert lib.ax_helm_f32(*nul, 8, 0, None) == _lib.AX_OK
    # NULL pointers with nelv > 0
    assert lib.ax_helm(*nul, 8, 5, None) == _lib.AX_EINVAL
    # lx out of range, negative nelv
    for lx in (0, 1, 17, 100):
        assert lib.ax_helm(*nul, lx, 0, None) == _lib.AX_EINVAL
    assert lib.ax_helm(*nul, 8, -1, None) == _lib.AX_EINVAL
    assert lib.ax_helm_bf16(*nul, 1, 3, None) == _lib.AX_EINVAL
    assert lib.ax_helm_variant(99, *[1] * 11, 8, 4, 0, None) == _lib.AX_EINVAL
    # the six-matrix and trilinear forms: same rules
    assert lib.ax_helm_xyz(*[None] * 15, 8, 0, None) == _lib.AX_OK
    assert lib.ax_helm_xyz(*[None] * 15, 8, 2, None) == _lib.AX_EINVAL
    assert lib.ax_helm_xyz(*[None] * 15, 17, 0, None) == _lib.AX_EINVAL
    assert lib.ax_helm_trilinear_f32(*[None] * 8, 8, 0, None) == _lib.AX_OK
    assert lib.ax_helm_trilinear_f32(*[None] * 8, 8, 2, None) == _lib.AX_EINVAL
    assert lib.ax_helm_trilinear_f32(*[None] * 8, 1, 0, None) == _lib.AX_EINVAL
    assert lib.ax_box_corners(0, 1, 1, None, None) == _lib.AX_EINVAL
    assert lib.ax_gll(1, None, None) == _lib.AX_EINVAL
    assert lib.ax_dmat(17, None, None) == _lib.AX_EINVAL


def test_tune_tables_save_and_load(tmp_path):
    """The tuning tables round-trip through a text file; a bad file applies
    nothing; a missing one is an I/O error."""
    saved = {(d, lx): ax.tune_get(d, lx) for d in (ax.AX_BATCH_F64, ax.AX_BATCH_F32)
             for lx in (5, 8)}
    saved_v = {lx: ax.tune_variant_get(lx) for lx in (6, 8)}
    try:
        ax.tune_set(ax.AX_BATCH_F64, 8, 3)
        ax.tune_set(ax.AX_BATCH_F32, 5, 7)
        ax.tune_variant_set(8, ax.AX_VARIANT_F64_DF)
        ax.tune_variant_set(6, ax.AX_VARIANT_F64_NATIVE)
        path = tmp_path / "tune.txt"
        ax.tune_save(str(path))
        text = path.read_text()
        assert "epb 1 8 3" in text and "epb 2 5 7" in text and "variant 8 2" in text
        for d, lx in saved:
            ax.tune_set(d, lx, 0)
        ax.tune_variant_set(8, 0)
        ax.tune_variant_set(6, 0)
        ax.tune_load(str(path))
        assert ax.tune_get(ax.AX_BATCH_F64, 8) == 3 and ax.tune_get(ax.AX_BATCH_F32, 5) == 7
        assert ax.tune_variant_get(8) == ax.AX_VARIANT_F64_DF
        assert ax.tune_variant_get(6) == ax.AX_VARIANT_F64_NATIVE
        # a refused entry (9 x 8 x 8 > 256 threads) after a valid one: nothing applied
        bad = tmp_path / "bad.txt"
        bad.write_text("epb 1 8 1\nepb 1 8 9\n")
        lib = _lib.lib()
        assert lib.ax_tune_load(str(bad).encode()) == _lib.AX_EINVAL
        assert ax.tune_get(ax.AX_BATCH_F64, 8) == 3
        bad.write_text("bogus 1 2\n")
        assert lib.ax_tune_load(str(bad).encode()) == _lib.AX_EINVAL
        assert lib.ax_tune_load(str(tmp_path / "missing.txt").encode()) == _lib.AX_EIO
        assert lib.ax_tune_load(None) == _lib.AX_EINVAL
    finally:
        for (d, lx), v in saved.items():
            ax.tune_set(d, lx, v)
        for lx, v in saved_v.items():
            ax.tune_variant_set(lx, v)


def test_header_is_a_c_abi(tmp_path):
    """The boundary is plain C: a C99 program includes the header, links the
    library and calls host entry points (GLL nodes for lx = 3 are -1, 0, 1
    with weights 1/3, 4/3, 1/3)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    _lib.lib()  # builds the library if needed
    lib_dir = os.path.dirname(_lib.LIB_PATH)
    src = tmp_path / "abi.c"
    src.write_text(
        '#include <math.h>\n#include <stdio.h>\n#include "axhelm.h"\n'
        "int main(void) {\n"
        "  double x[3], w[3];\n"
        "  if (ax_gll(3, x, w) != AX_OK) return 2;\n"
        "  if (fabs(x[0] + 1) > 1e-15 || fabs(x[1]) > 1e-15 || fabs(x[2] - 1) > 1e-15) return 3;\n"
        "  if (fabs(w[0] - 1.0 / 3) > 1e-15 || fabs(w[1] - 4.0 / 3) > 1e-15) return 4;\n"
        "  if (ax_helm(0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 8, 5, 0) != AX_EINVAL) return 5;\n"
        '  printf("%s\\n", ax_version());\n'
        "  return 0;\n}\n")
    exe = tmp_path / "abi"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(root, "include"),
                        str(src), "-L", lib_dir, "-laxhelm", "-lm", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, LD_LIBRARY_PATH=lib_dir + os.pathsep + os.environ.get("LD_LIBRARY_PATH", ""))
    run = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=60)
    assert run.returncode == 0, (run.returncode, run.stderr)
    assert "axhelm" in run.stdout
