"""The oracle and the CUDA path share no code: no module of the package
imports the oracle, the oracle imports nothing of the package, and the one
module both sides use (the seeded input generators) imports neither the
library binding nor the oracle."""
import ast
import glob
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            mod = node.module or ""
            names.add("." * node.level + mod)
            names.update(("." * node.level + mod + "." + a.name).lstrip(".") for a in node.names)
    return names


def test_package_does_not_import_the_oracle():
    for path in glob.glob(os.path.join(ROOT, "paper_2506_20994_gb300", "*.py")):
        assert not any("oracle" in n for n in _imports(path)), path


def test_oracle_does_not_import_the_package():
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        assert not any("paper_2506_20994_gb300" in n or n.startswith(".") and "synth" in n
                       for n in _imports(path)), path


def test_shared_input_module_holds_no_binding():
    names = _imports(os.path.join(ROOT, "paper_2506_20994_gb300", "synth.py"))
    assert not any("oracle" in n or "_lib" in n or "ctypes" in n or "torch" in n
                   for n in names), names


def test_missing_library_fails_loudly():
    """No fallback: without libaxhelm.so every device entry point raises
    (checked in a child interpreter with the library path pointed away)."""
    import subprocess
    import sys
    code = (
        "import paper_2506_20994_gb300 as ax\n"
        "from paper_2506_20994_gb300 import _lib\n"
        "_lib._lib = None\n"
        "_lib.LIB_PATH = '/nonexistent/libaxhelm.so'\n"
        "try:\n"
        "    _lib.lib()\n"
        "except RuntimeError as e:\n"
        "    print('raised:', e)\n"
        "else:\n"
        "    raise SystemExit(3)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and "raised:" in r.stdout, (r.returncode, r.stdout, r.stderr)
