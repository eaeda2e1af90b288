"""The oracle and the product path share no code: nothing in the package, the C ABI or the CUDA
sources imports, includes or names a file under oracle/, and the oracle imports nothing of the
package (the seeded input generators of synth.py are the only module both sides use, and they are
passed to the oracle by the tests, not imported by it)."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1603_02329_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out.update(a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            out.add(("." * node.level) + (node.module or ""))
    return out


def test_package_does_not_import_the_oracle():
    for path in glob.glob(os.path.join(PKG, "**", "*.py"), recursive=True):
        for name in _imports(path):
            assert not name.split(".")[0] == "oracle", (path, name)


def test_cuda_and_c_sources_do_not_reference_the_oracle():
    srcs = glob.glob(os.path.join(PKG, "csrc", "*")) + glob.glob(os.path.join(ROOT, "include", "*"))
    assert srcs
    for path in srcs:
        txt = open(path, errors="replace").read()
        assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", txt), path
        assert "pat_oracle" not in txt and "oracle/" not in txt, path


def test_oracle_imports_only_numpy_scipy_and_itself():
    allowed = {"numpy", "scipy", "__future__", "typing", "dataclasses", "math", "types", "functools",
               "itertools", "collections", "os", "sys", "warnings"}
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        for name in _imports(path):
            if name.startswith("."):
                continue                      # the oracle's own modules
            assert name.split(".")[0] in allowed, (path, name)
