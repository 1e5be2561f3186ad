"""The oracle and the CUDA library share no code (CPU, static checks).

The oracle imports nothing from the package; the package (Python binding, generator,
build script, CUDA sources) never imports, includes or reads the oracle. Only the test
suite, the smoke check and the benchmark's CPU legs may use the oracle.
"""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2510_02382_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module:
            names.add(node.module.split(".")[0])
    return names


def _files(top, exts):
    for d, _, fs in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_oracle_imports_nothing_from_the_package():
    for p in _files(os.path.join(ROOT, "oracle"), (".py",)):
        mods = _imports(p)
        assert "paper_2510_02382_gb300" not in mods, p
        assert mods <= {"__future__", "numpy", "torch"}, (p, mods)


def test_package_never_uses_the_oracle():
    for p in _files(PKG, (".py",)):
        assert "oracle" not in _imports(p), p
    for p in _files(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".cpp", ".h")):
        assert "oracle" not in open(p).read().lower(), p
    for p in _files(os.path.join(ROOT, "include"), (".h",)):
        assert "oracle" not in open(p).read().lower(), p


def test_benchmark_uses_the_oracle_only_in_its_cpu_legs():
    """bench.py imports the oracle inside the reference arm and the CPU-baseline legs only."""
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    allowed = {"run_reference", "cpu_baseline_sample", "cpu_oracle_timings"}
    for fn in [n for n in tree.body if isinstance(n, ast.FunctionDef)]:
        src = ast.get_source_segment(open(os.path.join(ROOT, "bench.py")).read(), fn)
        if "oracle" in src and "ctfmnmf_oracle" in src:
            assert fn.name in allowed, fn.name
    top = {n.module for n in tree.body if isinstance(n, ast.ImportFrom)} | \
          {a.name for n in tree.body if isinstance(n, ast.Import) for a in n.names}
    assert not any(m and m.startswith("oracle") for m in top)
