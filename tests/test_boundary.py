"""The separation between the product and the oracle, checked on the sources (CPU): no module of
the package imports the oracle; bench.py imports it only inside its CPU-baseline sampler (the
baseline and reference legs); the Python binding refuses to load without the built CUDA library
(no CPU fallback)."""
import ast
import os
import shutil
import subprocess
import sys

from conftest import ROOT


def _oracle_imports(path):
    tree = ast.parse(open(path).read())
    found = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            found += [(node.lineno, a.name) for a in node.names if a.name.split(".")[0] == "oracle"]
        elif isinstance(node, ast.ImportFrom) and node.module and node.module.split(".")[0] == "oracle":
            found.append((node.lineno, node.module))
    return found, tree


def test_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_0807_1949_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                found, _ = _oracle_imports(os.path.join(dirpath, f))
                assert not found, (f, found)


def test_bench_imports_the_oracle_only_in_its_sampler():
    """bench.py runs the oracle only to time it (the cpu_baseline / reference leg): the sampler
    (OracleSampler, oracle_timing) and its worker processes _ow_main."""
    found, tree = _oracle_imports(os.path.join(ROOT, "bench.py"))
    assert found
    inside = set()
    for n in ast.walk(tree):
        if (isinstance(n, ast.FunctionDef) and n.name in ("oracle_timing", "_ow_main")) or \
                (isinstance(n, ast.ClassDef) and n.name == "OracleSampler"):
            inside |= {m.lineno for m in ast.walk(n) if isinstance(m, (ast.Import, ast.ImportFrom))}
    assert all(line in inside for line, _ in found)


def test_binding_fails_loudly_without_the_library(tmp_path):
    dst = tmp_path / "paper_0807_1949_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_0807_1949_gb300"), dst,
                    ignore=shutil.ignore_patterns("_lib", "__pycache__", "*.so"))
    r = subprocess.run([sys.executable, "-c", "import paper_0807_1949_gb300.vtm"], cwd=tmp_path,
                       capture_output=True, text=True, env=dict(os.environ, PYTHONPATH=str(tmp_path)))
    assert r.returncode != 0 and "libvtm.so is not built" in r.stderr
