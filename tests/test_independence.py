"""The oracle and the product path are independent (no GPU).

* Nothing in the package (the CUDA sources, the binding and its helpers) imports, includes
  or loads anything under `oracle/`.
* The oracle includes none of the library's sources and imports from the package only
  the seeded input generators (`inputs`), which both sides take their inputs from.
* `inputs.py` imports neither side.
* `bench.py` reaches the oracle only in its CPU-baseline and reference-arm functions.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2306_09760_gb300")


def _files(top, exts):
    for d, dirs, names in os.walk(top):
        dirs[:] = [x for x in dirs if x not in ("__pycache__", "_build")]
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def _imports(path):
    """(module, enclosing function or None) for every import in a Python file."""
    tree = ast.parse(open(path).read())
    out = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            if isinstance(child, ast.Import):
                out.extend((a.name, fn) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                mod = ("." * child.level) + (child.module or "")
                out.extend((f"{mod}.{a.name}" if mod else a.name, fn) for a in child.names)
                out.append((mod, fn))
            visit(child, f)

    visit(tree, None)
    return out


def test_package_never_reaches_the_oracle():
    for path in _files(PKG, (".py",)):
        for mod, _ in _imports(path):
            assert not re.match(r"^(oracle)(\.|$)", mod), (path, mod)
        text = open(path).read()
        assert "liboracle" not in text and "oracle/" not in text, path
    for path in _files(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".h", ".cpp")):
        for line in open(path):
            if line.lstrip().startswith("#include"):
                assert "oracle" not in line, (path, line)


def test_oracle_shares_no_code_with_the_library():
    for path in _files(os.path.join(ROOT, "oracle"), (".cpp", ".h", ".c")):
        for line in open(path):
            if line.lstrip().startswith("#include"):
                assert "csrc" not in line and "wcns_" not in line and "paper_2306" not in line, (path, line)
    for path in _files(os.path.join(ROOT, "oracle"), (".py",)):
        for mod, _ in _imports(path):
            if mod.startswith("paper_2306_09760_gb300"):
                assert mod in ("paper_2306_09760_gb300", "paper_2306_09760_gb300.inputs"), (path, mod)


def test_inputs_import_neither_side():
    for mod, _ in _imports(os.path.join(PKG, "inputs.py")):
        assert not mod.startswith("oracle") and "wcns" not in mod and "build" not in mod, mod


def test_bench_uses_the_oracle_only_for_its_cpu_legs():
    uses = [(mod, fn) for mod, fn in _imports(os.path.join(ROOT, "bench.py")) if mod.split(".")[0] == "oracle"]
    assert uses, "the CPU baseline leg times the oracle"
    assert {fn for _, fn in uses} <= {"cpu_sample_rate", "run_reference"}, uses
