"""The oracle and the CUDA path share no code: the product package never
imports the oracle, the oracle imports nothing of the product, and the only
module both sides use is the seeded input generator, which holds no method
arithmetic (no operator, weights, solver or residual)."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1804_05522_gb300")


def _imports(path):
    tree = ast.parse(open(path).read())
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out |= {a.name for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            mod = node.module or ""
            out.add(mod)
            out |= {f"{mod}.{a.name}" for a in node.names}
    return out


def _py_files(d):
    for base, _, files in os.walk(d):
        if "__pycache__" in base or "_lib" in base:
            continue
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def test_product_never_imports_the_oracle():
    for f in _py_files(PKG):
        assert not any(m == "oracle" or m.startswith("oracle.") for m in _imports(f)), f
    for f in (os.path.join(PKG, "csrc", x) for x in os.listdir(os.path.join(PKG, "csrc"))):
        assert "oracle" not in open(f).read().lower(), f


def test_oracle_imports_nothing_of_the_product():
    for f in _py_files(os.path.join(ROOT, "oracle")):
        mods = _imports(f)
        assert not any(m.startswith("paper_1804_05522_gb300") for m in mods), (f, mods)


def test_shared_input_module_has_no_method_arithmetic():
    src = open(os.path.join(PKG, "inputs.py")).read()
    tree = ast.parse(src)
    names = {n.name for n in ast.walk(tree) if isinstance(n, (ast.FunctionDef, ast.ClassDef))}
    for forbidden in ("gl_weights", "fd_operator", "toeplitz", "sylvester", "residual", "solve", "hodlr", "aca"):
        assert not any(forbidden in n.lower() for n in names), (forbidden, names)


def test_only_tests_smoke_and_bench_baseline_use_the_oracle():
    """Outside tests/, only __graft_entry__.smoke() and bench.py's CPU-baseline and
    reference legs may import the oracle, and only inside those functions."""
    allowed = {"__graft_entry__.py": {"smoke"}, "bench.py": {"__init__"}}  # OracleSampler.__init__
    for f in _py_files(ROOT):
        rel = os.path.relpath(f, ROOT)
        if rel.startswith(("tests" + os.sep, "oracle" + os.sep, "_work" + os.sep, "baseline" + os.sep)):
            continue
        tree = ast.parse(open(f).read())
        for fn in [n for n in ast.walk(tree) if isinstance(n, (ast.FunctionDef, ast.Module))]:
            body_imports = [n for n in ast.walk(fn) if isinstance(n, (ast.Import, ast.ImportFrom))]
            uses = any((isinstance(n, ast.ImportFrom) and (n.module or "").startswith("oracle")) or
                       (isinstance(n, ast.Import) and any(a.name.startswith("oracle") for a in n.names))
                       for n in body_imports)
            if uses and isinstance(fn, ast.FunctionDef):
                assert fn.name in allowed.get(rel, set()), (rel, fn.name)
        top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
        assert not any((isinstance(n, ast.ImportFrom) and (n.module or "").startswith("oracle")) or
                       (isinstance(n, ast.Import) and any(a.name.startswith("oracle") for a in n.names))
                       for n in top), rel
