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
