"""The oracle is test infrastructure: the product path never reaches it, and
the oracle shares no code with the CUDA path (static checks, CPU only)."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1607_06156_gb300")


def _imports(path):
    """(module, enclosing function or None) for every import in a Python file."""
    tree = ast.parse(open(path).read(), path)
    out = []

    def visit(node, fn):
        for ch in ast.iter_child_nodes(node):
            f = ch.name if isinstance(ch, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            if isinstance(ch, ast.Import):
                out.extend((a.name.split(".")[0], fn) for a in ch.names)
            elif isinstance(ch, ast.ImportFrom) and ch.module:
                out.append((ch.module.split(".")[0], fn))
            visit(ch, f)

    visit(tree, None)
    return out


def test_package_never_imports_the_oracle():
    for py in glob.glob(os.path.join(PKG, "**", "*.py"), recursive=True):
        assert "oracle" not in [m for m, _ in _imports(py)], py
    for src in glob.glob(os.path.join(PKG, "csrc", "*")):
        assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", open(src).read()), src


def test_generators_hold_no_oracle_or_engine_code():
    for py in glob.glob(os.path.join(ROOT, "graphgen", "*.py")):
        mods = [m for m, _ in _imports(py)]
        assert "oracle" not in mods and "paper_1607_06156_gb300" not in mods, py


def test_oracle_never_imports_the_engine():
    for py in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        assert "paper_1607_06156_gb300" not in [m for m, _ in _imports(py)], py
    for c in glob.glob(os.path.join(ROOT, "oracle", "*.c")):
        incs = re.findall(r"#\s*include\s*[<\"]([^>\"]+)", open(c).read())
        assert all(not i.startswith("cc_gb300") and "csrc" not in i for i in incs), c


def test_bench_uses_the_oracle_only_in_its_cpu_legs():
    """bench.py imports the oracle only inside its cpu_baseline-leg helpers
    (the timed oracle and the label check); the timing helpers never call
    them, so no oracle work sits inside a timed region."""
    path = os.path.join(ROOT, "bench.py")
    legs = {"cpu_oracle_rate", "cpu_leg", "cpu_leg_check", "cpu_leg_batch", "cpu_leg_multi"}
    assert {fn for m, fn in _imports(path) if m == "oracle"} <= legs
    tree = ast.parse(open(path).read())
    callers = {}
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, ast.Call) and getattr(node.func, "id", None) in legs:
                    callers.setdefault(fn.name, set()).add(node.func.id)
    assert set(callers) <= {"run_reference", "main", "cpu_leg", "single_record", "batch_record", "learned_record",
                            "multi_start_record"}
    assert "timed_calls" not in callers and "profiled_calls" not in callers
