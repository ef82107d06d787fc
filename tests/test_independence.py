"""The oracle and the CUDA path share no code: nothing in the package imports oracle/,
nothing in oracle/ or workloads/ imports the package, workloads/ holds no oracle import
either, and bench.py reaches the oracle only in its CPU-baseline and reference legs."""
import ast
import glob
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    """(module name, enclosing function name or None) for every import in a file."""
    tree = ast.parse(open(path).read(), filename=path)
    out = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else func
            if isinstance(child, ast.Import):
                out.extend((a.name, f) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                mod = ("." * child.level) + (child.module or "")
                out.append((mod, f))
            visit(child, f)

    visit(tree, None)
    return out


def _py(*parts):
    return sorted(glob.glob(os.path.join(ROOT, *parts, "**", "*.py"), recursive=True))


def test_package_does_not_import_the_oracle():
    for path in _py("paper_2102_11536_gb300"):
        for mod, _ in _imports(path):
            assert not mod.split(".")[0] == "oracle", (path, mod)


def test_oracle_and_inputs_do_not_import_the_package():
    for path in _py("oracle") + _py("workloads"):
        for mod, _ in _imports(path):
            assert not mod.startswith("paper_2102_11536_gb300"), (path, mod)
    for path in _py("workloads"):
        for mod, _ in _imports(path):
            assert mod.split(".")[0] != "oracle", (path, mod)


def test_bench_uses_the_oracle_only_for_the_cpu_legs():
    allowed = {"oracle_setup", "run_cpu_baseline", "run_reference"}
    for mod, func in _imports(os.path.join(ROOT, "bench.py")):
        if mod.split(".")[0] == "oracle":
            assert func in allowed, (mod, func)
