"""The oracle and the CUDA path share no code: no module of the package imports
the oracle, the oracle imports nothing of the package (nor anything beyond
numpy, scipy and the standard library), no CUDA source includes anything from
the oracle, and the benchmark and the smoke check reach the oracle only from
their CPU-baseline legs, the reference arm and the smoke check itself."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1603_09493_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _py_files(d):
    for base, _, files in os.walk(d):
        if "_build" in base or "__pycache__" in base:
            continue
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def _imports(tree):
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name, 0
        elif isinstance(node, ast.ImportFrom):
            yield node.module or "", node.level


def test_the_package_never_imports_the_oracle():
    for f in _py_files(PKG):
        for mod, level in _imports(ast.parse(open(f).read())):
            assert level > 0 or not mod.split(".")[0] == "oracle", f


def test_the_oracle_imports_only_itself_numpy_scipy_and_the_standard_library():
    allowed = {"numpy", "scipy", "math", "__future__", "dataclasses", "typing", "functools", "itertools",
               "collections", "concurrent", "os", "multiprocessing"}
    for f in _py_files(ORACLE):
        for mod, level in _imports(ast.parse(open(f).read())):
            if level > 0:
                continue                                   # the oracle's own modules
            assert mod.split(".")[0] in allowed, (f, mod)


def test_no_cuda_source_includes_oracle_code():
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        for inc in re.findall(r'#include\s+[<"]([^>"]+)[>"]', txt):
            assert "oracle" not in inc, (f, inc)


def _functions_importing_the_oracle(path):
    tree = ast.parse(open(path).read())
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    for n in top:
        for mod, _ in _imports(ast.Module(body=[n], type_ignores=[])):
            assert mod.split(".")[0] != "oracle", f"{path}: the oracle is imported at module level"
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.FunctionDef):
            for mod, _ in _imports(node):
                if mod.split(".")[0] == "oracle":
                    out.add(node.name)
    return out


def test_bench_and_smoke_reach_the_oracle_only_from_their_baseline_legs():
    bench = _functions_importing_the_oracle(os.path.join(ROOT, "bench.py"))
    # the worker-pool functions and oracle_step_count serve cpu_baseline and the reference arm
    # (main_reference); measure_neb / measure_ego / measure_head_field time their own oracle baselines
    assert bench <= {"cpu_baseline", "_oracle_worker_init", "_oracle_worker_run", "oracle_step_count",
                     "measure_neb", "measure_ego", "measure_head_field", "main_reference"}, bench
    entry = _functions_importing_the_oracle(os.path.join(ROOT, "__graft_entry__.py"))
    assert entry <= {"smoke", "_smoke_surrogate"}, entry
