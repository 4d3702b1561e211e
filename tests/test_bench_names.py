"""Static check of bench.py: every name a function reads is defined somewhere (module level,
the function's own assignments or parameters, an enclosing function, or builtins).  The
modes that need a GPU cannot run here, so a renamed constant in one of them would only
show on the GPU machine."""
import ast
import builtins
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bound_names(node):
    names = set()
    for n in ast.walk(node):
        if isinstance(n, ast.Name) and isinstance(n.ctx, (ast.Store, ast.Del)):
            names.add(n.id)
        elif isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
            names.add(n.name)
        elif isinstance(n, ast.arg):
            names.add(n.arg)
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            for a in n.names:
                names.add((a.asname or a.name).split(".")[0])
        elif isinstance(n, ast.ExceptHandler) and n.name:
            names.add(n.name)
    return names


def test_bench_functions_read_only_defined_names():
    with open(os.path.join(ROOT, "bench.py")) as f:
        tree = ast.parse(f.read())
    module = _bound_names(tree) | set(dir(builtins)) | {"__file__", "__name__"}
    missing = []
    for fn in [n for n in tree.body if isinstance(n, (ast.FunctionDef, ast.ClassDef))]:
        local = _bound_names(fn)
        for n in ast.walk(fn):
            if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load) and n.id not in local and n.id not in module:
                missing.append(f"{fn.name}: {n.id} (line {n.lineno})")
    assert not missing, missing
