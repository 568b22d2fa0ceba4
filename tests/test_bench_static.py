"""Static check of the measurement scripts on CPU (bench.py and the timing
helpers of the package): every name a function reads is bound somewhere it
can see (module level, its arguments, its own assignments and imports, or
builtins).  Their GPU legs only run on a GPU, so a missing import there would
otherwise surface only when they are timed."""
import ast
import builtins
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bound_in(node):
    names = set()
    for n in ast.walk(node):
        if isinstance(n, (ast.Import, ast.ImportFrom)):
            for a in n.names:
                names.add((a.asname or a.name).split(".")[0])
        elif isinstance(n, ast.Name) and isinstance(n.ctx, (ast.Store, ast.Del)):
            names.add(n.id)
        elif isinstance(n, ast.arg):
            names.add(n.arg)
        elif isinstance(n, (ast.FunctionDef, ast.ClassDef, ast.Lambda)):
            if hasattr(n, "name"):
                names.add(n.name)
        elif isinstance(n, ast.ExceptHandler) and n.name:
            names.add(n.name)
    return names


def _check(fn, outer, missing):
    """Names read in fn (not in its nested functions) must be bound in fn or
    an enclosing scope; nested functions see fn's names as well."""
    local = _bound_in(fn) | outer
    nested = [n for n in ast.walk(fn) if n is not fn and isinstance(n, (ast.FunctionDef, ast.Lambda))]
    inner = set()
    for f in nested:
        inner |= {id(x) for x in ast.walk(f)}
    for n in ast.walk(fn):
        if id(n) in inner:
            continue
        if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load) and n.id not in local:
            missing.append(f"{getattr(fn, 'name', 'lambda')}: {n.id} (line {n.lineno})")
    for f in nested:
        # direct children only; deeper ones are reached from their parent
        parents = [g for g in nested if g is not f and any(x is f for x in ast.walk(g))]
        if not parents:
            _check(f, local, missing)


@pytest.mark.parametrize("path", ["bench.py", "paper_1309_7128_gb300/timepass.py",
                                  "paper_1309_7128_gb300/tolc_study.py"])
def test_functions_read_only_bound_names(path):
    tree = ast.parse(open(os.path.join(ROOT, path)).read())
    module = set(dir(builtins)) | {"__file__", "__name__"}
    for node in tree.body:
        if not isinstance(node, (ast.FunctionDef, ast.ClassDef)):
            module |= _bound_in(node)
        else:
            module.add(node.name)
    missing = []
    for node in ast.walk(tree):
        if isinstance(node, ast.FunctionDef) and (node in tree.body or any(
                node in c.body for c in tree.body if isinstance(c, ast.ClassDef))):
            _check(node, module, missing)
    assert not missing, missing
