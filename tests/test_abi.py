"""The C-ABI library builds, loads without a GPU, and exports every entry
point include/dd.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(dd_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libdd():
    from paper_2012_00357_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("dd_load_dataset", "dd_project_nearest", "dd_solve"):
        assert want in names


def test_library_exports_every_declared_symbol(libdd):
    out = subprocess.run(["nm", "-D", "--defined-only", libdd], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (dd_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libdd)
    for n in declared_functions():
        getattr(lib, n)


def test_binding_names_match_header(libdd):
    import paper_2012_00357_gb300 as P
    assert sorted(P.EXPORTS) == declared_functions()
    for n in P.EXPORTS:
        assert callable(getattr(P, n))


def test_no_cuda_device_is_reported_not_crashed(libdd):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2012_00357_gb300 as P
    with pytest.raises(P.DDError) as e:
        P.dd_create(0)
    assert e.value.status == P.DD_ERR_CUDA


def test_binding_functions_use_only_defined_names():
    """Every name a function of the binding reads is a parameter, a local, a
    module-level name or a builtin (the GPU calls cannot run here, so a
    misspelt argument would otherwise go unnoticed)."""
    import ast
    import builtins
    import os
    src = open(os.path.join(os.path.dirname(__file__), "..", "paper_2012_00357_gb300", "binding.py")).read()
    tree = ast.parse(src)
    glob = {n.id for n in ast.walk(tree) if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Store)}
    glob |= {f.name for f in tree.body if isinstance(f, (ast.FunctionDef, ast.ClassDef))}
    for node in tree.body:
        if isinstance(node, (ast.Import, ast.ImportFrom)):
            glob |= {(a.asname or a.name).split(".")[0] for a in node.names}
    bad = []
    for f in [n for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)]:
        known = {a.arg for a in f.args.args + f.args.kwonlyargs}
        known |= {n.id for n in ast.walk(f) if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Store)}
        known |= {a.arg for n in ast.walk(f) if isinstance(n, ast.Lambda) for a in n.args.args}
        for n in ast.walk(f):
            if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load) and n.id not in known | glob \
                    and not hasattr(builtins, n.id):
                bad.append((f.name, n.id))
    assert not bad
