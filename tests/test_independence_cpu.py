"""The oracle and the CUDA path share no code, and the product path has no
fallback: checked on the sources and by loading a missing library."""
import ast
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2203_02479_gb300")


def _files(top, exts):
    for dp, _, fns in os.walk(top):
        if "__pycache__" in dp:
            continue
        for fn in fns:
            if fn.endswith(exts):
                yield os.path.join(dp, fn)


def _code(path):
    """Source without comments and string literals (Python: the AST's
    imports; C/CUDA: the text with // and /* */ comments removed)."""
    txt = open(path, encoding="utf-8").read()
    if path.endswith(".py"):
        return txt
    txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)
    return re.sub(r"//[^\n]*", " ", txt)


def _imports(path):
    tree = ast.parse(open(path, encoding="utf-8").read())
    names = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names += [a.name for a in node.names]
        elif isinstance(node, ast.ImportFrom) and node.module:
            names.append(node.module)
    return names


def test_package_never_touches_the_oracle():
    for path in _files(PKG, (".py",)):
        assert not any(n.split(".")[0] == "oracle" for n in _imports(path)), path
    for path in list(_files(PKG, (".cu", ".cuh", ".h", ".py"))) + list(_files(os.path.join(ROOT, "include"), (".h",))):
        assert not re.search(r"wsoracle|_wsoracle", _code(path)), path


def test_oracle_never_touches_the_package():
    for path in _files(os.path.join(ROOT, "oracle"), (".py",)):
        assert not any(n.split(".")[0] in ("paper_2203_02479_gb300", "wiresim", "torch") for n in _imports(path)), path
    for path in _files(os.path.join(ROOT, "oracle"), (".c", ".h")):
        code = _code(path)
        assert not re.search(r'#include\s*"', code), path              # system headers only
        assert not re.search(r"wiresim|ws_internal|__global__", code), path


def _functions_importing_oracle(path):
    tree = ast.parse(open(path, encoding="utf-8").read())
    out = set()
    for fn in ast.walk(tree):
        if isinstance(fn, (ast.FunctionDef, ast.AsyncFunctionDef)):
            for node in ast.walk(fn):
                if isinstance(node, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in node.names):
                    out.add(fn.name)
                if isinstance(node, ast.ImportFrom) and (node.module or "").split(".")[0] == "oracle":
                    out.add(fn.name)
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    top_oracle = any((isinstance(n, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in n.names)) or
                     (isinstance(n, ast.ImportFrom) and (n.module or "").split(".")[0] == "oracle") for n in top)
    return out, top_oracle


def test_oracle_users_outside_tests():
    """bench.py runs the oracle only through oracle_unit (its CPU baselines,
    the error against the oracle and the reference arm); __graft_entry__
    only builds it and uses it in smoke()."""
    fns, top = _functions_importing_oracle(os.path.join(ROOT, "bench.py"))
    assert not top and fns == {"oracle_unit"}
    fns, top = _functions_importing_oracle(os.path.join(ROOT, "__graft_entry__.py"))
    assert not top and fns <= {"build", "smoke"}


def test_inputs_module_holds_no_method_arithmetic():
    """The only module both sides read draws numbers: it imports nothing of
    either side and nothing beyond numpy."""
    names = _imports(os.path.join(PKG, "inputs.py"))
    assert set(n.split(".")[0] for n in names) <= {"__future__", "dataclasses", "math", "numpy"}


def test_missing_library_fails_loudly():
    code = ("from paper_2203_02479_gb300 import wiresim\n"
            "try:\n"
            "    wiresim.load_library('/nonexistent/libwiresim.so')\n"
            "except wiresim.WiresimError as e:\n"
            "    print('raised', e.status)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "raised" in r.stdout, r.stderr
