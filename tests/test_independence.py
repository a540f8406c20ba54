"""The CUDA path and the oracle share no code, and neither calls the other.

Static checks over the sources (CPU):
* nothing in the package (Python binding, CUDA sources, internal headers) or
  in the public headers names the oracle;
* nothing in oracle/ names the package, its sources or the public headers,
  and the oracle's C++ includes standard headers only;
* the input generator igdata imports neither side (numpy only);
* bench.py imports the oracle only in its CPU-baseline and reference legs,
  and __graft_entry__ only in build() (compiling it) and smoke().
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_2507_14222_gb300"


def _sources(sub, exts):
    out = []
    for dirpath, dirnames, files in os.walk(os.path.join(ROOT, sub)):
        dirnames[:] = [d for d in dirnames if d not in ("_build", "__pycache__")]
        out += [os.path.join(dirpath, f) for f in files if f.endswith(exts)]
    assert out, sub
    return out


def _read(path):
    with open(path, encoding="utf-8") as f:
        return f.read()


def test_package_and_headers_never_name_the_oracle():
    for path in _sources(PKG, (".py", ".cu", ".cuh", ".h", ".cpp")) + _sources("include", (".h",)):
        assert not re.search(r"\boracle\b", _read(path), re.I), path


def test_oracle_never_names_the_package():
    for path in _sources("oracle", (".py", ".cpp", ".h")):
        src = _read(path)
        assert PKG not in src and "csrc" not in src, path
        assert not re.search(r"\big(_helpers)?\.h\b", src), path


def test_oracle_cpp_includes_standard_headers_only():
    for path in _sources("oracle", (".cpp", ".h")):
        for inc in re.findall(r"^\s*#\s*include\s*(\S+)", _read(path), re.M):
            assert inc.startswith("<"), (path, inc)


def _imports(tree):
    """(module name, enclosing top-level function or None) of every import."""
    found = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            here = fn
            if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) and fn is None:
                here = child.name
            if isinstance(child, ast.Import):
                found.extend((a.name.split(".")[0], here) for a in child.names)
            elif isinstance(child, ast.ImportFrom) and child.module:
                found.append((child.module.split(".")[0], here))
            visit(child, here)

    visit(tree, None)
    return found


def test_generator_imports_neither_side():
    for path in _sources("igdata", (".py",)):
        mods = {m for m, _ in _imports(ast.parse(_read(path)))}
        assert not mods & {"oracle", PKG}, (path, mods)


def test_bench_and_entry_import_the_oracle_only_where_allowed():
    allowed = {"bench.py": {"_oracle_pass", "cpu_baseline", "run_reference", "_reference_served"},
               "__graft_entry__.py": {"build", "smoke"}}
    for name, fns in allowed.items():
        where = {fn for m, fn in _imports(ast.parse(_read(os.path.join(ROOT, name))))
                 if m == "oracle"}
        assert where and where <= fns, (name, where)
