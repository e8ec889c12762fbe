"""The CUDA path and the oracle share nothing but the seeded input generator:

* nothing in the package imports or includes anything under oracle/;
* the oracle imports nothing from the package but workloads (inputs only);
* bench.py reaches the oracle only from its CPU-baseline legs (the functions
  named cpu_baseline* and the --impl reference arm);
* __graft_entry__ reaches it only from build() (compiling it) and smoke().
"""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2603_28907_gb300")


def _imports(tree):
    """(module name, enclosing top-level function or None) of every import."""
    out = []
    for top in tree.body:
        fn = top.name if isinstance(top, (ast.FunctionDef, ast.AsyncFunctionDef)) else None
        for node in ast.walk(top):
            if isinstance(node, ast.Import):
                out += [(a.name, fn) for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mod = node.module or ""
                out.append((mod, fn))
                if node.level == 0 and mod == "":
                    out += [(a.name, fn) for a in node.names]
    return out


def _parse(path):
    return ast.parse(open(path).read(), filename=path)


def test_package_does_not_reach_the_oracle():
    for path in glob.glob(os.path.join(PKG, "**", "*.py"), recursive=True):
        for mod, _ in _imports(_parse(path)):
            assert not mod.split(".")[0] == "oracle", (path, mod)
    for path in glob.glob(os.path.join(PKG, "csrc", "*")):
        txt = open(path, errors="replace").read()
        assert not re.search(r'#\s*include\s*[<"][^>"]*oracle', txt), path


def test_oracle_uses_only_the_input_generator():
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        for mod, _ in _imports(_parse(path)):
            if mod.startswith("paper_2603_28907_gb300"):
                assert mod == "paper_2603_28907_gb300.workloads", (path, mod)
    txt = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert "paper_2603_28907_gb300" not in txt and "csrc" not in txt


def test_bench_reaches_the_oracle_only_from_its_cpu_baseline_legs():
    seen = set()
    for mod, fn in _imports(_parse(os.path.join(ROOT, "bench.py"))):
        if mod.split(".")[0] == "oracle":
            assert fn is not None and (fn.startswith("cpu_baseline") or fn == "run_reference"), (mod, fn)
            seen.add(fn)
    assert "cpu_baseline" in seen and "run_reference" in seen


def test_entry_reaches_the_oracle_only_from_build_and_smoke():
    for mod, fn in _imports(_parse(os.path.join(ROOT, "__graft_entry__.py"))):
        if mod.split(".")[0] == "oracle":
            assert fn in ("build", "smoke"), (mod, fn)
