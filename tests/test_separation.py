"""The product path and the oracle stay apart: nothing in the package (Python
binding, pipelines, tuner, replicas, CUDA/C++ sources) imports, includes or
calls the oracle, and the oracle shares no code with the package except the
seeded input generators' module, which holds none of the pipelines'
arithmetic."""

import ast
import glob
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2012_07145_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            names.add(("." * node.level) + (node.module or ""))
    return names


def test_package_never_imports_the_oracle():
    for path in glob.glob(os.path.join(PKG, "*.py")):
        bad = [n for n in _imports(path) if n == "oracle" or n.startswith("oracle.")]
        assert not bad, f"{os.path.basename(path)} imports {bad}"
    for path in glob.glob(os.path.join(PKG, "csrc", "*")):
        text = open(path, errors="replace").read()
        assert "oracle" not in text.lower(), os.path.basename(path)


def test_oracle_imports_nothing_from_the_package():
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        for n in _imports(path):
            assert not n.startswith("paper_2012_07145_gb300"), f"{os.path.basename(path)} imports {n}"
            assert n in {"numpy", "math", "fractions", "itertools", "functools"} or n.startswith("."), \
                f"{os.path.basename(path)} imports {n}"


def test_input_generators_hold_no_pipeline_arithmetic():
    # synth.py draws numbers only: it imports numpy alone and defines no stage
    # operation (no stencil, pyramid, histogram, remap or compositing names)
    path = os.path.join(PKG, "synth.py")
    assert _imports(path) == {"numpy"}
    tree = ast.parse(open(path).read())
    funcs = {n.name for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)}
    for word in ("stencil_clamp", "downsample", "upsample", "histogram", "remap", "over", "harris", "unsharp"):
        assert word not in funcs
