"""The oracle and the CUDA path share nothing: the package never imports the oracle (so there
is no CPU fallback through it), the oracle imports nothing from the package or the input
generators, and the input generators import neither."""

import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            out.add("." if node.level else node.module.split(".")[0])
    return out


def _py_files(d):
    for dirpath, _, files in os.walk(os.path.join(ROOT, d)):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(dirpath, f)


def test_package_never_imports_the_oracle():
    for f in _py_files("paper_2505_23618_gb300"):
        assert "oracle" not in _imports(f), f


def test_oracle_imports_only_numpy_and_the_standard_library():
    for f in _py_files("oracle"):
        mods = _imports(f) - {"."}
        assert mods <= {"__future__", "math", "numpy"}, (f, mods)


def test_input_generators_hold_no_transform_code():
    for f in _py_files("synth"):
        mods = _imports(f)
        assert "oracle" not in mods and "paper_2505_23618_gb300" not in mods, (f, mods)
