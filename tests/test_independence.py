"""The oracle and the library share no code: nothing in the package (Python
binding, CUDA and C++ sources, build script) or in the input generators
imports or names the oracle, the oracle never imports the package or loads the
library, and the input generators import nothing but numpy and each other."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def files(sub, exts):
    for d, _, fs in os.walk(os.path.join(ROOT, sub)):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def imports(path):
    tree = ast.parse(open(path).read())
    out = set()
    for n in ast.walk(tree):
        if isinstance(n, ast.Import):
            out |= {a.name.split(".")[0] for a in n.names}
        elif isinstance(n, ast.ImportFrom):
            out.add("." if n.level else (n.module or "").split(".")[0])
    return out


def test_package_never_reaches_the_oracle():
    for p in files("paper_2509_22975_gb300", (".py", ".cu", ".cuh", ".cpp", ".h")):
        text = open(p).read()
        assert not re.search(r"\boracle\b", text), p
    for p in files("include", (".h",)):
        assert not re.search(r"\boracle\b", open(p).read()), p


def test_oracle_never_reaches_the_package():
    for p in files("oracle", (".py",)):
        assert not ({"paper_2509_22975_gb300", "ctypes", "torch"} & imports(p)), p
        assert "libmcd" not in open(p).read(), p


def test_input_generators_hold_no_method_code():
    for p in files("workloads", (".py",)):
        assert imports(p) <= {"__future__", "dataclasses", "numpy", "."}, (p, imports(p))
