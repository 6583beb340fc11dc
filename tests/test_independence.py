"""The oracle and the CUDA path share no code: no module of the package imports the oracle,
no oracle module imports the package, and the package's C/CUDA sources include nothing
from the oracle.  The input generator (workloads.py) is the one module both are fed from,
and it holds no arithmetic of the method (checked here for the kernel's ingredients)."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2607_06429_b300")
ORACLE = os.path.join(ROOT, "oracle")


def _imports(path):
    tree = ast.parse(open(path).read())
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names |= {a.name for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            names.add(("." * node.level) + (node.module or ""))
    return names


def _py(d):
    return [os.path.join(d, f) for f in sorted(os.listdir(d)) if f.endswith(".py")]


def test_package_never_imports_the_oracle():
    for path in _py(PKG):
        for name in _imports(path):
            assert not name.split(".")[0] == "oracle", (path, name)


def test_oracle_never_imports_the_package():
    for path in _py(ORACLE):
        for name in _imports(path):
            assert "paper_2607_06429_b300" not in name, (path, name)


def test_cuda_sources_include_nothing_from_the_oracle():
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        for inc in re.findall(r'#include\s+[<"]([^>"]+)[>"]', txt):
            assert "oracle" not in inc, (f, inc)


def test_input_generator_holds_no_kernel_arithmetic():
    txt = open(os.path.join(PKG, "workloads.py")).read()
    # the Green's function, its phase and the quadrature weights live on each side alone
    for pattern in (r"exp\(\s*1j", r"4\s*\*\s*math\.pi\s*\*\s*r", r"sincos", r"leggauss"):
        assert not re.search(pattern, txt), pattern
