"""Static checks of the separation between the CUDA path and the oracle: no
module of the package imports the oracle, the oracle imports nothing of the
package, the seeded input generator imports neither, and the CUDA sources
include no oracle file."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1307_8052_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            names.add(node.module.split(".")[0])
    return names


def _py_files(d):
    return [os.path.join(d, f) for f in sorted(os.listdir(d)) if f.endswith(".py")]


def test_package_does_not_import_the_oracle():
    files = _py_files(PKG)
    assert any(f.endswith("binding.py") for f in files)
    for f in files:
        assert "oracle" not in _imports(f), f


def test_oracle_does_not_import_the_package():
    for f in _py_files(os.path.join(ROOT, "oracle")):
        assert "paper_1307_8052_gb300" not in _imports(f), f


def test_input_generator_imports_neither_side():
    imp = _imports(os.path.join(PKG, "synthetic.py"))
    assert "oracle" not in imp and "paper_1307_8052_gb300" not in imp


def test_cuda_sources_include_no_oracle_file():
    csrc = os.path.join(PKG, "csrc")
    srcs = [f for f in os.listdir(csrc) if f.endswith((".cu", ".cpp", ".h"))]
    assert srcs
    for f in srcs:
        for line in open(os.path.join(csrc, f)):
            if line.lstrip().startswith("#include"):
                assert "oracle" not in line, (f, line)
