"""The oracle and the CUDA path share no code: the package never imports the
oracle, the oracle never loads the package or its library, the CUDA sources
include nothing from the oracle, and bench.py touches the oracle only in its
CPU-baseline and reference legs."""
import ast
import glob
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def imported_modules(path):
    tree = ast.parse(open(path).read())
    out = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out += [a.name.split(".")[0] for a in node.names]
        elif isinstance(node, ast.ImportFrom) and node.module:
            out.append(node.module.split(".")[0])
    return out


def test_package_never_imports_the_oracle():
    for path in glob.glob(os.path.join(ROOT, "paper_1109_1205_gb300", "*.py")):
        assert "oracle" not in imported_modules(path), path
    for path in glob.glob(os.path.join(ROOT, "paper_1109_1205_gb300", "csrc", "*")):
        text = open(path).read()
        includes = [ln for ln in text.splitlines() if ln.strip().startswith("#include")]
        assert not any("oracle" in ln for ln in includes), path
        assert "kg_oracle" not in text and "kgoracle" not in text, path


def test_oracle_never_loads_the_package():
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        assert "paper_1109_1205_gb300" not in imported_modules(path), path
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")) + glob.glob(os.path.join(ROOT, "oracle", "*.cpp")):
        text = open(path).read()
        assert "libkrylovgf" not in text and "krylovgf.h" not in text, path


def test_bench_uses_the_oracle_only_in_its_cpu_legs():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    users = set()
    for fn in [n for n in tree.body if isinstance(n, ast.FunctionDef)]:
        for node in ast.walk(fn):
            if isinstance(node, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in node.names):
                users.add(fn.name)
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    assert not any(isinstance(n, ast.Import) and any(a.name == "oracle" for a in n.names) for n in top)
    assert users <= {"cpu_baseline_sample", "run_reference"}, users
