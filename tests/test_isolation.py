"""The oracle and the CUDA path share no code: the package never imports the
oracle, the oracle never imports the package, and the seeded input
generators (workloads/) import neither. __graft_entry__ touches the oracle
only in smoke(). Checked on the import statements of every source file."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _py_files(sub):
    for dirpath, _, names in os.walk(os.path.join(ROOT, sub)):
        for n in names:
            if n.endswith(".py"):
                yield os.path.join(dirpath, n)


def _imports(path):
    """(top-level module name, enclosing function name or None) per import."""
    tree = ast.parse(open(path).read(), path)
    out = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else func
            if isinstance(child, ast.Import):
                out.extend((a.name.split(".")[0], func) for a in child.names)
            elif isinstance(child, ast.ImportFrom) and child.module and child.level == 0:
                out.append((child.module.split(".")[0], func))
            visit(child, f)

    visit(tree, None)
    return out


def test_package_and_workloads_never_import_the_oracle():
    for sub in ("paper_2505_08777_gb300", "workloads"):
        for f in _py_files(sub):
            assert "oracle" not in [m for m, _ in _imports(f)], f


def test_oracle_and_workloads_never_import_the_package():
    for sub in ("oracle", "workloads"):
        for f in _py_files(sub):
            assert "paper_2505_08777_gb300" not in [m for m, _ in _imports(f)], f


def test_graft_entry_uses_the_oracle_only_in_smoke():
    for mod, func in _imports(os.path.join(ROOT, "__graft_entry__.py")):
        if mod == "oracle":
            assert func == "smoke", func


def test_cuda_sources_include_only_their_own_headers():
    csrc = os.path.join(ROOT, "paper_2505_08777_gb300", "csrc")
    for n in os.listdir(csrc):
        if n.endswith((".cu", ".cuh", ".h")):
            for line in open(os.path.join(csrc, n)):
                if line.startswith("#include \""):
                    assert "oracle" not in line, (n, line)
