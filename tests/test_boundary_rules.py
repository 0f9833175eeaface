"""The product path is the CUDA library alone.

It never reaches the oracle: the package does not mention it, and the benchmark imports it
only in its CPU-baseline sample and in its reference arm, both of which time the oracle on
the host. And it fails loudly when its library is missing, since there is no CPU fallback.
"""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2104_00897_gb300")


def test_package_sources_never_reference_the_oracle():
    checked = 0
    for dirpath, dirnames, files in os.walk(PKG):
        dirnames[:] = [d for d in dirnames if d not in ("_build", "__pycache__")]
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp", ".c")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower(), os.path.join(dirpath, f)
                checked += 1
    assert checked >= 10


def _oracle_imports(node):
    for x in ast.walk(node):
        if isinstance(x, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in x.names):
            yield x
        elif isinstance(x, ast.ImportFrom) and (x.module or "").split(".")[0] == "oracle":
            yield x


def test_bench_imports_the_oracle_only_in_its_cpu_legs():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    allowed = {"oracle_sample", "run_reference"}
    seen = set()
    for node in tree.body:
        found = list(_oracle_imports(node))
        if not found:
            continue
        assert isinstance(node, ast.FunctionDef) and node.name in allowed, \
            f"oracle imported at line {found[0].lineno} outside {sorted(allowed)}"
        seen.add(node.name)
    assert seen == allowed


def test_missing_library_raises(monkeypatch, tmp_path):
    import paper_2104_00897_gb300 as fb
    monkeypatch.setattr(fb, "_lib", None)
    monkeypatch.setattr(fb._build, "LIB", str(tmp_path / "libftblas.so"))
    with pytest.raises(RuntimeError, match="not found"):
        fb.load(build_if_needed=False)


def test_torch_helpers_refuse_host_tensors_before_any_launch():
    """The C ABI takes raw device pointers: the torch helpers refuse host tensors up front
    (here, with no GPU, before any CUDA call is made)."""
    torch = pytest.importorskip("torch")
    import paper_2104_00897_gb300 as fb
    a = torch.zeros((4, 3), dtype=torch.float64)
    b = torch.zeros((3, 5), dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        fb.gemm(a, b)
    with pytest.raises(ValueError, match="CUDA tensor"):
        fb.dgemm(a, b)
    with pytest.raises(ValueError, match="CUDA tensor"):
        fb.gemm(a.to(torch.bfloat16), b.to(torch.bfloat16))
