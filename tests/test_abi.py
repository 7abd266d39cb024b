"""The C-ABI library builds, loads and exports every symbol include/*.h declares.

No compute call is made here (no GPU on the build host); only host-only
functions (version, status strings, default options) are exercised.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def clib():
    from paper_1408_1237_gb300.build import build
    build()
    from paper_1408_1237_gb300 import binding
    return binding.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(krr_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["krr_kernel_mvp", "krr_cg_solve", "krr_fgmres_solve", "krr_mll_grad",
                     "krr_fgmres_solve_batched", "krr_create", "krr_destroy"]:
        assert required in names


def test_every_declared_symbol_is_exported(clib):
    missing = [n for n in declared_functions() if not hasattr(clib, n)]
    assert not missing, f"not exported: {missing}"


def test_host_only_functions(clib):
    from paper_1408_1237_gb300 import binding
    assert clib.krr_version() >= 100
    assert binding.status_string(0) == "KRR_OK"
    assert binding.status_string(5) == "KRR_NOT_CONVERGED"
    o = binding.default_opts()
    # Sec. 6 defaults: outer tol 1e-6, delta and inner tol from the rules
    assert (o.restart, o.tol, o.delta, o.inner_tol) == (30, 1e-6, -1.0, -1.0)
    assert o.inner_maxit == 100 and o.inner_prec == 0


def test_struct_layouts_match_header(clib):
    from paper_1408_1237_gb300 import binding
    # krr_fgmres_opts: 2 ints, 3 doubles, 3 ints (with padding) -> 48 bytes
    assert ctypes.sizeof(binding.krr_fgmres_opts) == 48
    assert ctypes.sizeof(binding.krr_solve_info) == 48
    assert ctypes.sizeof(binding.krr_problem) == 40
    assert ctypes.sizeof(binding.krr_profile) == 40


def test_product_path_has_no_oracle_dependency():
    # The library package must not reach the oracle (test infrastructure).
    pkg = os.path.join(ROOT, "paper_1408_1237_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
            assert "krr_oracle" not in text, path
