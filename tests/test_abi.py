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
    assert o.use_graph == 1 and o.x0_given == 0


def test_struct_layouts_match_header(clib):
    from paper_1408_1237_gb300 import binding
    # krr_fgmres_opts: 2 ints, 3 doubles, 4 ints -> 48 bytes
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


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "libkrr.h"

int main(void) {
    krr_fgmres_opts o;
    krr_fgmres_default_opts(&o);
    if (o.restart != 30 || o.tol != 1e-6 || o.inner_maxit != 100 || o.x0_given != 0) return 2;
    if (sizeof(krr_fgmres_opts) != 48) return 10;
    if (strcmp(krr_status_string(KRR_NOT_CONVERGED), "KRR_NOT_CONVERGED") != 0) return 3;
    if (krr_version() < 100) return 4;
    if (krr_create(NULL) != KRR_ERR_INVALID_ARG) return 5;
    krr_handle h = NULL;
    krr_status s = krr_create(&h);          /* KRR_ERR_CUDA where no GPU is visible */
    if (s == KRR_OK) {
        if (krr_set_option(h, 999, 1) != KRR_ERR_INVALID_ARG) return 6;
        if (krr_destroy(h) != KRR_OK) return 7;
    } else if (s != KRR_ERR_CUDA || h != NULL) {
        return 8;
    }
    if (krr_kernel_mvp(NULL, NULL, 1, 3, 1.f, 0.f, NULL, 1, NULL, KRR_FP32, NULL)
        != KRR_ERR_INVALID_ARG) return 9;
    krr_points pts = NULL;
    if (krr_points_create(NULL, NULL, 1, 3, 1.f, &pts, NULL) != KRR_ERR_INVALID_ARG || pts != NULL)
        return 11;
    if (krr_kernel_mvp_points(NULL, NULL, NULL, 1, 0.f, NULL, KRR_FP32, NULL) != KRR_ERR_INVALID_ARG)
        return 12;
    if (krr_points_destroy(NULL, NULL) != KRR_ERR_INVALID_ARG) return 13;
    if (krr_tune_save(NULL, "x") != KRR_ERR_INVALID_ARG || krr_tune_load(NULL, "x") != KRR_ERR_INVALID_ARG)
        return 14;
    printf("ok %d\n", (int)s);
    return 0;
}
"""


def test_header_is_plain_c_and_links(clib, tmp_path):
    # The boundary is a C ABI: the header compiles as C99 with warnings as
    # errors, and a C program links against libkrr.so and runs its host-only
    # calls (no device work).
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.join(ROOT, "paper_1408_1237_gb300")
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-lkrr", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    assert out.stdout.startswith("ok")


def test_binding_constants_match_header():
    # Every enumerator of include/libkrr.h that the binding repeats has the
    # header's value (status codes, options, kernel families, precisions).
    from paper_1408_1237_gb300 import binding
    text = open(os.path.join(ROOT, "include", "libkrr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    enums = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(KRR_\w+)\s*=\s*(\d+)", text)}
    assert len(enums) >= 20
    repeated = [n for n in enums if hasattr(binding, n)]
    assert len(repeated) >= 18
    for name in repeated:
        assert getattr(binding, name) == enums[name], name
    prec = {"fp32": "KRR_FP32", "bf16": "KRR_BF16", "fp16": "KRR_FP16"}
    for key, name in prec.items():
        assert binding.PRECISION[key] == enums[name]
