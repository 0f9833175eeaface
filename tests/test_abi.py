"""The C ABI library builds, loads and exports every entry point include/ftblas.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

import paper_2104_00897_gb300 as fb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ftblas.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ftblas_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound():
    lib = fb.load()
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
        assert n in fb.SIGNATURES, f"binding lacks {n}"


def test_struct_sizes_match_the_header_layout():
    assert ctypes.sizeof(fb.FtErrorRecord) == 96
    assert fb.REPORT_BYTES == 6 * 8 + 4 + 4 + 64 * 96
    assert ctypes.sizeof(fb.FtInjectPoint) == 40
    assert ctypes.sizeof(fb.FtInject) == 8 + 10 * 4 + 16 * 40


@pytest.mark.parametrize("args,code", [
    ((100, 111, 111, 4, 4, 4, 1.0, 1, 4, 1, 4, 0.0, 1, 4), -1),
    ((102, 110, 111, 4, 4, 4, 1.0, 1, 4, 1, 4, 0.0, 1, 4), -2),
    ((102, 111, 113, 4, 4, 4, 1.0, 1, 4, 1, 4, 0.0, 1, 4), -3),
    ((102, 111, 111, -1, 4, 4, 1.0, 1, 4, 1, 4, 0.0, 1, 4), -4),
    ((102, 111, 111, 4, -1, 4, 1.0, 1, 4, 1, 4, 0.0, 1, 4), -5),
    ((102, 111, 111, 4, 4, -1, 1.0, 1, 4, 1, 4, 0.0, 1, 4), -6),
    ((102, 111, 111, 4, 4, 4, 1.0, None, 4, 1, 4, 0.0, 1, 4), -8),
    ((102, 111, 111, 4, 4, 4, 1.0, 1, 3, 1, 4, 0.0, 1, 4), -9),
    ((102, 111, 112, 4, 5, 4, 1.0, 1, 4, 1, 4, 0.0, 1, 4), -11),   # B^T stored 5 x 4 needs ldb >= 5
    ((102, 111, 111, 4, 4, 4, 1.0, 1, 4, 1, 4, 0.0, None, 4), -13),
    ((101, 111, 111, 4, 6, 4, 1.0, 1, 4, 1, 6, 0.0, 1, 5), -14),   # row-major C needs ldc >= N
])
def test_argument_validation_codes(args, code):
    # Invalid arguments are rejected on the host before any CUDA call.
    assert fb.ftblas_dgemm(*args, None, None) == code
    assert fb.ftblas_dgemm_noabft(*args, None) == code


def test_empty_problem_returns_without_gpu_work():
    # M == 0 / N == 0: quick return, no device memory touched (null pointers are fine).
    assert fb.ftblas_dgemm(102, 111, 111, 0, 4, 4, 1.0, None, 1, None, 4, 0.0, None, 1, None, None) == 0
    assert fb.ftblas_dgemm(102, 111, 111, 4, 0, 4, 1.0, None, 4, None, 4, 0.0, None, 4, None, None) == 0


def test_injection_config_validation_and_counter():
    assert fb.ftblas_set_injection(fb.make_injection(seed=3, every_n_launches=5, errors_per_launch=2)) == 0
    assert fb.ftblas_injection_launch_count() == 0
    bad = fb.make_injection(bit_lo=50, bit_hi=40, every_n_launches=1, errors_per_launch=1)
    assert fb.ftblas_set_injection(bad) == -1
    bad = fb.make_injection(every_n_launches=1, errors_per_launch=65)
    assert fb.ftblas_set_injection(bad) == -1
    assert fb.ftblas_set_injection(None) == 0


def test_verification_tile_and_engine_switch():
    assert fb.ftblas_verification_tile(fb.COL_MAJOR, fb.R_64F, 10, 10, 10) == (128, 128, 32)
    assert fb.ftblas_verification_tile(fb.ROW_MAJOR, fb.R_64F, 10, 10, 10) == (128, 128, 32)
    # The FP64 tile edge follows the waves of CTAs on 152 SMs (no device here): 64 where
    # 128-edge tiles leave most SMs idle, 128 where they fill the waves.
    expect = {(256, 256): 64, (300, 200): 64, (1024, 1024): 64, (2048, 2048): 64, (128, 8192): 64,
              (4096, 4096): 128, (8192, 8192): 128, (16384, 16384): 128, (32768, 1024): 128}
    for (m, n), e in expect.items():
        for layout in (fb.COL_MAJOR, fb.ROW_MAJOR):
            assert fb.ftblas_verification_tile(layout, fb.R_64F, m, n, 512) == (e, e, 32), (m, n)
    assert fb.ftblas_set_fp64_tile(128) == 0
    assert fb.ftblas_verification_tile(fb.COL_MAJOR, fb.R_64F, 1024, 1024, 1024) == (128, 128, 32)
    assert fb.ftblas_set_fp64_tile(64) == 128
    assert fb.ftblas_verification_tile(fb.COL_MAJOR, fb.R_64F, 8192, 8192, 8192) == (64, 64, 32)
    prev = fb.ftblas_set_fp64_engine(fb.ENGINE_DMMA)
    assert fb.ftblas_verification_tile(fb.COL_MAJOR, fb.R_64F, 1024, 1024, 1024) == (128, 128, 32)
    fb.ftblas_set_fp64_engine(prev)
    assert fb.ftblas_set_fp64_tile(96) == -1
    assert fb.ftblas_set_fp64_tile(0) == 64
    # tensor-core forms: 128 x 248 tiles (8 checksum columns), k-tile 64 BF16 or 128 E4M3
    for ct in (fb.R_32F, fb.R_16BF):
        assert fb.ftblas_verification_tile(fb.COL_MAJOR, ct, 8192, 8192, 8192) == (128, 248, 64)
        assert fb.ftblas_verification_tile(fb.ROW_MAJOR, ct, 8192, 8192, 8192) == (248, 128, 64)
    assert fb.ftblas_verification_tile(fb.COL_MAJOR, fb.R_8F_E4M3, 16384, 16384, 16384) == (128, 248, 128)
    prev = fb.ftblas_set_fp64_engine(fb.ENGINE_DMMA)
    assert fb.ftblas_set_fp64_engine(prev) == fb.ENGINE_DMMA
    assert fb.ftblas_set_fp64_engine(7) == -1
    # tensor-core kernel form: 0 (by call), 1 or 2; the verification tile does not depend on it
    assert fb.ftblas_set_tc_cta_group(3) == -1 and fb.ftblas_set_tc_cta_group(-1) == -1
    prev = fb.ftblas_set_tc_cta_group(2)
    assert prev == 0 and fb.tc_cta_group(True) == 2
    assert fb.ftblas_verification_tile(fb.COL_MAJOR, fb.R_16BF, 8192, 8192, 8192) == (128, 248, 64)
    assert fb.ftblas_set_tc_cta_group(prev) == 2
    assert fb.tc_cta_group(True) == 2 and fb.tc_cta_group(False) == 2


def test_every_declaration_cites_its_passage():
    """Each entry point's comment in the header names the passage of the paper that defines
    its operation, or says that the paper has no counterpart (controls, diagnostics)."""
    src = open(os.path.join(ROOT, "include", "ftblas.h")).read()
    decls = list(re.finditer(r"(/\*(?:(?!\*/).)*?\*/)\s*\n(?:int|const char\s*\*|void|int64_t)\s+(ftblas_\w+)\s*\(",
                             src, flags=re.S))
    assert len(decls) >= 20
    missing = [m.group(2) for m in decls
               if not re.search(r"Section|no counterpart", " ".join(re.sub(r"\n\s*\*", " ", m.group(1)).split()))]
    assert not missing, missing


C_CONSUMER = r"""
#include <stdio.h>
#include <string.h>
#include "ftblas.h"

int main(void) {
  int64_t tr = 0, tc = 0, bk = 0;
  /* argument validation returns -p (xerbla style) before any device work */
  int bad = ftblas_dgemm(FTBLAS_COL_MAJOR, FTBLAS_NO_TRANS, FTBLAS_NO_TRANS, -1, 4, 4, 1.0, 0, 1, 0, 4, 0.0, 0, 1,
                         0, 0);
  int rc = ftblas_verification_tile(FTBLAS_COL_MAJOR, FTBLAS_R_16BF, 256, 256, 256, &tr, &tc, &bk);
  printf("%s|%d|%d|%lld|%lld|%lld|%s\n", ftblas_version(), bad, rc, (long long)tr, (long long)tc, (long long)bk,
         ftblas_status_string(FTBLAS_STATUS_NOT_SUPPORTED));
  return 0;
}
"""


def test_header_is_plain_c_and_a_c_program_links_and_calls_the_library(tmp_path):
    """The boundary is a C ABI: the header compiles as C99 on its own, and a plain C program
    links against libftblas.so and calls entry points that need no GPU."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    inc = os.path.join(ROOT, "include")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-fsyntax-only", "-x", "c",
                        os.path.join(inc, "ftblas.h")], capture_output=True, text=True)
    assert r.returncode == 0 and not r.stderr.strip(), r.stderr
    fb.load()
    lib = fb.library_path()
    src = tmp_path / "consumer.c"
    src.write_text(C_CONSUMER)
    exe = tmp_path / "consumer"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-I", inc, str(src), "-o", str(exe), lib,
                        "-Wl,-rpath," + os.path.dirname(lib)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    version, bad, rc, tr, tc, bk, msg = r.stdout.strip().split("|")
    expected = fb.ftblas_version()
    assert version == (expected.decode() if isinstance(expected, bytes) else expected)
    assert int(bad) == -4  # M is argument 4
    assert int(rc) == 0 and (int(tr), int(tc), int(bk)) == (128, 248, 64)
    assert msg
