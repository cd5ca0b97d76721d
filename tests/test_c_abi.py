"""The boundary is a C ABI: include/mpm.h compiles as strict C99, and a C
program linked against the built library plans a filter and reads back
error strings without Python or a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "mpm.h"

int main(void) {
    /* two DNA patterns of length 8, row-major */
    const uint8_t P[16] = {'A','C','G','T','A','C','G','T', 'T','T','G','A','C','C','A','G'};
    mpm_params in, out;
    mpm_table_info info;
    memset(&in, 0, sizeof in);
    in.map_shift = -1;
    if (mpm_plan(P, 2, 8, 4, &in, &out, &info) != MPM_OK) return 1;
    if (out.q < 1 || out.k < 1 || info.positions < 1 || info.table_bytes == 0) return 2;
    if (mpm_plan(P, 0, 8, 4, &in, &out, &info) != MPM_EINVAL) return 3;
    if (mpm_last_error() != MPM_EINVAL) return 4;
    if (strcmp(mpm_strerror(MPM_OK), "ok") != 0) return 5;
    printf("q=%d sigma_r=%d k=%d positions=%d\n", out.q, out.sigma_r, out.k, info.positions);
    return 0;
}
"""


@pytest.fixture(scope="module")
def libdir():
    from paper_1405_5483_gb300 import build_lib
    build_lib.build()
    from paper_1405_5483_gb300 import _native
    return os.path.dirname(_native.LIB_PATH)


def test_header_is_strict_c99(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "hdr.c"
    src.write_text('#include "mpm.h"\nint main(void) { return 0; }\n')
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), "-fsyntax-only", str(src)], check=True)


def test_c_program_plans_through_the_library(tmp_path, libdir):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "plan.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "plan"
    subprocess.run([cc, "-std=c99", "-O1", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe), "-L", libdir, "-lmpm", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    assert out.stdout.startswith("q=")
