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


SEARCH_PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "mpm.h"

/* usage: search TEXT PATTERNS r m sigma OUT
   reads the text and the r x m pattern bytes, searches with automatic
   parameters through host buffers, writes z pairs (pos, pid) as uint32 */
static uint8_t* slurp(const char* path, size_t* n) {
    FILE* f = fopen(path, "rb");
    if (!f) return NULL;
    fseek(f, 0, SEEK_END);
    long len = ftell(f);
    fseek(f, 0, SEEK_SET);
    uint8_t* buf = (uint8_t*)malloc(len > 0 ? (size_t)len : 1);
    if (buf && len > 0 && fread(buf, 1, (size_t)len, f) != (size_t)len) { free(buf); buf = NULL; }
    fclose(f);
    *n = (size_t)len;
    return buf;
}

int main(int argc, char** argv) {
    if (argc != 7) return 10;
    size_t n = 0, pn = 0;
    uint8_t* T = slurp(argv[1], &n);
    uint8_t* P = slurp(argv[2], &pn);
    const size_t r = (size_t)atol(argv[3]), m = (size_t)atol(argv[4]);
    const int sigma = atoi(argv[5]);
    if (!T || !P || pn != r * m) return 11;
    mpm_handle* h = mpm_build(P, r, m, sigma, NULL);
    if (!h) { fprintf(stderr, "build: %s\n", mpm_strerror(mpm_last_error())); return 12; }
    free(P);  /* the handle keeps its own copy */
    /* too small an output: MPM_ECAPACITY with the count needed */
    size_t z = 1;
    uint32_t one_pos, one_pid;
    int rc = mpm_search(h, T, n, &one_pos, &one_pid, &z);
    if (rc != MPM_ECAPACITY && !(rc == MPM_OK && z <= 1)) return 13;
    const size_t cap = z + 16;
    uint32_t* pos = (uint32_t*)malloc(cap * 4);
    uint32_t* pid = (uint32_t*)malloc(cap * 4);
    for (int rep = 0; rep < 2; rep++) {
        size_t zz = cap;
        rc = mpm_search(h, T, n, pos, pid, &zz);
        if (rc != MPM_OK) { fprintf(stderr, "search: %s\n", mpm_strerror(rc)); return 14; }
        if (zz != z) return 15;
    }
    mpm_stats st;
    if (mpm_get_stats(h, &st) != MPM_OK || st.z != z || st.n != n) return 16;
    mpm_free(h);
    FILE* o = fopen(argv[6], "wb");
    if (!o) return 17;
    for (size_t i = 0; i < z; i++) {
        fwrite(&pos[i], 4, 1, o);
        fwrite(&pid[i], 4, 1, o);
    }
    fclose(o);
    printf("z=%zu\n", z);
    free(pos);
    free(pid);
    free(T);
    return 0;
}
"""


@pytest.mark.gpu
@pytest.mark.parametrize("alpha", ["dna", "protein"])
def test_c_program_searches_host_buffers_on_the_gpu(tmp_path, libdir, alpha):
    """A C program (no Python, no CUDA headers) builds a handle, searches a
    host text into host outputs twice and frees it; its list equals the
    oracle's."""
    import numpy as np
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from oracle import native
    from paper_1405_5483_gb300 import workloads as W
    native.build()
    c = (W.dna_case((1 << 22) + 5, 100, 16, 50) if alpha == "dna"
         else W.protein_case((1 << 22) + 3, 500, 32, 250))
    (tmp_path / "T.bin").write_bytes(c.T.tobytes())
    (tmp_path / "P.bin").write_bytes(np.ascontiguousarray(c.P).tobytes())
    src = tmp_path / "search.c"
    src.write_text(SEARCH_PROGRAM)
    exe = tmp_path / "search"
    subprocess.run([cc, "-std=c99", "-O1", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe), "-L", libdir, "-lmpm", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe), str(tmp_path / "T.bin"), str(tmp_path / "P.bin"),
                          str(c.r), str(c.m), str(c.sigma), str(tmp_path / "occ.bin")],
                         capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    got = np.fromfile(tmp_path / "occ.bin", np.uint32).reshape(-1, 2)
    want = native.aho_corasick(c.T, c.P, threads=8)
    assert got.shape[0] == want[0].size >= c.planted_offsets.size
    assert np.array_equal(got[:, 0], want[0]) and np.array_equal(got[:, 1], want[1])
