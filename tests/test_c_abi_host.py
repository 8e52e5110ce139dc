"""The C ABI from plain C: include/tm.h compiles as C11 and a C program linked against
libtm.so uses the host-only entry points (no GPU), agreeing with the Python binding."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1009_4975_gb300 import build
    return build.build()


def test_c_program_uses_the_host_entry_points(lib, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "host_tables")
    cuda_inc = "/usr/local/cuda/include"
    cmd = [cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc,
           os.path.join(ROOT, "tests", "c", "host_tables.c"), "-o", exe, lib, "-Wl,-rpath," + os.path.dirname(lib)]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    lines = out.stdout.strip().splitlines()
    import paper_1009_4975_gb300 as P
    leaves = [[k & 1, (k >> 1) & 1, (k >> 2) & 1, 1] for k in range(8)] + [[2, 0, 0, 0]]
    info, _ = P.tm_tables_build(2, 1, 1, 1, 1.0, leaves)
    assert lines[0] == (f"Ne {info['Ne']} Nn {info['Nn']} hanging {info['n_hanging']} free {info['n_free']} "
                        f"blocks {info['n_blocks']}")
    assert lines[1] == "adapt rc 0 leaves 16"      # 8 children of the refined base cell + 8 unchanged
    assert lines[2] == "bad mark rc 1"              # TM_EINVAL
    g = P.tm_tables_diag(2, 1, 1, 1, 1.0, leaves)
    h = np.where(np.arange(info["Ne"]) == info["Ne"] - 1, 1.0, 0.5)
    want = 0.0
    for nd in range(info["Nn"]):   # the same summation order as the C program
        for j in range(g["ptr"][nd], g["ptr"][nd + 1]):
            want += h[g["elem"][j]] * g["tab"][g["q"][j], 0]
    assert lines[3] == (f"diag rc 0 entries {g['elem'].size} triples {g['tab'].shape[0]} "
                        f"sum0 {want:.17g}")
