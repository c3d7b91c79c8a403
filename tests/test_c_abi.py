"""liblp from plain C: tests/c_abi_host_only.c is compiled with gcc against include/lp.h and
linked against the built liblp.so, then run on the host (LP_COMPILE_HOST_ONLY, no GPU). Its
printed CSR of Example 1 must equal the paper's arrays (tests/golden/example1.json), and a
solve on the host-only handle must be refused with a message."""
import json
import os
import shutil
import subprocess

import pytest

import paper_2009_10247_gb300 as lp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_consumer(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lib = lp.library_path()
    if not os.path.exists(lib):
        lp.load(build_if_missing=True)
    exe = str(tmp_path / "c_abi_host_only")
    libdir = os.path.dirname(lib)
    r = subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c_abi_host_only.c"), "-o", exe, "-L", libdir, "-l:liblp.so",
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stdout + run.stderr
    lines = dict(line.split(" ", 1) for line in run.stdout.strip().splitlines() if not line.startswith("host-only"))
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "example1.json")))
    assert [int(x) for x in lines["row_ptr"].split()] == g["csr_row_index"]
    assert [int(x) for x in lines["col"].split()] == g["csr_col_index"]
    thr = [int(x) for x in lines["threshold"].split()]
    rows = [i for i in range(len(thr)) for _ in range(g["csr_row_index"][i + 1] - g["csr_row_index"][i])]
    assert [1.0 / thr[i] for i in rows] == g["csr_value"]
    assert "host-only solve 1 with message" in run.stdout
