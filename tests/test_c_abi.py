"""liblp from plain C: tests/c_abi_host_only.c is compiled with gcc against include/lp.h and
linked against the built liblp.so, then run on the host (LP_COMPILE_HOST_ONLY, no GPU). Its
printed CSR of Example 1 must equal the paper's arrays (tests/golden/example1.json), and a
solve on the host-only handle must be refused with a message. tests/c_abi_device.c solves on the
GPU from plain C with host buffers: Example 1's least model (all five atoms after 3 theta
applications; only r, s from the fact s alone), Example 2's single stable model {t}, and the two
stable models of an even loop."""
import json
import os
import shutil
import subprocess

import pytest

import paper_2009_10247_gb300 as lp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build_and_run(tmp_path, name):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lib = lp.library_path()
    if not os.path.exists(lib):
        lp.load(build_if_missing=True)
    exe = str(tmp_path / name)
    libdir = os.path.dirname(lib)
    r = subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", name + ".c"), "-o", exe, "-L", libdir, "-l:liblp.so",
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return subprocess.run([exe], capture_output=True, text=True, timeout=120)


@pytest.mark.gpu
def test_plain_c_device_solves(tmp_path):
    run = _build_and_run(tmp_path, "c_abi_device")
    assert run.returncode == 0, run.stdout + run.stderr
    out = {line.split(" ", 1)[0] + " " + line.split(" ", 2)[1]: line.split() for line in run.stdout.splitlines()}
    # Example 1: every atom p q r s t (bits 0-4), 3 theta applications (Sec. 2.1)
    assert out["example1 least"] == ["example1", "least", "0", "model", str(0b11111), "iters", "3"]
    # from the fact s alone: s and r (r :- s); iterations: v0, r, no change
    assert out["example1 facts_s"] == ["example1", "facts_s", "0", "model", str((1 << 3) | (1 << 2)), "iters", "2"]
    # Example 2: t is a fact, so its barred atom is not guessed (k = 0); the one stable model is {t}
    assert out["example2 stable"] == ["example2", "stable", "0", "k", "0", "mask", "1", "n_stable", "1", "model",
                                      str(1 << 3)]
    # even loop: guess bit 0 = p-bar, bit 1 = q-bar (ascending atom id); {q} is g = 1 (p false),
    # {p} is g = 2 (q false); models in guess order: {q} = bit 1, then {p} = bit 0
    assert out["evenloop stable"] == ["evenloop", "stable", "0", "mask", str(0b0110), "n_stable", "2", "models",
                                      "2", "1"]


def test_plain_c_consumer(tmp_path):
    run = _build_and_run(tmp_path, "c_abi_host_only")
    assert run.returncode == 0, run.stdout + run.stderr
    lines = dict(line.split(" ", 1) for line in run.stdout.strip().splitlines() if not line.startswith("host-only"))
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "example1.json")))
    assert [int(x) for x in lines["row_ptr"].split()] == g["csr_row_index"]
    assert [int(x) for x in lines["col"].split()] == g["csr_col_index"]
    thr = [int(x) for x in lines["threshold"].split()]
    rows = [i for i in range(len(thr)) for _ in range(g["csr_row_index"][i + 1] - g["csr_row_index"][i])]
    assert [1.0 / thr[i] for i in rows] == g["csr_value"]
    assert "host-only solve 1 with message" in run.stdout
