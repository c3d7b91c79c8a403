"""C ABI checks that need no GPU: the library loads, exports every entry point that
include/lp.h declares, validates its inputs, and its host compiler (lp_compile with
LP_COMPILE_HOST_ONLY) builds exactly the standardized matrix the oracle builds."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2009_10247_gb300 as lp
from tests.helpers import golden
from workloads import normal_program, parse, small_definite, tiny_random, transitive_closure

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lp.h")


@pytest.fixture(scope="module")
def lib():
    return lp.load(build_if_missing=True)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lp_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "lp_compile" in names and "lp_least_model" in names and "lp_stable_models" in names
    raw = ctypes.CDLL(lp.library_path())
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, f"declared but not exported: {missing}"
    assert sorted(lp.EXPORTS) == sorted(n for n in names if n in lp.EXPORTS)


def _compare_with_oracle(prog):
    s = oracle.standardize(prog)
    with lp.Program.from_program(prog, host_only=True) as P:
        info = P.info
        m = P.export_matrix()
    assert info["n_prime"] == s.n_prime and info["nnz"] == s.nnz
    assert info["n_barred"] == s.n_barred and info["n_aux"] == s.n_aux
    assert info["k"] == len(s.guess_rows())
    assert np.array_equal(m["row_ptr"], s.row_ptr)
    assert np.array_equal(m["col"], s.col)
    assert np.array_equal(m["kind"], s.kind)
    # threshold t_i with a_ij = 1/t_i (rule rows) or 1 (OR rows, self-loops): the oracle's
    # exact values num/den must be 1/threshold on every entry, den = 1 for the rest
    rows = np.repeat(np.arange(s.n_prime), np.diff(s.row_ptr))
    vals = s.num / s.den[rows]
    assert np.allclose(vals, 1.0 / np.maximum(m["threshold"][rows], 1))
    empty = np.diff(s.row_ptr) == 0
    assert np.all(m["threshold"][empty] == 0) and np.all(m["threshold"][~empty] >= 1)


def test_example1_csr_arrays(lib):
    g = golden("example1.json")
    p = parse(g["program"], atoms=g["atoms"])
    with lp.Program.from_program(p, host_only=True) as P:
        m = P.export_matrix()
    assert m["row_ptr"].tolist() == g["csr_row_index"]
    assert m["col"].tolist() == g["csr_col_index"]
    rows = np.repeat(np.arange(7), np.diff(m["row_ptr"]))
    assert (1.0 / m["threshold"][rows]).tolist() == g["csr_value"]


def test_example2_matrix(lib):
    g = golden("example2.json")
    _compare_with_oracle(parse(g["program"], atoms=g["atoms"]))


@pytest.mark.parametrize("seed", range(30))
def test_compile_tiny_random(lib, seed):
    rng = np.random.default_rng(seed)
    _compare_with_oracle(tiny_random(seed, n_atoms=int(rng.integers(1, 14)), n_rules=int(rng.integers(0, 30)),
                                     max_body=5, p_fact=0.25, p_neg=0.2 if seed % 2 else 0.0))


@pytest.mark.parametrize("seed", range(12))
def test_compile_medium_random(lib, seed):
    # larger random programs than the brute-force ones: many heads with several rules, facts
    # that also head rules, repeated body atoms, negation on a third of the programs, and a few
    # long bodies (the parallel compiler splits every phase over its threads)
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(50, 400))
    _compare_with_oracle(tiny_random(900 + seed, n_atoms=n, n_rules=int(rng.integers(n, 6 * n)),
                                     max_body=int(rng.choice([3, 8, 40])), p_fact=float(rng.uniform(0.02, 0.3)),
                                     p_neg=0.15 if seed % 3 == 0 else 0.0))


def test_compile_generators(lib):
    _compare_with_oracle(small_definite(2))
    _compare_with_oracle(transitive_closure(40, 3.0, seed=2))
    _compare_with_oracle(normal_program(seed=4, n=3000, n_rules=9000, k=8, per_atom=3))


def test_compile_full_size_programs(lib):
    # the benchmark's programs at full size: the large definite program (5e6 rules) and the
    # 2^16-guess normal program, compiled by the parallel host compiler, equal the oracle's
    # standardization row for row (the internal order is checked by the solves on the GPU)
    from workloads import large_definite
    _compare_with_oracle(large_definite(seed=1))
    _compare_with_oracle(normal_program(seed=1))


def test_compile_rejects_malformed(lib):
    def compile_raw(n, head, off, atom, neg=None):
        return lp.Program(n, np.array(head), np.array(off), np.array(atom), neg, host_only=True)

    with pytest.raises(lp.LPError) as e:
        compile_raw(2, [0, 5], [0, 0, 1], [1])  # head out of range
    assert e.value.status == 1
    with pytest.raises(lp.LPError):
        compile_raw(2, [0], [0, 1], [7])  # body atom out of range
    with pytest.raises(lp.LPError):
        compile_raw(2, [0, 1], [0, 2, 1], [1, 1])  # decreasing offsets
    with pytest.raises(lp.LPError):
        compile_raw(2, [0], [1, 2], [1, 1])  # body_off[0] != 0
    with pytest.raises(lp.LPError):
        compile_raw(-1, [], [0], [])


def test_empty_program(lib):
    with lp.Program(0, np.zeros(0, np.int32), np.zeros(1, np.int64), np.zeros(0, np.int32), host_only=True) as P:
        assert P.info["n_prime"] == 0 and P.info["nnz"] == 0


def test_host_only_handle_refuses_solves(lib):
    p = parse("a. b :- a.")
    with lp.Program.from_program(p, host_only=True) as P:
        out = np.zeros(1, np.uint64)
        with pytest.raises(lp.LPError) as e:
            P.least_model(out)
        assert e.value.status == 1


def test_schedule_get_set_validates(lib):
    with lp.Program.from_program(small_definite(1), host_only=True) as P:
        assert P.schedule == {"fixpoint_kernel": 0, "fixpoint_blocks_per_sm": 0, "fixpoint_row_split": 0,
                              "fixpoint_chunk_batch": 0, "fixpoint_row_map": 0, "stable_tile_words": 0,
                              "stable_blocks_per_sm": 0, "stable_row_split": 0, "stable_frontier": 0,
                              "fixpoint_stage": 0}
        for m in (1, 2, 3):
            P.set_schedule(fixpoint_row_map=m)
            assert P.schedule["fixpoint_row_map"] == m
        for bad in ({"fixpoint_row_split": 2}, {"fixpoint_chunk_batch": 4}, {"fixpoint_kernel": 1}):
            with pytest.raises(lp.LPError):  # a thread-per-row map takes neither
                P.set_schedule(**bad)
        P.set_schedule(fixpoint_row_map=0)
        P.set_schedule(fixpoint_kernel=1, fixpoint_blocks_per_sm=2, stable_tile_words=8, stable_blocks_per_sm=1)
        assert P.schedule["stable_tile_words"] == 8 and P.schedule["fixpoint_kernel"] == 1
        for bad in ({"fixpoint_kernel": 4}, {"fixpoint_stage": 2}, {"stable_frontier": 3}, {"stable_frontier": -1},
                    {"stable_frontier": 1, "stable_row_split": 1}, {"stable_frontier": 2, "stable_row_split": 1}, {"stable_tile_words": 3}, {"stable_tile_words": 64},
                    {"fixpoint_row_split": 3}, {"fixpoint_row_split": 2},  # the second: kernel 1 is set
                    {"fixpoint_chunk_batch": 2}, {"fixpoint_chunk_batch": 4}, {"stable_row_split": 2},
                    {"fixpoint_blocks_per_sm": -1}, {"stable_blocks_per_sm": -2}, {"fixpoint_row_map": 4},
                    {"fixpoint_row_map": -1}, {"fixpoint_row_map": 1}):  # the last: kernel 1 is set
            with pytest.raises(lp.LPError):
                P.set_schedule(**bad)
        assert P.schedule["stable_tile_words"] == 8  # unchanged by the rejected calls
        for mode in (2, 1, 0):
            P.set_schedule(stable_frontier=mode)
            assert P.schedule["stable_frontier"] == mode
        with pytest.raises(lp.LPError):
            P.autotune()  # a host-only handle cannot run solves


def test_compile_flags_validate_without_gpu(lib):
    # LP_COMPILE_ON_DEVICE with a host flag and unknown flags fail before any device use; a small
    # program compiled on the host (one thread) gives the oracle's matrix
    out = ctypes.c_void_p()
    head = np.array([0, 1], np.int32)
    off = np.array([0, 0, 1], np.int64)
    atom = np.array([0], np.int32)
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    for flags in (lp.LP_COMPILE_ON_DEVICE | lp.LP_COMPILE_HOST_ONLY, lp.LP_COMPILE_ON_DEVICE | lp.LP_COMPILE_ON_HOST,
                  8, 16):
        assert lib.lp_compile(2, 2, ptr(head), ptr(off), ptr(atom), None, flags, None, ctypes.byref(out)) == 1
        assert not out.value
    prog = small_definite(3)
    with lp.Program.from_program(prog, host_only=True) as P:
        m = P.export_matrix()
    s = oracle.standardize(prog)
    assert np.array_equal(m["row_ptr"], s.row_ptr) and np.array_equal(m["col"], s.col)


def test_batch_entry_points_validate_without_gpu(lib):
    out = ctypes.c_void_p()
    one = np.array([2], np.int32)
    off = np.array([0, 1], np.int64)
    head = np.array([0], np.int32)
    boff = np.array([0, 0], np.int64)
    atom = np.zeros(1, np.int32)
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    assert lib.lp_compile_batch(1, ptr(one), ptr(off), ptr(head), ptr(boff), ptr(atom), None, 4, None,
                                ctypes.byref(out)) == 1  # unknown flag
    bad_off = np.array([1, 1], np.int64)
    assert lib.lp_compile_batch(1, ptr(one), ptr(bad_off), ptr(head), ptr(boff), ptr(atom), None, 0, None,
                                ctypes.byref(out)) == 1  # rule_off[0] must be 0
    assert lib.lp_compile_batch(1, ptr(one), ptr(off), ptr(head), ptr(boff), ptr(atom), None, 0, None, None) == 1
    assert lib.lp_batch_info(None, None, None, None, None, None) == 1
    assert lib.lp_batch_stable_models(None, None, None, None, 10, None) == 1
    lib.lp_batch_free(None)


@pytest.mark.parametrize("threads", ["1", "3"])
def test_compile_is_independent_of_thread_count(lib, threads):
    # the host compiler splits work by the team that runs it (one thread when lp_compile_batch
    # runs it inside its own parallel loop): the matrix must not depend on it
    import subprocess
    import sys
    code = (
        "import numpy as np, oracle, paper_2009_10247_gb300 as lp\n"
        "from workloads import large_definite, normal_program\n"
        "for prog in [normal_program(seed=2, n=3000, n_rules=9000, k=6),\n"
        "             large_definite(seed=2, n=20000, n_rules=100000, chain_levels=20, chain_width=10)]:\n"
        "    with lp.Program.from_program(prog, host_only=True) as P:\n"
        "        m = P.export_matrix()\n"
        "    s = oracle.standardize(prog)\n"
        "    assert np.array_equal(m['row_ptr'], s.row_ptr) and np.array_equal(m['col'], s.col)\n"
        "print('ok')\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, OMP_NUM_THREADS=threads, PYTHONPATH=root)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300, cwd=root)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr[-2000:]


def test_check_matrix_on_host_copies(lib):
    progs = [small_definite(1), normal_program(seed=3, n=2000, n_rules=6000, k=6),
             transitive_closure(30, 2.0, 1)] + [tiny_random(800 + s, n_atoms=20, n_rules=40, p_neg=0.1)
                                                for s in range(10)]
    for prog in progs:
        with lp.Program.from_program(prog, host_only=True) as P:
            assert P.check_matrix() == 0


def test_concurrent_host_compiles_and_thread_local_errors(lib):
    # the host compiler may run on several caller threads at once (each with its own OpenMP
    # team), and lp_last_error belongs to the calling thread
    import threading

    progs = [normal_program(seed=20 + i, n=2000, n_rules=6000, k=5) for i in range(4)]
    want = [oracle.standardize(p) for p in progs]
    results, errors = [None] * 4, [None] * 4
    barrier = threading.Barrier(5)

    def compile_one(i):
        barrier.wait()
        with lp.Program.from_program(progs[i], host_only=True) as P:
            results[i] = P.export_matrix()

    def fail_one():
        barrier.wait()
        for _ in range(20):
            try:
                lp.Program(2, np.array([0, 5]), np.array([0, 0, 1]), np.array([1]), None, host_only=True)
            except lp.LPError as e:
                errors[0] = str(e)
        errors[1] = lib.lp_last_error().decode()  # this thread's last error, not another thread's

    threads = [threading.Thread(target=compile_one, args=(i,)) for i in range(4)] + [threading.Thread(target=fail_one)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    for m, s in zip(results, want):
        assert m is not None
        assert np.array_equal(m["row_ptr"], s.row_ptr) and np.array_equal(m["col"], s.col)
    assert errors[0] and "out of range" in errors[0]
    assert "out of range" in errors[1]


def test_binding_rejects_strided_buffers(lib):
    # liblp reads and writes dense arrays: a strided view must not reach it
    import torch
    t = torch.zeros(8, dtype=torch.int64)
    with pytest.raises(ValueError):
        lp.lp._ptr(t[::2])
    with pytest.raises(ValueError):
        lp.lp._ptr(np.zeros(8, np.int64)[::2])
    assert lp.lp._ptr(t).value == t.data_ptr()


def test_autotune_cache_reuses_a_stored_schedule(lib, tmp_path):
    # a stored schedule is applied without tuning (a host-only handle cannot run the tuner);
    # a miss tunes, which a host-only handle refuses, and leaves the file as it was
    import json
    path = str(tmp_path / "schedules.json")
    with lp.Program.from_program(small_definite(1), host_only=True) as P:
        with pytest.raises(lp.LPError):
            P.autotune_cached(path)
        assert not os.path.exists(path)
        key = P.schedule_cache_key()
        assert "format=" in key and str(P.info["nnz"]) in key
        want = dict(P.schedule, fixpoint_row_map=3, stable_tile_words=8)
        json.dump({key: want}, open(path, "w"))
        assert P.autotune_cached(path) is True
        assert P.schedule == want
        # a schedule stored for another device or schedule format is not applied
        other = key.replace("format=", "format=9")
        json.dump({other: dict(want, fixpoint_row_map=1)}, open(path, "w"))
        with pytest.raises(lp.LPError):
            P.autotune_cached(path)
        # nor is one this build rejects: the handle tunes again (refused here)
        json.dump({key: dict(want, fixpoint_kernel=7)}, open(path, "w"))
        with pytest.raises(lp.LPError):
            P.autotune_cached(path)
        assert P.schedule == want
