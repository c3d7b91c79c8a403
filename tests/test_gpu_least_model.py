"""GPU parity of the least-model path (Algorithm 1 in liblp) against the CPU oracle.

Bit-exact comparison of every model bit and of the iteration count (theta applications),
under every row map of kernel 0, the sliced kernel 2 (vector prefix staged in shared memory or
not) and the one-block kernel 3 where the program fits it, on the paper's example, tiny random programs with ragged
sizes, every workload generator at test sizes, and the full-size large definite program in the
launch configuration the benchmark times."""
import numpy as np
import pytest

import oracle
import paper_2009_10247_gb300 as lp
from tests.helpers import golden, is_model
from workloads import (large_definite, parse, small_definite, tiny_random, transitive_closure)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import gpu_least_model  # noqa: E402


ROW_MAPS = (0, 1, 2, 3)  # the warp-per-word map and the three thread-per-row maps of kernel 0
# kernel 0 under each row map, then the sliced kernel with and without the staged prefix
# and the one-block kernel 3 (matrix in shared memory) wherever the program fits it
SCHEDULES = tuple(dict(fixpoint_kernel=0, fixpoint_row_map=m, fixpoint_stage=0) for m in ROW_MAPS) + (
    dict(fixpoint_kernel=2, fixpoint_row_map=0, fixpoint_stage=0),
    dict(fixpoint_kernel=2, fixpoint_row_map=0, fixpoint_stage=1),
    dict(fixpoint_kernel=3, fixpoint_row_map=0, fixpoint_stage=0))


def _apply(P, sc):
    """Set a schedule; False if it is kernel 3 and the program's matrix does not fit one block."""
    try:
        P.set_schedule(**sc)
        return True
    except lp.LPError as e:
        if sc["fixpoint_kernel"] == 3 and e.status == lp.ERR_INVALID:
            return False
        raise


def _parity(prog, init=None):
    # every schedule of the least-model solve must give the oracle's model and iteration count
    want, want_it = oracle.least_model(prog, init=init)
    with lp.Program.from_program(prog) as P:
        for sc in SCHEDULES:
            if not _apply(P, sc):
                continue
            got, it = gpu_least_model(P, init=init)
            assert np.array_equal(got, want), f"{sc}: {np.count_nonzero(got != want)} atoms differ"
            assert it == want_it, f"{sc}"
    return got, it


def test_example1():
    g = golden("example1.json")
    got, it = _parity(parse(g["program"], atoms=g["atoms"]))
    assert got.all() and it == 3


@pytest.mark.parametrize("seed", range(40))
def test_tiny_random(seed):
    rng = np.random.default_rng(seed)
    _parity(tiny_random(seed, n_atoms=int(rng.integers(1, 90)), n_rules=int(rng.integers(0, 200)),
                        max_body=6, p_fact=0.2))


@pytest.mark.parametrize("seed", range(6))
def test_fact_subsets(seed):
    p = small_definite(10 + seed)
    keep = p.fact_atoms() & (np.random.default_rng(seed).random(p.n_atoms) < 0.5)
    _parity(p, init=keep)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_small_definite(seed):
    got, it = _parity(small_definite(seed))
    assert it > 40


def test_transitive_closure_bfs_30():
    p = transitive_closure(30, 2.0, seed=7)
    got, _ = _parity(p)
    N, E = p.meta["n_nodes"], len(p.meta["edges"])
    adj = {x: [] for x in range(N)}
    for x, y in p.meta["edges"]:
        adj[int(x)].append(int(y))
    for x in range(N):
        seen, stack = set(), list(adj[x])
        while stack:
            y = stack.pop()
            if y not in seen:
                seen.add(y)
                stack.extend(adj[y])
        row = got[E + x * N:E + (x + 1) * N]
        assert set(np.nonzero(row)[0].tolist()) == seen


def test_transitive_closure_500():
    p = transitive_closure(500, 4.0, seed=1)
    want, want_it = oracle.least_model(p)
    with lp.Program.from_program(p) as P:
        for sc in SCHEDULES:
            if not _apply(P, sc):
                continue
            got, it = gpu_least_model(P)
            assert it == want_it and np.array_equal(got, want), f"{sc}"


def test_large_definite_scaled():
    _parity(large_definite(seed=2, n=100_000, n_rules=500_000, chain_levels=100, chain_width=20))


def test_large_definite_full_size():
    # the benchmark workload itself: 1e6 atoms, 5e6 rules, ~1000 iterations, under the default
    # schedule, every thread-per-row map, and the schedule the autotuner picks (which is what
    # the benchmark times)
    p = large_definite(seed=1)
    want, want_it = oracle.least_model(p)
    assert want_it > 1000
    assert is_model(p, want)
    with lp.Program.from_program(p) as P:
        for sc in SCHEDULES:
            if not _apply(P, sc):
                continue
            got, it = gpu_least_model(P)
            assert it == want_it and np.array_equal(got, want), f"{sc}"
        P.autotune(lp.LP_TUNE_LEAST, reps=1)
        got, it = gpu_least_model(P)
        assert it == want_it and np.array_equal(got, want), f"tuned {P.schedule}"


def test_rows_mode_matches_literal_algorithm1():
    p = small_definite(4)
    s = oracle.standardize(p)
    rng = np.random.default_rng(0)
    with lp.Program.from_program(p) as P:
        for trial in range(8):
            v0 = rng.random(s.n_prime) < 0.3
            want, want_it, ok = oracle.alg1(s, v0.astype(np.uint8), max_iters=500)
            assert _apply(P, SCHEDULES[trial % len(SCHEDULES)])
            if ok:
                got, it = gpu_least_model(P, init=v0, rows=True, max_iters=500)
                assert np.array_equal(got, want.astype(bool)) and it == want_it
            else:
                with pytest.raises(lp.LPError) as e:
                    gpu_least_model(P, init=v0, rows=True, max_iters=500)
                assert e.value.status == 4


def test_oscillation_reports_no_fixpoint():
    p = parse("p :- q. q :- p.")
    with lp.Program.from_program(p) as P:
        with pytest.raises(lp.LPError) as e:
            gpu_least_model(P, init=np.array([1, 0], bool), rows=True, max_iters=51)
        assert e.value.status == 4


def test_max_iters_too_small():
    p = small_definite(1)
    with lp.Program.from_program(p) as P:
        with pytest.raises(lp.LPError) as e:
            gpu_least_model(P, max_iters=5)
        assert e.value.status == 4


def test_init_must_be_subset_of_facts():
    p = parse("a. b :- a. c.")
    with lp.Program.from_program(p) as P:
        with pytest.raises(lp.LPError) as e:
            gpu_least_model(P, init=np.array([1, 1, 0], bool))
        assert e.value.status == 1
        got, it = gpu_least_model(P, init=np.array([0, 0, 1], bool))
        assert got.tolist() == [False, False, True]


def test_host_buffers_and_async_stats():
    p = small_definite(5)
    want, want_it = oracle.least_model(p)
    with lp.Program.from_program(p) as P:
        out = np.zeros(lp.words(p.n_atoms), np.uint64)
        it = P.least_model(out)  # host output: staged through device memory
        from tests.helpers import bits_to_bool
        assert np.array_equal(bits_to_bool(out, p.n_atoms), want) and it == want_it
        dev_out = torch.zeros(lp.words(p.n_atoms), dtype=torch.int64, device="cuda:0")
        assert P.least_model(dev_out, sync=False, timing=True) is None
        st = P.last_stats()
        assert st["status"] == 0 and st["iters"] == want_it and st["kernel_ms"] > 0 and st["launches"] == 1


def test_degenerate_programs():
    for text in ["a.", "a :- b.", "a :- a.", "a. a. a :- a.", "a :- b, c. b :- c. c :- a."]:
        _parity(parse(text))
    empty = type("E", (), dict(n_atoms=0, head=np.zeros(0, np.int32), body_off=np.zeros(1, np.int64),
                               body_atom=np.zeros(0, np.int32), body_neg=None))
    with lp.Program.from_program(empty) as P:
        out = torch.zeros(1, dtype=torch.int64, device="cuda:0")
        assert P.least_model(out) == 1


def test_ragged_word_boundaries():
    # n' just around multiples of 32 / 64 rows
    for n in (31, 32, 33, 63, 64, 65, 127, 129):
        rules = [(i, [i - 1]) for i in range(1, n)] + [(0, [])]
        from workloads import from_rules
        p = from_rules(n, rules)
        got, it = _parity(p)
        assert got.all() and it == n


def test_rows_longer_than_a_stage():
    # a rule with 7000 body atoms: its word's entries do not fit a shared-memory stage and
    # are read from global memory; a word with more than 1024 entries takes the long path
    from workloads import from_rules
    rules = [(0, list(range(1, 7001)))] + [(a, []) for a in range(1, 7001)] + [(7001, [0]), (7002, [0]), (7002, [7001])]
    got, it = _parity(from_rules(7003, rules))
    assert got.all()
    rules = [(0, list(range(1, 7001)))] + [(a, []) for a in range(1, 7000)] + [(7001, [0])]
    got, it = _parity(from_rules(7002, rules))
    assert not got[0] and not got[7001]


@pytest.mark.parametrize("stage_bytes", ["16", "65536"])
def test_sliced_kernel_stage_cap(stage_bytes, monkeypatch):
    # a cap on the staged prefix: where the gathered rows do not fit, every slice reads global memory
    monkeypatch.setenv("LP_SLICED_STAGE_BYTES", stage_bytes)
    for prog in (small_definite(5), large_definite(seed=6, n=200_000, n_rules=1_000_000, chain_levels=50,
                                                   chain_width=20)):
        want, want_it = oracle.least_model(prog)
        with lp.Program.from_program(prog) as P:
            P.set_schedule(fixpoint_kernel=2)
            got, it = gpu_least_model(P)
        assert it == want_it and np.array_equal(got, want)


def test_long_rows_and_mixed_slices():
    # rows of 1 to 64 entries, OR rows and facts mixed: slices of many widths, rows padded by
    # repeating their first entry, kernel 3's multi-chunk words
    rules = []
    n = 3000
    rng = np.random.default_rng(3)
    facts = list(range(200))
    rules += [(f, []) for f in facts]
    for h in range(200, 3000):
        ln = int(rng.choice([1, 2, 8, 31, 32, 33, 40, 64]))
        rules.append((h, [int(x) for x in rng.choice(h, size=min(ln, h), replace=False)]))
    for h in range(200, 3000, 7):  # a second rule: OR rows
        rules.append((h, [int(x) for x in rng.choice(h, size=2, replace=False)]))
    from workloads import from_rules
    _parity(from_rules(n, rules))


def test_block_kernel_used_where_it_fits_and_refused_elsewhere():
    # kernel 3 takes a program whose CSR fits one block's shared memory and refuses a larger one
    with lp.Program.from_program(small_definite(2)) as P:
        P.set_schedule(fixpoint_kernel=3)
        assert P.schedule["fixpoint_kernel"] == 3
    with lp.Program.from_program(large_definite(seed=2, n=100_000, n_rules=500_000, chain_levels=100,
                                                chain_width=20)) as P:
        with pytest.raises(lp.LPError) as e:
            P.set_schedule(fixpoint_kernel=3)
        assert e.value.status == lp.ERR_INVALID
