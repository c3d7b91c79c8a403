"""GPU parity of the stable-model path (Algorithms 2 and 3 in liblp) against the oracle.

The stable bit of every guess and every returned model are compared bit for bit with the
oracle's per-guess Algorithm 2/3 (and its Gelfond-Lifschitz check), on the paper's example,
textbook programs, tiny random normal programs, multi-tile runs, explicit guess lists, and
the full-size 2^16-guess workload in the configuration the benchmark times (every one of the
65,536 stable bits against the oracle's Algorithms 2/3, per-tile iteration counts, and a reduct
check of the models found)."""
import os

import numpy as np
import pytest

import oracle
import paper_2009_10247_gb300 as lp
from tests.helpers import golden, program_fingerprint
from workloads import normal_program, parse, small_definite, table1_program, tiny_random

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import dev_words, gpu_stable  # noqa: E402


def _parity(prog, guesses=None, max_models=64):
    # every schedule: the full sweep per tile, the frontier over all tiles from M_0, and the
    # frontier from the guess-independent fixpoint F (the default)
    st4, m4, _ = oracle.stable_models_alg23(prog, guesses=guesses)
    want_models = m4[st4]
    with lp.Program.from_program(prog) as P:
        for frontier in (0, 1, 2):
            P.set_schedule(stable_frontier=frontier)
            st, models, ns = gpu_stable(P, guesses=guesses, max_models=max_models)
            assert np.array_equal(st, st4), f"frontier={frontier}"
            assert ns == int(st4.sum()), f"frontier={frontier}"
            assert np.array_equal(models, want_models[:max_models]), f"frontier={frontier}"
    return st, models


def test_example2():
    g = golden("example2.json")
    st, models = _parity(parse(g["program"], atoms=g["atoms"]))
    assert st.tolist() == [True]
    assert models[0].tolist() == [a == "t" for a in g["atoms"]]


@pytest.mark.parametrize("text,n_models", [
    ("p :- not q. q :- not p.", 2), ("p :- not p.", 0), ("p :- not q.", 1),
    ("a :- not b. b :- not a. c :- a. c :- b.", 2), ("p :- not q. q :- not r. r :- not p.", 0),
])
def test_textbook(text, n_models):
    st, models = _parity(parse(text))
    assert st.sum() == n_models


@pytest.mark.parametrize("seed", range(30))
def test_tiny_random_normal(seed):
    rng = np.random.default_rng(2000 + seed)
    _parity(tiny_random(2000 + seed, n_atoms=int(rng.integers(2, 60)), n_rules=int(rng.integers(1, 120)),
                        max_body=4, p_fact=0.15, p_neg=0.1))


def test_definite_program_single_column():
    p = small_definite(2)
    st, models = _parity(p)
    assert st.tolist() == [True] and np.array_equal(models[0], oracle.least_model(p)[0])


@pytest.mark.parametrize("tile_bytes", [None, "1"])
def test_normal_program_all_guesses(tile_bytes, monkeypatch):
    # 1 byte of budget forces one 64-guess word per tile: many tiles, one launch
    if tile_bytes:
        monkeypatch.setenv("LP_TILE_BYTES", tile_bytes)
    p = normal_program(seed=5, n=3000, n_rules=9000, k=10, per_atom=3)
    _parity(p, max_models=8)


def test_choice_program_many_models():
    # k independent even loops a_i <- not b_i, b_i <- not a_i: 2^k stable models out of 4^k guesses
    k = 5
    text = " ".join(f"a{i} :- not b{i}. b{i} :- not a{i}. c :- a{i}." for i in range(k))
    st, models = _parity(parse(text), max_models=64)
    assert st.sum() == 2 ** k


def test_explicit_guesses():
    p = normal_program(seed=6, n=2000, n_rules=6000, k=12, per_atom=3)
    rng = np.random.default_rng(1)
    g = rng.integers(0, 1 << 12, 777).astype(np.uint64)
    g[:5] = g[0]  # duplicates are evaluated independently
    _parity(p, guesses=g, max_models=16)


def test_zero_guesses_and_host_buffers():
    p = parse("p :- not q. q :- not p.")
    with lp.Program.from_program(p) as P:
        mask = np.zeros(1, np.uint64)
        assert P.stable_models(mask, guesses=np.zeros(0, np.uint64), n_guesses=0) == 0
        models = np.zeros((4, 1), np.uint64)
        ns = P.stable_models(mask, models=models, max_models=4)
        assert ns == 2 and int(mask[0]) == 0b0110
        assert sorted(int(x) for x in models[:2, 0]) == [0b01, 0b10]


def test_full_size_2_16_guesses_sampled():
    # 1e5 atoms, 3e5 rules, k = 16: all 65,536 guesses on the GPU; the oracle checks a sample
    # of guesses with Algorithms 2/3 and every stable model found with the reduct.
    p = normal_program(seed=1)
    s = oracle.standardize(p)
    with lp.Program.from_program(p) as P:
        assert P.info["k"] == 16
        st, models, ns = gpu_stable(P, max_models=256)
        P.autotune(lp.LP_TUNE_STABLE, reps=1)  # the schedule the benchmark times
        st_t, models_t, ns_t = gpu_stable(P, max_models=256)
        assert np.array_equal(st_t, st) and ns_t == ns and np.array_equal(models_t, models)
    rng = np.random.default_rng(0)
    sample = np.unique(np.concatenate([rng.integers(0, 1 << 16, 96), np.nonzero(st)[0][:32], [0, 65535]]))
    st4, m4, _ = oracle.stable_models_alg23(p, guesses=sample.astype(np.uint64), std=s)
    assert np.array_equal(st[sample], st4)
    idx = np.nonzero(st)[0]
    assert ns == len(idx)
    if len(idx):
        st5, m5 = oracle.stable_models_gl(p, guesses=idx[:32].astype(np.uint64), std=s)
        assert st5.all()
        assert np.array_equal(models[:min(32, len(idx))], m5)


def _full_size_expected(prog):
    """Stable bits of all 2^16 guesses of normal_program(seed=1) by the oracle's Algorithms 2/3,
    and per 64-guess word the largest iteration count of its columns: stored by
    tests/golden/make_normal_program_stable.py, recomputed by the oracle (minutes) if the
    generator yields another program than the one stored."""
    g = golden("normal_program_seed1_stable.json")
    if g["fingerprint"] == program_fingerprint(prog):
        st = np.zeros(g["n_guesses"], dtype=bool)
        st[np.asarray(g["stable"], dtype=np.int64)] = True
        return st, np.asarray(g["word_max_iters"], dtype=np.int64)
    st, _, iters = oracle.stable_models_alg23(prog, want_models=False)
    return st, iters.reshape(-1, 64).max(axis=1)


def test_full_size_2_16_guesses_every_bit():
    # all 65,536 guesses in one call, default (frontier from F), full-sweep, tuned, frontier-from-
    # M_0 on the tuned width and frontier-from-F schedules: every stable bit equals the oracle's;
    # every tile's iteration count is the largest of its columns' counts (from M_0), or at most
    # that (from F)
    p = normal_program(seed=1)
    want, word_iters = _full_size_expected(p)
    assert len(want) == 1 << 16
    with lp.Program.from_program(p) as P:
        for variant in ("default", "full", "tuned", "frontier", "from_F"):
            if variant == "full":
                P.set_schedule(stable_frontier=0)
            if variant == "tuned":
                P.autotune(lp.LP_TUNE_STABLE, reps=1)  # the schedule the benchmark times
            if variant == "frontier":
                P.set_schedule(stable_frontier=1)  # on the tuned tile width
            if variant == "from_F":
                P.set_schedule(stable_frontier=2)
            st, _, ns = gpu_stable(P)
            assert np.array_equal(st, want), f"{variant}: {np.count_nonzero(st != want)} guesses differ"
            assert ns == int(want.sum())
            stats = P.last_stats()
            W = stats["tile_words"]
            per_tile = word_iters.reshape(-1, W).max(axis=1)
            assert stats["tiles"] == len(per_tile)
            if P.schedule["stable_frontier"] == 2:
                assert 1 <= stats["max_tile_iters"] <= per_tile.max()
                assert stats["sum_tile_iters"] <= per_tile.sum()
            else:
                assert stats["max_tile_iters"] == per_tile.max()
                assert stats["sum_tile_iters"] == per_tile.sum()
            if P.schedule["stable_frontier"] >= 1:  # re-evaluated rows: a few per cent of the full sweeps
                assert 0 < stats["frontier_rows"] < 0.2 * P.info["n_prime"] * per_tile.sum()


@pytest.mark.parametrize("W", [1, 2, 8, 32])
def test_frontier_schedule_matches_oracle(W):
    # the frontier schedule (after a tile's first iteration only rows with a changed input are
    # evaluated) gives the oracle's stable bits and models, and the full sweep's tile iterations
    progs = [normal_program(seed=4, n=3000, n_rules=9000, k=12, per_atom=2), parse("p :- not q. q :- not p."),
             parse("a :- not b. b :- not a. c :- a. c :- b."), small_definite(2)]
    rng = np.random.default_rng(9)
    progs += [tiny_random(7000 + s, n_atoms=int(rng.integers(2, 60)), n_rules=int(rng.integers(1, 120)), max_body=4,
                          p_fact=0.15, p_neg=0.1) for s in range(12)]
    for prog in progs:
        st4, m4, _ = oracle.stable_models_alg23(prog)
        with lp.Program.from_program(prog) as P:
            P.set_schedule(stable_tile_words=W, stable_frontier=0)
            _, _, _ = gpu_stable(P)
            full = P.last_stats()
            for mode in (1, 2):
                P.set_schedule(stable_frontier=mode)
                st, models, ns = gpu_stable(P, max_models=16)
                fr = P.last_stats()
                assert np.array_equal(st, st4) and ns == int(st4.sum()), mode
                assert np.array_equal(models, m4[st4][:16]), mode
                if mode == 1:  # Algorithm 2's iterates: its counts
                    assert (fr["max_tile_iters"], fr["sum_tile_iters"]) == (full["max_tile_iters"],
                                                                            full["sum_tile_iters"])
                else:  # from F: at most those
                    assert fr["max_tile_iters"] <= full["max_tile_iters"]
                    assert fr["sum_tile_iters"] <= full["sum_tile_iters"]


def _hub_program(seed, n=400, n_rules=1500, k=6):
    # normal program with hot atoms and long bodies: atoms 0-3 sit in every rule body (thousands of
    # dependents each), a third of the rules have 70-200 body atoms (rows a warp evaluates), the
    # rest 1-3; facts 10-39; k negated atoms as in the Table 5/6 programs
    rng = np.random.default_rng(seed)
    heads, bodies = [], []
    for a in range(10, 40):
        heads.append(a)
        bodies.append([])
    for r in range(n_rules):
        ln = int(rng.integers(70, 200)) if r % 3 == 0 else int(rng.integers(1, 4))
        body = set(rng.choice(np.arange(4, n), size=ln, replace=False).tolist()) | {r % 4}
        heads.append(int(rng.integers(0, n)))
        bodies.append(sorted(body))
    for a in range(4):  # the hubs become true early
        heads.append(a)
        bodies.append([10 + a])
    neg = rng.choice(np.arange(40, n), size=k, replace=False)
    text = []
    negated = set()
    for h, b in zip(heads, bodies):
        lits = []
        for x in b:
            if x in neg and x not in negated and len(b) > 1:
                negated.add(x)
                lits.append(f"not a{x}")
            else:
                lits.append(f"a{x}")
        text.append(f"a{h}." if not lits else f"a{h} :- {', '.join(lits)}.")
    return parse(" ".join(text), atoms=[f"a{i}" for i in range(n)])


@pytest.mark.parametrize("W", [1, 2, 4])
@pytest.mark.parametrize("wide_items", [None, "0", "3"])
def test_frontier_dense_rows_and_hot_atoms(W, wide_items, monkeypatch):
    # programs whose rows have up to ~200 entries (the long list: a warp per row) and whose atoms
    # have hundreds to thousands of dependents (pushed by the whole grid; with a wide list of 0 or
    # 3 slots the warps push what does not fit): the oracle's stable bits and models, and the full
    # sweep's tile iterations
    if wide_items is not None:
        monkeypatch.setenv("LP_FRONTIER_WIDE_ITEMS", wide_items)
    progs = [table1_program(61, 600, 1500, dense=True, k=6), table1_program(62, 1600, 4000, dense=True, k=8),
             _hub_program(63), _hub_program(64, k=8)]
    for prog in progs:
        st4, m4, _ = oracle.stable_models_alg23(prog)
        with lp.Program.from_program(prog) as P:
            P.set_schedule(stable_tile_words=W, stable_frontier=0)
            gpu_stable(P)
            full = P.last_stats()
            for mode in (1, 2, 1):  # a switch of mode rewrites the rest state in full
                P.set_schedule(stable_frontier=mode)
                for rep in range(2):  # the second solve starts from the rest state the first left
                    st, models, ns = gpu_stable(P, max_models=16)
                    fr = P.last_stats()
                    assert np.array_equal(st, st4) and ns == int(st4.sum()), (mode, rep)
                    assert np.array_equal(models, m4[st4][:16]), (mode, rep)
                    its = (fr["max_tile_iters"], fr["sum_tile_iters"])
                    if mode == 1:
                        assert its == (full["max_tile_iters"], full["sum_tile_iters"]), (mode, rep)
                    else:
                        assert its[0] <= full["max_tile_iters"] and its[1] <= full["sum_tile_iters"], rep


def test_frontier_schedule_explicit_guesses():
    p = normal_program(seed=6, n=2000, n_rules=6000, k=12, per_atom=3)
    g = np.random.default_rng(2).integers(0, 1 << 12, 500).astype(np.uint64)
    st4, _, _ = oracle.stable_models_alg23(p, guesses=g)
    with lp.Program.from_program(p) as P:
        P.set_schedule(stable_frontier=1)
        st, _, ns = gpu_stable(P, guesses=g)
    assert np.array_equal(st, st4) and ns == int(st4.sum())


def _frontier_tile_bytes(P, W):
    # one tile's share of the frontier buffers: two iterate buffers of W words per row, a stamp
    # and two list slots per row, the changed-row bitmap, a per-tile counter, the wide-item list
    # (n_pad / 16 + 64 slots) and 64 spare bytes
    n_pad = (P.info["n_prime"] + 63) // 64 * 64
    return 2 * n_pad * W * 8 + 12 * n_pad + (n_pad + 31) // 32 * 4 + 4 + (n_pad // 16 + 64) * 4 + 64


@pytest.mark.parametrize("mode", [1, 2])
def test_frontier_waves_and_rest_state(mode, monkeypatch):
    # One handle, many solves: all tiles in one wave, repeated (the buffers' rest state reused),
    # explicit guesses, waves of 1 and 3 tiles, a solve stopped by max_iters, another tile width,
    # from M_0 (mode 1) and from F (mode 2). Every solve gives the oracle's stable bits and models.
    prog = normal_program(seed=4, n=3000, n_rules=9000, k=12, per_atom=2)
    st_all, m_all, _ = oracle.stable_models_alg23(prog)
    g = np.random.default_rng(5).integers(0, 1 << 12, 700).astype(np.uint64)
    st_g, _, _ = oracle.stable_models_alg23(prog, guesses=g)

    def check_all(P, label):
        st, models, ns = gpu_stable(P, max_models=16)
        assert np.array_equal(st, st_all), label
        assert ns == int(st_all.sum()) and np.array_equal(models, m_all[st_all][:16]), label

    with lp.Program.from_program(prog) as P:
        P.set_schedule(stable_tile_words=2, stable_frontier=mode)  # 4096 guesses: 32 tiles of 2 words
        for rep in range(3):
            check_all(P, f"one wave, solve {rep}")
            assert P.last_stats()["tiles"] == 32
        st, _, ns = gpu_stable(P, guesses=g)
        assert np.array_equal(st, st_g) and ns == int(st_g.sum())
        check_all(P, "after explicit guesses")
        for c in (1, 3):
            monkeypatch.setenv("LP_FRONTIER_BYTES", str(c * _frontier_tile_bytes(P, 2)))
            check_all(P, f"waves of {c}")
            check_all(P, f"waves of {c}, again")
        monkeypatch.delenv("LP_FRONTIER_BYTES")
        mask = dev_words(1 << 12)
        with pytest.raises(lp.LPError) as e:
            P.stable_models(mask, max_iters=1)
        assert e.value.status == lp.ERR_NO_FIXPOINT
        check_all(P, "after a solve stopped by max_iters")
        P.set_schedule(stable_tile_words=8)
        check_all(P, "8-word tiles")
        P.set_schedule(stable_tile_words=2)
        check_all(P, "back to 2-word tiles")
