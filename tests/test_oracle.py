"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test compares the oracle with something other than itself: the matrices and arrays
the paper prints (Examples 1-4), hand derivations of Algorithm 1 on Example 1, brute force
over all interpretations of tiny programs, textbook stable-model cases, BFS reachability,
and invariants of the least fixpoint.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests.helpers import frac_matrix, golden, is_model
from workloads import (from_rules, normal_program, parse, small_definite, tiny_random,
                       transitive_closure)


def _exact_matrix(std):
    M = [[Fraction(0)] * std.n_prime for _ in range(std.n_prime)]
    for i in range(std.n_prime):
        for e in range(std.row_ptr[i], std.row_ptr[i + 1]):
            M[i][std.col[e]] = Fraction(int(std.num[e]), int(std.den[i]))
    return M


# ---------------------------------------------------------------- paper's worked examples

def test_example1_matrix_coo_csr():
    g = golden("example1.json")
    p = parse(g["program"], atoms=g["atoms"])
    s = oracle.standardize(p)
    assert s.n_prime == len(g["standardized_atoms"]) == 7
    assert _exact_matrix(s) == frac_matrix(g["matrix"])  # Example 1
    assert s.coo_rows().tolist() == g["coo_row_index"]  # Example 3
    assert s.col.tolist() == g["coo_col_index"] == g["csr_col_index"]
    assert s.values().tolist() == g["coo_value"] == g["csr_value"]
    assert s.row_ptr.tolist() == g["csr_row_index"]  # Example 4


def test_example2_matrix():
    g = golden("example2.json")
    p = parse(g["program"], atoms=g["atoms"])
    s = oracle.standardize(p)
    assert _exact_matrix(s) == frac_matrix(g["matrix"])  # Example 2, Def. 7
    assert s.n_barred == 1 and s.kind[6] == oracle.ORC_BARRED and s.owner[6] == 3


def test_example1_iterates_by_hand():
    # Algorithm 1 on Example 1, derived by hand from the printed matrix:
    # v0 = {s,t} (Def. 4); theta(M v0) = {q,r,s,t,v}; then {p,q,r,s,t,u,v}; then unchanged.
    g = golden("example1.json")
    p = parse(g["program"], atoms=g["atoms"])
    s = oracle.standardize(p)
    idx = {a: i for i, a in enumerate(g["standardized_atoms"])}
    vec = lambda atoms: np.array([1 if a in atoms else 0 for a in g["standardized_atoms"]], np.uint8)  # noqa
    v0 = oracle.initial_vector(s)
    assert v0.tolist() == vec("st").tolist()
    v1 = oracle.theta_step(s, v0)
    assert v1.tolist() == vec("qrstv").tolist()
    v2 = oracle.theta_step(s, v1)
    assert v2.tolist() == vec("pqrstuv").tolist()
    assert oracle.theta_step(s, v2).tolist() == v2.tolist()
    v, iters, ok = oracle.alg1(s, v0)
    assert ok and iters == 3 and v.tolist() == v2.tolist()
    assert idx["u"] == 5 and idx["v"] == 6


def test_example2_stable_model_is_t():
    g = golden("example2.json")
    p = parse(g["program"], atoms=g["atoms"])
    # t is a fact, so t-bar is forced to 0 (Def. 8 item 3): one column, h = 1.
    st, models, _ = oracle.stable_models_alg23(p)
    assert st.tolist() == [True]
    assert models[0].tolist() == [a == "t" for a in g["atoms"]]
    assert oracle.brute_stable_models(p) == [1 << g["atoms"].index("t")]


# ---------------------------------------------------------------- least model

@pytest.mark.parametrize("seed", range(60))
def test_least_model_three_ways(seed):
    rng = np.random.default_rng(seed)
    p = tiny_random(seed, n_atoms=int(rng.integers(1, 13)), n_rules=int(rng.integers(0, 25)),
                    max_body=4, p_fact=0.25)
    o3 = oracle.brute_least_model(p)
    o1, _ = oracle.tp_least_model(p)
    o2, iters = oracle.least_model(p)
    assert o1.tolist() == o3.tolist()
    assert o2.tolist() == o3.tolist()
    s = oracle.standardize(p)
    assert 1 <= iters <= s.n_prime + 1


@pytest.mark.parametrize("length", [1, 2, 7, 40])
def test_iteration_counts_in_closed_form(length):
    # a chain a_0. a_i <- a_{i-1}: a_i becomes true in theta application i, and one more
    # application shows no change, so length + 1 applications (Example 1 counts the same way)
    rules = [(0, [])] + [(i, [i - 1]) for i in range(1, length + 1)]
    got, iters = oracle.least_model(from_rules(length + 1, rules))
    assert got.all() and iters == length + 1
    # a rule joining the ends of two chains of lengths L and L // 2 fires one application
    # after the longer chain's end: L + 2 applications; a second rule for the same head that
    # also waits for that end turns it into an OR row over two new atoms, one more level: L + 3
    short = length // 2
    n = (length + 1) + (short + 1) + 1
    rules = ([(0, [])] + [(i, [i - 1]) for i in range(1, length + 1)] + [(length + 1, [])]
             + [(length + 1 + i, [length + i]) for i in range(1, short + 1)] + [(n - 1, [length, length + 1 + short])])
    got, iters = oracle.least_model(from_rules(n, rules))
    assert got.all() and iters == length + 2
    got, iters = oracle.least_model(from_rules(n, rules + [(n - 1, [length])]))
    assert got.all() and iters == length + 3


@pytest.mark.parametrize("seed", range(20))
def test_least_model_fact_subsets(seed):
    # An initial vector holding a subset of the facts computes the least model of the program
    # without the other fact rules (fact rows are self-loops, Def. 2 item 3).
    p = tiny_random(100 + seed, n_atoms=10, n_rules=20, max_body=3, p_fact=0.35)
    facts = p.fact_atoms()
    keep = facts & (np.random.default_rng(seed).random(p.n_atoms) < 0.5)
    o2, _ = oracle.least_model(p, init=keep)
    lens = np.diff(p.body_off)
    drop = (lens == 0) & ~keep[p.head]
    rules = [(int(p.head[r]), p.body_atom[p.body_off[r]:p.body_off[r + 1]].tolist())
             for r in range(p.n_rules) if not drop[r]]
    q = from_rules(p.n_atoms, rules)
    assert o2.tolist() == oracle.brute_least_model(q).tolist()


def test_fixpoint_invariants_small_definite():
    p = small_definite(3)
    s = oracle.standardize(p)
    v = oracle.initial_vector(s)
    prev = v
    iters = 0
    while True:
        u = oracle.theta_step(s, prev)
        iters += 1
        assert np.all(u >= prev), "iterates are monotone from the fact vector"
        if np.array_equal(u, prev):
            break
        prev = u
    vstar, it2, ok = oracle.alg1(s, v)
    assert ok and it2 == iters and np.array_equal(vstar, prev)
    assert np.array_equal(oracle.theta_step(s, vstar), vstar)  # T_P(I) = I
    model = vstar[: s.n].astype(bool)
    assert is_model(p, model)
    o1, _ = oracle.tp_least_model(p)
    assert np.array_equal(o1, model)
    assert iters >= 41  # 40 chain levels above the facts


def test_duplicate_body_atoms_are_a_set():
    # Footnote of Eq. 2 (distinct body atoms): p <- q & q must fire once q holds.
    p = from_rules(2, [(0, [1, 1]), (1, [])])
    assert oracle.least_model(p)[0].tolist() == [True, True]
    s = oracle.standardize(p)
    assert s.den[0] == 1 and s.row_ptr[1] - s.row_ptr[0] == 1


def test_exact_threshold_long_body():
    # Def. 5 with a_ij = 1/10: ten float additions of 0.1 fall short of 1, the exact sum does not.
    acc = 0.0
    for _ in range(10):
        acc += 0.1  # left-to-right float64 accumulation
    assert acc < 1.0
    rules = [(0, list(range(1, 11)))] + [(a, []) for a in range(1, 11)]
    p = from_rules(11, rules)
    assert oracle.least_model(p)[0][0]
    assert oracle.brute_least_model(p)[0]


def test_fact_that_heads_other_rules():
    # p <- (fact) and p <- q: the transform makes p an OR row over two new atoms.
    p = parse("p. p :- q. q :- r.", atoms=["p", "q", "r"])
    s = oracle.standardize(p)
    assert s.kind[0] == oracle.ORC_OR and s.n_aux == 2
    assert s.kind[3] == oracle.ORC_FACT and s.owner[3] == 0
    m, iters = oracle.least_model(p)
    assert m.tolist() == [True, False, False] and iters == 2


def test_oscillation_has_no_fixpoint_from_arbitrary_vector():
    # p <- q, q <- p from I = {p}: Algorithm 1 alternates {p},{q} (not an initial vector of
    # Def. 4, so the loop has no fixpoint to reach).
    p = parse("p :- q. q :- p.")
    s = oracle.standardize(p)
    v, iters, ok = oracle.alg1(s, np.array([1, 0], np.uint8), max_iters=50)
    assert not ok and iters == 50


def test_transitive_closure_matches_bfs():
    p = transitive_closure(30, 2.0, seed=7)
    N = p.meta["n_nodes"]
    E = len(p.meta["edges"])
    adj = [[] for _ in range(N)]
    for x, y in p.meta["edges"]:
        adj[x].append(y)
    reach = np.zeros((N, N), bool)
    for x in range(N):  # paths of length >= 1
        frontier = list(adj[x])
        seen = set()
        while frontier:
            y = frontier.pop()
            if y in seen:
                continue
            seen.add(y)
            frontier.extend(adj[y])
        for y in seen:
            reach[x, y] = True
    m, _ = oracle.least_model(p)
    assert np.array_equal(m[E:].reshape(N, N), reach)
    assert np.all(m[:E])


# ---------------------------------------------------------------- stable models

def _models_of(prog, st, models):
    return sorted(int(sum(1 << a for a in np.nonzero(models[i])[0])) for i in np.nonzero(st)[0])


@pytest.mark.parametrize("text,expected", [
    ("p :- not q. q :- not p.", [["p"], ["q"]]),
    ("p :- not p.", []),
    ("p :- not q.", [["p"]]),
    ("a. b :- a. c :- b, a.", [["a", "b", "c"]]),
    ("p :- not q. q :- not r. r :- not p.", []),
    ("a :- not b. b :- not a. c :- a. c :- b.", [["a", "c"], ["b", "c"]]),
])
def test_textbook_stable_models(text, expected):
    p = parse(text)
    names = p.names
    want = sorted(sum(1 << names.index(a) for a in m) for m in expected)
    st4, m4, _ = oracle.stable_models_alg23(p)
    st5, m5 = oracle.stable_models_gl(p)
    assert _models_of(p, st4, m4) == want
    assert _models_of(p, st5, m5) == want
    assert oracle.brute_stable_models(p) == want


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_stable_model_counts_in_closed_form(n):
    # n independent even loops a_i <- not b_i, b_i <- not a_i: each picks one atom, 2^n models
    # (every combination); adding n odd loops p_i <- not q_i, q_i <- not r_i, r_i <- not p_i
    # leaves none; adding instead f <- a_0, not f removes the models with a_0: 2^(n-1)
    pairs = " ".join(f"a{i} :- not b{i}. b{i} :- not a{i}." for i in range(n))
    p = parse(pairs)
    st, models, _ = oracle.stable_models_alg23(p)
    got = _models_of(p, st, models)
    names = p.names
    want = sorted(sum(1 << names.index((f"a{i}" if (c >> i) & 1 else f"b{i}")) for i in range(n))
                  for c in range(1 << n))
    assert got == want
    odd = " ".join(f"p{i} :- not q{i}. q{i} :- not r{i}. r{i} :- not p{i}." for i in range(n))
    st, _, _ = oracle.stable_models_alg23(parse(pairs + " " + odd))
    assert int(st.sum()) == 0
    p = parse(pairs + " f :- a0, not f.")
    st, models, _ = oracle.stable_models_alg23(p)
    assert int(st.sum()) == 1 << (n - 1)
    a0 = p.names.index("a0")
    assert not any(models[i][a0] for i in np.nonzero(st)[0])


@pytest.mark.parametrize("seed", range(40))
def test_stable_models_alg23_equals_gl_and_brute(seed):
    rng = np.random.default_rng(1000 + seed)
    p = tiny_random(1000 + seed, n_atoms=int(rng.integers(2, 11)), n_rules=int(rng.integers(1, 16)),
                    max_body=3, p_fact=0.2, p_neg=0.35)
    st4, m4, _ = oracle.stable_models_alg23(p)
    st5, m5 = oracle.stable_models_gl(p)
    assert np.array_equal(st4, st5)
    assert np.array_equal(m4, m5)  # same least model of P+ with the guess, for every guess
    assert _models_of(p, st4, m4) == oracle.brute_stable_models(p)


def test_definite_program_has_its_least_model_as_only_stable_model():
    p = small_definite(5)
    st, models, _ = oracle.stable_models_alg23(p)
    assert st.tolist() == [True]
    assert np.array_equal(models[0], oracle.least_model(p)[0])


def test_normal_program_generator_shape():
    p = normal_program(seed=3, n=2000, n_rules=6000, k=6, per_atom=2)
    s = oracle.standardize(p)
    assert len(s.guess_rows()) == 6 and s.n_barred == 6
    st4, m4, it4 = oracle.stable_models_alg23(p, guesses=np.arange(64, dtype=np.uint64))
    st5, m5 = oracle.stable_models_gl(p, guesses=np.arange(0, 64, 7, dtype=np.uint64))
    assert np.array_equal(st4[::7], st5) and np.array_equal(m4[::7], m5)


@pytest.mark.parametrize("seed", range(12))
def test_iteration_from_guess_independent_fixpoint(seed):
    # The reading behind the default stable schedule: F, the fixpoint from the fact rows with every
    # guessed row zero, lies below every column's least fixpoint, so Algorithm 2 started from F with
    # the guess's bits on the guessed rows reaches the column's fixpoint of Algorithm 2 from M_0 --
    # the same stable bits and models -- in at most as many iterations.
    rng = np.random.default_rng(900 + seed)
    prog = tiny_random(900 + seed, n_atoms=int(rng.integers(3, 40)), n_rules=int(rng.integers(2, 90)), max_body=4,
                       p_fact=0.15, p_neg=0.15)
    s = oracle.standardize(prog)
    rows = s.guess_rows()
    v0 = oracle.initial_vector(s)
    assert not v0[rows].any()  # guessed rows are zero in the fact vector
    F, _, ok = oracle.alg1(s, v0)
    assert ok
    st4, _, it4 = oracle.stable_models_alg23(prog)
    for g in range(1 << len(rows)):
        m0 = v0.copy()
        bits = np.array([(g >> j) & 1 for j in range(len(rows))], dtype=np.uint8)
        m0[rows] = bits
        fix0, it0, ok0 = oracle.alg1(s, m0)
        start = F.copy()
        start[rows] = bits
        assert np.all(m0 <= start) and np.all(start <= fix0)  # M_0 <= S <= the column's fixpoint
        fixF, itF, okF = oracle.alg1(s, start)
        assert ok0 and okF and np.array_equal(fixF, fix0), g
        assert itF <= it0 == it4[g]
        # Algorithm 3 on the fixpoint from F gives the oracle's stable bit
        q = np.nonzero(s.kind == oracle.ORC_BARRED)[0]
        atom_rows = s.owner[q]
        assert bool(np.all(fixF[atom_rows] != fixF[q])) == bool(st4[g])
