"""The standardization on the GPU (LP_COMPILE_ON_DEVICE, the default of lp_compile above 65,536
rules plus body literals) against the host compiler (LP_COMPILE_ON_HOST): the same matrix of Sec. 2.1-2.2 (Eq. 4 barred atoms, bodies as sets, OR
rules for heads with several rules, Def. 2 / Def. 7 rows) in the same internal order, array for
array, on programs that reach every branch: negation, facts, duplicate body atoms, multi-rule
heads, bodies long enough for the sorted-segment path, atoms that head nothing, empty programs;
and the same errors for malformed input."""
import numpy as np
import pytest

import oracle
import paper_2009_10247_gb300 as lp
from workloads import (from_rules, large_definite, normal_program, parse, small_definite, table1_program, tiny_random,
                       transitive_closure)
from workloads.programs import _pack

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import gpu_least_model, gpu_stable  # noqa: E402

INFO_KEYS = ("n_atoms", "n_rules", "n_prime", "nnz", "n_barred", "n_aux", "k", "n_fact_rows", "n_and_rows",
             "n_or_rows")


def _same_compile(prog):
    with lp.Program.from_program(prog, on_device=True) as D, lp.Program.from_program(prog, on_host=True) as H:
        for key in INFO_KEYS:
            assert D.info[key] == H.info[key], key
        for name in lp.Program.INTERNAL:
            a, b = D.debug_internal(name), H.debug_internal(name)
            assert a.shape == b.shape and np.array_equal(a, b), name
        md, mh = D.export_matrix(), H.export_matrix()
        for key in md:
            assert np.array_equal(md[key], mh[key]), key
        assert D.schedule == H.schedule


def _long_bodies(seed=3, n=5000):
    # bodies of 33 .. 2000 literals with repeats and negations, next to short ones
    rng = np.random.default_rng(seed)
    heads, lens, atoms, negs = [], [], [], []
    for r in range(400):
        m = int(rng.choice([0, 1, 3, 31, 32, 33, 40, 200, 2000]))
        heads.append(int(rng.integers(0, n)))
        lens.append(m)
        a = rng.integers(0, n // 3, m)  # many repeats
        atoms.append(a)
        negs.append((rng.random(m) < 0.05).astype(np.uint8))
    return _pack(n, np.array(heads), np.array(lens), np.concatenate(atoms), np.concatenate(negs))


PROGRAMS = {
    "chain": lambda: parse("a. b :- a. c :- a, b. d :- c. e :- d. f :- e, a. g :- f."),
    "negation": lambda: parse("p :- not q. q :- not p. r :- p. r :- q. t :- not t, r."),
    "choice": lambda: parse(" ".join(f"a{i} :- not b{i}. b{i} :- not a{i}. c :- a{i}." for i in range(5))),
    "small_definite": lambda: small_definite(2),
    "transitive_closure": lambda: transitive_closure(200, seed=3),
    "normal": lambda: normal_program(seed=4, n=3000, n_rules=9000, k=12, per_atom=2),
    "dense_table3": lambda: table1_program(6101, 1000, 5000, dense=True, k=7),
    "long_bodies": _long_bodies,
    "large_definite_1e5": lambda: large_definite(seed=2, n=100_000, n_rules=500_000, chain_levels=100,
                                                 chain_width=20),
    "no_rules": lambda: from_rules(5, []),
    "only_facts": lambda: from_rules(4, [(0, []), (2, []), (2, [])]),
}


@pytest.mark.parametrize("name", sorted(PROGRAMS))
def test_device_compile_equals_host_compile(name):
    _same_compile(PROGRAMS[name]())


def test_device_compile_equals_host_compile_tiny_random():
    rng = np.random.default_rng(11)
    for s in range(40):
        _same_compile(tiny_random(9000 + s, n_atoms=int(rng.integers(1, 40)), n_rules=int(rng.integers(0, 80)),
                                  max_body=5, p_fact=0.2, p_neg=0.2))


def test_empty_program():
    _same_compile(from_rules(0, []))


def test_solves_on_a_device_compiled_handle():
    # the least model and the stable set of programs compiled on the device, against the oracle
    for prog in (PROGRAMS["long_bodies"](), PROGRAMS["dense_table3"](), small_definite(3)):
        want, want_it = oracle.least_model(prog)
        with lp.Program.from_program(prog, on_device=True) as P:
            got, it = gpu_least_model(P)
        assert it == want_it and np.array_equal(got, want)
    prog = PROGRAMS["normal"]()
    st4, _, _ = oracle.stable_models_alg23(prog)
    with lp.Program.from_program(prog, on_device=True) as P:
        st, _, ns = gpu_stable(P)
    assert np.array_equal(st, st4) and ns == int(st4.sum())


@pytest.mark.parametrize("bad", ["head", "atom", "offsets"])
def test_malformed_program_same_error(bad):
    head = np.array([0, 1, 2], np.int32)
    off = np.array([0, 1, 3, 3], np.int64)
    atom = np.array([1, 0, 2], np.int32)
    if bad == "head":
        head[1] = 7
    elif bad == "atom":
        atom[2] = -1
    else:
        off[2] = 0
    msgs = []
    for kw in ({"on_device": True}, {"on_host": True}, {}):
        with pytest.raises(lp.LPError) as e:
            lp.Program(3, head, off, atom, **kw)
        assert e.value.status == lp.ERR_INVALID
        msgs.append(str(e.value))
    assert msgs[0] == msgs[1] == msgs[2]


def test_host_side_users_of_a_device_compile():
    # the streamed kernel's layout (built on the host from perm and the row kinds), the LP_ROWS
    # mode (the inverse permutation) and lp_export_matrix fetch the tables they need on demand
    prog = small_definite(5)
    want, want_it = oracle.least_model(prog)
    s = oracle.standardize(prog)
    with lp.Program.from_program(prog, on_device=True) as P, lp.Program.from_program(prog, on_host=True) as H:
        P.set_schedule(fixpoint_kernel=1, fixpoint_stage=0)
        got, it = gpu_least_model(P)
        assert it == want_it and np.array_equal(got, want)
        v0 = np.random.default_rng(1).random(s.n_prime) < 0.3
        want_rows, want_it_r, ok = oracle.alg1(s, v0.astype(np.uint8), max_iters=500)
        if ok:
            rows, it_r = gpu_least_model(P, init=v0, rows=True, max_iters=500)
            assert it_r == want_it_r and np.array_equal(rows, want_rows.astype(bool))
        md, mh = P.export_matrix(), H.export_matrix()
        assert all(np.array_equal(md[k], mh[k]) for k in md)


def test_small_program_default_compile():
    # a program of at most 16,384 rules plus body literals is standardized on one host thread by
    # default; the handle equals the device-compiled one and solves as the oracle does
    prog = small_definite(4)
    assert prog.n_rules + int(prog.body_off[-1]) <= 1 << 14
    want, want_it = oracle.least_model(prog)
    with lp.Program.from_program(prog) as P, lp.Program.from_program(prog, on_device=True) as D:
        for name in lp.Program.INTERNAL:
            assert np.array_equal(P.debug_internal(name), D.debug_internal(name)), name
        assert P.schedule == D.schedule
        got, it = gpu_least_model(P)
    assert it == want_it and np.array_equal(got, want)
