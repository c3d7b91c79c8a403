"""GPU parity of the many-program batch (lp_compile_batch / lp_batch_stable_models): every
program's stable bits over all 2^k guesses are compared bit for bit with the oracle's per-guess
Algorithms 2 and 3, on tiny random programs (with the degenerate ones: no rules, definite
programs, k = 0), on a reduced batch of the uneven-size workload, and, at the full 1000-program
size the benchmark times, against the oracle for every program and the single-program entry
point for a sample."""
import numpy as np
import pytest

import oracle
import paper_2009_10247_gb300 as lp
from tests.helpers import bits_to_bool
from workloads import Program, normal_program, parse, program_batch, small_definite, tiny_random

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import DEV, gpu_stable  # noqa: E402


def _run_batch(progs, host=False, max_iters=1 << 30, full_sweep=False, from_m0=False):
    with lp.Batch(progs, full_sweep=full_sweep, from_m0=from_m0) as B:
        n = B.n_programs
        if host:
            mask = np.zeros(max(B.total_mask_words, 1), dtype=np.uint64)
            ns = np.zeros(max(n, 1), dtype=np.int64)
            it = np.zeros(max(n, 1), dtype=np.int32)
            B.stable_models(mask, ns, it, max_iters=max_iters)
        else:
            mask_t = torch.zeros(max(B.total_mask_words, 1), dtype=torch.int64, device=DEV)
            ns_t = torch.zeros(max(n, 1), dtype=torch.int64, device=DEV)
            it_t = torch.zeros(max(n, 1), dtype=torch.int32, device=DEV)
            B.stable_models(mask_t, ns_t, it_t, max_iters=max_iters)
            torch.cuda.synchronize()
            mask, ns, it = mask_t.cpu().numpy().view(np.uint64), ns_t.cpu().numpy(), it_t.cpu().numpy()
        out = []
        for p in range(n):
            ng = 1 << B.k[p]
            w = (ng + 63) // 64
            out.append(bits_to_bool(mask[B.mask_offset[p]:B.mask_offset[p] + w], ng))
        return out, ns[:n], it[:n], B


def _check_oracle(progs, got, ns):
    for p, prog in enumerate(progs):
        st4, _, _ = oracle.stable_models_alg23(prog)
        assert np.array_equal(got[p], st4), f"program {p}"
        assert ns[p] == int(st4.sum())


@pytest.mark.parametrize("full_sweep", [False, True])
def test_tiny_random_programs(full_sweep):
    rng = np.random.default_rng(77)
    progs = []
    for s in range(60):
        progs.append(tiny_random(5000 + s, n_atoms=int(rng.integers(2, 50)), n_rules=int(rng.integers(1, 100)),
                                 max_body=4, p_fact=0.15, p_neg=0.12))
    progs += [parse("p :- not q. q :- not p."), parse("p :- not p."), small_definite(1),
              parse("a :- not b. b :- not a. c :- a. c :- b.")]
    got, ns, _, _ = _run_batch(progs, full_sweep=full_sweep)
    _check_oracle(progs, got, ns)


@pytest.mark.parametrize("full_sweep", [False, True])
def test_degenerate_programs(full_sweep):
    empty = Program(n_atoms=3, head=np.zeros(0, np.int64), body_off=np.zeros(1, np.int64),
                    body_atom=np.zeros(0, np.int64), body_neg=None)
    progs = [empty, parse("p."), parse("p :- not q. q :- not p."), empty]
    got, ns, it, _ = _run_batch(progs, full_sweep=full_sweep)
    _check_oracle(progs, got, ns)
    assert all(i >= 1 for i in it)


def test_empty_batch():
    got, ns, _, B = _run_batch([])
    assert got == [] and B.total_rows == 0


def test_host_buffers_match_device():
    progs = program_batch(seed=3, count=24, n_lo=50, n_hi=1500)
    a, na, ia, _ = _run_batch(progs)
    b, nb, ib, _ = _run_batch(progs, host=True)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert np.array_equal(na, nb) and np.array_equal(ia, ib)
    _check_oracle(progs, a, na)


@pytest.mark.parametrize("full_sweep", [False, True])
def test_reduced_uneven_batch_against_oracle(full_sweep):
    # the uneven-size workload's generator with smaller programs (oracle cost)
    progs = program_batch(seed=11, count=40, n_lo=100, n_hi=3000)
    got, ns, _, _ = _run_batch(progs, full_sweep=full_sweep)
    _check_oracle(progs, got, ns)


def _chain(length=20):
    # one guessed atom whose guess 1 makes a chain of `length` rules fire one after another: from
    # F (every guessed row zero) that column needs length + 2 iterations
    text = "p0 :- not q. " + " ".join(f"p{i + 1} :- p{i}." for i in range(length))
    return parse(text)


def test_no_fixpoint_reports_error():
    with pytest.raises(lp.LPError):  # Algorithm 2 from M_0: 86 theta applications
        _run_batch([small_definite(2)], max_iters=2, from_m0=True)
    with pytest.raises(lp.LPError):  # from F: more than 20 in the guessed column
        _run_batch([_chain()], max_iters=2)
    got, ns, it, _ = _run_batch([_chain(), small_definite(2)])
    assert it[0] > 20 and it[1] == 1  # a definite program is at F already: one confirming pass
    _check_oracle([_chain(), small_definite(2)], got, ns)


def test_too_many_guesses_rejected():
    # 17 negated atoms that are not facts: k = 17 > 16
    p = parse(" ".join(f"p{i} :- not q{i}." for i in range(17)))
    with pytest.raises(lp.LPError):
        lp.Batch([parse("p :- not q."), p])


def test_full_uneven_batch():
    # the benchmark's workload: 1000 programs, 100..20000 atoms, 3 rules per atom, k in 4..8;
    # every program against the oracle (about 30 s of CPU), and every 20th against the
    # single-program entry point
    progs = program_batch(seed=1)
    got, ns, it, B = _run_batch(progs)
    assert B.n_programs == 1000
    _check_oracle(progs, got, ns)
    for p in range(0, 1000, 20):
        with lp.Program.from_program(progs[p]) as P:
            st, _, n1 = gpu_stable(P)
        assert np.array_equal(got[p], st), f"program {p}"
        assert ns[p] == n1


def test_more_programs_than_one_launch():
    # 4100 programs: two cooperative launches (up to 4096 programs each)
    rng = np.random.default_rng(5)
    progs = [tiny_random(9000 + s, n_atoms=int(rng.integers(2, 30)), n_rules=int(rng.integers(1, 50)), max_body=3,
                         p_fact=0.2, p_neg=0.15) for s in range(4100)]
    got, ns, it, _ = _run_batch(progs)
    _check_oracle(progs, got, ns)
    assert np.all(it >= 1)


@pytest.mark.parametrize("full_sweep", [False, True])
def test_single_and_few_large_programs(full_sweep):
    # one program alone takes the whole batch's work: it runs as one job on many blocks that
    # meet at the job's barrier; two programs of very different sizes split the blocks
    one = [normal_program(seed=21, n=4000, n_rules=12000, k=7, per_atom=2)]
    got, ns, it, _ = _run_batch(one, full_sweep=full_sweep)
    _check_oracle(one, got, ns)
    two = [normal_program(seed=22, n=6000, n_rules=18000, k=8, per_atom=2), parse("p :- not q. q :- not p.")]
    got, ns, it, _ = _run_batch(two, full_sweep=full_sweep)
    _check_oracle(two, got, ns)
    assert np.all(it >= 1)


def test_frontier_equals_full_sweep():
    # the frontier schedule (programs with k <= 8) against the full sweep on the same programs:
    # from M_0 the same stable masks and the same per-program iteration counts, from F (the
    # default) the same masks in at most as many iterations; programs of k = 9 and 10 (rows wider
    # than 32 bytes, full sweep in all three) mixed in; and the frontier evaluates far fewer rows
    # than the full sweeps would
    progs = program_batch(seed=13, count=60, n_lo=100, n_hi=4000)
    progs += [normal_program(seed=31, n=2000, n_rules=6000, k=9, per_atom=2),
              normal_program(seed=32, n=1500, n_rules=4500, k=10, per_atom=2)]
    a, na, ia, _ = _run_batch(progs, from_m0=True)
    b, nb, ib, _ = _run_batch(progs, full_sweep=True)
    f, nf, itf, _ = _run_batch(progs)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert all(np.array_equal(x, y) for x, y in zip(f, b))
    assert np.array_equal(na, nb) and np.array_equal(ia, ib) and np.array_equal(nf, nb)
    assert np.all(itf >= 1) and np.all(itf <= ib) and np.array_equal(itf[-2:], ib[-2:])
    _check_oracle(progs[-2:], a[-2:], na[-2:])
    with lp.Batch(progs[:60]) as B:
        m = torch.zeros(max(B.total_mask_words, 1), dtype=torch.int64, device=DEV)
        B.stable_models(m)
        torch.cuda.synchronize()
        rows = B.last_stats()["rows_evaluated"]
    full_rows = sum(int(i) * inf["n_prime"] for i, inf in zip(ib[:60], B.info))
    assert 0 < rows < full_rows


def test_frontier_no_fixpoint_reports_error():
    with pytest.raises(lp.LPError):
        _run_batch([normal_program(seed=21, n=400, n_rules=1200, k=5, per_atom=2)], max_iters=1, from_m0=True)


def _solve(B, max_iters=1 << 30):
    n = B.n_programs
    mask_t = torch.zeros(max(B.total_mask_words, 1), dtype=torch.int64, device=DEV)
    ns_t = torch.zeros(max(n, 1), dtype=torch.int64, device=DEV)
    it_t = torch.zeros(max(n, 1), dtype=torch.int32, device=DEV)
    B.stable_models(mask_t, ns_t, it_t, max_iters=max_iters)
    torch.cuda.synchronize()
    return mask_t.cpu().numpy().copy(), ns_t.cpu().numpy()[:n].copy(), it_t.cpu().numpy()[:n].copy()


@pytest.mark.parametrize("from_m0", [True, False])
def test_frontier_repeated_solves_keep_rest_state(from_m0):
    # one handle, several solves: the frontier's buffers rest between solves (at M_0's guess-
    # independent part, or at F) and each solve restores the rows it changed; a solve stopped by
    # max_iters leaves the handle usable
    progs = program_batch(seed=17, count=30, n_lo=100, n_hi=3000) + [_chain()]
    with lp.Batch(progs, full_sweep=True) as F:
        ref = _solve(F)
    assert ref[2].max() > 2

    def same(got):
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
        if from_m0:
            assert np.array_equal(got[2], ref[2])
        else:
            assert np.all(got[2] >= 1) and np.all(got[2] <= ref[2])

    with lp.Batch(progs, from_m0=from_m0) as B:
        for _ in range(3):
            same(_solve(B))
        with pytest.raises(lp.LPError):
            _solve(B, max_iters=2)
        for _ in range(2):
            same(_solve(B))
