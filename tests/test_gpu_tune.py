"""Schedules and the autotuner on the GPU: every schedule (both least-model kernels at several
residencies, every stable tile width) gives the oracle's least model and stable bits, and
lp_autotune keeps the fastest candidate it timed, after checking that all candidates agree."""
import numpy as np
import pytest

import oracle
import paper_2009_10247_gb300 as lp
from workloads import large_definite, normal_program, small_definite, table1_program, tiny_random

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import gpu_least_model, gpu_stable  # noqa: E402


@pytest.mark.parametrize("kernel,bpsm,split,xn,rmap", [
    (0, 0, 1, 1, 0), (0, 2, 1, 1, 0), (0, 1, 1, 1, 0), (0, 0, 2, 1, 0), (0, 0, 4, 1, 0), (0, 3, 8, 1, 0),
    (0, 0, 1, 4, 0), (0, 0, 2, 4, 0), (0, 2, 8, 4, 0), (0, 0, 1, 1, 1), (0, 1, 1, 1, 1), (0, 0, 1, 1, 2),
    (0, 1, 1, 1, 2), (0, 0, 1, 1, 3), (0, 1, 1, 1, 3), (1, 0, 1, 1, 0), (1, 1, 1, 1, 0), (2, 0, 1, 1, 0),
    (2, 0, 1, 1, -1)])
def test_least_model_every_schedule(kernel, bpsm, split, xn, rmap):
    # the dense Table 1 shaped program has rows of about 50 entries: the thread-per-row maps
    # take their multi-pass paths there; the others fill fewer words than there are warps
    progs = [small_definite(2), tiny_random(77, n_atoms=40, n_rules=90, max_body=4, p_fact=0.2),
             large_definite(seed=3, n=20_000, n_rules=100_000, chain_levels=60, chain_width=20),
             table1_program(31, 1000, 5000, dense=True), table1_program(32, 1600, 24000)]
    for prog in progs:
        want, want_it = oracle.least_model(prog)
        with lp.Program.from_program(prog) as P:
            # rmap -1: kernel 2 gathering from global memory (no staged prefix)
            P.set_schedule(fixpoint_kernel=kernel, fixpoint_blocks_per_sm=bpsm, fixpoint_row_split=split,
                           fixpoint_chunk_batch=xn, fixpoint_row_map=max(rmap, 0), fixpoint_stage=int(rmap < 0))
            got, it = gpu_least_model(P)
        assert it == want_it and np.array_equal(got, want)


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("W", [1, 2, 4, 8, 16, 32])
def test_stable_models_every_tile_width(W, split):
    progs = [normal_program(seed=4, n=3000, n_rules=9000, k=12, per_atom=2),
             table1_program(6101, 1000, 5000, dense=True, k=7)]
    for prog in progs:
        st4, _, _ = oracle.stable_models_alg23(prog)
        with lp.Program.from_program(prog) as P:
            P.set_schedule(stable_tile_words=W, stable_blocks_per_sm=0 if W < 8 else 1, stable_row_split=split,
                           stable_frontier=0)
            st, _, ns = gpu_stable(P)
        assert np.array_equal(st, st4) and ns == int(st4.sum())


def test_autotune_keeps_fastest_and_stays_exact():
    prog = normal_program(seed=5, n=4000, n_rules=12000, k=10, per_atom=2)
    st4, _, _ = oracle.stable_models_alg23(prog)
    want, want_it = oracle.least_model(prog)
    with lp.Program.from_program(prog) as P:
        recs = P.autotune(lp.LP_TUNE_LEAST | lp.LP_TUNE_STABLE, reps=2)
        sched = P.schedule
        least = [r for r in recs if r["solve"] == "least"]
        stable = [r for r in recs if r["solve"] == "stable"]
        assert len(least) >= 10 and len(stable) >= 2 and all(r["ms"] >= 0 for r in recs)
        assert {r["fixpoint_row_split"] for r in least} == {1, 2, 4, 8}
        assert {r["fixpoint_row_map"] for r in least} == {0, 1, 2, 3}
        assert {0, 1, 2} <= {r["fixpoint_kernel"] for r in least}
        bl, bs = min(least, key=lambda r: r["ms"]), min(stable, key=lambda r: r["ms"])
        keys = ("fixpoint_kernel", "fixpoint_blocks_per_sm", "fixpoint_row_split", "fixpoint_chunk_batch",
                "fixpoint_row_map", "fixpoint_stage")
        assert all(sched[k] == bl[k] for k in keys)
        assert (sched["stable_tile_words"], sched["stable_blocks_per_sm"]) == (bs["stable_tile_words"],
                                                                              bs["stable_blocks_per_sm"])
        # k = 10: 16 guess words, so tiles wider than 16 words are not candidates
        assert max(r["stable_tile_words"] for r in stable) == 16
        st, _, ns = gpu_stable(P)
        got, it = gpu_least_model(P)
    assert np.array_equal(st, st4) and ns == int(st4.sum())
    assert it == want_it and np.array_equal(got, want)


def test_autotune_choice_is_min_of_records():
    prog = large_definite(seed=4, n=50_000, n_rules=200_000, chain_levels=40, chain_width=30)
    with lp.Program.from_program(prog) as P:
        recs = P.autotune(lp.LP_TUNE_LEAST, reps=2)
        best = min(recs, key=lambda r: r["ms"])
        s = P.schedule
        assert (s["fixpoint_kernel"], s["fixpoint_blocks_per_sm"]) == (best["fixpoint_kernel"],
                                                                      best["fixpoint_blocks_per_sm"])
        assert {r["fixpoint_kernel"] for r in recs} == {0, 1, 2}  # too large for kernel 3


def test_autotune_includes_block_kernel_where_it_fits():
    # kernel 3 (one block, matrix in shared memory) is a candidate exactly when the program fits it
    for prog, fits in ((small_definite(3), True),
                       (large_definite(seed=4, n=50_000, n_rules=200_000, chain_levels=40, chain_width=30), False)):
        want, want_it = oracle.least_model(prog)
        with lp.Program.from_program(prog) as P:
            recs = P.autotune(lp.LP_TUNE_LEAST, reps=1)
            assert (3 in {r["fixpoint_kernel"] for r in recs}) == fits
            got, it = gpu_least_model(P)
        assert it == want_it and np.array_equal(got, want)
