"""Failure detection without a GPU fault: the bounded grid barrier that every persistent
kernel meets once per iteration gives up after its limit when blocks never arrive, reports
LP_ERR_TIMEOUT through the device status, and leaves the context usable (a solve right after
it is still exact)."""
import numpy as np
import pytest

import oracle
import paper_2009_10247_gb300 as lp
from workloads import small_definite

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import gpu_least_model  # noqa: E402

LP_OK, LP_ERR_TIMEOUT = 0, 6


def test_barrier_completes_when_every_block_arrives():
    for blocks in (1, 2, 152, 304):
        st, ms = lp.check_grid_barrier(blocks, 0, 100_000)
        assert st == LP_OK and ms < 50


@pytest.mark.parametrize("blocks,absent", [(2, 1), (152, 1), (304, 37), (152, 151)])
def test_missing_blocks_time_out_and_context_survives(blocks, absent):
    st, ms = lp.check_grid_barrier(blocks, absent, 20_000)  # 20 ms limit
    assert st == LP_ERR_TIMEOUT
    assert 15 <= ms < 1000
    prog = small_definite(3)
    want, want_it = oracle.least_model(prog)
    with lp.Program.from_program(prog) as P:
        got, it = gpu_least_model(P)
    assert it == want_it and np.array_equal(got, want)


def test_rejects_non_resident_grid():
    with pytest.raises(lp.LPError):
        lp.check_grid_barrier(1 << 20, 0, 1000)


def test_check_matrix_on_device_copies():
    from workloads import normal_program, transitive_closure
    for prog in [small_definite(1), normal_program(seed=3, n=2000, n_rules=6000, k=6), transitive_closure(30, 2.0, 1)]:
        with lp.Program.from_program(prog) as P:
            assert P.check_matrix() == 0


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_injected_allocation_failures_leak_nothing():
    # every allocation of lp_compile in turn fails: the call returns LP_ERR_OOM and frees what
    # it had allocated; the process keeps working
    from workloads import normal_program, program_batch
    prog = normal_program(seed=3, n=2000, n_rules=6000, k=6)
    with lp.Program.from_program(prog) as P:  # warm the CUDA context and caches
        P.stable_models(torch.zeros(1, dtype=torch.int64, device="cuda:0"))
    free0 = _free_bytes()
    failures = 0
    try:
        for after in range(0, 40):
            lp.debug_fail_alloc(after)
            try:
                with lp.Program.from_program(prog):
                    pass
            except lp.LPError as e:
                assert "OOM" in str(e)
                failures += 1
        for after in range(0, 30):
            lp.debug_fail_alloc(after)
            try:
                with lp.Batch(program_batch(seed=5, count=5, n_lo=50, n_hi=300)):
                    pass
            except lp.LPError as e:
                assert "OOM" in str(e)
                failures += 1
    finally:
        lp.debug_fail_alloc(-1)
    assert failures >= 10
    assert abs(_free_bytes() - free0) < (64 << 20)
    # solves: the first stable-model call allocates its tiles; make that allocation fail
    with lp.Program.from_program(prog) as P:
        mask = torch.zeros(1, dtype=torch.int64, device="cuda:0")
        lp.debug_fail_alloc(0)
        try:
            with pytest.raises(lp.LPError):
                P.stable_models(mask)
        finally:
            lp.debug_fail_alloc(-1)
        st4, _, _ = oracle.stable_models_alg23(prog)
        ns = P.stable_models(mask)  # the handle is still usable
        assert ns == int(st4.sum())
    want, want_it = oracle.least_model(small_definite(3))
    with lp.Program.from_program(small_definite(3)) as P:
        got, it = gpu_least_model(P)
    assert it == want_it and np.array_equal(got, want)
