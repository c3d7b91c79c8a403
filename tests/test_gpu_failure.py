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
