"""Reuse of small device buffers and pinned control blocks across handles.

liblp keeps the blocks (up to 256 KiB each) of a freed handle for later handles instead of
returning them to the driver. A reused block holds whatever the last handle left in it, so
handles compiled into reused blocks must still solve exactly as the oracle does; repeated
compile-solve-free rounds must not grow the memory in use; and with LP_ALLOC_CACHE=0 every
buffer is the driver's again."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import paper_2009_10247_gb300 as lp
from workloads import normal_program, small_definite, transitive_closure

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import gpu_least_model, gpu_stable  # noqa: E402


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_reused_blocks_give_exact_solves():
    progs = [small_definite(11), transitive_closure(120, 3.0, 2), small_definite(12),
             normal_program(seed=8, n=1500, n_rules=4500, k=8, per_atom=2)]
    want = [(oracle.least_model(prog), oracle.stable_models_alg23(prog)[0]) for prog in progs]
    free0 = None
    for rep in range(6):
        if rep == 1:  # after one round: modules loaded, the caches (liblp's, torch's, the pool) warm
            free0 = _free_bytes()
        for prog, ((lm, it), st4) in zip(progs, want):
            with lp.Program.from_program(prog) as P:
                got, got_it = gpu_least_model(P)
                assert got_it == it and np.array_equal(got, lm), rep
                st, _, ns = gpu_stable(P)
                assert np.array_equal(st, st4) and ns == int(st4.sum()), rep
    assert abs(_free_bytes() - free0) < (40 << 20)  # later rounds reuse what the first one kept


def test_cache_off_and_device_compile_in_a_fresh_process():
    code = (
        "import numpy as np, oracle, paper_2009_10247_gb300 as lp\n"
        "from tests.gpu_util import gpu_least_model\n"
        "from workloads import small_definite\n"
        "prog = small_definite(13)\n"
        "want, want_it = oracle.least_model(prog)\n"
        "for kw in ({}, {'on_device': True}, {'on_host': True}):\n"
        "    for _ in range(3):\n"
        "        with lp.Program.from_program(prog, **kw) as P:\n"
        "            got, it = gpu_least_model(P)\n"
        "        assert it == want_it and np.array_equal(got, want)\n"
        "print('ok')\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, LP_ALLOC_CACHE="0", PYTHONPATH=root)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stderr[-2000:]
