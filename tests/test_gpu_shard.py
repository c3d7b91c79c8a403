"""The sharded stable-model path with liblp doing each range (one rank here; the multi-rank
host logic is covered on CPU): guess ranges through explicit guess lists gather to the same
mask as one call over all 2^k guesses, through a gloo group and through an NCCL group (the
backend the multi-GPU benchmark opens, which gathers device tensors)."""
import os
import socket

import numpy as np
import pytest

import paper_2009_10247_gb300 as lp
from paper_2009_10247_gb300.shard import guess_range, stable_models_sharded
from workloads import normal_program

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("backend", ["gloo", "nccl"])
def test_sharded_equals_unsharded(backend):
    import torch.distributed as dist

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    if backend == "nccl":
        dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", 0))
    else:
        dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        prog = normal_program(seed=6, n=5000, n_rules=15000, k=12, per_atom=2)
        with lp.Program.from_program(prog) as P:
            full = torch.zeros(lp.words(1 << 12), dtype=torch.int64, device="cuda:0")
            P.stable_models(full)
            got = stable_models_sharded(P)
            # the ranges a 3-rank run would take, solved one after another here
            parts = []
            for r in range(3):
                lo, hi = guess_range(1 << 12, r, 3)
                g = torch.arange(lo, hi, dtype=torch.int64, device="cuda:0")
                m = torch.zeros(lp.words(hi - lo), dtype=torch.int64, device="cuda:0")
                P.stable_models(m, guesses=g, n_guesses=hi - lo)
                parts.append(m.cpu().numpy().view(np.uint64))
        want = full.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want)
        assert np.array_equal(np.concatenate(parts), want)
    finally:
        dist.destroy_process_group()
