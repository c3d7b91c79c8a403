"""Host logic of the sharded stable-model path, on CPU: the guess ranges cover every guess once,
on word boundaries and balanced; and two gloo ranks that each solve their own range (the
oracle stands in for the per-rank GPU solve) gather exactly the oracle's full stable mask."""
import os
import socket

import numpy as np
import pytest

from paper_2009_10247_gb300.shard import guess_range, program_range


@pytest.mark.parametrize("n", [0, 1, 63, 64, 65, 1000, 1 << 16])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_guess_ranges(n, world):
    spans = [guess_range(n, r, world) for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == n
    for (a, b), (c, d) in zip(spans, spans[1:]):
        assert b == c
    assert all(lo % 64 == 0 for lo, _ in spans)
    words = [(hi - lo + 63) // 64 for lo, hi in spans]
    assert max(words) - min(words) <= 1


def test_program_ranges():
    spans = [program_range(1000, r, 3) for r in range(3)]
    assert spans == [(0, 333), (333, 666), (666, 1000)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    from paper_2009_10247_gb300.shard import stable_models_sharded
    from workloads import normal_program

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prog = normal_program(seed=9, n=600, n_rules=1800, k=9, per_atom=2)
    std = oracle.standardize(prog)

    class Info:
        info = {"k": len(std.guess_rows())}

    def solve_range(lo, hi):
        st, _, _ = oracle.stable_models_alg23(prog, guesses=np.arange(lo, hi, dtype=np.uint64), std=std,
                                              want_models=False)
        return np.packbits(np.pad(st, (0, (-len(st)) % 64)).astype(np.uint8), bitorder="little").view(np.uint64)

    full = stable_models_sharded(Info(), solve_range=solve_range)
    np.save(os.path.join(out_dir, f"mask{rank}.npy"), full)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_the_full_mask(tmp_path):
    import torch.multiprocessing as mp

    import oracle
    from workloads import normal_program

    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:
        if p.is_alive():
            p.kill()
    assert all(p.exitcode == 0 for p in procs)
    prog = normal_program(seed=9, n=600, n_rules=1800, k=9, per_atom=2)
    st, _, _ = oracle.stable_models_alg23(prog, want_models=False)
    want = np.packbits(np.pad(st, (0, (-len(st)) % 64)).astype(np.uint8), bitorder="little").view(np.uint64)
    for r in range(2):
        got = np.load(tmp_path / f"mask{r}.npy")
        assert np.array_equal(got, want)


def _relaxed_worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    from oracle.relaxed import RelaxedProgram
    from paper_2009_10247_gb300.shard import allreduce_weight_grad, batch_range
    from workloads import small_definite

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    R = RelaxedProgram(small_definite(4))
    rng = np.random.default_rng(3)
    w = rng.uniform(0.5, 1.5, R.n_rules)
    v0 = rng.uniform(0.0, 1.0, (R.n_prime, 10))
    c = rng.uniform(-1.0, 1.0, (R.n_prime, 10))
    lo, hi = batch_range(10, rank, world)
    vs = R.forward(w, v0[:, lo:hi], 8, 0.2)
    dw, dv0 = R.backward(w, vs, c[:, lo:hi], 0.2)
    t = torch.from_numpy(dw.copy())
    allreduce_weight_grad(t)
    np.save(os.path.join(out_dir, f"dw{rank}.npy"), t.numpy())
    np.save(os.path.join(out_dir, f"dv{rank}.npy"), dv0)
    dist.barrier()
    dist.destroy_process_group()


def test_relaxed_columns_and_weight_allreduce(tmp_path):
    import torch.multiprocessing as mp

    from oracle.relaxed import RelaxedProgram
    from workloads import small_definite

    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_relaxed_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:
        if p.is_alive():
            p.kill()
    assert all(p.exitcode == 0 for p in procs)
    R = RelaxedProgram(small_definite(4))
    rng = np.random.default_rng(3)
    w = rng.uniform(0.5, 1.5, R.n_rules)
    v0 = rng.uniform(0.0, 1.0, (R.n_prime, 10))
    c = rng.uniform(-1.0, 1.0, (R.n_prime, 10))
    dw, dv0 = R.backward(w, R.forward(w, v0, 8, 0.2), c, 0.2)
    for r in range(2):
        assert np.allclose(np.load(tmp_path / f"dw{r}.npy"), dw, rtol=1e-12, atol=1e-14)
    assert np.allclose(np.concatenate([np.load(tmp_path / "dv0.npy"), np.load(tmp_path / "dv1.npy")], axis=1), dv0,
                       rtol=1e-12, atol=1e-14)


def test_collective_device_follows_backend(monkeypatch):
    # NCCL takes device tensors only; gloo takes host tensors
    import torch
    import torch.distributed as dist

    from paper_2009_10247_gb300 import shard

    monkeypatch.setattr(torch.cuda, "current_device", lambda: 3)
    monkeypatch.setattr(dist, "get_backend", lambda group=None: "nccl")
    assert shard.collective_device() == torch.device("cuda", 3)
    monkeypatch.setattr(dist, "get_backend", lambda group=None: "gloo")
    assert shard.collective_device() == torch.device("cpu")
