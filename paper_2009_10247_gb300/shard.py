"""Stable models and relaxed batches sharded over ranks, one GPU per rank.

The 2^k guesses of Algorithm 2 are independent columns (Def. 8), so ranks take contiguous
guess ranges and need no exchange while they iterate; the only collective is one gather of the
stable masks at the end. Ranges start on multiples of 64 guesses, so each rank's mask words
concatenate without shifting. Programs of a batch shard the same way (contiguous program
ranges). The per-range solve runs in liblp (`Program.stable_models` on an explicit guess list);
this module only splits ranges and gathers results. Relaxed batches split by columns; their
rule-weight gradients meet in one all-reduce per backward pass.
"""
from typing import Callable, Optional, Tuple

import numpy as np


def guess_range(n_guesses: int, rank: int, world: int) -> Tuple[int, int]:
    """[lo, hi) of rank's guesses: contiguous, disjoint, covering, lo a multiple of 64, and the
    ranks' word counts differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    n_words = (n_guesses + 63) // 64
    w0 = n_words * rank // world
    w1 = n_words * (rank + 1) // world
    return min(64 * w0, n_guesses), min(64 * w1, n_guesses)


def program_range(n_programs: int, rank: int, world: int) -> Tuple[int, int]:
    """[lo, hi) of rank's programs of a batch (contiguous, balanced by count)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    return n_programs * rank // world, n_programs * (rank + 1) // world


def collective_device(group=None):
    """Device of the tensors a collective on `group` takes: the current CUDA device for an NCCL
    group (NCCL moves device memory only), the CPU for gloo and the others."""
    import torch
    import torch.distributed as dist

    if dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def gather_mask(local_words: np.ndarray, n_guesses: int, group=None) -> np.ndarray:
    """Concatenate every rank's mask words (rank order) into the full mask of n_guesses bits,
    on every rank. local_words: uint64 words of this rank's guess_range. The gather runs on
    the group's collective device (collective_device)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    n_words = (n_guesses + 63) // 64
    counts = []
    for r in range(world):
        lo, hi = guess_range(n_guesses, r, world)
        counts.append((hi - lo + 63) // 64)
    width = max(counts) if counts else 0
    mine = np.zeros(max(width, 1), dtype=np.uint64)
    mine[:len(local_words)] = local_words
    t = torch.from_numpy(mine.view(np.int64).copy()).to(collective_device(group))
    parts = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    full = np.concatenate([p.cpu().numpy().view(np.uint64)[:c] for p, c in zip(parts, counts)]) if world else np.zeros(0)
    assert len(full) == n_words
    return full


def stable_models_sharded(prog, group=None, solve_range: Optional[Callable] = None) -> np.ndarray:
    """Stable mask of all 2^k guesses of `prog` (a liblp Program, or any object whose
    solve_range is given), computed as this rank's guess range plus one gather.
    solve_range(lo, hi) -> uint64 mask words of guesses lo..hi-1; by default liblp's
    lp_stable_models on the explicit guess list lo..hi-1 on the current CUDA device."""
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    k = prog.info["k"]
    n = 1 << k
    lo, hi = guess_range(n, rank, world)
    if solve_range is None:
        solve_range = _liblp_range(prog)
    local = solve_range(lo, hi) if hi > lo else np.zeros(0, dtype=np.uint64)
    return gather_mask(np.asarray(local, dtype=np.uint64), n, group)


def _liblp_range(prog):
    import torch

    from .lp import words

    def run(lo, hi):
        dev = torch.device("cuda", torch.cuda.current_device())
        g = torch.arange(lo, hi, dtype=torch.int64, device=dev)
        mask = torch.zeros(words(hi - lo), dtype=torch.int64, device=dev)
        prog.stable_models(mask, guesses=g, n_guesses=hi - lo)
        return mask.cpu().numpy().view(np.uint64)

    return run


def batch_range(batch: int, rank: int, world: int) -> Tuple[int, int]:
    """[lo, hi) of rank's columns of a relaxed batch (contiguous, balanced)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    return batch * rank // world, batch * (rank + 1) // world


def allreduce_weight_grad(dweights, group=None):
    """Sum of the per-rank rule-weight gradients, in place on every rank: the weight gradient
    is a sum over batch columns, so ranks that hold disjoint column ranges of one batch meet in
    this single all-reduce per backward pass (the initial-vector gradients stay per rank)."""
    import torch.distributed as dist

    dist.all_reduce(dweights, op=dist.ReduceOp.SUM, group=group)
    return dweights
