"""Helpers for the GPU parity tests: run liblp through its C ABI (Python binding) on cuda:0
and decode the bit-packed results. No model is computed here."""
import numpy as np

import paper_2009_10247_gb300 as lp
from tests.helpers import bits_to_bool, bool_to_bits

try:
    import torch
except ImportError:  # pragma: no cover
    torch = None

DEV = "cuda:0"


def dev_words(n_bits):
    return torch.zeros(lp.words(n_bits), dtype=torch.int64, device=DEV)


def to_dev_bits(x):
    return torch.from_numpy(bool_to_bits(x).view(np.int64)).to(DEV)


def from_dev_bits(t, n):
    return bits_to_bool(t.cpu().numpy().view(np.uint64), n)


def gpu_least_model(P, init=None, max_iters=1 << 30, rows=False):
    n = P.info["n_prime"] if rows else P.info["n_atoms"]
    out = dev_words(n)
    it = P.least_model(out, init=None if init is None else to_dev_bits(init), max_iters=max_iters, rows=rows)
    torch.cuda.synchronize()
    return from_dev_bits(out, n), it


def gpu_stable(P, guesses=None, max_models=0):
    k = P.info["k"]
    n = P.info["n_atoms"]
    ng = (1 << k) if guesses is None else len(guesses)
    mask = dev_words(ng)
    models = torch.zeros((max(max_models, 1), lp.words(n)), dtype=torch.int64, device=DEV) if max_models else None
    g = None if guesses is None else torch.from_numpy(np.asarray(guesses, dtype=np.uint64).view(np.int64)).to(DEV)
    ns = P.stable_models(mask, guesses=g, n_guesses=ng, models=models, max_models=max_models)
    torch.cuda.synchronize()
    st = from_dev_bits(mask, ng)
    mod = None
    if max_models:
        mm = models.cpu().numpy().view(np.uint64)
        mod = np.stack([bits_to_bool(mm[i], n) for i in range(min(ns, max_models))]) if ns else np.zeros((0, n), bool)
    return st, mod, ns
