"""Test helpers: decoding bit-packed vectors and checking properties of models.

Nothing here computes the fixpoint; these are independent property checks written from
the definitions of Sec. 2.1 (model of a program) and the bit layout of the C ABI.
"""
import json
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def frac_matrix(rows):
    return [[Fraction(x) for x in r] for r in rows]


def bits_to_bool(words, n: int) -> np.ndarray:
    """Unpack little-endian 64-bit words: bit i of the array (word i//64, bit i%64) = item i."""
    w = np.ascontiguousarray(np.asarray(words).reshape(-1).view(np.uint64))
    b = np.unpackbits(w.view(np.uint8), bitorder="little")
    return b[:n].astype(bool)


def bool_to_bits(x) -> np.ndarray:
    x = np.asarray(x, dtype=bool).reshape(-1)
    nw = max(1, (len(x) + 63) // 64)
    b = np.zeros(nw * 64, dtype=np.uint8)
    b[: len(x)] = x
    return np.packbits(b, bitorder="little").view(np.uint64).copy()


def is_model(prog, I) -> bool:
    """Sec. 2.1: I is a model iff every rule whose body is contained in I has its head in I
    (definite programs)."""
    I = np.asarray(I, dtype=bool)
    cs = np.concatenate([[0], np.cumsum(~I[prog.body_atom])])
    body_true = (cs[prog.body_off[1:]] - cs[prog.body_off[:-1]]) == 0
    return bool(np.all(~body_true | I[prog.head]))


def program_fingerprint(prog) -> str:
    """SHA-256 over a program's arrays (atom count, heads, body offsets, atoms, negation marks):
    a stored expected value applies only to the program it was computed on."""
    import hashlib

    h = hashlib.sha256()
    h.update(np.int64(prog.n_atoms).tobytes())
    for a, dt in ((prog.head, np.int32), (prog.body_off, np.int64), (prog.body_atom, np.int32)):
        h.update(np.ascontiguousarray(a, dtype=dt).tobytes())
    if getattr(prog, "body_neg", None) is not None:
        h.update(np.ascontiguousarray(prog.body_neg, dtype=np.uint8).tobytes())
    return h.hexdigest()
