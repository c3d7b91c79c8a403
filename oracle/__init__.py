"""Plain CPU oracle for the sparse linear-algebraic fixpoint of logic programs.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are the only callers. It imports nothing from the CUDA library's package
and shares no code with it.

What it computes, and from which passage of the paper (Nguyen, Inoue, Sakama, ICLP 2020):

* ``standardize``      -- Sec. 2.1 standardization, Eq. 4 positive form, Def. 2 / Def. 7
                          program matrix, Sec. 3.2 CSR arrays (C: orc_standardize_*).
* ``initial_vector``   -- Def. 4 (optionally restricted to a subset of the facts).
* ``alg1``             -- Algorithm 1 with theta of Def. 5, exact rational row sums.
* ``least_model``      -- O2: Algorithm 1 on the standardized matrix, projected on B_P.
* ``tp_least_model``   -- O1: the T_P operator of Sec. 2.1 iterated from the empty set.
* ``brute_least_model``-- O3: all 2^n interpretations, keep the models (Sec. 2.1), intersect.
* ``stable_models_alg23`` -- O4: Def. 8 initial matrix, Algorithm 2, Algorithm 3 per guess.
* ``stable_models_gl`` -- O5: Gelfond-Lifschitz reduct check of each guess (the criterion of
                          Alferes et al. quoted in Sec. 2.2 makes it equal to O4).
* ``brute_stable_models`` -- all 2^n interpretations I with I = lm(P^I).
"""
import ctypes

import numpy as np

from . import build as _build

ORC_EMPTY, ORC_AND, ORC_OR, ORC_FACT, ORC_BARRED = 0, 1, 2, 3, 4
ERR_INVALID, ERR_NO_FIXPOINT, ERR_NEGATION = 1, 4, 7

_lib = None


def load(path):
    """Load an oracle shared library and declare its C signatures."""
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    L.orc_standardize_size.argtypes = [i32, i64, P, P, P, P, P]
    L.orc_standardize_fill.argtypes = [i32, i64, P, P, P, P, P, P, P, P, P, P]
    L.orc_theta_step.argtypes = [i64, P, P, P, P, P, P]
    L.orc_theta_step.restype = None
    L.orc_alg1.argtypes = [i64, P, P, P, P, P, i64, P, P]
    L.orc_tp_least_model.argtypes = [i32, i64, P, P, P, P, P, P, P, P]
    L.orc_alg23_batch.argtypes = [i32, i64, P, P, P, P, P, P, i64, P, i64, P, i64, P, P, P]
    L.orc_num_threads.restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(_build.build())
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _prog_arrays(prog):
    head = np.ascontiguousarray(prog.head, dtype=np.int32)
    off = np.ascontiguousarray(prog.body_off, dtype=np.int64)
    atom = np.ascontiguousarray(prog.body_atom, dtype=np.int32)
    neg = None
    if getattr(prog, "body_neg", None) is not None:
        neg = np.ascontiguousarray(prog.body_neg, dtype=np.uint8)
    return int(prog.n_atoms), len(head), head, off, atom, neg


def num_threads() -> int:
    return int(lib().orc_num_threads())


class Standardized:
    """The standardized positive form P' and its program matrix M_P as CSR.

    Rows: the n original atoms, then the barred atoms (ascending atom id), then the new atoms
    (rule order). Entry e of row i has the exact value num[e] / den[i].
    """

    def __init__(self, n, row_ptr, col, num, den, kind, owner, n_barred, n_aux):
        self.n = n
        self.row_ptr, self.col, self.num, self.den = row_ptr, col, num, den
        self.kind, self.owner = kind, owner
        self.n_barred, self.n_aux = n_barred, n_aux
        self.n_prime = len(den)
        self.nnz = len(col)

    def values(self):
        """Sec. 3.2 'value' array, as float64 (exact for the 1/m of Def. 2)."""
        rows = np.repeat(np.arange(self.n_prime), np.diff(self.row_ptr))
        return self.num.astype(np.float64) / self.den[rows].astype(np.float64)

    def dense(self):
        """M_P as a dense float64 matrix (small programs only)."""
        M = np.zeros((self.n_prime, self.n_prime))
        rows = np.repeat(np.arange(self.n_prime), np.diff(self.row_ptr))
        M[rows, self.col] = self.values()
        return M

    def coo_rows(self):
        """Sec. 3.2 COO row-index array."""
        return np.repeat(np.arange(self.n_prime), np.diff(self.row_ptr))

    def fact_atoms(self):
        """Original atoms q with a fact q <- in P (a FACT row owned by q)."""
        f = np.zeros(self.n, dtype=bool)
        f[self.owner[self.kind == ORC_FACT]] = True
        return f

    def guess_rows(self):
        """Barred rows enumerated by Def. 8 item 3 (their atom is not a fact), ascending."""
        facts = self.fact_atoms()
        rows = np.nonzero(self.kind == ORC_BARRED)[0]
        return rows[~facts[self.owner[rows]]].astype(np.int64)


def standardize(prog) -> Standardized:
    n, nr, head, off, atom, neg = _prog_arrays(prog)
    L = lib()
    sizes = np.zeros(4, dtype=np.int64)
    rc = L.orc_standardize_size(n, nr, _p(head), _p(off), _p(atom), _p(neg), _p(sizes))
    if rc:
        raise ValueError(f"oracle: invalid program (code {rc})")
    np_, nnz = int(sizes[0]), int(sizes[1])
    row_ptr = np.zeros(np_ + 1, dtype=np.int64)
    col = np.zeros(max(nnz, 1), dtype=np.int64)
    num = np.zeros(max(nnz, 1), dtype=np.int32)
    den = np.zeros(max(np_, 1), dtype=np.int32)
    kind = np.zeros(max(np_, 1), dtype=np.int8)
    owner = np.zeros(max(np_, 1), dtype=np.int64)
    rc = L.orc_standardize_fill(n, nr, _p(head), _p(off), _p(atom), _p(neg), _p(row_ptr), _p(col),
                                _p(num), _p(den), _p(kind), _p(owner))
    if rc:
        raise ValueError(f"oracle: invalid program (code {rc})")
    return Standardized(n, row_ptr, col[:nnz], num[:nnz], den[:np_], kind[:np_], owner[:np_],
                        int(sizes[2]), int(sizes[3]))


def initial_vector(std: Standardized, init=None) -> np.ndarray:
    """Def. 4: v0_i = 1 iff row i is a fact. ``init`` (bool over the n original atoms) keeps
    only the facts of those atoms; it must be a subset of the fact atoms."""
    v0 = (std.kind == ORC_FACT).astype(np.uint8)
    if init is not None:
        init = np.asarray(init, dtype=bool)
        if np.any(init & ~std.fact_atoms()):
            raise ValueError("initial atoms must be facts")
        v0 &= init[std.owner].astype(np.uint8)
    return v0


def theta_step(std: Standardized, v) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.uint8)
    u = np.zeros(std.n_prime, dtype=np.uint8)
    lib().orc_theta_step(std.n_prime, _p(std.row_ptr), _p(std.col), _p(std.num), _p(std.den), _p(v), _p(u))
    return u


def alg1(std: Standardized, v0, max_iters: int = 1 << 40):
    """Algorithm 1 from v0. Returns (v, iters, converged)."""
    v0 = np.ascontiguousarray(v0, dtype=np.uint8)
    v = np.zeros(max(std.n_prime, 1), dtype=np.uint8)
    it = np.zeros(1, dtype=np.int64)
    rc = lib().orc_alg1(std.n_prime, _p(std.row_ptr), _p(std.col), _p(std.num), _p(std.den), _p(v0),
                        int(max_iters), _p(v), _p(it))
    if rc not in (0, ERR_NO_FIXPOINT):
        raise RuntimeError(f"oracle alg1 failed ({rc})")
    return v[: std.n_prime], int(it[0]), rc == 0


def least_model(prog, init=None, max_iters: int = 1 << 40, std: Standardized = None):
    """O2: least model via Algorithm 1 on the standardized matrix, projected on the n
    original atoms (the first n rows). Returns (model bool[n], iters)."""
    std = std or standardize(prog)
    v, it, ok = alg1(std, initial_vector(std, init), max_iters)
    if not ok:
        raise RuntimeError("no fixpoint within max_iters")
    return v[: std.n].astype(bool), it


def tp_least_model(prog, keep_fact=None, assume_true=None):
    """O1: T_P iterated from the empty set on the original rules. Returns (I bool[n], iters)."""
    n, nr, head, off, atom, neg = _prog_arrays(prog)
    kf = None if keep_fact is None else np.ascontiguousarray(keep_fact, dtype=np.uint8)
    at = None if assume_true is None else np.ascontiguousarray(assume_true, dtype=np.uint8)
    out = np.zeros(max(n, 1), dtype=np.uint8)
    it = np.zeros(1, dtype=np.int64)
    rc = lib().orc_tp_least_model(n, nr, _p(head), _p(off), _p(atom), _p(neg), _p(kf), _p(at), _p(out), _p(it))
    if rc:
        raise ValueError(f"oracle T_P failed (code {rc})")
    return out[:n].astype(bool), int(it[0])


def all_guesses(k: int) -> np.ndarray:
    return np.arange(1 << k, dtype=np.uint64)


def stable_models_alg23(prog, guesses=None, max_iters: int = 1 << 40, std: Standardized = None,
                        want_models: bool = True):
    """O4: Def. 8 column per guess, Algorithm 2 to the fixpoint, Algorithm 3 check.
    Bit j of a guess is the value of the barred atom ``std.guess_rows()[j]`` in M_0.
    Returns (stable bool[h], models bool[h, n] or None, iters int64[h])."""
    std = std or standardize(prog)
    rows = np.ascontiguousarray(std.guess_rows(), dtype=np.int64)
    k = len(rows)
    g = all_guesses(k) if guesses is None else np.ascontiguousarray(guesses, dtype=np.uint64)
    h = len(g)
    stable = np.zeros(max(h, 1), dtype=np.uint8)
    iters = np.zeros(max(h, 1), dtype=np.int64)
    models = np.zeros((max(h, 1), max(std.n, 1)), dtype=np.uint8) if want_models else None
    rc = lib().orc_alg23_batch(std.n, std.n_prime, _p(std.row_ptr), _p(std.col), _p(std.num), _p(std.den),
                               _p(std.kind), _p(std.owner), k, _p(rows), h, _p(g), int(max_iters),
                               _p(stable), _p(models), _p(iters))
    if rc:
        raise RuntimeError(f"oracle alg2/3 failed ({rc})")
    m = None if models is None else models[:h, : std.n].astype(bool)
    return stable[:h].astype(bool), m, iters[:h]


def stable_models_gl(prog, guesses=None, std: Standardized = None):
    """O5: for each guess, the assumed-true negated atoms A (barred value 0; facts are forced
    to 0 by Def. 8 item 3); L = lm(P^A) by T_P on the reduct; stable iff L agrees with A on
    every negated atom. Returns (stable bool[h], models bool[h, n])."""
    std = std or standardize(prog)
    rows = std.guess_rows()
    owners = std.owner[rows]
    negated = np.zeros(std.n, dtype=bool)
    negated[std.owner[std.kind == ORC_BARRED]] = True
    k = len(rows)
    g = all_guesses(k) if guesses is None else np.asarray(guesses, dtype=np.uint64)
    stable = np.zeros(len(g), dtype=bool)
    models = np.zeros((len(g), std.n), dtype=bool)
    base = negated & std.fact_atoms()
    for t, gv in enumerate(g):
        A = base.copy()
        bits = (int(gv) >> np.arange(k)) & 1
        A[owners] = bits == 0
        L, _ = tp_least_model(prog, assume_true=A)
        models[t] = L
        stable[t] = bool(np.all(L[negated] == A[negated]))
    return stable, models


# ----------------------------------------------------------------------------------------
# Brute force over all 2^n interpretations (n <= 16), vectorised over the interpretations.
# ----------------------------------------------------------------------------------------

def _rules(prog):
    n, nr, head, off, atom, neg = _prog_arrays(prog)
    out = []
    for r in range(nr):
        lits = [(int(atom[e]), bool(neg[e]) if neg is not None else False) for e in range(off[r], off[r + 1])]
        out.append((int(head[r]), lits))
    return n, out


def brute_least_model(prog):
    """O3: the models of Sec. 2.1 (body true implies head true, for every rule) among all
    2^n interpretations; the least model is their intersection (it is itself a model)."""
    n, rules = _rules(prog)
    if n > 16:
        raise ValueError("brute force limited to 16 atoms")
    I = np.arange(1 << n, dtype=np.int64)
    is_model = np.ones(1 << n, dtype=bool)
    for h, lits in rules:
        if any(neg for _, neg in lits):
            raise ValueError("definite programs only")
        body = np.ones(1 << n, dtype=bool)
        for a, _ in lits:
            body &= ((I >> a) & 1).astype(bool)
        is_model &= ~body | ((I >> h) & 1).astype(bool)
    models = I[is_model]
    least = np.bitwise_and.reduce(models) if len(models) else 0
    assert is_model[least], "intersection of models must be a model"
    return np.array([(least >> a) & 1 for a in range(n)], dtype=bool)


def brute_stable_models(prog):
    """All I subset of B_P with I = lm(P^I) (Gelfond-Lifschitz), n <= 16. Returns the sorted
    list of stable models as int bitmasks over the atoms."""
    n, rules = _rules(prog)
    if n > 16:
        raise ValueError("brute force limited to 16 atoms")
    I = np.arange(1 << n, dtype=np.int64)
    L = np.zeros(1 << n, dtype=np.int64)  # least model of P^I, for every I at once
    while True:
        nxt = np.zeros(1 << n, dtype=np.int64)
        for h, lits in rules:
            fires = np.ones(1 << n, dtype=bool)
            for a, neg in lits:
                if neg:
                    fires &= ((I >> a) & 1) == 0  # kept in P^I iff a not in I
                else:
                    fires &= ((L >> a) & 1) == 1
            nxt |= fires.astype(np.int64) << h
        if np.array_equal(nxt, L):
            break
        L = nxt
    return sorted(int(x) for x in I[L == I])

