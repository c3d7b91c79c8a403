"""Seeded program generators (inputs only; no part of the fixpoint method lives here).

A program is a list of rules ``head <- body``; body literals are atoms, optionally negated.
Arrays: ``head[r]``; literals ``body_atom[body_off[r]:body_off[r+1]]``; ``body_neg`` marks
"not b". An empty body is a fact. Generators follow the shapes the paper describes (Sec. 4:
random programs after Table 1, normal programs with k negated atoms, transitive closure of a
graph) at the sizes of the benchmark configurations.
"""
from dataclasses import dataclass, field
import re
from typing import List, Optional, Sequence

import numpy as np


@dataclass
class Program:
    n_atoms: int
    head: np.ndarray  # int32 [n_rules]
    body_off: np.ndarray  # int64 [n_rules + 1]
    body_atom: np.ndarray  # int32 [n_literals]
    body_neg: Optional[np.ndarray] = None  # uint8 [n_literals] or None (definite)
    names: Optional[List[str]] = None
    meta: dict = field(default_factory=dict)

    @property
    def n_rules(self) -> int:
        return len(self.head)

    @property
    def n_literals(self) -> int:
        return len(self.body_atom)

    def is_definite(self) -> bool:
        return self.body_neg is None or not np.any(self.body_neg)

    def fact_atoms(self) -> np.ndarray:
        f = np.zeros(self.n_atoms, dtype=bool)
        f[self.head[np.diff(self.body_off) == 0]] = True
        return f


def _pack(n_atoms, heads, lens, atoms, negs=None, **meta) -> Program:
    lens = np.asarray(lens, dtype=np.int64)
    off = np.zeros(len(lens) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    neg = None if negs is None else np.ascontiguousarray(negs, dtype=np.uint8)
    return Program(int(n_atoms), np.ascontiguousarray(heads, dtype=np.int32), off,
                   np.ascontiguousarray(atoms, dtype=np.int32), neg, meta=dict(meta))


def from_rules(n_atoms: int, rules: Sequence, names=None) -> Program:
    """rules: [(head, [lit, ...]), ...]; a literal is an atom id, or ``~a`` for "not a"."""
    heads, lens, atoms, negs = [], [], [], []
    for h, body in rules:
        heads.append(h)
        lens.append(len(body))
        for lit in body:
            atoms.append(~lit if lit < 0 else lit)
            negs.append(1 if lit < 0 else 0)
    p = _pack(n_atoms, heads, lens, np.array(atoms, dtype=np.int64), negs if any(negs) else None)
    p.names = names
    return p


def parse(text: str, atoms: Optional[Sequence[str]] = None) -> Program:
    """Parse ``"p :- q, r. s. t :- not u."`` (``<-`` also accepted). Atom ids follow ``atoms``
    when given (every atom must be listed), else the order of first appearance."""
    names = list(atoms) if atoms is not None else []
    index = {a: i for i, a in enumerate(names)}

    def aid(a):
        if a not in index:
            if atoms is not None:
                raise ValueError(f"atom {a!r} not in the given atom list")
            index[a] = len(names)
            names.append(a)
        return index[a]

    rules = []
    for stmt in [s.strip() for s in text.split(".") if s.strip()]:
        parts = re.split(r":-|<-", stmt)
        h = aid(parts[0].strip())
        body = []
        if len(parts) > 1 and parts[1].strip():
            for lit in parts[1].split(","):
                lit = lit.strip()
                if lit.startswith("not "):
                    body.append(~aid(lit[4:].strip()))
                else:
                    body.append(aid(lit))
        rules.append((h, body))
    return from_rules(len(names), rules, names=names)


def _permute_rules(rng, heads, lens, atoms, negs=None):
    """Shuffle rule order (variable-length bodies moved with their rule)."""
    lens = np.asarray(lens, dtype=np.int64)
    off = np.zeros(len(lens) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    order = rng.permutation(len(lens))
    nl = lens[order]
    starts = off[:-1][order]
    # gather index: for each new rule, starts + 0..len-1
    new_off = np.zeros(len(nl) + 1, dtype=np.int64)
    np.cumsum(nl, out=new_off[1:])
    idx = np.repeat(starts - new_off[:-1], nl) + np.arange(new_off[-1], dtype=np.int64)
    out_negs = None if negs is None else np.asarray(negs)[idx]
    return np.asarray(heads)[order], nl, np.asarray(atoms)[idx], out_negs


def _zipf_ranks(rng, n: int, a: float, size: int) -> np.ndarray:
    """Ranks 0..n-1 with P(rank r) proportional to (r+1)^-a (bounded Zipf)."""
    w = np.arange(1, n + 1, dtype=np.float64) ** (-a)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(size)
    return np.minimum(np.searchsorted(cdf, u, side="right"), n - 1)


def _geom_lengths(rng, size, mean=3.0, cap=8):
    return np.minimum(rng.geometric(1.0 / mean, size), cap).astype(np.int64)


def _chain_rules(rng, facts, chain, lens):
    """Layered chain: chain[d] (d = 0..L-1) are the heads of level d+1. Each body holds one
    atom of the previous level (the facts for d = 0) and len-1 atoms from the facts and all
    lower levels, so the level-d atoms are derived exactly at step d+1."""
    L, W = chain.shape
    pool = np.concatenate([facts, chain.reshape(-1)])
    nf = len(facts)
    lens = lens.reshape(L, W)
    atoms = []
    for d in range(L):
        prev = facts if d == 0 else chain[d - 1]
        first = prev[rng.integers(0, len(prev), W)]
        rest_n = int(lens[d].sum() - W)
        rest = pool[rng.integers(0, nf + d * W, rest_n)] if rest_n else np.zeros(0, dtype=pool.dtype)
        # interleave: rule w gets first[w] then its len-1 others
        o = np.zeros(W + 1, dtype=np.int64)
        np.cumsum(lens[d] - 1, out=o[1:])
        for w in range(W):
            atoms.append(first[w:w + 1])
            atoms.append(rest[o[w]:o[w + 1]])
    return chain.reshape(-1), lens.reshape(-1), np.concatenate(atoms) if atoms else np.zeros(0, np.int64)


def small_definite(seed: int = 1, n: int = 1000, n_rules: int = 2000, n_facts: int = 50,
                   chain_levels: int = 40, chain_width: int = 5, max_body: int = 5) -> Program:
    """Small definite program: n atoms, n_rules rules, body length U{1..max_body}, body atoms
    uniform; n_facts facts; chain_levels x chain_width chain rules with unique heads that force
    about chain_levels iterations; the remaining rules are random."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    facts = perm[:n_facts]
    nc = chain_levels * chain_width
    chain = perm[n_facts:n_facts + nc].reshape(chain_levels, chain_width)
    others = perm[n_facts + nc:]
    c_heads, c_lens, c_atoms = _chain_rules(rng, facts, chain, rng.integers(1, max_body + 1, nc))
    nr = n_rules - n_facts - nc
    r_lens = rng.integers(1, max_body + 1, nr)
    r_atoms = rng.integers(0, n, int(r_lens.sum()))
    r_heads = others[rng.integers(0, len(others), nr)]
    heads = np.concatenate([facts, c_heads, r_heads])
    lens = np.concatenate([np.zeros(n_facts, np.int64), c_lens, r_lens])
    atoms = np.concatenate([c_atoms, r_atoms])
    h, l, a, _ = _permute_rules(rng, heads, lens, atoms)
    return _pack(n, h, l, a, name="small_definite", seed=seed)


def large_definite(seed: int = 1, n: int = 1_000_000, n_rules: int = 5_000_000, fact_frac: float = 0.01,
                   chain_levels: int = 1000, chain_width: int = 50, zipf_a: float = 1.1,
                   mean_body: float = 3.0, max_body: int = 8) -> Program:
    """Large definite program: body length Geom(mean 3) capped at 8, body atoms Zipf(1.1)
    over a seeded permutation of the atoms, fact_frac of the atoms are facts, and a layered
    chain of chain_levels x chain_width unique heads forcing about chain_levels iterations."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    nf = max(1, int(round(n * fact_frac)))
    nc = chain_levels * chain_width
    facts = perm[:nf]
    chain = perm[nf:nf + nc].reshape(chain_levels, chain_width)
    others = perm[nf + nc:]
    c_heads, c_lens, c_atoms = _chain_rules(rng, facts, chain, _geom_lengths(rng, nc, mean_body, max_body))
    nr = n_rules - nf - nc
    r_lens = _geom_lengths(rng, nr, mean_body, max_body)
    zperm = rng.permutation(n)
    r_atoms = zperm[_zipf_ranks(rng, n, zipf_a, int(r_lens.sum()))]
    r_heads = others[rng.integers(0, len(others), nr)]
    heads = np.concatenate([facts, c_heads, r_heads])
    lens = np.concatenate([np.zeros(nf, np.int64), c_lens, r_lens])
    atoms = np.concatenate([c_atoms, r_atoms])
    h, l, a, _ = _permute_rules(rng, heads, lens, atoms)
    return _pack(n, h, l, a, name="large_definite", seed=seed)


def transitive_closure(n_nodes: int = 500, mean_outdeg: float = 4.0, seed: int = 1) -> Program:
    """Ground transitive closure of a random digraph (out-degree Poisson(mean), no
    self-loops): edge atoms are facts; path(x,y) <- edge(x,y) for every edge and
    path(x,y) <- edge(x,z) & path(z,y) for every edge (x,z) and every node y.
    Atom ids: edge e -> e, path(x,y) -> |E| + x*n_nodes + y."""
    rng = np.random.default_rng(seed)
    src, dst = [], []
    for x in range(n_nodes):
        d = min(int(rng.poisson(mean_outdeg)), n_nodes - 1)
        cand = rng.choice(n_nodes - 1, size=d, replace=False)
        cand = np.where(cand >= x, cand + 1, cand)  # skip x itself
        src.extend([x] * d)
        dst.extend(sorted(cand.tolist()))
    return _ground_closure(n_nodes, np.array(src, dtype=np.int64), np.array(dst, dtype=np.int64), seed)


def transitive_closure_edges(n_nodes: int, n_edges: int, seed: int = 1) -> Program:
    """The same grounding on a random digraph with exactly n_edges distinct edges (no
    self-loops), drawn uniformly: a stand-in for a named graph of which only the node and edge
    counts are known (the paper's Table 4)."""
    rng = np.random.default_rng(seed)
    n_edges = min(n_edges, n_nodes * (n_nodes - 1))
    flat = rng.choice(n_nodes * (n_nodes - 1), size=n_edges, replace=False)
    src = flat // (n_nodes - 1)
    dst = flat % (n_nodes - 1)
    dst = np.where(dst >= src, dst + 1, dst)
    order = np.lexsort((dst, src))
    return _ground_closure(n_nodes, src[order].astype(np.int64), dst[order].astype(np.int64), seed)


def transitive_closure_pairs(n_nodes: int, n_edges: int, seed: int = 1) -> Program:
    """Transitive closure grounded over every ordered pair and triple of distinct nodes, the
    grounding the paper's Table 4 sizes imply: atoms edge(x,y) and path(x,y) for all x != y
    (n = 2 |V| (|V|-1)); facts edge(x,y) for the |E| edges of a uniform random digraph;
    path(x,y) <- edge(x,y) for all x != y; path(x,y) <- edge(x,z) & path(z,y) for all distinct
    x, z, y. Atom ids: edge(x,y) -> pair(x,y), path(x,y) -> |V|(|V|-1) + pair(x,y), pairs in
    row-major order skipping x = y."""
    rng = np.random.default_rng(seed)
    N = n_nodes
    NP = N * (N - 1)
    n_edges = min(n_edges, NP)
    flat = np.sort(rng.choice(NP, size=n_edges, replace=False))  # edge = pair index
    src = flat // (N - 1)
    dst = flat % (N - 1)
    dst = np.where(dst >= src, dst + 1, dst)

    def pair(x, y):  # x != y
        return x * (N - 1) + np.where(y > x, y - 1, y)

    x, z, y = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    keep = (x != z) & (z != y) & (x != y)
    x, z, y = x[keep], z[keep], y[keep]
    px, py = np.repeat(np.arange(N), N - 1), None
    py = np.array([v for u in range(N) for v in range(N) if v != u], dtype=np.int64)
    base_heads = NP + pair(px, py)
    heads = [flat, base_heads, NP + pair(x, y)]
    lens = [np.zeros(n_edges, np.int64), np.ones(NP, np.int64), np.full(len(x), 2, np.int64)]
    rec = np.empty(2 * len(x), dtype=np.int64)
    rec[0::2] = pair(x, z)
    rec[1::2] = NP + pair(z, y)
    atoms = [pair(px, py), rec]
    return _pack(2 * NP, np.concatenate(heads), np.concatenate(lens), np.concatenate(atoms),
                 name="transitive_closure_pairs", seed=seed, n_nodes=N, edges=np.stack([src, dst], 1))


def _ground_closure(n_nodes: int, src: np.ndarray, dst: np.ndarray, seed: int) -> Program:
    E = len(src)
    N = n_nodes
    n_atoms = E + N * N
    path = lambda x, y: E + x * N + y  # noqa: E731
    eids = np.arange(E, dtype=np.int64)
    # facts, base rules, recursive rules (edge e=(x,z), all y)
    heads = [eids, path(src, dst), np.repeat(path(src, 0), N) + np.tile(np.arange(N), E)]
    lens = [np.zeros(E, np.int64), np.ones(E, np.int64), np.full(E * N, 2, np.int64)]
    rec_body = np.empty(2 * E * N, dtype=np.int64)
    rec_body[0::2] = np.repeat(eids, N)
    rec_body[1::2] = np.repeat(path(dst, 0), N) + np.tile(np.arange(N), E)
    atoms = [eids, rec_body]
    return _pack(n_atoms, np.concatenate(heads), np.concatenate(lens), np.concatenate(atoms),
                 name="transitive_closure", seed=seed, n_nodes=N, edges=np.stack([src, dst], 1))


def normal_program(seed: int = 1, n: int = 100_000, n_rules: int = 300_000, fact_frac: float = 0.01,
                   body_lo: int = 1, body_hi: int = 6, k: int = 16, per_atom: int = 4) -> Program:
    """Normal program: body length U{body_lo..body_hi}, atoms uniform, fact_frac facts; k
    distinct non-fact atoms each put negated into per_atom random bodies (replacing a literal)."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    nf = max(1, int(round(n * fact_frac)))
    facts = perm[:nf]
    nonfacts = perm[nf:]
    nr = n_rules - nf
    r_lens = rng.integers(body_lo, body_hi + 1, nr)
    r_atoms = rng.integers(0, n, int(r_lens.sum()))
    r_heads = nonfacts[rng.integers(0, len(nonfacts), nr)]
    heads = np.concatenate([facts, r_heads])
    lens = np.concatenate([np.zeros(nf, np.int64), r_lens])
    atoms = r_atoms.copy()
    negs = np.zeros(len(atoms), dtype=np.uint8)
    off = np.zeros(nr + 1, dtype=np.int64)
    np.cumsum(r_lens, out=off[1:])
    q_atoms = rng.choice(nonfacts, size=k, replace=False)
    sites = rng.choice(nr, size=k * per_atom, replace=False)  # distinct rules
    for j, r in enumerate(sites):
        pos = off[r] + rng.integers(0, r_lens[r])
        atoms[pos] = q_atoms[j // per_atom]
        negs[pos] = 1
    h, l, a, ng = _permute_rules(rng, heads, lens, atoms, negs)
    return _pack(n, h, l, a, ng, name="normal_program", seed=seed, negated=np.sort(q_atoms))


def program_batch(seed: int = 1, count: int = 1000, n_lo: int = 100, n_hi: int = 20000,
                  rules_per_atom: int = 3, k_lo: int = 4, k_hi: int = 8, per_atom: int = 2) -> List[Program]:
    """Many normal programs of uneven size: n log-uniform in [n_lo, n_hi], rules = 3n,
    k ~ U{k_lo..k_hi} negated atoms (the range of the paper's normal-program experiments)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        k = int(rng.integers(k_lo, k_hi + 1))
        out.append(normal_program(seed=int(rng.integers(1 << 31)), n=n, n_rules=rules_per_atom * n,
                                  k=k, per_atom=per_atom))
    return out


# Share of the non-fact rules by body length 1..8 (the paper's Table 1).
TABLE1_LENGTH_SHARE = (0.04, 0.04, 0.10, 0.40, 0.35, 0.04, 0.02, 0.01)


def table1_program(seed: int, n: int, m: int, dense: bool = False, k: int = 0) -> Program:
    """Random program shaped like the paper's experiments (Sec. 4, Table 1): m rules over n
    atoms. Facts: a seeded share u*n of the atoms, u ~ U(0.1, 1/3) (the table allows fewer than
    n/3); each fact atom heads only its fact. Other heads are uniform over the non-fact atoms,
    body atoms uniform over all atoms, distinct within a body. Body lengths follow Table 1; with
    dense=True the lengths 1 and 2 keep their 4 % shares and every other rule takes each atom
    with probability 0.05 (a body of about 5 % of n), the lower-sparsity programs of Tables 3
    and 6. k > 0 negates one body occurrence of each of k distinct non-fact atoms (Tables 5, 6)."""
    rng = np.random.default_rng(seed)
    n_f = int(round(n * rng.uniform(0.1, 1.0 / 3.0)))
    perm = rng.permutation(n)
    facts, nonfacts = perm[:n_f], perm[n_f:]
    nr = m - n_f
    if dense:
        u = rng.random(nr)
        kind = np.where(u < 0.04, 1, np.where(u < 0.08, 2, 0))  # 0: about 5 % of n
        short = np.nonzero(kind > 0)[0]
        bodies = [None] * nr
        for r in short:
            bodies[r] = rng.choice(n, size=int(kind[r]), replace=False)
        wide = np.nonzero(kind == 0)[0]
        chunk = max(1, (64 << 20) // max(n, 1))
        for c0 in range(0, len(wide), chunk):
            rows = wide[c0:c0 + chunk]
            sel = rng.random((len(rows), n), dtype=np.float32) < 0.05
            sel[np.arange(len(rows)), rng.integers(0, n, len(rows))] = True  # never empty
            rr, cc = np.nonzero(sel)
            splits = np.searchsorted(rr, np.arange(1, len(rows)))
            for r, body in zip(rows, np.split(cc, splits)):
                bodies[r] = body
        lens = np.array([len(x) for x in bodies], dtype=np.int64)
        atoms = np.concatenate(bodies) if nr else np.zeros(0, np.int64)
        off = np.zeros(nr + 1, dtype=np.int64)
        np.cumsum(lens, out=off[1:])
    else:
        lens = np.minimum(rng.choice(np.arange(1, 9), size=nr, p=np.array(TABLE1_LENGTH_SHARE)), n).astype(np.int64)
        off = np.zeros(nr + 1, dtype=np.int64)
        np.cumsum(lens, out=off[1:])
        atoms = rng.integers(0, n, int(off[-1]))
        rule_of = np.repeat(np.arange(nr), lens)
        for _ in range(64):  # redraw repeated atoms of a body
            key = rule_of * n + atoms
            order = np.argsort(key, kind="stable")
            dup = np.zeros(len(key), dtype=bool)
            dup[order[1:]] = key[order[1:]] == key[order[:-1]]
            if not dup.any():
                break
            atoms[dup] = rng.integers(0, n, int(dup.sum()))
    heads = np.concatenate([facts, nonfacts[rng.integers(0, len(nonfacts), nr)]])
    all_lens = np.concatenate([np.zeros(n_f, np.int64), lens])
    negs = None
    if k > 0:
        negs = np.zeros(len(atoms), dtype=np.uint8)
        q = rng.choice(nonfacts, size=k, replace=False)
        for a in q:
            pos = np.nonzero(atoms == a)[0]
            if len(pos) == 0:  # the atom occurs in no body: put it into a random body
                pos = np.array([off[int(rng.integers(nr))]])
                atoms[pos[0]] = a
            negs[pos[int(rng.integers(len(pos)))]] = 1
    h, ln, a, ng = _permute_rules(rng, heads, all_lens, atoms, negs)
    return _pack(n, h, ln, a, ng, name="table1_dense" if dense else "table1", seed=seed, k=k)


def tiny_random(seed: int, n_atoms: int = 8, n_rules: int = 12, max_body: int = 3, p_fact: float = 0.2,
                p_neg: float = 0.0) -> Program:
    """Tiny random program for brute-force checks: heads and body atoms uniform (so facts may
    also head other rules, bodies may repeat an atom, heads may appear in their own body)."""
    rng = np.random.default_rng(seed)
    heads, lens, atoms, negs = [], [], [], []
    for _ in range(n_rules):
        heads.append(int(rng.integers(n_atoms)))
        m = 0 if rng.random() < p_fact else int(rng.integers(1, max_body + 1))
        lens.append(m)
        for _ in range(m):
            atoms.append(int(rng.integers(n_atoms)))
            negs.append(1 if rng.random() < p_neg else 0)
    return _pack(n_atoms, heads, lens, np.array(atoms, dtype=np.int64), negs if p_neg > 0 else None,
                 name="tiny_random", seed=seed)


def random_fact_subsets(prog: Program, b: int, seed: int = 1, p: float = 0.5) -> np.ndarray:
    """b initial interpretations, each keeping every fact atom independently with prob. p.
    Returns bool [b, n_atoms]."""
    rng = np.random.default_rng(seed)
    f = prog.fact_atoms()
    keep = rng.random((b, prog.n_atoms)) < p
    return keep & f[None, :]
