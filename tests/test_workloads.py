"""Shape of the seeded generators that stand in for the paper's random programs (Sec. 4,
Table 1): body-length shares, facts, the denser variant's 5 % bodies, negated atoms, and the
standardized size n' against the sizes the paper prints for the same (n, m)."""
import numpy as np
import pytest

import oracle
from workloads import TABLE1_LENGTH_SHARE, table1_program


def _lens(p):
    return np.diff(p.body_off)


def test_table1_length_shares():
    p = table1_program(1, 2000, 40000)
    L = _lens(p)
    body = L[L > 0]
    share = np.bincount(body, minlength=9)[1:9] / len(body)
    assert np.allclose(share, TABLE1_LENGTH_SHARE, atol=0.01)
    # facts: fewer than n/3, each heading only its fact
    facts = p.head[L == 0]
    assert 0.1 * 2000 - 1 <= len(facts) < 2000 / 3
    assert len(np.unique(facts)) == len(facts)
    assert not np.isin(p.head[L > 0], facts).any()


def test_bodies_are_sets():
    for dense in (False, True):
        p = table1_program(3, 1000, 5000, dense=dense)
        for r in range(0, p.n_rules, 97):
            b = p.body_atom[p.body_off[r]:p.body_off[r + 1]]
            assert len(np.unique(b)) == len(b)


def test_dense_bodies_are_about_five_percent():
    p = table1_program(2, 2000, 10000, dense=True)
    L = _lens(p)
    body = L[L > 0]
    wide = body[body > 2]
    assert abs(wide.mean() / 2000 - 0.05) < 0.003
    assert abs((body <= 2).mean() - 0.08) < 0.02


def test_negated_atoms():
    p = table1_program(4, 1000, 5000, k=7)
    negated = np.unique(p.body_atom[p.body_neg.astype(bool)])
    assert len(negated) == 7
    facts = p.head[_lens(p) == 0]
    assert not np.isin(negated, facts).any()
    assert oracle.standardize(p).n_barred == 7


@pytest.mark.parametrize("n,m,n_prime", [(1000, 5000, 5788), (1000, 10000, 10799), (1600, 24000, 25198),
                                         (2000, 40000, 41936)])
def test_standardized_size_close_to_paper(n, m, n_prime):
    # Table 2 prints n' for each (n, m); the generator's fact share is drawn, so allow 3 %
    s = oracle.standardize(table1_program(7, n, m))
    assert abs(s.n_prime - n_prime) / n_prime < 0.03


def test_transitive_closure_edges_shape():
    from workloads import transitive_closure_edges
    for nv, ne in [(65, 95), (28, 217), (5, 20)]:
        p = transitive_closure_edges(nv, ne, seed=3)
        e = p.meta["edges"]
        assert len(e) == min(ne, nv * (nv - 1))
        assert len({(int(a), int(b)) for a, b in e}) == len(e)  # distinct
        assert not np.any(e[:, 0] == e[:, 1])                   # no self-loops
        assert p.n_atoms == len(e) + nv * nv
        assert p.n_rules == 2 * len(e) + len(e) * nv            # facts, base rules, recursive rules


@pytest.mark.parametrize("nv,ne,n,m,n_prime", [(28, 217, 1512, 20629, 21924), (62, 159, 7564, 230861, 238266),
                                               (77, 254, 11704, 445006, 456456)])
def test_pair_grounding_reproduces_table4_sizes(nv, ne, n, m, n_prime):
    # Table 4 prints n, m and n' per graph; grounding over all ordered pairs / triples of
    # distinct nodes gives exactly those sizes
    from workloads import transitive_closure_pairs
    p = transitive_closure_pairs(nv, ne, seed=1)
    assert (p.n_atoms, p.n_rules) == (n, m)
    assert oracle.standardize(p).n_prime == n_prime
