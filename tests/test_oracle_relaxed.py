"""Pins of the FP64 relaxed-fixpoint oracle (no GPU): a hand closed form, hardening to the
exact Algorithm 1 iterates as tau -> 0, and central finite differences of its forward pass
against its reverse-mode gradients."""
import numpy as np
import pytest

import oracle
from oracle.relaxed import RelaxedProgram
from workloads import parse, small_definite, tiny_random


def test_closed_form_rule_row():
    # p <- q & r with q = 1, r = 1/2 (self-loops): x_p = 3/4, x - 1 + 1/(2m) = 0, so u_p = 1/2
    # for every weight and temperature.
    p = parse("p :- q, r. q. r.", atoms=["p", "q", "r"])
    R = RelaxedProgram(p)
    v0 = np.array([[0.0], [1.0], [0.5]])
    for tau in (0.05, 1.0):
        vs = R.forward(np.array([1.7, 1.0, 1.0]), v0, 1, tau)
        assert vs[1][0, 0] == pytest.approx(0.5, abs=1e-15)
        assert vs[1][1, 0] == 1.0 and vs[1][2, 0] == 0.5  # self-loops keep their value


def test_closed_form_or_row():
    # p <- q and p <- r: p is an OR row over two new atoms a <- q, b <- r (m = 1).
    p = parse("p :- q. p :- r. q. r.", atoms=["p", "q", "r"])
    R = RelaxedProgram(p)
    assert list(R.kind[:3]) == [oracle.ORC_OR, oracle.ORC_FACT, oracle.ORC_FACT]
    v0 = np.array([[0.0], [1.0], [0.0], [0.0], [0.0]])
    tau, w = 0.5, np.array([2.0, 3.0, 1.0, 1.0])
    vs = R.forward(w, v0, 2, tau)
    sig = lambda z: 1.0 / (1.0 + np.exp(-z))  # noqa: E731
    a = sig(2.0 * (1.0 - 1.0 + 0.5) / tau)  # new atom of p <- q
    b = sig(3.0 * (0.0 - 1.0 + 0.5) / tau)  # new atom of p <- r
    assert vs[1][3, 0] == pytest.approx(a) and vs[1][4, 0] == pytest.approx(b)
    assert vs[2][0, 0] == pytest.approx(sig((a + b - 0.5) / tau))


@pytest.mark.parametrize("seed", range(8))
def test_hardening_matches_algorithm1(seed):
    prog = small_definite(seed + 1) if seed < 2 else tiny_random(seed, n_atoms=12, n_rules=25, max_body=4, p_fact=0.3)
    R = RelaxedProgram(prog)
    s = R.std
    v = oracle.initial_vector(s)
    w = np.random.default_rng(seed).uniform(0.5, 1.5, R.n_rules)
    T = 20
    vs = R.forward(w, v.astype(np.float64)[:, None], T, 1e-3)
    for t in range(T):
        v = oracle.theta_step(s, v)
        assert np.array_equal(vs[t + 1][:, 0] > 0.5, v.astype(bool)), f"step {t + 1}"
        assert np.all(np.minimum(vs[t + 1][:, 0], 1 - vs[t + 1][:, 0]) < 1e-6)


@pytest.mark.parametrize("seed", range(6))
def test_finite_differences(seed):
    rng = np.random.default_rng(seed)
    prog = tiny_random(50 + seed, n_atoms=9, n_rules=16, max_body=3, p_fact=0.25)
    R = RelaxedProgram(prog)
    b, T, tau = 2, 6, 0.4
    w = rng.uniform(0.5, 1.5, R.n_rules)
    v0 = rng.uniform(0.0, 1.0, (R.n_prime, b))
    c = rng.uniform(-1.0, 1.0, (R.n_prime, b))

    def loss(w_, v0_):
        return float(np.sum(c * R.forward(w_, v0_, T, tau)[-1]))

    dw, dv0 = R.backward(w, R.forward(w, v0, T, tau), c, tau)
    h = 1e-6
    num_w = np.array([(loss(w + h * e, v0) - loss(w - h * e, v0)) / (2 * h) for e in np.eye(len(w))])
    num_v = np.zeros_like(v0)
    for i in range(v0.shape[0]):
        for j in range(b):
            d = np.zeros_like(v0)
            d[i, j] = h
            num_v[i, j] = (loss(w, v0 + d) - loss(w, v0 - d)) / (2 * h)
    assert np.allclose(dw, num_w, rtol=1e-5, atol=1e-8)
    assert np.allclose(dv0, num_v, rtol=1e-5, atol=1e-8)
    facts = np.diff(prog.body_off) == 0
    assert np.all(dw[facts] == 0.0)  # facts carry no weight
