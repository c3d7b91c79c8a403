"""GPU parity of the relaxed (differentiable) fixpoint against the FP64 oracle.

Forward values and both gradient groups (rule weights, initial vectors) must match the FP64
reference within a relative error of 1e-4 (||g - g_ref|| / ||g_ref|| per group); the result must
not depend on the checkpoint interval; at tau = 1e-3 the relaxed iterates are the exact
Algorithm 1 iterates; and the torch.autograd path returns the same gradients."""
import numpy as np
import pytest

import oracle
from oracle.relaxed import RelaxedProgram
import paper_2009_10247_gb300 as lp
from workloads import large_definite, small_definite, tiny_random

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2009_10247_gb300.relaxed import relaxed_fixpoint  # noqa: E402

DEV = "cuda:0"


def _rel(a, b):
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def _run(prog, w, v0, c, T, tau, ckpt):
    P = lp.Program.from_program(prog)
    b = v0.shape[1]
    wt = torch.tensor(w, dtype=torch.float32, device=DEV)
    v0t = torch.tensor(v0, dtype=torch.float32, device=DEV)
    ck, sc = P.relaxed_workspace(b, T, ckpt)
    ckb = torch.empty(ck, dtype=torch.float32, device=DEV)
    vT = torch.empty_like(v0t)
    P.relaxed_forward(wt, v0t, b, T, tau, ckpt, ckb, vT)
    scratch = torch.empty(sc, dtype=torch.float32, device=DEV)
    dw = torch.empty_like(wt)
    dv0 = torch.empty_like(v0t)
    P.relaxed_backward(wt, torch.tensor(c, dtype=torch.float32, device=DEV), b, T, tau, ckpt, ckb, scratch, dw, dv0)
    torch.cuda.synchronize()
    P.close()
    return vT.cpu().numpy(), dw.cpu().numpy(), dv0.cpu().numpy()


def _case(prog, seed, b, T, tau, v0_binary=False):
    rng = np.random.default_rng(seed)
    R = RelaxedProgram(prog)
    w = rng.uniform(0.5, 1.5, R.n_rules)
    if v0_binary:
        v0 = np.repeat((R.kind == oracle.ORC_FACT).astype(np.float64)[:, None], b, axis=1)
        v0 *= rng.random(v0.shape) < 0.5
    else:
        v0 = rng.uniform(0.0, 1.0, (R.n_prime, b))
    c = rng.uniform(-1.0, 1.0, (R.n_prime, b))
    vs = R.forward(w, v0, T, tau)
    dw_ref, dv0_ref = R.backward(w, vs, c, tau)
    return R, w, v0, c, vs[-1], dw_ref, dv0_ref


@pytest.mark.parametrize("seed", range(6))
def test_tiny_programs(seed):
    prog = tiny_random(300 + seed, n_atoms=int(10 + 7 * seed), n_rules=int(20 + 15 * seed), max_body=4, p_fact=0.25)
    R, w, v0, c, vT_ref, dw_ref, dv0_ref = _case(prog, seed, b=5, T=10, tau=0.3)
    vT, dw, dv0 = _run(prog, w, v0, c, 10, 0.3, 4)
    assert np.max(np.abs(vT - vT_ref)) < 1e-5
    assert _rel(dw, dw_ref) < 1e-4
    assert _rel(dv0, dv0_ref) < 1e-4


def test_small_definite_batch_40():
    prog = small_definite(3)
    R, w, v0, c, vT_ref, dw_ref, dv0_ref = _case(prog, 7, b=40, T=16, tau=0.1, v0_binary=True)
    vT, dw, dv0 = _run(prog, w, v0, c, 16, 0.1, 8)
    assert np.max(np.abs(vT - vT_ref)) < 1e-4
    assert _rel(dw, dw_ref) < 1e-4
    assert _rel(dv0, dv0_ref) < 1e-4


def test_checkpoint_interval_does_not_change_results():
    prog = small_definite(4)
    R, w, v0, c, _, _, _ = _case(prog, 3, b=33, T=13, tau=0.2)
    ref = _run(prog, w, v0, c, 13, 0.2, 13)
    for ck in (1, 3, 8):
        got = _run(prog, w, v0, c, 13, 0.2, ck)
        for a, b_ in zip(got, ref):
            assert np.array_equal(a, b_)


def test_hardening_reproduces_exact_iterates():
    prog = small_definite(5)
    R = RelaxedProgram(prog)
    s = R.std
    T = 30
    v = oracle.initial_vector(s)
    v0 = np.repeat(v.astype(np.float64)[:, None], 3, axis=1)
    w = np.random.default_rng(0).uniform(0.5, 1.5, R.n_rules)
    vT, _, _ = _run(prog, w, v0, np.zeros_like(v0), T, 1e-3, 8)
    for _ in range(T):
        v = oracle.theta_step(s, v)
    for j in range(3):
        assert np.array_equal(vT[:, j] > 0.5, v.astype(bool))
    assert np.all(np.minimum(vT, 1 - vT) < 1e-4)


def test_full_size_hardening_equals_least_model():
    # the relaxed workload's program and launch shape (1e5 atoms, 4e5 rules, chain depth 12;
    # T = 32, checkpoint every 8, 256 columns of fact subsets kept with probability 1/2), hardened
    # at tau = 1e-3: every column of v_32 is within 1e-4 of 0 or 1 and, thresholded at 1/2, equals
    # the exact Algorithm 1 iterate v_32 from that column. Where Algorithm 1 reaches its fixpoint
    # within 32 steps (most columns), that is the least model of the program with the column's
    # fact subset, which the oracle's least model confirms.
    prog = large_definite(seed=5, n=100_000, n_rules=400_000, chain_levels=12, chain_width=50)
    R = RelaxedProgram(prog)
    s = R.std
    rng = np.random.default_rng(1)
    b, T = 256, 32
    w = rng.uniform(0.5, 1.5, R.n_rules)
    fact = np.nonzero(s.kind == oracle.ORC_FACT)[0]
    v0 = np.zeros((R.n_prime, b))
    v0[fact] = rng.random((len(fact), b)) < 0.5
    vT, _, _ = _run(prog, w, v0, np.zeros_like(v0), T, 1e-3, 8)
    assert np.all(np.minimum(vT, 1 - vT) < 1e-4)
    converged = []
    for j in range(b):
        v, it, ok = oracle.alg1(s, v0[:, j].astype(np.uint8), max_iters=T)  # v = v_T, or the fixpoint
        assert np.array_equal(vT[:, j] > 0.5, v.astype(bool)), f"column {j} differs from Algorithm 1"
        if ok:
            converged.append(j)
    assert len(converged) >= 0.9 * b, f"only {len(converged)} of {b} columns reach the fixpoint within {T} steps"
    for j in converged[:: max(1, len(converged) // 8)]:  # the reference: the least model of the fact subset
        subset = np.zeros(s.n, dtype=bool)
        subset[s.owner[fact[v0[fact, j] > 0.5]]] = True
        lm, _ = oracle.least_model(prog, init=subset, std=s)
        assert np.array_equal(vT[: s.n, j] > 0.5, lm)


def test_autograd_function():
    prog = small_definite(6)
    R, w, v0, c, vT_ref, dw_ref, dv0_ref = _case(prog, 11, b=8, T=12, tau=0.2)
    P = lp.Program.from_program(prog)
    wt = torch.tensor(w, dtype=torch.float32, device=DEV, requires_grad=True)
    v0t = torch.tensor(v0, dtype=torch.float32, device=DEV, requires_grad=True)
    vT = relaxed_fixpoint(P, wt, v0t, 12, 0.2, 4)
    loss = (torch.tensor(c, dtype=torch.float32, device=DEV) * vT).sum()
    loss.backward()
    assert np.max(np.abs(vT.detach().cpu().numpy() - vT_ref)) < 1e-5
    assert _rel(wt.grad.cpu().numpy(), dw_ref) < 1e-4
    assert _rel(v0t.grad.cpu().numpy(), dv0_ref) < 1e-4
    P.close()


def test_full_size_program_reduced_batch():
    # the relaxed workload's program (1e5 atoms, 4e5 rules, chain depth 12), T = 32, tau = 0.05,
    # checkpoint every 8; batch of 8 columns of random fact subsets (the oracle's cost)
    prog = large_definite(seed=5, n=100_000, n_rules=400_000, chain_levels=12, chain_width=50)
    R, w, v0, c, vT_ref, dw_ref, dv0_ref = _case(prog, 1, b=8, T=32, tau=0.05, v0_binary=True)
    vT, dw, dv0 = _run(prog, w, v0, c, 32, 0.05, 8)
    assert np.max(np.abs(vT - vT_ref)) < 1e-3
    assert _rel(dw, dw_ref) < 1e-4
    assert _rel(dv0, dv0_ref) < 1e-4


def test_full_size_bench_batch_sampled_columns():
    # the benchmark's launch configuration: the relaxed workload's program with a batch of 256
    # columns (float4 rows, one 256-column warp pass), T = 32, tau = 0.05, checkpoint every 8.
    # Columns are independent in the forward pass, so the oracle checks a sample S of them; the
    # cotangent is zero outside S, so dL/dw is the oracle's sum over S and dL/dv0 vanishes
    # outside S.
    prog = large_definite(seed=5, n=100_000, n_rules=400_000, chain_levels=12, chain_width=50)
    R = RelaxedProgram(prog)
    rng = np.random.default_rng(11)
    b, T, tau = 256, 32, 0.05
    w = rng.uniform(0.5, 1.5, R.n_rules)
    v0 = np.repeat((R.kind == oracle.ORC_FACT).astype(np.float64)[:, None], b, axis=1)
    v0 *= rng.random(v0.shape) < 0.5
    S = np.array([0, 3, 127, 128, 200, 255])
    c = np.zeros((R.n_prime, b))
    c[:, S] = rng.uniform(-1.0, 1.0, (R.n_prime, len(S)))
    vT, dw, dv0 = _run(prog, w, v0, c, T, tau, 8)
    vs = R.forward(w, v0[:, S], T, tau)
    dw_ref, dv0_ref = R.backward(w, vs, c[:, S], tau)
    assert np.max(np.abs(vT[:, S] - vs[-1])) < 1e-3
    assert _rel(dw, dw_ref) < 1e-4
    assert _rel(dv0[:, S], dv0_ref) < 1e-4
    rest = np.setdiff1d(np.arange(b), S)
    assert not np.any(dv0[:, rest])


@pytest.mark.parametrize("b,T,ck", [(1, 1, 1), (1, 5, 100), (4, 1, 8), (7, 6, 6), (2, 9, 4)])
def test_edge_sizes(b, T, ck):
    # one column, one step, a checkpoint interval longer than the run, T a multiple of it
    prog = small_definite(7)
    R, w, v0, c, vT_ref, dw_ref, dv0_ref = _case(prog, 20 + T, b=b, T=T, tau=0.25)
    vT, dw, dv0 = _run(prog, w, v0, c, T, 0.25, ck)
    assert np.max(np.abs(vT - vT_ref)) < 1e-5
    assert _rel(dw, dw_ref) < 1e-4
    assert _rel(dv0, dv0_ref) < 1e-4


def test_rejects_host_buffers_and_bad_arguments():
    prog = small_definite(2)
    with lp.Program.from_program(prog) as P:
        n_prime = P.info["n_prime"]
        ck, sc = P.relaxed_workspace(4, 8, 4)
        w = torch.ones(len(prog.head), dtype=torch.float32, device=DEV)
        v0 = torch.zeros((n_prime, 4), dtype=torch.float32, device=DEV)
        ckpt = torch.empty(ck, dtype=torch.float32, device=DEV)
        vT = torch.empty_like(v0)
        with pytest.raises(lp.LPError):  # host input
            P.relaxed_forward(w, v0.cpu().numpy(), 4, 8, 0.1, 4, ckpt, vT)
        with pytest.raises(lp.LPError):  # tau must be positive
            P.relaxed_forward(w, v0, 4, 8, 0.0, 4, ckpt, vT)
        with pytest.raises(lp.LPError):  # at least one step
            P.relaxed_forward(w, v0, 4, 0, 0.1, 4, ckpt, vT)
        P.relaxed_forward(w, v0, 4, 8, 0.1, 4, ckpt, vT)  # still usable after the rejections
        torch.cuda.synchronize()
        assert torch.isfinite(vT).all()
