"""lp_least_model_static -- the allocation-free least-model entry point -- against
lp_least_model.

Some callers cannot call cudaMalloc: code that runs under another framework's fixed device
memory pool or budget, or a latency-critical loop that cannot take the synchronisation an
allocation may cause. They keep the matrix in their own device buffers and call
lp_least_model_static, whose only scratch is a fixed array compiled into liblp. These tests
call it through the C ABI twice in a row on different programs (the second call starts
from whatever the first left in that array) and require each result, bit for bit, and its
iteration count to equal those of the handle-based lp_least_model (LP_ROWS mode) on the
same matrix and initial vector."""
import numpy as np
import pytest

import oracle
import paper_2009_10247_gb300 as lp
from workloads import large_definite, small_definite, transitive_closure

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import dev_words, from_dev_bits, to_dev_bits  # noqa: E402


def _reference_and_inputs(prog):
    """Canonical CSR + fact vector, and the existing entry point's fixpoint on them."""
    with lp.Program.from_program(prog) as P:
        m = P.export_matrix()
        n = P.info["n_prime"]
        v0 = m["kind"] == 3  # fact rows (Def. 4)
        ref = dev_words(n)
        ref_it = P.least_model(ref, init=to_dev_bits(v0), rows=True)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).to("cuda:0")  # noqa: E731
    return n, dev(m["row_ptr"]), dev(m["col"]), dev(m["threshold"]), to_dev_bits(v0), ref, ref_it


def test_static_entry_point_two_calls_in_a_row():
    cases = [large_definite(seed=3, n=200_000, n_rules=1_000_000, chain_levels=200, chain_width=20),
             small_definite(7)]
    inputs = [_reference_and_inputs(p) for p in cases]
    torch.cuda.synchronize()
    for n, row_ptr, col, thr, v0, ref, ref_it in inputs:  # two calls back to back
        out = dev_words(n)
        it = lp.least_model_static(n, row_ptr, col, thr, v0, out)
        torch.cuda.synchronize()
        assert it == ref_it
        assert torch.equal(out, ref), "fixpoint differs from lp_least_model"


def test_static_entry_point_in_place_and_after_larger_call():
    n, row_ptr, col, thr, v0, ref, ref_it = _reference_and_inputs(transitive_closure(60, 3.0, seed=2))
    buf = v0.clone()  # out may be v0 itself
    assert lp.least_model_static(n, row_ptr, col, thr, buf, buf) == ref_it
    torch.cuda.synchronize()
    assert torch.equal(buf, ref)


def test_static_entry_point_rejects_oversize_and_host_buffers():
    with pytest.raises(lp.LPError) as e:
        lp.least_model_static((1 << 24) + 1, None, None, None, None, None)
    assert e.value.status == 1 and "static scratch" in str(e.value)
    rp = np.zeros(2, np.int32)
    with pytest.raises(lp.LPError) as e:
        lp.least_model_static(1, rp, rp, rp, np.zeros(1, np.uint64), np.zeros(1, np.uint64))
    assert e.value.status == 1


def test_static_entry_point_equals_oracle():
    # the same fixpoint as the CPU oracle's Algorithm 1 (exact rational row sums) on the same
    # canonical matrix and fact vector, twice in a row
    prog = small_definite(8)
    s = oracle.standardize(prog)
    v0 = oracle.initial_vector(s)
    want, want_it, ok = oracle.alg1(s, v0)
    assert ok
    n, row_ptr, col, thr, v0_dev, _, _ = _reference_and_inputs(prog)
    assert n == s.n_prime
    for _ in range(2):
        out = dev_words(n)
        it = lp.least_model_static(n, row_ptr, col, thr, v0_dev, out)
        torch.cuda.synchronize()
        assert it == want_it
        assert np.array_equal(from_dev_bits(out, n), want.astype(bool))
