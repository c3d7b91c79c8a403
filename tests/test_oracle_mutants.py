"""The oracle's pins catch plausible mistakes.

Each case copies the oracle's C source, plants one mistake (a wrong comparison, a transposed
operand, a dropped step, an off-by-one), compiles the copy on the CPU and runs the pins of
test_oracle.py against it: at least one pin must fail. The committed oracle is not touched.
"""
import multiprocessing
import os
import shutil
import subprocess
import tempfile

import pytest

import oracle
from tests import test_oracle as pins

HERE = os.path.dirname(os.path.abspath(oracle.__file__))

MUTANTS = {
    "theta strict >": ("u[i] = s >= den[i] ? 1 : 0;", "u[i] = s > den[i] ? 1 : 0;"),
    "theta transposed operand": ("s += (int64_t)num[e] * v[col[e]];", "s += (int64_t)num[e] * v[i];"),
    "body not reduced to a set": ("if (u == 0 || buf[u - 1] != buf[i]) buf[u++] = buf[i];", "buf[u++] = buf[i];"),
    "AND weight 1/(m+1)": ("den[row] = (int32_t)m;", "den[row] = (int32_t)m + 1;"),
    "fact row not a self-loop": ("      col[cur[row]] = row;\n      num[cur[row]++] = 1;\n      den[row] = 1;",
                                 "      col[cur[row]] = 0;\n      num[cur[row]++] = 1;\n      den[row] = 1;"),
    "iteration count starts at 1": ("int64_t iters = 0;\n  for (;;) {\n    if (iters >= max_iters)",
                                    "int64_t iters = 1;\n  for (;;) {\n    if (iters >= max_iters)"),
    "barred row keeps guess of facts": ("v[i] = kind[i] == ORC_FACT ? 1 : 0;", "v[i] = kind[i] != ORC_EMPTY ? 1 : 0;"),
    "Algorithm 3 compares with 0": ("v[owner[j]] + v[j] != 1", "v[owner[j]] + v[j] == 0"),
    "reduct keeps the wrong rules": ("if (assume_true[body_atom[e]]) fires = 0;", "if (!assume_true[body_atom[e]]) fires = 0;"),
    "T_P ignores a body literal": ("} else if (!out[body_atom[e]]) {", "} else if (e > body_off[r] && !out[body_atom[e]]) {"),
    "new atoms before barred atoms": ("p->aux[r] = p->cnt[head[r]] >= 2 ? (int64_t)n + p->n_barred + p->n_aux++ : -1;",
                                      "p->aux[r] = p->cnt[head[r]] >= 2 ? (int64_t)n + p->n_aux++ : -1;"),
}

PIN_CASES = [
    lambda: pins.test_example1_matrix_coo_csr(),
    lambda: pins.test_example2_matrix(),
    lambda: pins.test_example1_iterates_by_hand(),
    lambda: pins.test_example2_stable_model_is_t(),
    lambda: [pins.test_least_model_three_ways(s) for s in range(20)],
    lambda: pins.test_duplicate_body_atoms_are_a_set(),
    lambda: pins.test_fact_that_heads_other_rules(),
    lambda: [pins.test_textbook_stable_models(t, e) for t, e in [
        ("p :- not q. q :- not p.", [["p"], ["q"]]), ("p :- not p.", []),
        ("a :- not b. b :- not a. c :- a. c :- b.", [["a", "c"], ["b", "c"]])]],
    lambda: [pins.test_stable_models_alg23_equals_gl_and_brute(s) for s in range(20)],
    lambda: pins.test_transitive_closure_matches_bfs(),
]


def _build_mutant(tmp, old, new):
    src = open(os.path.join(HERE, "oracle.c")).read()
    assert src.count(old) == 1, f"mutation site not unique/absent: {old!r}"
    open(os.path.join(tmp, "oracle.c"), "w").write(src.replace(old, new))
    shutil.copy(os.path.join(HERE, "oracle.h"), tmp)
    so = os.path.join(tmp, "libmutant.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", os.path.join(tmp, "oracle.c"), "-o", so],
                   check=True, capture_output=True)
    return so


def _run_pins(so_path):
    """Child process: load the given oracle library and run every pin case; return the
    names of the exceptions raised."""
    import oracle as o
    from tests import test_oracle_mutants as m
    o._lib = o.load(so_path)
    caught = []
    for case in m.PIN_CASES:
        try:
            case()
        except Exception as e:  # AssertionError or an error the mutant provokes
            caught.append(type(e).__name__)
    return caught


def _pins_against(so_path, timeout=20.0):
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(1) as pool:
        res = pool.apply_async(_run_pins, (so_path,))
        try:
            return res.get(timeout=timeout)
        except multiprocessing.TimeoutError:
            return ["Timeout"]  # a mutant that never reaches a fixpoint is caught too


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    old, new = MUTANTS[name]
    with tempfile.TemporaryDirectory() as tmp:
        caught = _pins_against(_build_mutant(tmp, old, new))
    assert caught, f"no pin caught the planted mistake: {name}"


def test_unmutated_copy_passes_all_pins():
    with tempfile.TemporaryDirectory() as tmp:
        caught = _pins_against(_build_mutant(tmp, "int orc_num_threads(void) {", "int orc_num_threads(void) {"))
    assert caught == []
