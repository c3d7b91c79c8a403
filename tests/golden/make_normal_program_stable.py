"""Writes tests/golden/normal_program_seed1_stable.json: the oracle's Algorithms 2 + 3 (one
guess at a time, OpenMP over guesses) on every one of the 2^16 guesses of the 1e5-atom normal
program (300,000 rules, k = 16 negated atoms), the benchmark's stable-model workload.

Stored: the program's fingerprint (the test recomputes the mask with the oracle if the generator
ever yields another program), the stable guess indices, and per 64-guess word the largest
Algorithm 2 iteration count of its columns. Only oracle/ and workloads/ are called.

    python tests/golden/make_normal_program_stable.py      # about two CPU-core-hours (OpenMP)
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from tests.helpers import program_fingerprint  # noqa: E402
from workloads import normal_program  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "normal_program_seed1_stable.json")


def compute(prog):
    std = oracle.standardize(prog)
    st, _, iters = oracle.stable_models_alg23(prog, std=std, want_models=False)
    return std, st, iters


def main():
    t0 = time.time()
    prog = normal_program(seed=1)
    std, st, iters = compute(prog)
    k = len(std.guess_rows())
    rec = {
        "what": "Algorithms 2 + 3 (oracle O4) on all 2^k guesses of normal_program(seed=1)",
        "cite": "Sec. 2.2, Def. 8, Algorithms 2 and 3",
        "fingerprint": program_fingerprint(prog),
        "n_prime": int(std.n_prime),
        "k": int(k),
        "n_guesses": int(len(st)),
        "stable": [int(i) for i in np.nonzero(st)[0]],
        "word_max_iters": [int(x) for x in iters.reshape(-1, 64).max(axis=1)],
        "oracle_threads": oracle.num_threads(),
        "oracle_seconds": round(time.time() - t0, 1),
    }
    with open(OUT, "w") as f:
        json.dump(rec, f)
    print(f"wrote {OUT}: {len(rec['stable'])} stable of {rec['n_guesses']} in {rec['oracle_seconds']} s")


if __name__ == "__main__":
    main()
