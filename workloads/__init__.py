"""Seeded synthetic logic programs shaped like the paper's workloads.

This module only draws inputs: it holds no part of the fixpoint method. Both the CUDA
library's tests/benchmark and the CPU oracle take their programs from here.
"""
from .programs import (  # noqa: F401
    Program,
    from_rules,
    parse,
    tiny_random,
    small_definite,
    large_definite,
    transitive_closure,
    transitive_closure_edges,
    transitive_closure_pairs,
    normal_program,
    program_batch,
    table1_program,
    TABLE1_LENGTH_SHARE,
    random_fact_subsets,
)
