"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This package only draws inputs (tables, graphs, basic graph patterns); it holds
none of the join arithmetic.
"""
from .rng import Rng, mix64, zipf_ranks  # noqa: F401
from .tables import Table, pairwise_uniform, skewed_two_key, uneven_batch, random_table  # noqa: F401
from .university import university_graph, PREDICATES, N_PREDICATES  # noqa: F401
