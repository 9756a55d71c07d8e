"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark.  This package holds only random-number generation and shaping of
ratings matrices; none of the factorisation method's arithmetic lives here.
"""
from .ratings import (  # noqa: F401
    Ratings, CONFIGS, make_config, make_ratings, init_factors, rank_degrees,
    sample_distinct, half_star_values, make_dense, foldin_requests, make_batch, c4_problems, C4_NF,
    TABLE_SHAPES, TABLE_DENSITY, table_problem,
)
from .scale_gpu import SCALE_STEPS, make_scale_gpu  # noqa: F401,E402
