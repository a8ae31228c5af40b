"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench."""
from .rmat import EdgeLog, make_log, max_out_degree_vertex, random_small_log, rmat_endpoints  # noqa: F401
from .configs import (SSSP, SSWP, BFS, SSNP, TYPE_NAMES, Query, small_rmat, rmat20, rmat22, rmat24,  # noqa: F401
                      scaled_rmat, rmat20_queries, batch_queries, rmat24_queries, serve_requests)
