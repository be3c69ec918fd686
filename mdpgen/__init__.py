"""Seeded synthetic MDP inputs shared by the tests, the benchmark and the oracle checks.

Only input generation lives here (Philox4x32-10 draws and the workload
shapes); nothing in this package computes Bellman operators, policies or
values.
"""
from .philox import philox4x32, stream, uniform53
from .generators import (MDPData, random_sparse, ragged_sparse, banded_birth_death, pendulum_grid, maze,
                         quantize_rows, random_value_vector, regenerate_rows, request_header, serving_request,
                         serving_request_philox, workload)

__all__ = ["philox4x32", "stream", "uniform53", "MDPData", "random_sparse", "ragged_sparse", "banded_birth_death",
           "pendulum_grid", "maze", "quantize_rows", "request_header", "serving_request", "serving_request_philox",
           "random_value_vector", "regenerate_rows", "workload"]
