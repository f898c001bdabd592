"""Seeded synthetic particle sets shaped like the workloads of the range-separated
tensor method (protein-like clusters, ionic lattices, serving traffic).

This package holds input generation only: positions, charges, arrival times and
the per-workload parameter files.  It contains none of the method's arithmetic
(no quadrature, factors, splitting, compression or potential evaluation), so both
the CPU oracle and the CUDA path may consume it.
"""
from .generate import (  # noqa: F401
    WORKLOADS, load_config, make_particles, make_serving_requests, seed_for,
)
