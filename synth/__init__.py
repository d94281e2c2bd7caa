"""Seeded synthetic inputs for the mini-batch quasi-Newton proximal method.

This module is shared by the FP64 oracle, the tests and the benchmark.  It
holds geometry and random draws only: phantoms, illumination directions,
subset partitions, raw noise draws and the named workload configurations.
It contains none of the method's arithmetic (no Green's function, no solver,
no TV, no metric).  Every array is produced in float64/complex128 on the host
from ``numpy.random.default_rng`` (PCG64), so both implementations receive
identical bytes after casting.

Seeds: phantom = 1000*config_id + 0, noise = +1, strategy-II draws = +2,
power-iteration start vector = +3.
"""
from .workloads import (  # noqa: F401
    Workload,
    WORKLOADS,
    workload,
    phantom,
    illumination_dirs,
    subsets,
    noise_draws,
    strategy2_draws,
    power_start,
    uneven_requests,
    small,
)
