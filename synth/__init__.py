"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This package holds no arithmetic of the factorization itself: it only draws the
matrices and right-hand sides that the workloads are defined on.
"""
from .generators import (  # noqa: F401
    SEED_BASE,
    seed_for,
    normals,
    uniforms,
    dominant_spd,
    paper_spd,
    rbf_spd,
    gram_spd,
    wide_range_spd,
    rhs,
    known_factor,
)
