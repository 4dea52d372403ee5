"""Seeded synthetic-input generators shared by the tests, the benchmark and the oracle
harness.  They draw random numbers only; none of the HOPE method's arithmetic lives here.
"""
from .inputs import noise_field, bump_centres, fd_direction, perturb_h  # noqa: F401
