"""Seeded synthetic workloads shared by the oracle, the tests and the benchmark."""
from .synthetic import *  # noqa: F401,F403
