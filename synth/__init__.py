"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the bench.

This package draws random numbers and lays out arrays; it contains none of the
periodogram arithmetic, so both sides of every parity check can use it.
"""
from .workloads import *  # noqa: F401,F403
