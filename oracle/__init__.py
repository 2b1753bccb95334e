"""FP64 CPU oracle for the Red-Green-Gray edge classification.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import GREEN, GRAY, RED, _load  # noqa: F401
