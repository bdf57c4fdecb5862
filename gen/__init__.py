"""Seeded input generators shared by the tests, the bench and the oracle's
callers.  Holds no solver arithmetic."""
from . import problems  # noqa: F401
