"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

Holds no analysis arithmetic: event columns (events.py) and plain-data
analysis descriptions (analyses.py) only.
"""
from .events import Columns, SEMILEP, DILEP, gen_semilep, gen_dilep, concat  # noqa: F401
from . import analyses  # noqa: F401
