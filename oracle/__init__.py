"""Plain FP64 CPU oracle of the GameDev collision step (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs
may import this package.  See oracle/gdo.c for the implementation and citations.
"""
from . import gdo  # noqa: F401
