"""FP64 CPU oracle for the sparse w-projection hot path.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check in
__graft_entry__.py and by the CPU-baseline leg of bench.py, never by the
product package.  See wproj_oracle.py for the model and the paper's passages.
"""
from . import wproj_oracle  # noqa: F401
