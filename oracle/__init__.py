"""FP64 CPU oracle for Pinv-Recon: test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package. The library in paper_2410_06129_gb300/ never does.
"""
from .pinv_oracle import *  # noqa: F401,F403
