"""CPU oracle for the ChFSI hot path (TEST INFRASTRUCTURE).

Plain FP64 NumPy/SciPy restatement of the method, used only by the tests, the package
smoke check and the benchmark's CPU-baseline leg.  The GPU library never imports it.
"""
from .chfsi_oracle import *  # noqa: F401,F403
