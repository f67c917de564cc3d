"""Oracle for the APM level solve (Passy & Bryan, arXiv:1410.0010).

TEST INFRASTRUCTURE ONLY.  A plain, slow FP64 CPU statement of the method,
used to check the CUDA path.  Only tests, the smoke check and the benchmark's
CPU-baseline leg import it; the product package never does, and nothing here
imports the product.

Functions whose result is not pinned by an independent check in the test suite
say so in their docstring ("parity unpinned").
"""
from .apm_oracle import *  # noqa: F401,F403
