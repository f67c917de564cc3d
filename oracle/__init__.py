"""Oracle for the APM level solve (Passy & Bryan, arXiv:1410.0010).

TEST INFRASTRUCTURE ONLY.  A plain, slow FP64 CPU statement of the method,
used to check the CUDA path.  Only tests, the smoke check and the benchmark's
CPU-baseline leg import it; the product package never does, and nothing here
imports the product.

Every function's result is pinned by an independent check in the test suite
(closed forms, brute force, the paper's printed values, or, for the influence
function of Eq. influence, the real-space minimiser of the mesh-force error
that defines it).
"""
from .apm_oracle import *  # noqa: F401,F403
