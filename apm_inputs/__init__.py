"""Seeded synthetic inputs shaped like the test problems of Passy & Bryan
(arXiv:1410.0010, Sec. 3) and the benchmark workloads built on them.

This package holds none of the method's arithmetic (no deposit, Green's
function, FFT convolution, differencing or interpolation): only random draws,
analytic density fields and grid layouts.  Both the oracle-side and the
CUDA-side code receive their inputs from here.
"""
from .workloads import *  # noqa: F401,F403
