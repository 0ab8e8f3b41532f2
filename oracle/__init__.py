"""CPU oracle for shape-adaptive motion estimation -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded C restatement of the paper's method (Fig. 1,
Sec. 3.1, Sec. 3.2, Eqs. 2-5) plus an exhaustive search that judges it.  Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
legs of ``bench.py`` may import this package.  The product path
(``paper_1002_1168_gb300``) never imports it; the two share no code.
"""
from .oracle import (  # noqa: F401
    OracleParams,
    build_oracle,
    classify_frame,
    compensate,
    compensate4,
    estimate_pair,
    estimate_pair4,
    estimate_sequence,
    estimate_sequence4,
    full_search,
    gradient_step,
    gradient_step_block,
    interp,
    psnr,
    shape_sad,
    texture_sad,
    valid_range,
)
