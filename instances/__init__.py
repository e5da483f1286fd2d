"""Seeded synthetic arrowhead LP instances.

This package only draws random data and builds the block pieces of an
arrowhead LP (the problem statement of Sec. 3.2, eq. (fig:blockstructure),
restricted to equality rows and x >= 0).  It holds none of the interior-point
method's arithmetic, so both the CPU oracle and the CUDA path may use it.
"""
from .generate import (  # noqa: F401
    BlockLP,
    random_block_lp,
    config0,
    config1,
    config2,
    config3,
    config4,
    tiny_lp,
    prefix,
    window,
    general_block_lp,
    CONFIGS,
)
