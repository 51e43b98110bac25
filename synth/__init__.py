"""Seeded synthetic string networks: the inputs shared by the oracle and the GPU path.

This package only draws random configurations (string node positions, velocities,
tangents, Burden-loop parameters, shell geometry).  It contains none of the map
arithmetic of the method: no light-cone solve, no pixel directions, no Eq. (1)
sums.  Everything is drawn from ``numpy.random.Generator(PCG64(seed))``.
"""
from .strings import (  # noqa: F401
    Workload,
    NROWS,
    LOOP_PARAMS,
    MODE_LINEAR,
    MODE_BURDEN,
    burden_loop_params,
    burden_nodes,
    random_walk_strings,
    config,
    CONFIG_NAMES,
)
from .stacking import StackWorkload, base_pixel_centres, stack_config  # noqa: F401
