"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This package holds geometry and parameter generation only (water boxes, rock-salt
lattices, random charge vectors).  It contains none of the electrostatics or
dynamics arithmetic: both the CUDA path and the CPU oracle receive the arrays it
produces and compute from them independently.
"""

from .serving import serving_stream  # noqa: F401
from .water import (  # noqa: F401
    WaterBox,
    water_box,
    water_box_length,
    serving_mesh_size,
    random_neutral_charges,
    rocksalt_lattice,
    simple_cubic_lattice,
    O_MASS,
    H_MASS,
    WATER_DENSITY,
)
