"""Seeded synthetic inputs for the solar-tomography projector and its solver.

This package builds the *inputs* of the hot path — density cubes shaped like
the solar corona, observer pointing tables, pixel masks and noise draws — for
the workloads the projector is measured on.  It holds none of the method's
arithmetic (no ray construction, no Siddon walk, no solver): both the CUDA
path and the FP64 oracle consume what it produces, and nothing here calls
either of them.

The paper's own examples use STEREO/EUVI and STEREO/COR1 FITS data
(Section 5); those files are not available, so every recipe here is a seeded
stand-in with the shapes, sizes and structure of those workloads.
"""

from .geometry import (POINTING_COLUMNS, cube_geom, pointing_table,
                       cdelt_for_fov, voxel_centres)
from .corona import (radial_exp, radial_power, add_structures, random_axes,
                     uniform_noise, corona_cube, corona_frames)
from .masks import occulter_mask, shell_map_mask, height_weights
from .configs import (CONFIGS, make_config, noise_draw, add_noise,
                      problem_seeds_batched)

__all__ = [
    "POINTING_COLUMNS", "cube_geom", "pointing_table", "cdelt_for_fov",
    "voxel_centres", "radial_exp", "radial_power", "add_structures",
    "random_axes", "uniform_noise", "corona_cube", "corona_frames", "occulter_mask", "shell_map_mask", "height_weights",
    "CONFIGS", "make_config", "noise_draw", "add_noise",
    "problem_seeds_batched",
]
