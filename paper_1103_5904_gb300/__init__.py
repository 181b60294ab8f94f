"""GB300-native Siddon projector, transpose and CG solver for solar
rotational tomography (the hot path of TomograPy, Barbey, Guennou & Auchere).

The compute lives in ``libtomo.so`` (CUDA for sm_103a, C ABI declared in
``include/tomo.h``); ``tomo`` is its thin binding and ``autograd`` wraps the
projector as a differentiable PyTorch operation.  Build the library with
``paper_1103_5904_gb300.build.build()``.
"""

from . import tomo  # noqa: F401
from .tomo import (Context, TomoError, default_context, load_library,  # noqa
                   tomo_project, tomo_backproject, tomo_solve,
                   tomo_prior_apply, tomo_count_segments,
                   tomo_project_batched, tomo_backproject_batched,
                   tomo_solve_batched, tomo_autotune,
                   tomo_set_plane_rules, tomo_walk_plan, project,
                   backproject, solve, prior_apply, count_segments)
from .autograd import TomoProject  # noqa: F401
