"""GB300 SPH neighbour search with Neighbour Recycling (arXiv:1810.09898).

The compute path is the CUDA library ``_build/libsphgrp.so`` (C ABI in
``include/sphgrp.h``); this package only marshals arguments to it.  Nothing here falls
back to a CPU implementation: if the library is missing or no GPU is present the
calls raise.
"""

from .binding import (  # noqa: F401
    BATCH_BACKWARD,
    BATCH_GRAPH,
    CENTRE_BOX,
    Batch,
    CENTRE_FIRST,
    DENSITY,
    GROUP_COUNT,
    GROUP_RADIUS,
    GROUP_TREE,
    GROUPED,
    HYDRO,
    INDIVIDUAL,
    ITER_IN_GROUP,
    ITER_PASSES,
    ITER_RECYCLE,
    SphgrpError,
    Context,
    kernel_launches,
    library_path,
    sfc_keys_sort_static,
    load_library,
)
from .autograd import SPHForces, sph_forces  # noqa: F401,E402
