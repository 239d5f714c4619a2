"""GB300-native constrained forward-dynamics step (Kamino, arXiv 2603.16536).

The compute path is the CUDA library built from ``csrc/`` (C ABI in ``include/kamino.h``);
``kamino`` is its Python binding.  Build with ``paper_2603_16536_gb300.build.build()``.
"""
from .kamino import (  # noqa: F401
    FP32, FP64, MIXED, WARM_CACHED, WARM_COLD, WARM_EXTERNAL, KaminoError, Model, State, SolverParams,
    load_library, make_params,
)
