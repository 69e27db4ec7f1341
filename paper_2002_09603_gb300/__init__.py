"""GB300 (sm_103a) solver for the stabilized, hybridized Q1-RT0-P0
poromechanics system of arXiv:2002.09603 behind the C ABI of
``include/mhfp.h``.

The compute path is the CUDA library ``libmhfp.so`` (built in-tree by
``paper_2002_09603_gb300.build``); this package only marshals arguments.
"""
from ._lib import (Batch, MhfpError, Options, Solver, default_options, load,  # noqa: F401
                   prepare, launch_count, solve_batch, EXPORTS, LIB_PATH)
