"""FP64 CPU oracle for the subset-correlation hot path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library never does, and the two
share no code: see ``dic_oracle`` for what is computed and which passage of the
paper each step follows.
"""
from .dic_oracle import *  # noqa: F401,F403
from .dic_oracle import (AFFINE, BICUBIC, BSPLINE3, DEFAULT_PARAMS, GAUSS_NEWTON, LEVENBERG_MARQUARDT, N_PARAMS, NSSD,  # noqa: F401
                         QUADRATIC, RIGID, SSD, ZNSSD, Plane,
                         ReferenceSubset, bspline_coefficients, correlate, correlate_sequence, grid, icgn,
                         interpolate, keys, seed_search)
from . import fft_oracle, incremental_oracle, strain_oracle  # noqa: F401
