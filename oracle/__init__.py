"""FP64 CPU oracle of the cut chain and reconstruction -- TEST INFRASTRUCTURE.

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  The product path (the CUDA library and its binding)
never touches it.
"""
from .oracle import (build, load, run, records, best_of, unit, philox4x32_10, unit_normals,  # noqa: F401
                     w_pz, w_pz_both, hadtop, ttbar, real_roots, dilep_pairing, hist_bin, mass)
from . import hl  # noqa: F401,E402
