"""GB300-native (sm_103a, FP64) asynchrony-tolerant finite differences (Aditya & Donzis, arXiv:1702.00496).

The computation lives in libatfd.so (CUDA kernels behind the C ABI of include/at.h); this package is
its ctypes binding plus device-memory plumbing.  There is no CPU fallback: if the library cannot be
built or loaded, the calls raise.
"""
from .binding import (AT_AT, AT_AT_SPACE1, AT_AT_SPACE2, AT_ASYNC_STD, AT_SYNC, ATError, Config,  # noqa: F401
                      at_coeffs, at_delay, at_destroy, at_error_stats, at_error_stats_ref, at_init, at_last_error,
                      at_num_sides, at_ring_slots, at_solve_stencil,
                      at_reset, at_set_fusion, at_set_launch, at_state, at_stencil_taps, at_step, at_sync, load)
from .solver import Ensemble, Solver  # noqa: F401
from .autograd import ATForward, at_forward  # noqa: F401
