"""GB300 tree-tensor-network trajectory simulator for color-code circuits.

Thin Python binding over the C ABI in include/ttn.h (libttn.so, built in-tree
by `paper_2511_05719_gb300.build.build()`).  The binding only marshals
arguments; every step of the simulation runs in the library's CUDA kernels.
Importing the package does not load the library; the first call does, and
raises if it is missing.
"""
from ._lib import (  # noqa: F401
    NOISE, PRECISION, LAYOUT, TTNError, Circuit, run_trajectories, logical_error_rate,
    decode, debug_state, philox_uniforms, load_library, library_path,
    profile_begin, profile_end, KERNEL_CLASSES, grad, logical_error_rate_fn, decode_noalloc,
    run_mixed, newton_crossing, crossing, threshold_fit, grad_sums, gram_exact, eig_gram, Pipeline,
)
