"""GB300-native shifted Green's-function solver (order-N electronic structure).

Solves (z_k S - H) x = e_j for many complex shifts and unit right-hand sides
with a shifted COCG of the library's own design, on hand-written sm_103a CUDA
kernels behind the C ABI in ``include/gbgreen.h``; Python only marshals
arguments (``_binding``).
"""
from ._binding import (  # noqa: F401
    EXPORTED,
    GB_FP64,
    GB_MIXED,
    GBError,
    Matrix,
    block_factor_to_host,
    add_sinv_terms,
    fermi_density,
    forces,
    wavepacket,
    bsr_to_host,
    load,
    pattern_offsets,
    shifted_solve,
    shifted_solve_batched,
    shifted_solve_static,
    solve_plan,
    true_residual,
    workspace_bytes,
)
