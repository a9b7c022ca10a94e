"""CPU oracle for the shifted Green's-function path — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  The library under
``paper_1603_09616_gb300`` never calls it and shares no code with it.

It computes the plain definition the paper's order-N method rests on
(Introduction: the generalized shifted linear equations (zS - H) x = b, used
instead of the generalized eigenproblem H y = lambda S y): for every energy
shift z_k and unit right-hand side b = e_j, x = (z_k S - H)^{-1} e_j, i.e. the
column j of the Green's function G(z_k) = (z_k S - H)^{-1}, by a dense complex
LU factorisation per shift (FP64 / complex128), and then the Green's-function
reductions (local DOS, density-matrix and energy-density elements on the
sparsity pattern, local charge and local energy).  The paper itself notes that
a direct O(N^3) solver is the numerically exact complement of the order-N
solver (Introduction), which is why a direct solve serves as the reference.
"""
from . import fermi, forces, wavepacket  # noqa: F401
from .green import (  # noqa: F401
    green_columns,
    green_columns_sparse,
    project_columns,
    reduce_outputs,
    solve_outputs,
    pattern_offsets,
)
