"""Seeded synthetic tight-binding inputs for the shifted Green's-function path.

This package only *draws inputs*: sparse real-symmetric Hamiltonians H, SPD
overlaps S, energy shifts z_k, quadrature weights and right-hand-side column
lists.  It contains none of the solver's arithmetic, so both the CUDA library
(through its Python binding) and the CPU oracle may take their inputs from it
without sharing any method code.

The workloads stand in for the organic-polymer systems of the paper's
quantum-MD section (a PPV bundle of 169 chains x 50 monomers, Sec. "Quantum
molecular dynamics simulation"); the real structures are not public, so the
geometry here is a synthetic planar 14-atom phenylene-vinylene unit.
"""
from .tb import (  # noqa: F401
    TBSystem,
    align_blocks,
    displace,
    model_gradients,
    pole_weights,
    chain_4orb,
    ppv_chain,
    ppv_bundle,
    uneven_chains,
    uneven_batch,
    shift_grid,
    fermi_weights,
    random_columns,
    workload,
)
