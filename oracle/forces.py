"""Atomic forces from the density and energy-density matrices.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The quantum molecular dynamics of the paper moves the atoms with forces from
the electronic structure of each step (Quantum molecular dynamics simulation).
For a non-orthogonal tight-binding model at fixed chemical potential the force
on atom a is the derivative of the grand potential, which by the
Hellmann-Feynman argument for the generalized eigenproblem H y = lambda S y is

    F_a = -Tr[rho dH/dR_a] + Tr[P^E dS/dR_a],

with rho and the energy-density matrix P^E exactly the two matrices the
shifted solve reduces to (rho = sum_l f_l y_l y_l^T times the spin factor,
P^E the same with lambda_l f_l).  dH/dR_a and dS/dR_a are nonzero only on the
sparsity pattern: entry (i, j) between two different atoms depends on the
positions of both, with gradient g_ij with respect to the atom of row i and
-g_ij with respect to the atom of column j (two-center elements).

`forces` evaluates the two traces entry by entry from the packed pattern
outputs of a solve of every orbital; `grand_potential` and `eigen_density`
give the exact (eigenvalue) quantities the finite-difference pin uses.
"""
from __future__ import annotations

import numpy as np

from .fermi import fermi
from .green import pattern_offsets


def forces(system, rho, edm, cols, grad_h, grad_s):
    """F [n_atoms, 3] from packed rho / P^E of columns ``cols`` (every orbital
    once) and the per-entry gradients grad_h, grad_s [3, nnz] (CSR order, with
    respect to the atom of the entry's row).

    Tr[rho dH/dR_a] = sum over pattern entries (i, j) of rho_ij dH_ij/dR_a,
    where dH_ij/dR_a = g_ij if atom(i) = a, -g_ij if atom(j) = a (a different
    atom), and 0 otherwise; rho_ij is read from column j of the packed output.
    """
    cols = np.asarray(cols)
    if np.sort(cols).tolist() != list(range(system.n)):
        raise ValueError("forces need every orbital solved once")
    off = pattern_offsets(system.row_ptr, cols)
    n_atoms = int(system.orb_atom.max()) + 1
    F = np.zeros((n_atoms, 3))
    for c, j in enumerate(cols):
        lo, hi = int(system.row_ptr[j]), int(system.row_ptr[j + 1])
        aj = int(system.orb_atom[j])
        for t, e in enumerate(range(lo, hi)):
            i = int(system.col_idx[e])  # entry (j, i) of the CSR; by symmetry (i, j) has the same value
            ai = int(system.orb_atom[i])
            if ai == aj:
                continue
            r_ij = rho[off[c] + t]  # rho_ij of column j
            p_ij = edm[off[c] + t]
            # the element (i, j) equals the CSR element (j, i): its gradient with
            # respect to atom(j) is grad[:, e], with respect to atom(i) it is -grad[:, e]
            g_h, g_s = grad_h[:, e], grad_s[:, e]
            F[aj] -= r_ij * g_h - p_ij * g_s
            F[ai] -= -(r_ij * g_h - p_ij * g_s)
    return F


def grand_potential(system, mu, kT, spin=2.0):
    """Omega(mu) = -spin kT sum_l log(1 + exp(-(lambda_l - mu) / kT)) from the
    generalized eigenvalues (the band grand potential at fixed mu)."""
    import scipy.linalg as sla

    H, S = system.dense()
    lam = sla.eigh(H, S, eigvals_only=True)
    x = -(lam - mu) / kT
    return float(-spin * kT * np.sum(np.logaddexp(0.0, x)))


def eigen_density(system, mu, kT, spin=2.0):
    """Dense rho = spin sum_l f_l y_l y_l^T and P^E = spin sum_l f_l lambda_l y_l y_l^T."""
    import scipy.linalg as sla

    H, S = system.dense()
    lam, Y = sla.eigh(H, S)
    f = fermi((lam - mu) / kT)
    rho = spin * (Y * f) @ Y.T
    edm = spin * (Y * (f * lam)) @ Y.T
    return rho, edm


def pack(system, dense, cols):
    """A dense matrix on the pattern, packed like the solve's rho (column j, rows R_j)."""
    cols = np.asarray(cols)
    off = pattern_offsets(system.row_ptr, cols)
    out = np.zeros(int(off[-1]))
    for c, j in enumerate(cols):
        rows = system.col_idx[system.row_ptr[j] : system.row_ptr[j + 1]]
        out[off[c] : off[c + 1]] = dense[rows, j]
    return out
