"""Wavepacket propagation, d/dt Psi = -i H Psi in a non-orthogonal basis.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's transport simulations propagate a hole wavepacket with a
Schroedinger-type equation, starting from an eigenstate such as the HOMO
(Quantum wavepacket dynamics).  In the tight-binding basis with overlap S the
coefficients obey i S dc/dt = H c (time in units of hbar / eV), so
c(t) = exp(-i t S^-1 H) c(0).  With the generalized eigenpairs H y_l =
lambda_l S y_l, y_l^T S y_m = delta_lm, this is the plain spectral sum
    c(t) = sum_l y_l exp(-i lambda_l t) (y_l^T S c(0)).
"""
from __future__ import annotations

import numpy as np


def propagate(system, c0, t):
    """c(t) for every column of c0 [n, w] (complex), t in hbar / eV."""
    import scipy.linalg as sla

    H, S = system.dense()
    lam, Y = sla.eigh(H, S)
    c0 = np.asarray(c0, dtype=np.complex128)
    proj = Y.T @ (S @ c0)  # y_l^T S c(0)
    return Y @ (np.exp(-1j * lam * t)[:, None] * proj)


def s_norm(system, c):
    """c^H S c per column (conserved by the propagation)."""
    H, S = system.dense()
    c = np.asarray(c, dtype=np.complex128)
    return np.real(np.einsum("iw,ij,jw->w", c.conj(), S, c))


def homo(system, n_electrons, spin=2.0):
    """The highest occupied generalized eigenvector (S-normalised) and its energy."""
    import scipy.linalg as sla

    H, S = system.dense()
    lam, Y = sla.eigh(H, S)
    k = int(np.ceil(n_electrons / spin)) - 1
    return Y[:, k], lam[k]
