"""Chemical potential from the electron count, and the Fermi-weighted density
and energy-density matrices from the same Green's-function columns.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The order-N method obtains the density matrix of the molecular dynamics from
the Green's-function columns (Introduction; Quantum molecular dynamics
simulation: electronic structure at every MD step).  The occupation needs the
chemical potential mu, fixed by the electron count.  On an evenly spaced
real-axis shift grid z_k = eps_k + i eta (spacing d), with the Fermi function
f(x) = 1 / (1 + exp(x)) and spin degeneracy s:
  c_k(mu)   = -(s / pi) f((eps_k - mu) / kT) d        (density weights)
  c^E_k(mu) = eps_k c_k(mu)                           (energy-density weights)
  N(mu)     = sum_j q_j = sum_k c_k(mu) Im sum_j (G(z_k) S)_jj
            = -pi sum_k c_k(mu) D_k,   D_k = sum_j ldos[k, j]  (all orbitals j)
N is increasing in mu (every D_k > 0 for eta > 0), so mu solving N(mu) = N_e
is found by bisection.  rho_ij and P^E_ij then follow from the same G_ij(z_k)
through the reductions of green.reduce_outputs with these weights.
"""
from __future__ import annotations

import numpy as np

from .green import green_columns, project_columns, reduce_outputs


def fermi(x):
    """f(x) = 1 / (1 + e^x), evaluated without overflow."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    pos = x >= 0
    e = np.exp(-x[pos])
    out[pos] = e / (1.0 + e)
    out[~pos] = 1.0 / (1.0 + np.exp(x[~pos]))
    return out


def grid_spacing(eps):
    """Spacing of an evenly spaced grid (raises if it is not evenly spaced)."""
    eps = np.asarray(eps, dtype=np.float64)
    if len(eps) < 2:
        raise ValueError("need at least two shifts")
    d = (eps[-1] - eps[0]) / (len(eps) - 1)
    if not np.allclose(np.diff(eps), d, rtol=1e-9, atol=0.0) or not d > 0:
        raise ValueError("the real parts of the shifts must be evenly spaced and increasing")
    return d


def weights(eps, mu, kT, spin=2.0):
    """(c_k, c^E_k) of the real-axis rule at chemical potential mu."""
    eps = np.asarray(eps, dtype=np.float64)
    d = grid_spacing(eps)
    c = -(spin / np.pi) * fermi((eps - mu) / kT) * d
    return c.astype(np.complex128), (eps * c).astype(np.complex128)


def electron_count(eps, dos, mu, kT, spin=2.0):
    """N(mu) = -pi sum_k c_k(mu) D_k for the total DOS D_k = sum_j ldos[k, j]."""
    c, _ = weights(eps, mu, kT, spin)
    return float(-np.pi * np.sum(c.real * dos))


def fermi_level(eps, ldos, n_electrons, kT, spin=2.0, iters=200):
    """mu with N(mu) = n_electrons by bisection; ldos [K, n] over all orbitals."""
    eps = np.asarray(eps, dtype=np.float64)
    dos = np.asarray(ldos, dtype=np.float64).sum(axis=1)
    lo, hi = eps[0] - 40.0 * kT, eps[-1] + 40.0 * kT
    if not electron_count(eps, dos, lo, kT, spin) <= n_electrons <= electron_count(eps, dos, hi, kT, spin):
        raise ValueError("the electron count is outside what the shift grid can hold")
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if electron_count(eps, dos, mid, kT, spin) < n_electrons:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def fermi_outputs(system, z, n_electrons, kT, spin=2.0):
    """Solve every column (dense LU), find mu, and reduce with its weights."""
    z = np.asarray(z)
    cols = np.arange(system.n)
    H, S = system.dense()
    X = green_columns(H, S, z, cols)
    g = project_columns(system, X, cols)
    zero = np.zeros(len(z), dtype=np.complex128)
    ldos = reduce_outputs(system, g, cols, zero, zero)["ldos"]
    mu = fermi_level(z.real, ldos, n_electrons, kT, spin)
    c, ce = weights(z.real, mu, kT, spin)
    out = reduce_outputs(system, g, cols, c, ce)
    out["mu"] = mu
    out["g_proj"] = g
    return out


def sinv_terms(system, cols):
    """S^-1 and S^-1 H S^-1 on the pattern, packed like rho (dense inverse)."""
    from .forces import pack

    H, S = system.dense()
    Sinv = np.linalg.inv(S)
    return pack(system, Sinv, cols), pack(system, Sinv @ H @ Sinv, cols)


def outputs_with_sinv(system, z, cols, c_rho, c_edm, a_rho, b_edm, c_shs):
    """Shifted-solve reductions with weights (c_rho, c_edm), plus a_rho S^-1 in
    rho and b_edm S^-1 + c_shs S^-1 H S^-1 in P^E (the terms of a pole
    expansion of the Fermi function that are not resolvents); q and e_loc
    from the completed rho."""
    cols = np.asarray(cols)
    H, S = system.dense()
    X = green_columns(H, S, np.asarray(z), cols)
    g = project_columns(system, X, cols)
    out = reduce_outputs(system, g, cols, c_rho, c_edm)
    si, shs = sinv_terms(system, cols)
    out["rho"] = out["rho"] + a_rho * si
    out["edm"] = out["edm"] + b_edm * si + c_shs * shs
    off = out["off"]
    for c, j in enumerate(cols):
        lo, hi = int(system.row_ptr[j]), int(system.row_ptr[j + 1])
        r = out["rho"][off[c] : off[c + 1]]
        out["q"][c] = np.sum(r * system.s_val[lo:hi])
        out["e_loc"][c] = np.sum(r * system.h_val[lo:hi])
    return out
