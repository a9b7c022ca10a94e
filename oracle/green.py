"""Plain FP64 oracle: dense LU per shift, then the Green's-function reductions.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Nothing here is tuned:
one LU factorisation of z_k S - H per shift, one triangular solve per block of
unit columns, and the reductions written out as sums over the pattern.

Definitions (the paper fixes only the equation (zS - H) x = b, Introduction;
the reductions are the standard Green's-function outputs of an order-N
electronic-structure code):
  G(z)            = (z S - H)^{-1}                       complex symmetric
  x^k_j           = G(z_k) e_j                            solution column
  R_j             = { i : (j, i) in the sparsity pattern }  (row set of column j)
  ldos[k, c]      = -(1/pi) Im (G(z_k) S)_{jj} = -(1/pi) Im sum_{i in R_j} G_ij S_ij
  rho_ij          = sum_k Im( c^rho_k G_ij(z_k) ),   i in R_j
  edm_ij          = sum_k Im( c^E_k  G_ij(z_k) ),    i in R_j
  q_j             = sum_{i in R_j} rho_ij S_ij       (local charge)
  e_j             = sum_{i in R_j} rho_ij H_ij       (local energy)
(G S)_jj only needs i in R_j because S_ij = 0 outside the pattern.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def pattern_offsets(row_ptr: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """Offsets of each requested column's pattern block in the packed outputs.

    Column c (orbital j = cols[c]) owns entries [off[c], off[c+1]) of the
    packed rho / edm arrays, in the pattern's (sorted) row order.
    """
    m = (row_ptr[cols + 1] - row_ptr[cols]).astype(np.int64)
    off = np.zeros(len(cols) + 1, dtype=np.int64)
    np.cumsum(m, out=off[1:])
    return off


def green_columns(H: np.ndarray, S: np.ndarray, z: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """Dense solve of (z_k S - H) X = E[:, cols] for every shift (Introduction).

    Returns X with shape [n_shift, n, n_cols], complex128.
    """
    n = H.shape[0]
    cols = np.asarray(cols)
    E = np.zeros((n, len(cols)), dtype=np.complex128)
    E[cols, np.arange(len(cols))] = 1.0
    X = np.empty((len(z), n, len(cols)), dtype=np.complex128)
    for k, zk in enumerate(z):
        A = zk * S.astype(np.complex128) - H.astype(np.complex128)
        lu = sla.lu_factor(A, check_finite=False)
        X[k] = sla.lu_solve(lu, E, check_finite=False)
    return X


def green_columns_sparse(system, z: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """Sparse direct solve (SuperLU) of (z_k S - H) x = e_j, for large systems.

    Same definition as :func:`green_columns`; returns only the projected rows
    R_j of each column, shape [n_shift] list of packed arrays (pattern order).
    """
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    Hs = system.h_csr().astype(np.complex128)
    Ss = system.s_csr().astype(np.complex128)
    cols = np.asarray(cols)
    off = pattern_offsets(system.row_ptr, cols)
    out = np.empty((len(z), int(off[-1])), dtype=np.complex128)
    n = system.n
    for k, zk in enumerate(z):
        A = sp.csc_matrix(zk * Ss - Hs)
        lu = spla.splu(A)
        for c, j in enumerate(cols):
            b = np.zeros(n, dtype=np.complex128)
            b[j] = 1.0
            x = lu.solve(b)
            out[k, off[c] : off[c + 1]] = x[system.row_cols(int(j))]
    return out


def project_columns(system, X: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """Keep only rows R_j of each solved column: packed [n_shift, sum_j m_j]."""
    cols = np.asarray(cols)
    off = pattern_offsets(system.row_ptr, cols)
    out = np.empty((X.shape[0], int(off[-1])), dtype=np.complex128)
    for c, j in enumerate(cols):
        out[:, off[c] : off[c + 1]] = X[:, system.row_cols(int(j)), c]
    return out


def reduce_outputs(system, G_proj: np.ndarray, cols: np.ndarray, w_rho, w_edm) -> dict:
    """Green's-function reductions from the projected columns (module docstring).

    G_proj[k, off[c] + t] = G_{i j}(z_k) with j = cols[c] and i the t-th entry
    of R_j.  Returns ldos [n_shift, n_cols], gs_diag (complex (G S)_jj),
    rho / edm (packed like G_proj's second axis), q and e_loc [n_cols].
    """
    cols = np.asarray(cols)
    off = pattern_offsets(system.row_ptr, cols)
    n_shift = G_proj.shape[0]
    gs = np.zeros((n_shift, len(cols)), dtype=np.complex128)
    rho = np.zeros(int(off[-1]))
    edm = np.zeros(int(off[-1]))
    q = np.zeros(len(cols))
    e_loc = np.zeros(len(cols))
    for c, j in enumerate(cols):
        lo, hi = int(system.row_ptr[j]), int(system.row_ptr[j + 1])
        s_row = system.s_val[lo:hi]
        h_row = system.h_val[lo:hi]
        g = G_proj[:, off[c] : off[c + 1]]  # [n_shift, m_j]
        for k in range(n_shift):
            gs[k, c] = np.sum(g[k] * s_row)
        r = np.zeros(hi - lo)
        e = np.zeros(hi - lo)
        for k in range(n_shift):
            r += np.imag(w_rho[k] * g[k])
            e += np.imag(w_edm[k] * g[k])
        rho[off[c] : off[c + 1]] = r
        edm[off[c] : off[c + 1]] = e
        q[c] = np.sum(r * s_row)
        e_loc[c] = np.sum(r * h_row)
    ldos = -np.imag(gs) / np.pi
    return dict(ldos=ldos, gs_diag=gs, rho=rho, edm=edm, q=q, e_loc=e_loc, off=off)


def solve_outputs(system, z, cols, w_rho, w_edm, keep_full: bool = False) -> dict:
    """Dense-LU solve of every (shift, column) pair followed by the reductions."""
    H, S = system.dense()
    X = green_columns(H, S, np.asarray(z), np.asarray(cols))
    G_proj = project_columns(system, X, cols)
    out = reduce_outputs(system, G_proj, cols, w_rho, w_edm)
    out["g_proj"] = G_proj
    if keep_full:
        out["x_full"] = X
    return out
