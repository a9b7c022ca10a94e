"""Plain reference of the per-orbital environment descriptor — TEST INFRASTRUCTURE ONLY.

64 features per orbital j (atom a, species s_a, orbital slot o) from the
pattern row j of (H, S) and the atom positions; r_ab distances in nm,
w(r) = (cos(pi r / 0.5) + 1) / 2 for r < 0.5 nm:
  0-15   sum over carbon neighbour atoms b of w(r) exp(-((r - mu_t) / 0.03)^2),
         mu_t = 0.1 + 0.4 t / 15
  16-31  the same over hydrogen neighbour atoms
  32-39  per shell k (r in [k, k+1) * 0.125 nm, last shell closed at 0.5):
         |sum_b w u_b|^2 and ||sum_b w (u_b u_b^T - I/3)||_F^2, u_b = unit vector
  40-41  species one-hot, 42-45 orbital-slot one-hot (slot capped at 3)
  46 H_jj, 47 S_jj
  48-55  sum_{i != j} H_ji^2 exp(-((H_ii - c_t) / 0.75)^2), c_t = -3 + 6 t / 7
  56 sum H_ji^2, 57 sum S_ji^2, 58 sum H_ji S_ji, 59 sum H_ji^2 H_ii,
  60 sum |H_ji|, 61 |R_j| / 100, 62 sum S_ji H_ii (sums over i != j), 63 = 1
Neighbour atoms are the atoms of the row's orbitals (each counted once, the
own atom excluded).
"""
from __future__ import annotations

import numpy as np


def descriptors(system, species):
    pos = system.positions
    orb_atom = system.orb_atom
    first = np.zeros(len(system.atom_norb) + 1, dtype=np.int64)
    np.cumsum(system.atom_norb, out=first[1:])
    diag = np.array([system.h_val[system.row_ptr[i] + np.searchsorted(system.row_cols(i), i)] for i in range(system.n)])
    out = np.zeros((system.n, 64))
    for j in range(system.n):
        a = orb_atom[j]
        f = out[j]
        rows = system.row_cols(j)
        lo = system.row_ptr[j]
        dip = np.zeros((4, 3))
        quad = np.zeros((4, 3, 3))
        seen = set()
        for t, i in enumerate(rows):
            h = system.h_val[lo + t]
            s = system.s_val[lo + t]
            if i == j:
                f[46], f[47] = h, s
                continue
            hii = diag[i]
            for k in range(8):
                c = -3.0 + 6.0 * k / 7.0
                f[48 + k] += h * h * np.exp(-(((hii - c) / 0.75) ** 2))
            f[56] += h * h
            f[57] += s * s
            f[58] += h * s
            f[59] += h * h * hii
            f[60] += abs(h)
            f[62] += s * hii
            b = orb_atom[i]
            if b == a or b in seen:
                continue
            seen.add(b)
            d = pos[b] - pos[a]
            r = np.linalg.norm(d)
            if not (r > 1e-6) or r >= 0.5:
                continue
            w = 0.5 * (np.cos(np.pi * r / 0.5) + 1.0)
            base = 16 if species[b] else 0
            for k in range(16):
                mu = 0.1 + 0.4 * k / 15.0
                f[base + k] += w * np.exp(-(((r - mu) / 0.03) ** 2))
            sh = min(3, int(r / 0.125))
            u = d / r
            dip[sh] += w * u
            quad[sh] += w * (np.outer(u, u) - np.eye(3) / 3.0)
        for k in range(4):
            f[32 + 2 * k] = np.dot(dip[k], dip[k])
            f[33 + 2 * k] = np.sum(quad[k] * quad[k])
        f[40 + (1 if species[a] else 0)] = 1.0
        f[42 + min(3, j - first[a])] = 1.0
        f[61] = len(rows) / 100.0
        f[63] = 1.0
    return out
