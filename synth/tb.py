"""Seeded synthetic tight-binding systems, shift grids and quadrature weights.

Every function here is deterministic in its ``seed`` and draws with
``numpy.random.default_rng``.  Matrices come back as one CSR pattern shared by
H and S (sorted columns, symmetric pattern, full per-atom orbital blocks,
explicit zeros kept), which is the input format of both the CUDA library's
builder and the oracle.

Matrix-element rules (the "distance-decay" rules of the workloads):
  * onsite block of atom a: H diagonal ~ N(0, 1) eV, H off-diagonal 0;
    S = identity (before the diagonal-dominance fix below);
  * atom pair (a, b), a != b, at reduced distance d: every orbital pair gets
    H = -2.7 * exp(-(d - 1)) * U(0.5, 1) and S = 0.1 * exp(-d) * U(0, 1),
    drawn once for a < b and mirrored (H_ba = H_ab^T, same for S);
  * S is then made strictly diagonally dominant,
    S_ii = max(1, 1.01 * sum_{j != i} |S_ij|), hence SPD by Gershgorin.
For the 4-orbital chain, d is the site separation |i - j| (1..3); for the
polymer geometries d = r / r0 with r0 = 0.14 nm (a C-C bond).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

R0_NM = 0.14  # reference bond length for the reduced distance d = r / r0
PPV_REPEAT_NM = 0.66  # monomer repeat length along the chain axis


@dataclass
class TBSystem:
    """A sparse tight-binding pair (H, S) on one shared CSR pattern."""

    n: int
    row_ptr: np.ndarray  # int64 [n+1]
    col_idx: np.ndarray  # int32 [nnz]
    h_val: np.ndarray  # float64 [nnz]
    s_val: np.ndarray  # float64 [nnz]
    orb_atom: np.ndarray  # int32 [n] atom index of each orbital
    name: str = ""
    positions: np.ndarray | None = None  # float64 [n_atoms, 3] (nm), if geometric
    atom_norb: np.ndarray | None = None  # int32 [n_atoms]
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def h_csr(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.h_val, self.col_idx, self.row_ptr), shape=(self.n, self.n))

    def s_csr(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.s_val, self.col_idx, self.row_ptr), shape=(self.n, self.n))

    def dense(self):
        return self.h_csr().toarray(), self.s_csr().toarray()

    def row_cols(self, j: int) -> np.ndarray:
        """Orbitals i with (j, i) in the pattern (= the row set of column j)."""
        return self.col_idx[self.row_ptr[j] : self.row_ptr[j + 1]]


def _assemble(atom_norb, pair_a, pair_b, pair_d, rng, name, positions=None):
    """Build the shared-pattern CSR of H and S from atoms and interacting pairs."""
    atom_norb = np.asarray(atom_norb, dtype=np.int64)
    n_atoms = atom_norb.shape[0]
    off = np.zeros(n_atoms + 1, dtype=np.int64)
    np.cumsum(atom_norb, out=off[1:])
    n = int(off[-1])
    orb_atom = np.repeat(np.arange(n_atoms, dtype=np.int32), atom_norb)

    onsite_h = rng.standard_normal(n)

    pair_a = np.asarray(pair_a, dtype=np.int64)
    pair_b = np.asarray(pair_b, dtype=np.int64)
    pair_d = np.asarray(pair_d, dtype=np.float64)
    order = np.lexsort((pair_b, pair_a))
    pair_a, pair_b, pair_d = pair_a[order], pair_b[order], pair_d[order]
    na = atom_norb[pair_a]
    nb = atom_norb[pair_b]
    cnt = na * nb
    total = int(cnt.sum())
    u_h = rng.uniform(0.5, 1.0, total)
    u_s = rng.uniform(0.0, 1.0, total)

    # expand every pair block into orbital-pair entries (row-major inside the block)
    pid = np.repeat(np.arange(pair_a.shape[0]), cnt)
    start = np.zeros(pair_a.shape[0] + 1, dtype=np.int64)
    np.cumsum(cnt, out=start[1:])
    local = np.arange(total, dtype=np.int64) - start[pid]
    nb_e = nb[pid]
    r_loc = local // nb_e
    c_loc = local % nb_e
    rows_p = off[pair_a[pid]] + r_loc
    cols_p = off[pair_b[pid]] + c_loc
    d_e = pair_d[pid]
    h_p = -2.7 * np.exp(-(d_e - 1.0)) * u_h
    s_p = 0.1 * np.exp(-d_e) * u_s

    # onsite blocks: full na x na pattern, diagonal values only
    cnt_on = atom_norb * atom_norb
    tot_on = int(cnt_on.sum())
    aid = np.repeat(np.arange(n_atoms), cnt_on)
    st_on = np.zeros(n_atoms + 1, dtype=np.int64)
    np.cumsum(cnt_on, out=st_on[1:])
    loc_on = np.arange(tot_on, dtype=np.int64) - st_on[aid]
    na_on = atom_norb[aid]
    r_on = off[aid] + loc_on // na_on
    c_on = off[aid] + loc_on % na_on
    diag = r_on == c_on
    h_on = np.where(diag, onsite_h[r_on], 0.0)
    s_on = np.where(diag, 1.0, 0.0)

    rows = np.concatenate([r_on, rows_p, cols_p])
    cols = np.concatenate([c_on, cols_p, rows_p])
    hv = np.concatenate([h_on, h_p, h_p])
    sv = np.concatenate([s_on, s_p, s_p])
    o = np.lexsort((cols, rows))
    rows, cols, hv, sv = rows[o], cols[o], hv[o], sv[o]
    if rows.shape[0] > 1:
        dup = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if dup.any():
            raise ValueError("duplicate orbital pair in the interaction list")

    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    np.cumsum(row_ptr, out=row_ptr)

    # diagonal dominance of S: S_ii = max(1, 1.01 * sum_{j != i} |S_ij|)
    offd = np.where(rows != cols, np.abs(sv), 0.0)
    rsum = np.zeros(n)
    np.add.at(rsum, rows, offd)
    is_diag = rows == cols
    sv[is_diag] = np.maximum(1.0, 1.01 * rsum[rows[is_diag]])

    return TBSystem(
        n=n,
        row_ptr=row_ptr,
        col_idx=cols.astype(np.int32),
        h_val=hv,
        s_val=sv,
        orb_atom=orb_atom,
        name=name,
        positions=positions,
        atom_norb=atom_norb.astype(np.int32),
    )


def chain_4orb(n_sites: int = 200, seed: int = 0, reach: int = 3) -> TBSystem:
    """1-D chain of ``n_sites`` sites x 4 orbitals; sites |i-j| <= reach couple.

    The 800-orbital case (200 sites) is the plain-FP64 parity workload.
    """
    rng = np.random.default_rng(seed)
    a, b, d = [], [], []
    for i in range(n_sites):
        for s in range(1, reach + 1):
            if i + s < n_sites:
                a.append(i)
                b.append(i + s)
                d.append(float(s))
    return _assemble(np.full(n_sites, 4), a, b, d, rng, name=f"chain4orb_{n_sites}")


def _ppv_monomer():
    """Planar 14-atom phenylene-vinylene unit: 8 C (4 orbitals) then 6 H (1 orbital).

    Positions in nm, chain axis x, molecular plane xy; repeat length 0.66 nm.
    """
    ang = np.deg2rad(np.arange(0, 360, 60))
    ring = np.stack([0.14 * np.cos(ang), 0.14 * np.sin(ang), np.zeros(6)], axis=1)
    c7 = np.array([0.265, 0.035, 0.0])
    c8 = np.array([0.395, -0.035, 0.0])
    carbons = np.vstack([ring, c7, c8])
    h_ring = [np.array([0.248 * np.cos(t), 0.248 * np.sin(t), 0.0]) for t in ang[[1, 2, 4, 5]]]
    h7 = np.array([0.250, 0.140, 0.0])
    h8 = np.array([0.410, -0.140, 0.0])
    hydrogens = np.vstack(h_ring + [h7, h8])
    pos = np.vstack([carbons, hydrogens])
    norb = np.array([4] * 8 + [1] * 6)
    return pos, norb


def _pairs_within(pos: np.ndarray, cutoff: float):
    from scipy.spatial import cKDTree

    pairs = cKDTree(pos).query_pairs(cutoff, output_type="ndarray")
    if pairs.shape[0] == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0)
    a = np.minimum(pairs[:, 0], pairs[:, 1]).astype(np.int64)
    b = np.maximum(pairs[:, 0], pairs[:, 1]).astype(np.int64)
    r = np.linalg.norm(pos[a] - pos[b], axis=1)
    return a, b, r


def ppv_chain(n_mono: int = 50, seed: int = 1, disorder: float = 0.02, cutoff: float = 0.4) -> TBSystem:
    """Single synthetic PPV-like chain of ``n_mono`` monomers (38 orbitals each).

    ``disorder`` is the Gaussian positional noise as a fraction of r0 = 0.14 nm.
    """
    rng = np.random.default_rng(seed)
    mono, norb = _ppv_monomer()
    pos = np.vstack([mono + np.array([m * PPV_REPEAT_NM, 0.0, 0.0]) for m in range(n_mono)])
    pos = pos + rng.normal(0.0, disorder * R0_NM, pos.shape)
    atom_norb = np.tile(norb, n_mono)
    a, b, r = _pairs_within(pos, cutoff)
    sys_ = _assemble(atom_norb, a, b, r / R0_NM, rng, name=f"ppv_{n_mono}", positions=pos)
    sys_.meta.update(n_mono=n_mono, cutoff=cutoff, disorder=disorder)
    return sys_


def align_blocks(system: TBSystem) -> TBSystem:
    """The same system with its orbitals renumbered so that every 4-orbital
    atom starts on a multiple of 4 (one whole 4x4 block of the BSR format).

    Atoms keep their order except that, wherever a 4-orbital atom would start
    off a block boundary, 1-orbital atoms from the next few that follow move
    in front of it until the boundary is reached, choosing those whose
    couplings reach least far forward (for the PPV chains: two hydrogens of
    every odd monomer move ahead of its carbons).  H and S are
    permuted as P H P^T, P S P^T, so the physics is unchanged; the locality of
    the numbering (and the band of S) is kept.
    """
    norb = np.asarray(system.atom_norb)
    n_atoms = norb.shape[0]
    off = np.zeros(n_atoms + 1, dtype=np.int64)
    np.cumsum(norb, out=off[1:])
    # furthest orbital each atom couples to (its first orbital's pattern row)
    reach = system.col_idx[system.row_ptr[off[1:]] - 1] if n_atoms else np.zeros(0, np.int64)
    placed = np.zeros(n_atoms, dtype=bool)
    order = []
    pos = 0
    for a in range(n_atoms):
        if placed[a]:
            continue
        if norb[a] == 4 and pos % 4 != 0:
            # the next few unplaced 1-orbital atoms are candidates; those that
            # reach least far forward move (the band of S grows least)
            cand = []
            b = a + 1
            while b < n_atoms and len(cand) < 8:
                if not placed[b] and norb[b] == 1:
                    cand.append(b)
                b += 1
            need = (4 - pos % 4) % 4
            for b in sorted(cand, key=lambda x: (reach[x], x))[:need]:
                order.append(b)
                placed[b] = True
                pos += 1
        order.append(a)
        placed[a] = True
        pos += int(norb[a])
    perm = np.concatenate([np.arange(off[a], off[a + 1]) for a in order])  # perm[new] = old orbital
    H = system.h_csr()[perm][:, perm].tocsr()
    S = system.s_csr()[perm][:, perm].tocsr()
    H.sort_indices()
    S.sort_indices()
    if not (np.array_equal(H.indptr, S.indptr) and np.array_equal(H.indices, S.indices)):
        raise ValueError("H and S must share one pattern")
    inv_atom = np.empty(n_atoms, dtype=np.int64)
    inv_atom[np.asarray(order)] = np.arange(n_atoms)
    out = TBSystem(n=system.n, row_ptr=H.indptr.astype(np.int64), col_idx=H.indices.astype(np.int32),
                   h_val=H.data.astype(np.float64), s_val=S.data.astype(np.float64),
                   orb_atom=inv_atom[system.orb_atom[perm]].astype(np.int32), name=system.name + "_aligned",
                   positions=None if system.positions is None else system.positions[np.asarray(order)],
                   atom_norb=norb[np.asarray(order)].astype(np.int32), meta=dict(system.meta))
    out.meta["orbital_perm"] = perm
    return out


def _interatomic(system: TBSystem):
    """Per CSR entry: row and column atoms, and the mask of entries between two
    different atoms (the only entries that depend on positions; requires the
    diagonal of S to sit at 1, i.e. the diagonal-dominance fix inactive)."""
    if system.positions is None:
        raise ValueError("the system has no atomic positions")
    rows = np.repeat(np.arange(system.n), np.diff(system.row_ptr))
    ai = system.orb_atom[rows].astype(np.int64)
    aj = system.orb_atom[system.col_idx].astype(np.int64)
    s_diag = system.s_val[rows == system.col_idx]
    if not np.all(s_diag == 1.0):
        raise ValueError("S's diagonal depends on positions for this system (diagonal-dominance fix active)")
    return ai, aj, ai != aj


def model_gradients(system: TBSystem):
    """Gradients of H_ij and S_ij with respect to the position of the atom of
    orbital i, per CSR entry ([3, nnz] each, nm^-1 units times the element).

    Both decay rules are exponentials in d = r / r0, so dH_ij/dr = -H_ij / r0 and
    dS_ij/dr = -S_ij / r0 along the unit vector from the column atom to the row
    atom; entries within one atom do not depend on positions (zero).  These are
    inputs of the force calculation, like H and S themselves.
    """
    ai, aj, inter = _interatomic(system)
    d = system.positions[ai] - system.positions[aj]  # [nnz, 3]
    r = np.linalg.norm(d, axis=1)
    unit = np.zeros_like(d)
    unit[inter] = d[inter] / r[inter, None]
    gh = (-system.h_val / R0_NM)[:, None] * unit
    gs = (-system.s_val / R0_NM)[:, None] * unit
    gh[~inter] = 0.0
    gs[~inter] = 0.0
    return np.ascontiguousarray(gh.T), np.ascontiguousarray(gs.T)


def displace(system: TBSystem, atom: int, delta) -> TBSystem:
    """The same system with one atom moved by ``delta`` (nm): every element
    between that atom and another is rescaled by exp(-(r' - r) / r0), the
    decay rules' dependence on distance (the random factors stay)."""
    ai, aj, inter = _interatomic(system)
    pos = np.array(system.positions, dtype=np.float64, copy=True)
    r_old = np.linalg.norm(pos[ai] - pos[aj], axis=1)
    pos[atom] += np.asarray(delta, dtype=np.float64)
    r_new = np.linalg.norm(pos[ai] - pos[aj], axis=1)
    touched = inter & ((ai == atom) | (aj == atom))
    f = np.ones(system.nnz)
    f[touched] = np.exp(-(r_new[touched] - r_old[touched]) / R0_NM)
    return TBSystem(n=system.n, row_ptr=system.row_ptr, col_idx=system.col_idx, h_val=system.h_val * f,
                    s_val=system.s_val * f, orb_atom=system.orb_atom, name=system.name + "_displaced",
                    positions=pos, atom_norb=system.atom_norb, meta=dict(system.meta))


def ppv_bundle(
    n_side: int = 13,
    n_mono: int = 50,
    spacing: float = 0.45,
    sigma: float = 0.05,
    cutoff: float = 0.5,
    seed: int = 3,
) -> TBSystem:
    """``n_side`` x ``n_side`` bundle of PPV-like chains along x (condensed polymer).

    Chains sit on a square lattice of ``spacing`` nm in the (y, z) plane, each
    rotated about its axis by a random angle and shifted along it by a random
    fraction of a repeat; every atom then gets N(0, sigma) nm noise per axis.
    """
    rng = np.random.default_rng(seed)
    mono, norb = _ppv_monomer()
    chain = np.vstack([mono + np.array([m * PPV_REPEAT_NM, 0.0, 0.0]) for m in range(n_mono)])
    blocks = []
    for iy in range(n_side):
        for iz in range(n_side):
            th = rng.uniform(0.0, 2.0 * np.pi)
            shift = rng.uniform(0.0, PPV_REPEAT_NM)
            c, s = np.cos(th), np.sin(th)
            rot = np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
            p = chain @ rot.T + np.array([shift, iy * spacing, iz * spacing])
            blocks.append(p)
    pos = np.vstack(blocks)
    pos = pos + rng.normal(0.0, sigma, pos.shape)
    atom_norb = np.tile(norb, n_mono * n_side * n_side)
    a, b, r = _pairs_within(pos, cutoff)
    sys_ = _assemble(atom_norb, a, b, r / R0_NM, rng, name=f"bundle_{n_side}x{n_side}x{n_mono}", positions=pos)
    sys_.meta.update(n_side=n_side, n_mono=n_mono, spacing=spacing, sigma=sigma, cutoff=cutoff)
    return sys_


def uneven_chains(n_chains: int = 512, seed: int = 2, mono_range=(2, 50), shift_range=(32, 256)):
    """Independent chains of uneven size, each with its own shift count.

    Returns a list of (TBSystem, n_shift) with monomer counts uniform in
    ``mono_range`` and shift counts uniform in ``shift_range`` (inclusive).
    """
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_chains):
        n_mono = int(rng.integers(mono_range[0], mono_range[1] + 1))
        n_shift = int(rng.integers(shift_range[0], shift_range[1] + 1))
        sub_seed = int(rng.integers(0, 2**31 - 1))
        out.append((ppv_chain(n_mono, seed=sub_seed), n_shift))
    return out


def uneven_batch(n_chains: int = 512, cols_per_chain: int = 2, seed: int = 2, eta: float = 0.02,
                 tol: float = 1e-6, maxit: int = 16000, align: bool = False):
    """The uneven-chain batch with sampled right-hand sides per chain.

    Chains as in ``uneven_chains`` (2..50 monomers, 32..256 shifts each on
    [-15, 10] eV + i*eta); each chain gets ``cols_per_chain`` distinct random
    unit right-hand sides (always including its first orbital), Fermi weights
    and the common tolerance / iteration cap.  With ``align`` every chain is
    renumbered by align_blocks (same draws otherwise).  Returns (systems,
    problems).
    """
    rng = np.random.default_rng(seed + 7919)
    systems, problems = [], []
    for sysm, k in uneven_chains(n_chains, seed=seed):
        if align:
            sysm = align_blocks(sysm)
        z = shift_grid(-15.0, 10.0, k, eta)
        w_rho, w_edm = fermi_weights(z)
        extra = rng.choice(np.arange(1, sysm.n), size=cols_per_chain - 1, replace=False)
        cols = np.sort(np.concatenate([[0], extra])).astype(np.int32)
        systems.append(sysm)
        problems.append(dict(z=z, cols=cols, w_rho=w_rho, w_edm=w_edm, tol=tol, maxit=maxit))
    return systems, problems


def shift_grid(e_min: float, e_max: float, n_shift: int, eta: float) -> np.ndarray:
    """Energy shifts z_k = eps_k + i*eta, eps_k evenly spaced on [e_min, e_max]."""
    return np.linspace(e_min, e_max, n_shift) + 1j * eta


def fermi_weights(z: np.ndarray, mu: float = 0.0, kT: float = 0.1):
    """Complex quadrature weights for the density and energy-density matrices.

    Real-axis rule with spin degeneracy 2 on the (evenly spaced) shift grid:
    c_rho_k = -(2/pi) f(eps_k) d_eps and c_edm_k = eps_k * c_rho_k, with f the
    Fermi function at chemical potential ``mu`` and temperature ``kT`` (eV).
    The library only forms sum_k Im(c_k G(z_k)); it never picks mu or kT.
    """
    eps = z.real
    de = (eps[-1] - eps[0]) / max(len(eps) - 1, 1)
    f = 0.5 * (1.0 - np.tanh((eps - mu) / (2.0 * kT)))
    c_rho = (-(2.0 / np.pi) * f * de).astype(np.complex128)
    c_edm = (eps * c_rho.real).astype(np.complex128)
    return c_rho, c_edm


def pole_weights(mu: float = 0.0, kT: float = 0.1, n_poles: int = 40, spin: float = 2.0):
    """Shifts and weights of a pole expansion of the Fermi function (a complex
    shift set for the same solve, instead of the real-axis grid).

    The continued fraction of tanh truncated at depth 2 n_poles gives
    f(x) = 1 / (1 + e^x) ~= 1/2 + sum_p R_p [1 / (x - i a_p) + 1 / (x + i a_p)]
    with a_p = 1 / b_p and R_p = -v_p,1^2 / (4 b_p^2) from the positive
    eigenvalues b_p (eigenvectors v_p) of the symmetric tridiagonal matrix with
    off-diagonal 1 / (2 sqrt((2m - 1)(2m + 1))), m = 1 .. 2 n_poles - 1.  With
    x = (eps - mu) / kT the poles are w_p = mu + i kT a_p (the first at
    i pi kT) and, for the generalized problem,
      rho / s = 1/2 S^-1 - 2 kT sum_p R_p Re G(w_p),
      P^E / s = 1/2 S^-1 H S^-1 + 2 kT (sum_p R_p) S^-1 - 2 kT sum_p R_p Re(w_p G(w_p)).
    Returns (z, c_rho, c_edm, a_rho, b_edm, c_edm_shs): the shifts w_p, the
    library weights with sum_k Im(c_k G(z_k)) equal to the pole sums, and the
    coefficients of S^-1 in rho, of S^-1 in P^E and of S^-1 H S^-1 in P^E.
    """
    m2 = 2 * n_poles
    B = np.zeros((m2, m2))
    for m in range(1, m2):
        B[m - 1, m] = B[m, m - 1] = 1.0 / (2.0 * np.sqrt((2 * m - 1) * (2 * m + 1)))
    b, V = np.linalg.eigh(B)
    pos = b > 0
    bp, v1 = b[pos], V[0, pos]
    a = 1.0 / bp
    R = -(v1 ** 2) / (4.0 * bp ** 2)
    order = np.argsort(a)
    a, R = a[order], R[order]
    z = mu + 1j * kT * a
    c_rho = (-2.0 * kT * spin * R) * 1j
    c_edm = (-2.0 * kT * spin * R) * 1j * z
    return z, c_rho.astype(np.complex128), c_edm.astype(np.complex128), 0.5 * spin, 2.0 * kT * spin * R.sum(), \
        0.5 * spin


def random_columns(n: int, count: int, seed: int = 7) -> np.ndarray:
    """``count`` distinct orbital indices in [0, n), sorted."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(count, n), replace=False)).astype(np.int32)


def workload(name: str) -> dict:
    """Named workloads (system, shifts, weights, columns, tol, maxit, precision).

    chain800   : 200 sites x 4 orbitals, 64 shifts on [-12, 12] + 0.05i, all
                 800 columns, tol 1e-10, maxit 800, plain FP64.
    ppv1900    : 50-monomer PPV-like chain (N = 1900), 128 shifts on
                 [-15, 10] + 0.02i, all columns, mixed precision, tol 1e-6.
    bundle169  : 13 x 13 bundle of 50-monomer chains (N = 321,100), 64 shifts
                 on [-15, 10] + 0.02i, 4096 random columns, maxit 300.
    The PPV systems are numbered with align_blocks (every carbon on one whole
    4x4 block).
    """
    if name == "chain800":
        sys_ = chain_4orb(200, seed=0)
        z = shift_grid(-12.0, 12.0, 64, 0.05)
        cols = np.arange(sys_.n, dtype=np.int32)
        tol, maxit, prec = 1e-10, 800, "fp64"
    elif name == "ppv1900":
        sys_ = align_blocks(ppv_chain(50, seed=1))
        z = shift_grid(-15.0, 10.0, 128, 0.02)
        cols = np.arange(sys_.n, dtype=np.int32)
        # tol 1e-6 with a 1e-6 inner tolerance keeps every output within ~1e-7 of the
        # converged FP64 solution (relative to each output's largest magnitude)
        tol, maxit, prec = 1e-6, 16000, "mixed"
    elif name == "bundle169":
        sys_ = align_blocks(ppv_bundle(seed=3))
        z = shift_grid(-15.0, 10.0, 64, 0.02)
        cols = random_columns(sys_.n, 4096, seed=7)
        tol, maxit, prec = 1e-8, 300, "mixed"
    else:
        raise KeyError(name)
    w_rho, w_edm = fermi_weights(z)
    itol = 1e-6 if name == "ppv1900" else 0.0
    return dict(system=sys_, z=z, w_rho=w_rho, w_edm=w_edm, cols=cols, tol=tol, maxit=maxit, prec=prec, name=name,
                inner_tol=itol)
