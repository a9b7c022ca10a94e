"""Input generators: determinism, symmetry, SPD overlap, sizes of the workloads."""
import numpy as np

from synth import chain_4orb, fermi_weights, ppv_chain, random_columns, shift_grid, uneven_chains


def test_chain800_sizes_and_determinism():
    a = chain_4orb(200, seed=0)
    b = chain_4orb(200, seed=0)
    assert a.n == 800
    # 200 sites, site blocks |i-j| <= 3: 200*7 - 12 = 1388 blocks of 4x4
    assert a.nnz == 1388 * 16
    for f in ("row_ptr", "col_idx", "h_val", "s_val"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    c = chain_4orb(200, seed=1)
    assert not np.array_equal(a.h_val, c.h_val)


def test_symmetric_pattern_and_spd_overlap():
    for sysm in (chain_4orb(40, seed=2), ppv_chain(6, seed=3)):
        H, S = sysm.dense()
        assert np.array_equal(H, H.T)
        assert np.array_equal(S, S.T)
        assert np.linalg.eigvalsh(S).min() > 0.5
        # pattern sorted, diagonal present in every row
        for i in range(sysm.n):
            cols = sysm.row_cols(i)
            assert np.all(np.diff(cols) > 0)
            assert i in cols
        # Gershgorin: S strictly diagonally dominant
        off = np.abs(S).sum(1) - np.abs(np.diag(S))
        assert np.all(np.diag(S) > off)


def test_ppv_composition():
    p = ppv_chain(50, seed=1)
    assert p.n == 50 * 38  # 8 C x 4 orbitals + 6 H x 1 orbital per monomer
    assert np.bincount(p.orb_atom).max() == 4
    p2 = ppv_chain(2, seed=1)
    assert p2.n == 76


def test_grids_and_weights():
    z = shift_grid(-12, 12, 64, 0.05)
    assert z.shape == (64,) and np.allclose(z.imag, 0.05)
    assert np.isclose(z.real[0], -12) and np.isclose(z.real[-1], 12)
    w_rho, w_edm = fermi_weights(z, mu=0.0, kT=0.1)
    assert np.all(w_rho.real <= 0) and np.allclose(w_edm, z.real * w_rho)
    cols = random_columns(1000, 64, seed=1)
    assert len(np.unique(cols)) == 64 and cols.max() < 1000


def test_uneven_chain_ranges():
    chains = uneven_chains(12, seed=2)
    for sysm, k in chains:
        assert 2 * 38 <= sysm.n <= 50 * 38
        assert 32 <= k <= 256


def test_uneven_batch_is_deterministic():
    # the GPU correction tests address chains of this batch by index
    from synth import uneven_batch

    systems, problems = uneven_batch(eta=0.02)
    assert len(systems) == 512
    assert (systems[331].n, len(problems[331]["z"])) == (228, 115)
    assert (systems[69].n, len(problems[69]["z"])) == (570, 183)
    for s, p in zip(systems[:20], problems[:20]):
        assert 76 <= s.n <= 1900 and 32 <= len(p["z"]) <= 256
        assert p["cols"][0] == 0 and len(set(p["cols"].tolist())) == 2
        assert np.allclose(p["z"].imag, 0.02)
    again, _ = uneven_batch(eta=0.02)
    assert np.array_equal(again[331].h_val, systems[331].h_val)


def test_align_blocks_is_a_permutation_that_aligns_every_carbon():
    from synth import align_blocks

    p = ppv_chain(7, seed=3)
    a = align_blocks(p)
    perm = a.meta["orbital_perm"]
    assert np.array_equal(np.sort(perm), np.arange(p.n))
    H, S = p.dense()
    H2, S2 = a.dense()
    assert np.array_equal(H[np.ix_(perm, perm)], H2)
    assert np.array_equal(S[np.ix_(perm, perm)], S2)
    # every 4-orbital atom occupies one whole aligned block
    starts = np.concatenate([[0], np.cumsum(a.atom_norb)[:-1]])
    assert np.all(starts[a.atom_norb == 4] % 4 == 0)
    assert np.array_equal(np.bincount(a.orb_atom), a.atom_norb)
    # the band of S stays within the 63 of the block factor
    Sc = a.s_csr().tocoo()
    assert np.abs(Sc.row - Sc.col).max() <= 63
