"""Host-side checks of the C ABI library: it loads, exports every declared
entry point, and its CSR -> 4x4 block builder is exact (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1603_09616_gb300 as gbg
from synth import TBSystem, chain_4orb, ppv_bundle, ppv_chain

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names.update(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(gb_\w+)\s*\(", txt, flags=re.M))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = gbg.load()
    names = declared_entry_points()
    assert "gb_shifted_solve" in names and "gb_build_bsr" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(gbg.EXPORTED) <= set(names)
    assert lib.gb_abi_version() == 1


def dense_from_blocks(b, n):
    nb = b["nb"]
    H = np.zeros((4 * nb, 4 * nb))
    S = np.zeros((4 * nb, 4 * nb))
    for I in range(nb):
        for e in range(b["blk_ptr"][I], b["blk_ptr"][I + 1]):
            J = b["blk_col"][e]
            H[4 * I : 4 * I + 4, 4 * J : 4 * J + 4] = b["blk_h"][e]
            S[4 * I : 4 * I + 4, 4 * J : 4 * J + 4] = b["blk_s"][e]
    return H[:n, :n], S[:n, :n], H, S


@pytest.mark.parametrize("maker", [lambda: chain_4orb(20, seed=1), lambda: ppv_chain(3, seed=2)])
def test_bsr_round_trip_is_exact(maker):
    system = maker()
    b = gbg.bsr_to_host(system)
    H, S = system.dense()
    Hb, Sb, Hfull, Sfull = dense_from_blocks(b, system.n)
    assert np.array_equal(Hb, H) and np.array_equal(Sb, S)
    # padding rows/columns beyond n are zero
    assert not Hfull[system.n :].any() and not Sfull[:, system.n :].any()
    assert b["nb"] == (system.n + 3) // 4
    # block columns sorted and unique in each block row
    for I in range(b["nb"]):
        cols = b["blk_col"][b["blk_ptr"][I] : b["blk_ptr"][I + 1]]
        assert np.all(np.diff(cols) > 0)


def test_chain800_block_count():
    b = gbg.bsr_to_host(chain_4orb(200, seed=0))
    assert b["nb"] == 200 and b["nnzb"] == 1388


def _mutated(system, **kw):
    s = TBSystem(system.n, system.row_ptr.copy(), system.col_idx.copy(), system.h_val.copy(),
                 system.s_val.copy(), system.orb_atom)
    for k, v in kw.items():
        setattr(s, k, v)
    return s


def test_builder_rejects_bad_input():
    base = chain_4orb(4, seed=3)
    with pytest.raises(gbg.GBError, match="EINVAL"):
        h = base.h_val.copy()
        h[1] += 1.0  # breaks symmetry
        gbg.bsr_to_host(_mutated(base, h_val=h))
    with pytest.raises(gbg.GBError, match="EINVAL"):
        c = base.col_idx.copy()
        c[0], c[1] = c[1], c[0]  # unsorted row
        gbg.bsr_to_host(_mutated(base, col_idx=c))
    with pytest.raises(gbg.GBError, match="EINVAL"):
        c = base.col_idx.copy()
        c[3] = base.n + 5
        gbg.bsr_to_host(_mutated(base, col_idx=c))
    with pytest.raises(gbg.GBError, match="EINVAL"):
        h = base.h_val.copy()
        h[0] = np.nan
        gbg.bsr_to_host(_mutated(base, h_val=h))
    with pytest.raises(gbg.GBError, match="ENOTSPD"):
        s = base.s_val.copy()
        s[0] = -1.0  # a diagonal block that is not positive definite
        gbg.bsr_to_host(_mutated(base, s_val=s))


def test_builder_rejects_missing_diagonal():
    rp = np.array([0, 1, 2], np.int64)
    ci = np.array([1, 0], np.int32)
    v = np.array([1.0, 1.0])
    with pytest.raises(gbg.GBError, match="diagonal"):
        gbg.bsr_to_host(TBSystem(2, rp, ci, v, v, np.array([0, 1], np.int32)))


def test_gpu_entry_points_fail_loudly_without_a_device():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    with pytest.raises(RuntimeError, match="no CUDA device"):
        gbg.Matrix(chain_4orb(4, seed=0))


@pytest.mark.parametrize("maker", [lambda: chain_4orb(9, seed=1), lambda: ppv_chain(3, seed=4)])
def test_band_cholesky_factor_reproduces_s(maker):
    # the factor the flags-bit-3 inner solve uses: L L^T = S on the padded size
    # (identity past n), band layout by columns (up) and rows (row) consistent
    system = maker()
    f = gbg.band_cholesky_to_host(system)
    _, S = system.dense()
    n = system.n
    n4 = 4 * ((n + 3) // 4)
    rows, cols = np.nonzero(np.tril(S))
    assert f["bw"] == int((rows - cols).max())
    bw = f["bw"]
    L = np.zeros((n4, n4))
    for i in range(n4):
        L[i, i] = 1.0 / float(f["invd"][i])
        for t in range(bw):
            if i - 1 - t >= 0:
                L[i, i - 1 - t] = f["row"][i, t]
    for i in range(n4):
        for t in range(bw):
            if i + 1 + t < n4:
                assert f["up"][i, t] == np.float32(L[i + 1 + t, i])
    assert not f["up"][:, bw:].any() and not f["row"][:, bw:].any()
    Sp = np.eye(n4)
    Sp[:n, :n] = S
    assert np.abs(L @ L.T - Sp).max() < 1e-5 * np.abs(Sp).max()
    # solving with the FP32 factor is accurate to FP32 (the level's accuracy)
    r = np.random.default_rng(0).standard_normal(n4)
    x = np.linalg.solve(L.T, np.linalg.solve(L, r))
    ref = np.linalg.solve(Sp, r)
    assert np.abs(x - ref).max() < 1e-5 * np.abs(ref).max()


def test_band_cholesky_reports_wide_band_unavailable():
    bundle = ppv_bundle(n_side=2, n_mono=2, seed=1)
    _, S = bundle.dense()
    rows, cols = np.nonzero(np.tril(S))
    assert (rows - cols).max() > 63
    f = gbg.band_cholesky_to_host(bundle)
    assert f["bw"] == 0
    assert not f["up"].any() and not f["row"].any() and not f["invd"].any()
