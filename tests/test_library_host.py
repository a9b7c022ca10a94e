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
    assert lib.gb_abi_version() == 2


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


def block_solve_host(f, rhs):
    """Applies the factor the exact inner solve uses, in the order the kernel
    does: t_i = Dinv_i r_i, y_i = t_i - E_i y_{i-1}; u_i = DinvT_i y_i,
    x_i = u_i - F_i x_{i+1} (64-row blocks, k-major storage)."""
    nblk = f["nblk"]
    n64 = 64 * nblk
    r = np.zeros((n64,) + rhs.shape[1:])
    r[: rhs.shape[0]] = rhs
    blk = lambda v, i: v[64 * i : 64 * i + 64]
    # entry (r, k) of a block at [k, r]: the block's matrix is the transpose
    y = np.zeros_like(r)
    for i in range(nblk):
        t = f["dinv"][i].T @ blk(r, i)
        if i > 0:
            t = t - f["e"][i].T @ blk(y, i - 1)
        y[64 * i : 64 * i + 64] = t
    x = np.zeros_like(r)
    for i in reversed(range(nblk)):
        u = f["dinvt"][i].T @ blk(y, i)
        if i + 1 < nblk:
            u = u - f["f"][i].T @ blk(x, i + 1)
        x[64 * i : 64 * i + 64] = u
    return x[: rhs.shape[0]]


@pytest.mark.parametrize("maker", [lambda: chain_4orb(9, seed=1), lambda: ppv_chain(3, seed=4),
                                   lambda: ppv_chain(7, seed=2), lambda: chain_4orb(41, seed=3)])
def test_block_factor_solves_s_exactly(maker):
    # The exact inner solve's factor: the block recurrences reproduce S^-1 r to
    # FP64 rounding on the padded size (identity past n), the half-bandwidth
    # is S's, the factor blocks have the triangular / band structure the
    # kernel's loops rely on, and several 64-row blocks (ragged last block) occur.
    system = maker()
    f = gbg.block_factor_to_host(system)
    _, S = system.dense()
    n = system.n
    n4 = 4 * ((n + 3) // 4)
    rows, cols = np.nonzero(np.tril(S))
    bw = int((rows - cols).max())
    assert f["bw"] == bw and f["nblk"] == (n4 + 63) // 64
    Sp = np.eye(n4)
    Sp[:n, :n] = S
    rhs = np.random.default_rng(0).standard_normal((n4, 3))
    x = block_solve_host(f, rhs)
    ref = np.linalg.solve(Sp, rhs)
    assert np.abs(x - ref).max() < 1e-13 * np.abs(ref).max()
    for i in range(f["nblk"]):
        dinv = f["dinv"][i].T  # entry (r, k)
        assert not np.triu(dinv, 1).any()  # lower triangular
        assert np.array_equal(f["dinvt"][i], dinv)  # DinvT stored k-major is Dinv row-major
        assert not f["e"][i][: 64 - bw].any()  # E only in the last bw columns (k >= 64 - bw)
        assert not f["f"][i][bw:].any()  # F only in the first bw columns (k < bw)
    assert not f["e"][0].any() and not f["f"][-1].any()


def test_block_factor_reports_wide_band_unavailable():
    bundle = ppv_bundle(n_side=2, n_mono=2, seed=1)
    _, S = bundle.dense()
    rows, cols = np.nonzero(np.tril(S))
    assert (rows - cols).max() > 63
    f = gbg.block_factor_to_host(bundle)
    assert f["bw"] == 0 and f["nblk"] == 0
