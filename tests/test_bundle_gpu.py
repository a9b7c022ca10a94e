"""Condensed-bundle scale: 13 x 13 PPV-like chains x 50 monomers (N = 321,100).

* SpMM at full size, element by element, against SciPy's CSR product.
* Shifted solves on a smaller bundle from the same generator (4 x 4 chains x
  6 monomers, N = 3,648) against the dense-LU oracle.
* At full size, a property that holds for any size: G is complex symmetric, so
  for sampled columns i, j solved independently with i in R_j and j in R_i,
  the projected outputs must agree: G_ij(z) = G_ji(z).
"""
import numpy as np
import pytest

import oracle
from synth import fermi_weights, ppv_bundle, random_columns, shift_grid

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
gbg = pytest.importorskip("paper_1603_09616_gb300")


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.fixture(scope="module")
def bundle():
    torch.cuda.set_device(0)
    system = ppv_bundle(seed=3)
    mat = gbg.Matrix(system)
    yield system, mat
    mat.close()


def test_bundle_spmm_full_size(bundle):
    system, mat = bundle
    rng = np.random.default_rng(1)
    w = 8
    x = rng.standard_normal((system.n, w)) + 1j * rng.standard_normal((system.n, w))
    xt = torch.from_numpy(x).cuda()
    for which, A in ((0, system.h_csr()), (1, system.s_csr())):
        ref = A @ x
        y = mat.spmm(which, xt, prec="fp64").cpu().numpy()
        assert rel(y, ref) < 1e-13
        y32 = mat.spmm(which, xt, prec="fp32").cpu().numpy()
        assert rel(y32, ref) < 5e-6
    # narrow FP32 panels take the block-row-per-warp kernel
    for w in (1, 2, 4):
        x = rng.standard_normal((system.n, w)) + 1j * rng.standard_normal((system.n, w))
        y32 = mat.spmm(0, torch.from_numpy(x).cuda(), prec="fp32").cpu().numpy()
        assert rel(y32, system.h_csr() @ x) < 5e-6, w


def test_small_bundle_solves_match_oracle():
    torch.cuda.set_device(0)
    system = ppv_bundle(n_side=4, n_mono=6, seed=5)
    z = shift_grid(-8.0, 4.0, 16, 0.3)
    w_rho, w_edm = fermi_weights(z)
    cols = random_columns(system.n, 24, seed=2)
    mat = gbg.Matrix(system)
    ref = oracle.solve_outputs(system, z, cols, w_rho, w_edm)
    for prec, bound in (("fp64", 1e-10), ("mixed", 1e-6)):
        out = gbg.shifted_solve(mat, z, cols, tol=1e-12 if prec == "fp64" else 1e-10, maxit=6000, prec=prec,
                                w_rho=w_rho, w_edm=w_edm, want_g=True)
        assert out["status"] == 0, (prec, out["message"])
        assert rel(out["g_proj"].cpu().numpy(), ref["g_proj"]) < bound, prec
        for key in ("ldos", "rho", "edm", "q", "e_loc"):
            assert rel(out[key].cpu().numpy(), ref[key]) < bound, (prec, key)
    mat.close()


def test_bundle_full_size_complex_symmetry(bundle):
    system, mat = bundle
    z = shift_grid(-6.0, 3.0, 4, 1.0)
    # sampled columns with many pattern neighbours among themselves: a few
    # seeds plus every fourth orbital of their pattern rows
    seeds = random_columns(system.n, 2, seed=9)  # 69 columns, 1,164 symmetric pairs
    cols = np.unique(np.concatenate([system.row_cols(int(j))[::4] for j in seeds]).astype(np.int32))
    out = gbg.shifted_solve(mat, z, cols, tol=1e-8, maxit=2000, prec="mixed", want_g=True)
    assert out["status"] == 0, out["message"]
    g = out["g_proj"].cpu().numpy()
    off = out["off"]
    pos = {int(j): c for c, j in enumerate(cols)}
    checked, worst, scale = 0, 0.0, np.abs(g).max()
    for c, j in enumerate(cols):
        rows = system.row_cols(int(j))
        for t, i in enumerate(rows):
            ci = pos.get(int(i))
            if ci is None or i == j:
                continue
            rows_i = system.row_cols(int(i))
            s = np.searchsorted(rows_i, j)
            gij = g[:, off[c] + t]
            gji = g[:, off[ci] + s]
            worst = max(worst, np.abs(gij - gji).max())
            checked += 1
    assert checked > 40
    assert worst < 1e-6 * scale, (worst, scale, checked)
