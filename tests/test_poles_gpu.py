"""Pole expansion of the Fermi function (a complex shift set): the library's
S^-1 terms (gb_add_sinv_terms) against the oracle's dense inverse, and the
full density / energy-density matrices from 40 poles against the
eigen-decomposition at finite temperature."""
import numpy as np
import pytest

from oracle import fermi as ofermi
from oracle import forces as oforces
from synth import pole_weights, ppv_chain

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
gbg = pytest.importorskip("paper_1603_09616_gb300")


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def test_sinv_terms_match_dense_inverse():
    torch.cuda.set_device(0)
    system = ppv_chain(3, seed=4)  # N = 114: not a multiple of 32 columns
    cols = np.arange(system.n, dtype=np.int32)
    mat = gbg.Matrix(system)
    si, shs = ofermi.sinv_terms(system, cols)
    f64 = dict(dtype=torch.float64, device="cuda")
    for a, b, c, want_rho, want_edm in ((1.0, 0.0, 0.0, si, 0 * si), (0.0, 2.0, 0.5, 0 * si, 2.0 * si + 0.5 * shs)):
        solved = dict(rho=torch.zeros(len(si), **f64), edm=torch.zeros(len(si), **f64),
                      q=torch.zeros(system.n, **f64), e_loc=torch.zeros(system.n, **f64))
        gbg.add_sinv_terms(mat, cols, solved, a, b, c)
        got_rho, got_edm = solved["rho"].cpu().numpy(), solved["edm"].cpu().numpy()
        if a:
            assert rel(got_rho, want_rho) < 1e-12
        else:
            assert np.abs(got_rho).max() == 0.0
        if b or c:
            assert rel(got_edm, want_edm) < 1e-12
        else:
            assert np.abs(got_edm).max() == 0.0
        # q and e_loc follow the completed rho
        q_ref = np.array([np.sum(got_rho[o0:o1] * system.s_val[system.row_ptr[j]:system.row_ptr[j + 1]])
                          for j, o0, o1 in zip(cols, np.r_[0, np.cumsum(np.diff(system.row_ptr))][:-1],
                                               np.cumsum(np.diff(system.row_ptr)))])
        assert np.abs(solved["q"].cpu().numpy() - q_ref).max() < 1e-12 * max(np.abs(q_ref).max(), 1.0)
    mat.close()


@pytest.mark.parametrize("prec,tol,bound", [("fp64", 1e-12, 1e-10), ("mixed", 1e-10, 1e-6)])
def test_pole_expansion_matches_eigen_decomposition(prec, tol, bound):
    torch.cuda.set_device(0)
    system = ppv_chain(3, seed=4)
    mu, kT = 0.2, 0.1
    cols = np.arange(system.n, dtype=np.int32)
    z, c, ce, a, b, cs = pole_weights(mu=mu, kT=kT, n_poles=40)
    mat = gbg.Matrix(system)
    out = gbg.shifted_solve(mat, z, cols, tol=tol, maxit=4000, prec=prec, w_rho=c, w_edm=ce)
    assert out["status"] == 0, out["message"]
    gbg.add_sinv_terms(mat, cols, out, a, b, cs)
    rho_e, edm_e = oforces.eigen_density(system, mu, kT)
    assert rel(out["rho"].cpu().numpy(), oforces.pack(system, rho_e, cols)) < bound
    assert rel(out["edm"].cpu().numpy(), oforces.pack(system, edm_e, cols)) < bound
    H, S = system.dense()
    assert abs(out["q"].sum().item() - np.trace(rho_e @ S)) < bound * system.n
    mat.close()
