"""Atomic forces from the solve's density and energy-density matrices
(gb_forces) against the oracle (oracle/forces.py): the same contraction on the
same packed inputs to rounding, and end to end (solve + forces) within the
FP64 and mixed bounds; the forces sum to zero."""
import numpy as np
import pytest

import oracle
from oracle import forces as oforces
from synth import fermi_weights, model_gradients, ppv_chain, shift_grid

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
gbg = pytest.importorskip("paper_1603_09616_gb300")


def atom_offsets(system):
    return np.concatenate([[0], np.cumsum(system.atom_norb)]).astype(np.int64)


@pytest.mark.parametrize("prec,tol,bound", [("fp64", 1e-12, 1e-10), ("mixed", 1e-9, 1e-6)])
def test_forces_match_oracle(prec, tol, bound):
    torch.cuda.set_device(0)
    system = ppv_chain(3, seed=4)  # N = 114, 42 atoms
    z = shift_grid(-12.0, 8.0, 64, 0.1)
    w_rho, w_edm = fermi_weights(z)
    cols = np.arange(system.n, dtype=np.int32)
    gh, gs = model_gradients(system)
    mat = gbg.Matrix(system)
    out = gbg.shifted_solve(mat, z, cols, tol=tol, maxit=20000, prec=prec, w_rho=w_rho, w_edm=w_edm)
    assert out["status"] == 0, out["message"]
    F = gbg.forces(mat, cols, out["rho"], out["edm"], gh, gs, atom_offsets(system)).cpu().numpy()
    rho, edm = out["rho"].cpu().numpy(), out["edm"].cpu().numpy()
    # the contraction alone: the oracle on the device's own rho / P^E
    F_same = oforces.forces(system, rho, edm, cols, gh, gs)
    scale = np.abs(F_same).max()
    assert np.abs(F - F_same).max() < 1e-12 * scale
    # end to end: the oracle's solve and forces
    ref = oracle.solve_outputs(system, z, cols, w_rho, w_edm)
    F_ref = oforces.forces(system, ref["rho"], ref["edm"], cols, gh, gs)
    assert np.abs(F - F_ref).max() < bound * np.abs(F_ref).max()
    assert np.abs(F.sum(axis=0)).max() < 1e-10 * scale * len(F)
    mat.close()


def test_forces_reject_partial_columns_and_bad_atoms():
    torch.cuda.set_device(0)
    system = ppv_chain(2, seed=1)
    z = shift_grid(-12.0, 8.0, 16, 0.1)
    w_rho, w_edm = fermi_weights(z)
    cols = np.arange(system.n, dtype=np.int32)
    gh, gs = model_gradients(system)
    mat = gbg.Matrix(system)
    out = gbg.shifted_solve(mat, z, cols, tol=1e-10, maxit=4000, prec="fp64", w_rho=w_rho, w_edm=w_edm)
    ao = atom_offsets(system)
    with pytest.raises(gbg.GBError, match="EINVAL"):
        gbg.forces(mat, cols[:-1], out["rho"], out["edm"], gh, gs, ao)
    bad = ao.copy()
    bad[-1] -= 1
    with pytest.raises(gbg.GBError, match="EINVAL"):
        gbg.forces(mat, cols, out["rho"], out["edm"], gh, gs, bad)
    mat.close()
