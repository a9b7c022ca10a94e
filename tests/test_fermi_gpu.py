"""Chemical potential and Fermi-weighted density matrices from one solve
(gb_fermi_density) against the oracle's bisection on the same quadrature
(oracle/fermi.py), FP64 and mixed, and the exact electron count."""
import numpy as np
import pytest

from oracle import fermi as ofermi
from synth import chain_4orb, ppv_chain

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
gbg = pytest.importorskip("paper_1603_09616_gb300")


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.mark.parametrize("maker,prec,tol,bound", [(lambda: chain_4orb(6, seed=3), "fp64", 1e-12, 1e-10),
                                                  (lambda: ppv_chain(2, seed=5), "mixed", 1e-9, 1e-6)])
def test_fermi_level_and_density_match_oracle(maker, prec, tol, bound):
    # Every orbital solved once on a 160-point grid, filling 0.8 electrons per
    # orbital (inside a band, where dN/dmu is 10..25 per eV for these chains):
    # mu, rho, P^E, q and E must match the oracle's bisection on the same rule,
    # Tr[rho S] must be the electron count, and mu must sit within eta of the
    # sharp-level (eigenvalue) Fermi level of the same electron count.
    torch.cuda.set_device(0)
    system = maker()
    H, S = system.dense()
    import scipy.linalg as sla
    import scipy.optimize as so

    lam = sla.eigh(H, S, eigvals_only=True)
    eta, kT = 0.1, 0.1
    eps = np.linspace(lam.min() - 2.0, lam.max() + 2.0, 160)
    z = eps + 1j * eta
    cols = np.arange(system.n, dtype=np.int32)
    n_e = 0.8 * system.n
    mat = gbg.Matrix(system)
    solved = gbg.shifted_solve(mat, z, cols, tol=tol, maxit=20000, prec=prec, want_g=True)
    assert solved["status"] == 0, solved["message"]
    fd = gbg.fermi_density(mat, z, cols, solved, n_e, kT)
    ref = ofermi.fermi_outputs(system, z, n_e, kT)
    dos = ref["ldos"].sum(axis=1)
    assert abs(ofermi.electron_count(eps, dos, fd["mu"], kT) - n_e) < 10 * bound * n_e
    assert abs(fd["mu"] - ref["mu"]) < (1e-9 if prec == "fp64" else 1e-4), (fd["mu"], ref["mu"])
    for key in ("rho", "edm", "q", "e_loc"):
        assert rel(fd[key].cpu().numpy(), ref[key]) < bound, key
    assert abs(fd["q"].sum().item() - n_e) < 10 * bound * n_e
    mu_eig = so.brentq(lambda mu: np.sum(2.0 * ofermi.fermi((lam - mu) / kT)) - n_e, lam.min() - 5, lam.max() + 5)
    assert abs(fd["mu"] - mu_eig) < eta
    mat.close()


def test_fermi_rejects_partial_columns_and_uneven_grid():
    torch.cuda.set_device(0)
    system = chain_4orb(4, seed=1)
    mat = gbg.Matrix(system)
    z = np.linspace(-6, 6, 40) + 0.1j
    cols = np.arange(system.n, dtype=np.int32)
    solved = gbg.shifted_solve(mat, z, cols, tol=1e-10, maxit=5000, prec="fp64", want_g=True)
    with pytest.raises(gbg.GBError, match="EINVAL"):
        gbg.fermi_density(mat, z, cols[:-1], solved, 8.0, 0.1)
    zu = z.copy()
    zu[3] += 0.01
    with pytest.raises(gbg.GBError, match="EINVAL"):
        gbg.fermi_density(mat, zu, cols, solved, 8.0, 0.1)
    mat.close()


def test_fermi_density_tends_to_the_eigen_decomposition_limit():
    # Small eta on a fine grid (256 shifts, spacing 1.5 eta) over a compressed
    # spectrum (H scaled by 0.1, span 2.7 eV): the device's mu and rho approach
    # the sharp-level values mu_eig (sum_l 2 f((lambda_l - mu) / kT) = N_e) and
    # 2 sum_l f y_l y_l^T, and equal the oracle on the same rule to FP64 rounding.
    import dataclasses

    import scipy.linalg as sla

    torch.cuda.set_device(0)
    base = chain_4orb(4, seed=12)  # N = 16
    system = dataclasses.replace(base, h_val=base.h_val * 0.1)
    H, S = system.dense()
    lam, Y = sla.eigh(H, S)
    eta, kT = 0.01, 0.1
    z = np.linspace(lam.min() - 0.6, lam.max() + 0.6, 256) + 1j * eta
    n_e = float(system.n)
    lo, hi = lam.min() - 10, lam.max() + 10
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if 2 * ofermi.fermi((lam - mid) / kT).sum() < n_e:
            lo = mid
        else:
            hi = mid
    mu_eig = 0.5 * (lo + hi)
    cols = np.arange(system.n, dtype=np.int32)
    mat = gbg.Matrix(system)
    solved = gbg.shifted_solve(mat, z, cols, tol=1e-12, maxit=4000, prec="fp64", want_g=True)
    assert solved["status"] == 0, solved["message"]
    fd = gbg.fermi_density(mat, z, cols, solved, n_e, kT)
    ref = ofermi.fermi_outputs(system, z, n_e, kT)
    assert abs(fd["mu"] - ref["mu"]) < 1e-9
    assert rel(fd["rho"].cpu().numpy(), ref["rho"]) < 1e-10
    assert abs(fd["mu"] - mu_eig) < 5e-3, (fd["mu"], mu_eig)
    P = 2 * (Y * ofermi.fermi((lam - mu_eig) / kT)) @ Y.T
    rho = fd["rho"].cpu().numpy()
    off = fd["off"]
    err = max(np.abs(rho[off[c] : off[c + 1]] - P[system.row_cols(int(j)), j]).max() for c, j in enumerate(cols))
    assert err < 5e-2, err
    mat.close()
