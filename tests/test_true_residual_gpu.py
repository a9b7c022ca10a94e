"""FP64 true-residual check of the shifted solve (gb_true_residual).

The recurrence reports the recursive estimate ||rt_n|| / |pi^k_n| of
||e_j - (z_k S - H) x^k||; the check forms x^k on every row from the kept
history and evaluates the residual from H and S in FP64.
  * With an exact inner solve (the FP64 factor solve) the two agree to
    rounding at any iteration count: stopped early, far from convergence,
    they match pair by pair.
  * With H p as an unrefined FP32 product (flags bit 5) the estimate drifts
    below the true residual: columns meet tol by the estimate while the true
    residual misses it.  The check reports the failing pairs from the true
    residual (written into resid), marks their columns unconverged in the
    outputs, and the FP64 correction solve then brings every pair to tol and
    the outputs to the oracle.
"""
import numpy as np
import pytest

import oracle
from synth import chain_4orb, fermi_weights, ppv_chain, shift_grid

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
gbg = pytest.importorskip("paper_1603_09616_gb300")


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.mark.parametrize("maker,panel", [(lambda: ppv_chain(3, seed=7), 4), (lambda: chain_4orb(20, seed=2), 0)])
def test_true_residual_equals_estimate_with_exact_inner_solve(maker, panel):
    torch.cuda.set_device(0)
    system = maker()
    z = shift_grid(-8, 6, 24, 0.05)
    w_rho, w_edm = fermi_weights(z)
    cols = np.arange(0, system.n, 9, dtype=np.int32)
    mat = gbg.Matrix(system)
    out = gbg.shifted_solve(mat, z, cols, tol=1e-14, maxit=25, prec="fp64", w_rho=w_rho, w_edm=w_edm,
                            panel=panel, verify=True, raise_on=())
    assert out["status"] == gbg._binding.GB_ENOCONV  # stopped early on purpose
    est = out["resid"].cpu().numpy()
    true = out["resid_true"].cpu().numpy()
    assert true.shape == est.shape
    assert (est > 1e-6).any()  # far from convergence
    assert np.abs(true - est).max() <= 1e-9 * est.max() + 1e-13
    mat.close()


def test_true_residual_check_drives_the_correction():
    # Mixed path with H p as an unrefined FP32 product (flags bit 5): the
    # recursive estimate reaches tol 1e-8 while true residuals stay above 1e-6.
    # The FP64 check writes the true residual into resid, marks exactly the
    # columns that miss tol by it, and the FP64 correction then brings every
    # pair to tol and the outputs to the oracle.
    torch.cuda.set_device(0)
    system = ppv_chain(3, seed=8)
    z = shift_grid(-10, 6, 32, 0.05)
    w_rho, w_edm = fermi_weights(z)
    cols = np.arange(0, system.n, 13, dtype=np.int32)
    mat = gbg.Matrix(system)
    kw = dict(tol=1e-8, maxit=3000, prec="mixed", w_rho=w_rho, w_edm=w_edm, panel=4, flags=32)
    # without the check the solve reports success: every pair meets tol by its estimate
    plain = gbg.shifted_solve(mat, z, cols, raise_on=(), **kw)
    assert plain["status"] == 0, plain["message"]
    assert (plain["resid"].cpu().numpy() <= 1e-8).all()
    checked = gbg.shifted_solve(mat, z, cols, raise_on=(), verify=True, **kw)
    est = checked["resid"].cpu().numpy()
    true = checked["resid_true"].cpu().numpy()
    assert checked["status"] == gbg._binding.GB_ENOCONV
    assert true.max() > 1e-6
    failing = (true > 1e-8).any(axis=0)
    assert checked["flagged"] == int(failing.sum()) >= 1
    assert np.array_equal(failing, (est > 1e-8).any(axis=0))
    fixed = gbg.shifted_solve(mat, z, cols, raise_on=(), verify=True, correct=True, **kw)
    assert fixed["status"] == 0, fixed["message"]
    assert fixed["corrected"] == checked["flagged"]
    assert fixed["converged"].cpu().numpy().all()
    assert (fixed["resid"].cpu().numpy() <= 1e-8).all()
    ref = oracle.solve_outputs(system, z, cols, w_rho, w_edm)
    for key in ("ldos", "rho", "edm", "q", "e_loc"):
        assert rel(fixed[key].cpu().numpy(), ref[key]) < 1e-6, key
    mat.close()


def test_stalled_columns_stop_early_and_the_correction_fixes_them():
    # Chain 331 of the uneven batch at eta 0.02 (N = 228, 115 shifts): its
    # second column stalls above tol 1e-6 in the mixed path (near-gap shifts)
    # and runs to maxit 16000; with flags bit 6 it stops once no open shift has
    # halved its best residual for 3000 iterations (col_status 4 | 32).  The
    # column that converges is untouched (same iterations, same outputs), and
    # the correction then brings the stopped column to tol and to the oracle.
    from synth import uneven_batch

    torch.cuda.set_device(0)
    systems, problems = uneven_batch(eta=0.02)
    system, pr = systems[331], problems[331]
    mat = gbg.Matrix(system)
    maxit = pr["maxit"]
    kw = dict(tol=pr["tol"], maxit=maxit, prec="mixed", w_rho=pr["w_rho"], w_edm=pr["w_edm"], panel=2, raise_on=())
    full = gbg.shifted_solve(mat, pr["z"], pr["cols"], **kw)
    early = gbg.shifted_solve(mat, pr["z"], pr["cols"], flags=gbg._binding.FLAG_STALL, **kw)
    st = early["col_status"].cpu().numpy()
    its_e = early["iters"].cpu().numpy()
    its_f = full["iters"].cpu().numpy()
    stalled = (st & 32) != 0
    assert stalled.any() and not stalled.all()
    assert np.all(st[stalled] & 4)
    assert np.all(its_e[stalled] < maxit)
    assert np.all(its_f[stalled] == maxit)  # running on did not reach tol either
    ok = ~stalled
    assert np.array_equal(its_e[ok], its_f[ok])
    q_e, q_f = early["q"].cpu().numpy(), full["q"].cpu().numpy()
    assert np.array_equal(q_e[ok], q_f[ok])
    fixed = gbg.shifted_solve(mat, pr["z"], pr["cols"], correct=True, **kw)
    assert fixed["status"] == 0, fixed["message"]
    assert fixed["converged"].cpu().numpy().all()
    ref = oracle.solve_outputs(system, pr["z"], pr["cols"], pr["w_rho"], pr["w_edm"])
    for key in ("ldos", "rho", "edm", "q", "e_loc"):
        assert rel(fixed[key].cpu().numpy(), ref[key]) < 1e-6, key
    mat.close()
