"""Batched uneven systems in one persistent launch (gb_shifted_solve_batched).

Independent PPV-like chains of different length, each with its own shift
count and all of its unit right-hand sides, solved together; every system is
checked against the dense-LU oracle and against a single-system solve with
the same panel width (the per-panel arithmetic is identical, so the results
must agree to rounding).  The panel autotuner must return one of its
candidates.
"""
import numpy as np
import pytest

import oracle
from synth import fermi_weights, ppv_chain, shift_grid, uneven_batch

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
gbg = pytest.importorskip("paper_1603_09616_gb300")


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def make_batch(seed=4, n=6):
    rng = np.random.default_rng(seed)
    systems, problems = [], []
    for i in range(n):
        sysm = ppv_chain(int(rng.integers(2, 6)), seed=int(rng.integers(1, 10**6)))
        K = int(rng.integers(16, 49))
        z = shift_grid(-10.0, 6.0, K, 0.05)
        w_rho, w_edm = fermi_weights(z)
        systems.append(sysm)
        problems.append(dict(z=z, cols=np.arange(sysm.n, dtype=np.int32), w_rho=w_rho, w_edm=w_edm))
    return systems, problems


# FP64 with the exact factor inner solve reaches tol 1e-11 on every chain (a
# few pairs stall between 1e-12 and 1e-11, FP64 COCG's attainable accuracy at
# eta 0.05), and the outputs then meet the FP64 bound 1e-10
@pytest.mark.parametrize("prec,tol,bound", [("fp64", 1e-11, 1e-10), ("mixed", 1e-9, 1e-6)])
def test_batched_matches_oracle_and_single_solves(prec, tol, bound):
    torch.cuda.set_device(0)
    systems, problems = make_batch()
    for pr in problems:
        pr.update(tol=tol, maxit=8000)
    mats = [gbg.Matrix(s) for s in systems]
    res, info = gbg.shifted_solve_batched(mats, problems, prec=prec, panel=8, want_g=True)
    assert info["status"] == 0, info["message"]
    for s, (mat, sysm, pr, out) in enumerate(zip(mats, systems, problems, res)):
        ref = oracle.solve_outputs(sysm, pr["z"], pr["cols"], pr["w_rho"], pr["w_edm"])
        assert rel(out["g_proj"].cpu().numpy(), ref["g_proj"]) < bound, s
        for key in ("ldos", "rho", "edm", "q", "e_loc"):
            assert rel(out[key].cpu().numpy(), ref[key]) < bound, (s, key)
        single = gbg.shifted_solve(mat, pr["z"], pr["cols"], tol=tol, maxit=8000, prec=prec, w_rho=pr["w_rho"],
                                   w_edm=pr["w_edm"], panel=8)
        for key in ("ldos", "rho", "q", "resid"):
            assert rel(out[key].cpu().numpy(), single[key].cpu().numpy()) == 0.0, (s, key)
        assert np.array_equal(out["iters"].cpu().numpy(), single["iters"].cpu().numpy())
    for m in mats:
        m.close()


def test_batched_autotuner_picks_a_candidate():
    torch.cuda.set_device(0)
    systems, problems = make_batch(seed=9, n=5)
    for pr in problems:
        pr.update(tol=1e-8, maxit=4000)
    mats = [gbg.Matrix(s) for s in systems]
    res, info = gbg.shifted_solve_batched(mats, problems, prec="mixed", tune_probe_maxit=40)
    assert info["tuned_panel"] in (8, 16, 32)
    assert info["status"] == 0, info["message"]
    assert all(t > 0 for t in info["tune_times_ms"])
    for out in res:
        assert out["converged"].cpu().numpy().all()
    for m in mats:
        m.close()


def test_batched_512_uneven_chains_sampled_columns():
    # The uneven-chain configuration at full structure: 512 chains of 76..1900
    # orbitals with 32..256 shifts each (eta 0.05, tol 1e-6, mixed), two unit
    # right-hand sides per chain, in one persistent launch.  Every pair must
    # converge; the four chains cheapest for the dense oracle and the cheapest
    # one with N >= 1500 are checked against it element by element.
    # (At eta 0.02 a few chains have a shift near the gap where shifted COCG
    # stagnates above tol; that case has no retry yet.)
    torch.cuda.set_device(0)
    systems, problems = uneven_batch(eta=0.05)
    assert len(systems) == 512
    mats = [gbg.Matrix(s) for s in systems]
    res, info = gbg.shifted_solve_batched(mats, problems, prec="mixed", panel=2)
    assert info["status"] == 0, info["message"]
    for out in res:
        assert out["converged"].cpu().numpy().all()
    cost = np.array([s.n**3 * len(p["z"]) for s, p in zip(systems, problems)], dtype=np.float64)
    order = np.argsort(cost, kind="stable")
    pick = list(order[:4]) + [i for i in order if systems[i].n >= 1500][:1]
    assert systems[pick[-1]].n >= 1500
    for i in pick:
        pr = problems[i]
        ref = oracle.solve_outputs(systems[i], pr["z"], pr["cols"], pr["w_rho"], pr["w_edm"])
        for key in ("ldos", "rho", "edm", "q", "e_loc"):
            assert rel(res[i][key].cpu().numpy(), ref[key]) < 1e-6, (int(i), key)
    for m in mats:
        m.close()


def test_batched_correction_solve():
    # Two chains of the uneven batch at eta 0.02 whose mixed solve with the
    # iterative (Chebyshev, flags bit 4) inner solve stagnates on one column
    # each (331: N = 228, 115 shifts; 69: N = 570, 183 shifts), in one launch;
    # the per-system correction must bring every pair to tol.
    torch.cuda.set_device(0)
    systems, problems = uneven_batch(eta=0.02)
    pick = [331, 69]
    systems = [systems[i] for i in pick]
    problems = [problems[i] for i in pick]
    mats = [gbg.Matrix(s) for s in systems]
    res, info = gbg.shifted_solve_batched(mats, problems, prec="mixed", panel=2, flags=16)
    assert info["status"] == gbg._binding.GB_ENOCONV
    res, info = gbg.shifted_solve_batched(mats, problems, prec="mixed", panel=2, correct=True, flags=16)
    assert info["status"] == 0, info["message"]
    assert info["corrected"] >= 2
    for sysm, pr, out in zip(systems, problems, res):
        assert out["converged"].cpu().numpy().all()
        ref = oracle.solve_outputs(sysm, pr["z"], pr["cols"], pr["w_rho"], pr["w_edm"])
        for key in ("ldos", "rho", "edm", "q", "e_loc"):
            assert rel(out[key].cpu().numpy(), ref[key]) < 1e-6, key
    for m in mats:
        m.close()


def test_batched_512_uneven_chains_eta002_with_correction():
    # The uneven-chain batch at eta 0.02 (the damping of the 1900-orbital
    # workload): one mixed launch, then the FP64 correction of every column
    # that missed tol (exact factor inner solve, switched seed).  Every pair of
    # all 512 chains must then meet tol, chain 344 (the near-gap case of the
    # iterative inner solve) included, and five chains match the oracle.
    torch.cuda.set_device(0)
    systems, problems = uneven_batch(eta=0.02)
    mats = [gbg.Matrix(s) for s in systems]
    res, info = gbg.shifted_solve_batched(mats, problems, prec="mixed", panel=2, correct=True)
    assert info["status"] == 0, info["message"]
    for out in res:
        assert out["converged"].cpu().numpy().all()
        assert (out["resid"].cpu().numpy() <= 1e-6).all()
    cost = np.array([s.n**3 * len(p["z"]) for s, p in zip(systems, problems)], dtype=np.float64)
    order = np.argsort(cost, kind="stable")
    pick = list(order[:3]) + [i for i in order if systems[i].n >= 1500][:1] + [344]
    for i in pick:
        pr = problems[i]
        ref = oracle.solve_outputs(systems[i], pr["z"], pr["cols"], pr["w_rho"], pr["w_edm"])
        for key in ("ldos", "rho", "edm", "q", "e_loc"):
            assert rel(res[i][key].cpu().numpy(), ref[key]) < 1e-6, (int(i), key)
    for m in mats:
        m.close()
