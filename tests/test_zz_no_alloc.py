"""gb_shifted_solve_static: the solve for callers that may not allocate.

Some callers cannot allocate device memory while they run (their GPU memory
belongs to another runtime's pool, or cudaMalloc's implicit synchronisation is
not allowed in their loop).  For them the library offers an entry point whose
scratch is a fixed array inside the library.  This test calls it through the C
ABI twice in a row (the second call finds the first call's leftovers in the
shared scratch) and compares every output with the allocating entry point
gb_shifted_solve, within the FP64 tolerance of the other parity tests.  It
lives in a file collected last so that a failing run has already run every
other test.
"""
import numpy as np
import pytest

from synth import fermi_weights, ppv_chain, shift_grid, workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
gbg = pytest.importorskip("paper_1603_09616_gb300")

FP64_BOUND = 1e-10


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_static_entry_point_matches_allocating_one():
    torch.cuda.set_device(0)
    system = ppv_chain(3, seed=8)  # N = 114
    z = shift_grid(-10, 6, 24, 0.05)
    w_rho, w_edm = fermi_weights(z)
    cols = np.arange(0, system.n, 6, dtype=np.int32)
    mat = gbg.Matrix(system)
    kw = dict(tol=1e-12, maxit=3000, prec="fp64", w_rho=w_rho, w_edm=w_edm, want_g=True)
    ref = gbg.shifted_solve(mat, z, cols, **kw)
    assert ref["status"] == 0, ref["message"]
    for call in range(2):
        out = gbg.shifted_solve_static(mat, z, cols, **kw)
        torch.cuda.synchronize()
        assert out["status"] == 0, (call, out["message"])
        for key in ("g_proj", "ldos", "rho", "edm", "q", "e_loc", "resid"):
            assert rel(out[key].cpu().numpy(), ref[key].cpu().numpy()) <= FP64_BOUND, (call, key)
        assert np.array_equal(out["iters"].cpu().numpy(), ref["iters"].cpu().numpy())
        assert np.array_equal(out["converged"].cpu().numpy(), ref["converged"].cpu().numpy())
    mat.close()


def test_static_entry_point_rejects_oversized_problems():
    torch.cuda.set_device(0)
    lib = gbg.load()
    limit = lib.gb_static_scratch_bytes()
    assert limit == 32 << 20
    wl = workload("ppv1900")
    mat = gbg.Matrix(wl["system"])
    out = gbg.shifted_solve_static(mat, wl["z"], wl["cols"], tol=wl["tol"], maxit=wl["maxit"], prec="mixed",
                                   w_rho=wl["w_rho"], w_edm=wl["w_edm"])
    assert out["status"] == gbg._binding.GB_ENOMEM
    assert "static scratch" in out["message"]
    mat.close()
