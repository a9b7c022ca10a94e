"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances: plain FP64 path <= 1e-10 (the bound for the FP64 solver)
relative to the largest reference magnitude of each output array; the
reduced-precision path <= 1e-6.
"""
import numpy as np
import pytest

import oracle
from synth import chain_4orb, fermi_weights, ppv_chain, shift_grid, uneven_batch

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
gbg = pytest.importorskip("paper_1603_09616_gb300")


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def to_np(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def dev():
    torch.cuda.set_device(0)
    return torch.device("cuda", 0)


# ------------------------------------------------------------------ SpMM
@pytest.mark.parametrize("system_fn", [lambda: chain_4orb(37, seed=2), lambda: ppv_chain(5, seed=4)])
@pytest.mark.parametrize("w", [1, 2, 3, 4, 8, 16, 32, 64])
def test_spmm_fp64_and_fp32(dev, system_fn, w):
    system = system_fn()
    mat = gbg.Matrix(system)
    H, S = system.dense()
    rng = np.random.default_rng(w)
    x = rng.standard_normal((system.n, w)) + 1j * rng.standard_normal((system.n, w))
    xt = torch.from_numpy(x).to(dev)
    for which, A in ((0, H), (1, S)):
        y = to_np(mat.spmm(which, xt, prec="fp64"))
        assert rel(y, A @ x) < 1e-14
        y32 = to_np(mat.spmm(which, xt, prec="fp32"))
        assert rel(y32, A @ x) < 2e-6
    mat.close()


@pytest.mark.parametrize("w", [1, 2, 4, 8, 16])
def test_spmm_fp32_unaligned_x_matches_aligned(dev, w):
    # x starting 8 bytes past a 16-byte boundary cannot take the float4-gather
    # kernels of the FP32 panels; both kernels must give the product
    # (n % 4 == 0 here, so x is read in place, not through a padded copy)
    system = chain_4orb(37, seed=2)
    assert system.n % 4 == 0
    mat = gbg.Matrix(system)
    H, _ = system.dense()
    rng = np.random.default_rng(10 + w)
    x = rng.standard_normal((system.n, w)) + 1j * rng.standard_normal((system.n, w))
    buf = torch.zeros(system.n * w + 1, dtype=torch.complex64, device=dev)
    xa = buf[: system.n * w].view(system.n, w)
    xu = buf[1 : system.n * w + 1].view(system.n, w)
    assert xa.data_ptr() % 16 == 0 and xu.data_ptr() % 16 == 8
    xa.copy_(torch.from_numpy(x))
    ya = to_np(mat.spmm(0, xa, prec="fp32"))
    xu.copy_(torch.from_numpy(x))
    yu = to_np(mat.spmm(0, xu, prec="fp32"))
    assert rel(ya, H @ x) < 2e-6
    assert rel(yu, H @ x) < 2e-6
    mat.close()


# ------------------------------------------------------------------ shifted solve
def run_case(dev, system, z, cols, prec, tol, maxit, panel=0, want_g=True, seed_shift=-1, flags=0):
    w_rho, w_edm = fermi_weights(z)
    mat = gbg.Matrix(system)
    out = gbg.shifted_solve(mat, z, cols, tol=tol, maxit=maxit, prec=prec, w_rho=w_rho, w_edm=w_edm,
                            panel=panel, want_g=want_g, seed_shift=seed_shift, flags=flags)
    torch.cuda.synchronize()
    ref = oracle.solve_outputs(system, z, cols, w_rho, w_edm)
    mat.close()
    return out, ref


def check_outputs(out, ref, bound, want_g=True):
    assert out["status"] == 0, out["message"]
    errs = {}
    if want_g:
        errs["g"] = rel(to_np(out["g_proj"]), ref["g_proj"])
    for key in ("ldos", "rho", "edm", "q", "e_loc"):
        errs[key] = rel(to_np(out[key]), ref[key])
    for key, e in errs.items():
        assert e < bound, (key, e, errs)
    assert to_np(out["converged"]).all()
    assert (to_np(out["resid"]) <= 1.0).all()
    return errs


@pytest.mark.parametrize("panel", [1, 4, 32])
def test_fp64_chain_small_all_columns(dev, panel):
    system = chain_4orb(16, seed=3)  # N = 64
    z = shift_grid(-5, 5, 24, 0.1)
    cols = np.arange(system.n, dtype=np.int32)
    out, ref = run_case(dev, system, z, cols, "fp64", 1e-12, 3000, panel=panel)
    check_outputs(out, ref, 1e-10)


def test_fp64_ragged_ppv_subset(dev):
    system = ppv_chain(3, seed=7)  # N = 114: not a multiple of 4, hydrogen blocks
    z = shift_grid(-10, 6, 40, 0.05)
    cols = np.array([0, 1, 5, 31, 32, 33, 37, 60, 100, 113], np.int32)  # 10 columns: ragged last panel
    out, ref = run_case(dev, system, z, cols, "fp64", 1e-12, 5000, panel=4)
    check_outputs(out, ref, 1e-10)


def test_fp64_single_shift_single_column(dev):
    system = chain_4orb(9, seed=1)
    z = np.array([0.3 + 0.5j])
    cols = np.array([system.n - 1], np.int32)
    out, ref = run_case(dev, system, z, cols, "fp64", 1e-12, 1000)
    check_outputs(out, ref, 1e-10)


def test_fp64_seed_choice_does_not_change_results(dev):
    system = chain_4orb(12, seed=6)
    z = shift_grid(-4, 4, 33, 0.08)
    cols = np.arange(0, system.n, 5, dtype=np.int32)
    a, ref = run_case(dev, system, z, cols, "fp64", 1e-12, 3000, seed_shift=0)
    b, _ = run_case(dev, system, z, cols, "fp64", 1e-12, 3000, seed_shift=32)
    check_outputs(a, ref, 1e-10)
    check_outputs(b, ref, 1e-10)


def test_mixed_small(dev):
    system = ppv_chain(3, seed=8)
    z = shift_grid(-10, 6, 48, 0.05)
    cols = np.arange(0, system.n, 7, dtype=np.int32)
    out, ref = run_case(dev, system, z, cols, "mixed", 1e-10, 8000, panel=8)
    check_outputs(out, ref, 1e-6)


@pytest.mark.parametrize("flags", [0, 4, 6, 16, 18])
def test_mixed_inner_method_and_placement(dev, flags):
    # default: exact factor solves on the FP32 inner levels; bit 2: CG, bit 4:
    # Chebyshev instead; bit 1: the iterations' vectors in shared memory (they
    # fit at this size; the factor solve uses its own shared buffers).  Every
    # combination must reach the oracle; the plan reports the placement.
    system = ppv_chain(4, seed=9)  # N = 152
    z = shift_grid(-10, 6, 40, 0.05)
    cols = np.arange(1, system.n, 9, dtype=np.int32)  # 17 columns: ragged last panel
    mat = gbg.Matrix(system)
    plan = gbg.solve_plan(mat, z, cols, prec="mixed", panel=4, flags=flags)
    mat.close()
    assert plan["cg_smem"] == bool(flags & 2 and flags & (4 | 16))
    out, ref = run_case(dev, system, z, cols, "mixed", 1e-10, 8000, panel=4, flags=flags)
    check_outputs(out, ref, 1e-6)


def test_maxit_exhaustion_reports_noconv(dev):
    system = chain_4orb(30, seed=2)
    z = shift_grid(-3, 3, 16, 0.01)
    cols = np.array([0, 17, 50], np.int32)
    w_rho, w_edm = fermi_weights(z)
    mat = gbg.Matrix(system)
    out = gbg.shifted_solve(mat, z, cols, tol=1e-12, maxit=5, prec="fp64", w_rho=w_rho, w_edm=w_edm)
    assert out["status"] == gbg._binding.GB_ENOCONV
    conv = to_np(out["converged"])
    res = to_np(out["resid"])
    assert not conv.all()
    assert np.all((res <= 1e-12) == (conv == 1))
    assert (to_np(out["iters"]) == 5).all()
    mat.close()


def test_invalid_parameters_rejected(dev):
    system = chain_4orb(6, seed=2)
    mat = gbg.Matrix(system)
    z = np.array([0.1 + 0.1j])
    with pytest.raises(gbg.GBError, match="EINVAL"):
        gbg.shifted_solve(mat, np.array([0.1 - 0.1j]), [0], tol=1e-8, maxit=10)
    with pytest.raises(gbg.GBError, match="EINVAL"):
        gbg.shifted_solve(mat, z, [system.n], tol=1e-8, maxit=10)
    with pytest.raises(gbg.GBError, match="EINVAL"):
        gbg.shifted_solve(mat, z, [0], tol=1e-8, maxit=0)
    with pytest.raises(gbg.GBError, match="EINVAL"):
        gbg.shifted_solve(mat, z, [0], tol=1e-8, maxit=10, panel=3)
    mat.close()


def test_indefinite_overlap_reported(dev):
    system = chain_4orb(10, seed=4)
    s = system.s_val.copy()
    rows = np.repeat(np.arange(system.n), np.diff(system.row_ptr))
    off = rows != system.col_idx
    s[off] *= 30.0  # diagonal blocks stay SPD, the whole S does not
    system.s_val = s
    assert np.linalg.eigvalsh(system.dense()[1]).min() < 0
    mat = gbg.Matrix(system)
    out = gbg.shifted_solve(mat, np.array([0.2 + 0.3j]), [0, 7], tol=1e-10, maxit=50,
                            raise_on=())
    assert out["status"] == gbg._binding.GB_ENOTSPD
    mat.close()


def test_correction_solve_fixes_stagnating_column(dev):
    # Chain 331 of the uneven batch at eta 0.02 (N = 228, 115 shifts): with the
    # iterative (Chebyshev, flags bit 4) inner solve the mixed path's residual
    # for one column stagnates near a gap shift above tol 1e-6.
    # gb_correct_unconverged re-solves that column in FP64 with the stalled
    # shift as the seed; every pair must then meet tol and match the oracle.
    systems, problems = uneven_batch(eta=0.02)
    sysm, pr = systems[331], problems[331]
    assert sysm.n == 228 and len(pr["z"]) == 115
    mat = gbg.Matrix(sysm)
    kw = dict(tol=1e-6, maxit=16000, prec="mixed", w_rho=pr["w_rho"], w_edm=pr["w_edm"], panel=2, want_g=True,
              flags=16)
    first = gbg.shifted_solve(mat, pr["z"], pr["cols"], **kw)
    assert first["status"] == gbg._binding.GB_ENOCONV
    out = gbg.shifted_solve(mat, pr["z"], pr["cols"], correct=True, **kw)
    mat.close()
    assert out["status"] == 0, out["message"]
    assert out["corrected"] >= 1
    assert to_np(out["converged"]).all()
    assert (to_np(out["resid"]) <= 1e-6).all()
    ref = oracle.solve_outputs(sysm, pr["z"], pr["cols"], pr["w_rho"], pr["w_edm"])
    check_outputs(out, ref, 1e-6)


@pytest.mark.parametrize("prec,panel,tol,per", [("mixed", 4, 1e-10, 4), ("mixed", 8, 1e-8, 3), ("mixed", 8, 1e-6, 2),
                                                ("fp64", 4, 1e-12, 1), ("fp64", 32, 1e-12, 1)])
def test_exact_factor_inner_solve(dev, prec, panel, tol, per):
    # The default inner solve where S's half-bandwidth is <= 63 (53 here): the
    # block-bidiagonal Cholesky factor, one solve per FP64 application; the
    # mixed path refines FP32 solves around float-float residuals, two levels
    # for tol >= 1e-6, three down to 1e-9 and four below.  The inner count is levels x (outer
    # iterations + the initial S^-1 b); outputs match the oracle at each
    # path's bound.  N = 152: three 64-row blocks, ragged last.
    system = ppv_chain(4, seed=9)
    z = shift_grid(-10, 6, 40, 0.05)
    cols = np.arange(1, system.n, 9, dtype=np.int32)
    bound = 1e-6 if prec == "mixed" else 1e-10
    out, ref = run_case(dev, system, z, cols, prec, tol, 8000, panel=panel)
    check_outputs(out, ref, bound)
    it = to_np(out["iters"])
    inner = to_np(out["inner_iters"])
    for p0 in range(0, len(cols), panel):
        assert inner[p0] == per * (it[p0 : p0 + panel].max() + 1)


@pytest.mark.parametrize("w", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("maker", [lambda: ppv_chain(7, seed=2), lambda: chain_4orb(41, seed=3)])
def test_apply_sinv_exact(dev, maker, w):
    # the factor solve alone: FP64 to rounding, one FP32 solve (TF32 tensor
    # cores, three-term split) to ~2e-6 (several 64-row blocks, ragged last
    # block, every panel width)
    system = maker()
    mat = gbg.Matrix(system)
    _, S = system.dense()
    rng = np.random.default_rng(w)
    x = rng.standard_normal((system.n, w)) + 1j * rng.standard_normal((system.n, w))
    ref = np.linalg.solve(S, x)
    xt = torch.from_numpy(x).to(dev)
    y = to_np(mat.apply_sinv(xt, prec="fp64"))
    assert rel(y, ref) < 1e-13
    y32 = to_np(mat.apply_sinv(xt, prec="fp32"))
    assert rel(y32, ref) < 5e-6
    mat.close()


def test_fp64_cg_inner_solve_still_matches(dev):
    # flags bit 2 keeps the iterative inner CG (the path for wide-band S)
    system = ppv_chain(3, seed=7)
    z = shift_grid(-10, 6, 24, 0.05)
    cols = np.arange(0, system.n, 11, dtype=np.int32)
    out, ref = run_case(dev, system, z, cols, "fp64", 1e-12, 5000, panel=4, flags=4)
    check_outputs(out, ref, 1e-10)


def test_misaligned_complex_double_buffers_are_rejected(dev):
    # a complex-double array 8 bytes off its 16-byte boundary is GB_EINVAL
    # before any launch (the kernels read it as 16-byte vectors)
    import ctypes as C

    system = chain_4orb(8, seed=1)
    mat = gbg.Matrix(system)
    lib = gbg._binding.load()
    buf = torch.zeros(4 * system.n + 4, dtype=torch.float64, device=dev)
    out = torch.zeros(2 * system.n, dtype=torch.complex128, device=dev)
    st = lib.gb_spmm(mat.handle, 0, gbg._binding.GB_FP64, 1, C.c_void_p(buf.data_ptr() + 8),
                     C.c_void_p(out.data_ptr()), None)
    assert st == gbg._binding.GB_EINVAL
    assert "aligned" in lib.gb_last_error().decode()
    psi = C.c_void_p(buf.data_ptr() + 8)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
    st = lib.gb_wavepacket(mat.handle, 1, psi, 1, 0.1, -10.0, 10.0, None, C.c_void_p(ws.data_ptr()),
                           C.c_size_t(ws.numel()), None)
    assert st == gbg._binding.GB_EINVAL
    mat.close()
