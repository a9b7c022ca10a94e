"""Pins of the CPU oracle against results fixed by mathematics, not by itself.

The oracle solves (z S - H) x = e_j by dense LU (Introduction: generalized
shifted linear equations).  Each test below checks it against an independent
statement: the spectral closed form from the generalized eigenproblem
H y = lambda S y (the direct-solver complement named in the Introduction), the
complex symmetry of G, the trace identity, the sum rule, a 2-site analytic
case, brute-force inversion, and the spectral form of the reductions.  The
last tests plant mistakes in the oracle's inputs/outputs and check that a pin
catches each one.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from synth import TBSystem, chain_4orb, fermi_weights, ppv_chain, shift_grid


def spectral(system):
    H, S = system.dense()
    lam, Y = sla.eigh(H, S)  # Y^T S Y = I
    return H, S, lam, Y


def g_closed(lam, Y, z):
    return (Y / (z - lam)) @ Y.T


def small_systems():
    return [chain_4orb(30, seed=11), ppv_chain(4, seed=5)]


@pytest.mark.parametrize("which", [0, 1])
def test_lu_matches_spectral_closed_form(which):
    system = small_systems()[which]
    H, S, lam, Y = spectral(system)
    assert np.allclose(Y.T @ S @ Y, np.eye(system.n), atol=1e-10)
    z = shift_grid(lam.min() - 1, lam.max() + 1, 7, 0.05)
    cols = np.arange(system.n)
    X = oracle.green_columns(H, S, z, cols)
    for k, zk in enumerate(z):
        G = g_closed(lam, Y, zk)
        err = np.abs(X[k] - G).max() / np.abs(G).max()
        assert err < 1e-11, (k, err)


def test_complex_symmetry():
    system = ppv_chain(3, seed=2)
    H, S = system.dense()
    z = np.array([0.3 + 0.02j, -4.0 + 0.02j, 2.5 + 0.5j])
    X = oracle.green_columns(H, S, z, np.arange(system.n))
    for k in range(len(z)):
        G = X[k]
        assert np.abs(G - G.T).max() <= 1e-11 * np.abs(G).max()
        # and it is not Hermitian (the bilinear, not sesquilinear, symmetry)
        assert np.abs(G - G.conj().T).max() > 1e-3 * np.abs(G).max()


def test_trace_identity_full_column_set():
    system = chain_4orb(25, seed=4)
    H, S, lam, Y = spectral(system)
    z = shift_grid(-6, 6, 9, 0.05)
    cols = np.arange(system.n)
    w0 = np.zeros(len(z), complex)
    out = oracle.solve_outputs(system, z, cols, w0, w0)
    tr = out["gs_diag"].sum(axis=1)  # sum_j (G S)_jj
    exact = np.array([np.sum(1.0 / (zk - lam)) for zk in z])
    assert np.abs(tr - exact).max() <= 1e-10 * np.abs(exact).max()
    # the local DOS is -(1/pi) Im of the same diagonal
    assert np.allclose(out["ldos"], -np.imag(out["gs_diag"]) / np.pi)


def test_sum_rule_on_window():
    system = chain_4orb(6, seed=8)  # N = 24
    H, S, lam, Y = spectral(system)
    eta = 0.05
    a, b = -2.0, 2.5
    h = eta / 40
    eps = np.arange(a, b + h / 2, h)
    z = eps + 1j * eta
    cols = np.arange(system.n)
    w0 = np.zeros(len(z), complex)
    out = oracle.solve_outputs(system, z, cols, w0, w0)
    dos = out["ldos"].sum(axis=1)  # -(1/pi) Im Tr[G S]
    # composite Simpson on the evenly spaced grid (odd number of points)
    if len(eps) % 2 == 0:
        eps, dos = eps[:-1], dos[:-1]
        b = eps[-1]
    wts = np.ones(len(eps))
    wts[1:-1:2] = 4
    wts[2:-1:2] = 2
    integral = (eps[1] - eps[0]) / 3 * np.sum(wts * dos)
    exact = np.sum((np.arctan((b - lam) / eta) - np.arctan((a - lam) / eta)) / np.pi)
    assert abs(integral - exact) < 1e-6 * system.n, (integral, exact)
    # and the full-axis limit counts every state once (sum rule = N)
    wide = np.sum((np.arctan((1e9 - lam) / eta) - np.arctan((-1e9 - lam) / eta)) / np.pi)
    assert abs(wide - system.n) < 1e-6


def two_site(e, t, s):
    row_ptr = np.array([0, 2, 4], np.int64)
    col_idx = np.array([0, 1, 0, 1], np.int32)
    h = np.array([e, t, t, e], float)
    sv = np.array([1.0, s, s, 1.0])
    return TBSystem(2, row_ptr, col_idx, h, sv, np.array([0, 1], np.int32), name="two_site")


@pytest.mark.parametrize("e,t,s", [(0.0, -2.7, 0.1), (1.3, -1.1, 0.3), (-0.5, 0.8, -0.2)])
def test_two_site_analytic(e, t, s):
    system = two_site(e, t, s)
    z = np.array([0.1 + 0.05j, -3.0 + 0.02j, 2.0 + 1.0j, (e + t) / (1 + s) + 0.01j])
    cols = np.array([0, 1])
    w_rho = np.array([0.3, -0.2, 0.1 + 0.4j, 1.0])
    w_edm = np.array([0.0, 1.0, 0.5j, -0.25])
    out = oracle.solve_outputs(system, z, cols, w_rho, w_edm, keep_full=True)
    a = z - e
    c = z * s - t
    det = a * a - c * c
    G00 = a / det
    G01 = -c / det
    for k in range(len(z)):
        G = out["x_full"][k]
        assert np.allclose(G, [[G00[k], G01[k]], [G01[k], G00[k]]], rtol=1e-13, atol=0)
    gs00 = (a - c * s) / det
    assert np.allclose(out["gs_diag"][:, 0], gs00, rtol=1e-13)
    assert np.allclose(out["ldos"][:, 1], -np.imag(gs00) / np.pi, rtol=1e-12)
    # density / energy density on the pattern of column 0: rows (0, 1)
    rho0 = np.sum(np.imag(w_rho * G00))
    rho1 = np.sum(np.imag(w_rho * G01))
    edm1 = np.sum(np.imag(w_edm * G01))
    assert np.allclose(out["rho"][:2], [rho0, rho1], rtol=1e-12, atol=1e-15)
    assert np.isclose(out["edm"][1], edm1, rtol=1e-12, atol=1e-15)
    assert np.isclose(out["q"][0], rho0 + s * rho1, rtol=1e-12, atol=1e-15)
    assert np.isclose(out["e_loc"][0], e * rho0 + t * rho1, rtol=1e-12, atol=1e-15)
    # generalized eigenvalues of the 2-site pencil
    lam = np.sort(sla.eigh(*system.dense(), eigvals_only=True))
    assert np.allclose(lam, np.sort([(e + t) / (1 + s), (e - t) / (1 - s)]), rtol=1e-13)


def test_brute_force_tiny():
    rng = np.random.default_rng(3)
    for n in range(1, 9):
        A = rng.standard_normal((n, n))
        H = A + A.T
        B = 0.2 * rng.standard_normal((n, n))
        S = np.eye(n) + 0.5 * (B + B.T) * (n > 1)
        S += np.eye(n) * max(0.0, 0.1 - np.linalg.eigvalsh(S).min())
        z = np.array([0.4 + 0.1j, -1.0 + 0.3j])
        cols = np.arange(n)[::-1]
        X = oracle.green_columns(H, S, z, cols)
        for k, zk in enumerate(z):
            inv = np.linalg.inv(zk * S - H)
            assert np.allclose(X[k], inv[:, cols], rtol=1e-12, atol=1e-13)


def test_reductions_match_spectral_form():
    system = ppv_chain(3, seed=9)
    H, S, lam, Y = spectral(system)
    z = shift_grid(-8, 4, 24, 0.1)
    w_rho, w_edm = fermi_weights(z, mu=-1.0, kT=0.2)
    w_rho = w_rho + 0.05j * np.cos(np.arange(len(z)))  # complex weights too
    cols = np.array([0, 7, 33, system.n - 1])
    out = oracle.solve_outputs(system, z, cols, w_rho, w_edm)
    off = out["off"]
    for c, j in enumerate(cols):
        R = system.row_cols(int(j))
        # G_ij(z) = sum_l y_il y_jl / (z - lambda_l)
        Gz = np.array([(Y[R] * Y[j]) @ (1.0 / (zk - lam)) for zk in z])  # [K, m_j]
        rho = np.sum(np.imag(w_rho[:, None] * Gz), axis=0)
        edm = np.sum(np.imag(w_edm[:, None] * Gz), axis=0)
        assert np.allclose(out["rho"][off[c] : off[c + 1]], rho, rtol=1e-10, atol=1e-13)
        assert np.allclose(out["edm"][off[c] : off[c + 1]], edm, rtol=1e-10, atol=1e-13)
        lo, hi = system.row_ptr[j], system.row_ptr[j + 1]
        assert np.isclose(out["q"][c], np.sum(rho * system.s_val[lo:hi]), rtol=1e-10, atol=1e-13)
        assert np.isclose(out["e_loc"][c], np.sum(rho * system.h_val[lo:hi]), rtol=1e-10, atol=1e-13)
        # imaginary part of G from the Lorentzian form, for real weights
        imG = np.array([-(0.1) * (Y[R] * Y[j]) @ (1.0 / ((zk.real - lam) ** 2 + 0.01)) for zk in z])
        assert np.allclose(np.imag(Gz), imG, rtol=1e-10, atol=1e-13)


def test_density_matrix_small_eta_limit():
    """With eta -> 0 and Fermi weights the density matrix tends to
    2 sum_l f(lambda_l) y_il y_jl (spin-degenerate occupation of eigenstates)."""
    system = chain_4orb(4, seed=12)  # N = 16
    H, S, lam, Y = spectral(system)
    mu, kT, eta = 0.0, 0.2, 2e-3
    eps = np.arange(lam.min() - 3.0, mu + 3.0, eta / 4)
    z = eps + 1j * eta
    w_rho, _ = fermi_weights(z, mu=mu, kT=kT)
    cols = np.arange(system.n)
    out = oracle.solve_outputs(system, z, cols, w_rho, np.zeros_like(w_rho))
    f = 0.5 * (1 - np.tanh((lam - mu) / (2 * kT)))
    P = 2 * (Y * f) @ Y.T
    off = out["off"]
    err = 0.0
    for c, j in enumerate(cols):
        R = system.row_cols(int(j))
        err = max(err, np.abs(out["rho"][off[c] : off[c + 1]] - P[R, j]).max())
    assert err < 2e-2, err
    # the electron count sum_j q_j = Tr[rho S] -> 2 sum_l f(lambda_l)
    assert abs(out["q"].sum() - 2 * f.sum()) < 2e-2 * system.n


# ---------------------------------------------------------------- planted mistakes
def test_planted_sign_error_is_caught():
    system = chain_4orb(8, seed=1)
    H, S, lam, Y = spectral(system)
    z = np.array([0.3 + 0.05j])
    bad = oracle.green_columns(-H, -S, z, np.arange(system.n))  # solves (H - zS) x = b
    G = g_closed(lam, Y, z[0])
    assert np.abs(bad[0] - G).max() > 1e-2 * np.abs(G).max()


def test_planted_dropped_overlap_in_ldos_is_caught():
    system = chain_4orb(8, seed=1)
    H, S, lam, Y = spectral(system)
    z = shift_grid(-3, 3, 5, 0.05)
    cols = np.arange(system.n)
    X = oracle.green_columns(H, S, z, cols)
    Gp = oracle.project_columns(system, X, cols)
    import copy

    bad_sys = copy.deepcopy(system)
    bad_sys.s_val = np.where(system.col_idx == np.repeat(np.arange(system.n), np.diff(system.row_ptr)), 1.0, 0.0)
    w0 = np.zeros(len(z), complex)
    bad = oracle.reduce_outputs(bad_sys, Gp, cols, w0, w0)  # uses G_jj instead of (G S)_jj
    exact = np.array([np.sum(1.0 / (zk - lam)) for zk in z])
    assert np.abs(bad["gs_diag"].sum(axis=1) - exact).max() > 1e-3 * np.abs(exact).max()


def test_planted_column_shift_is_caught():
    rng = np.random.default_rng(0)
    n = 6
    A = rng.standard_normal((n, n))
    H = A + A.T
    S = np.eye(n)
    cols = np.arange(n)
    z = np.array([0.2 + 0.1j])
    X = oracle.green_columns(H, S, z, (cols + 1) % n)  # wrong right-hand sides
    inv = np.linalg.inv(z[0] * S - H)
    assert not np.allclose(X[0], inv[:, cols], rtol=1e-6)


def test_planted_real_part_in_density_is_caught():
    system = ppv_chain(2, seed=4)
    H, S, lam, Y = spectral(system)
    z = shift_grid(-5, 3, 12, 0.1)
    w_rho, w_edm = fermi_weights(z)
    cols = np.array([0, 10])
    X = oracle.green_columns(H, S, z, cols)
    Gp = oracle.project_columns(system, X, cols)
    # a real-part mistake: feed i*G so that Im(c * iG) = Re(c * G)
    bad = oracle.reduce_outputs(system, 1j * Gp, cols, w_rho, w_edm)
    R = system.row_cols(0)
    Gz = np.array([(Y[R] * Y[0]) @ (1.0 / (zk - lam)) for zk in z])
    rho = np.sum(np.imag(w_rho[:, None] * Gz), axis=0)
    assert not np.allclose(bad["rho"][: len(R)], rho, rtol=1e-3)


def test_sparse_oracle_matches_closed_form():
    system = ppv_chain(3, seed=6)
    H, S, lam, Y = spectral(system)
    z = np.array([-1.0 + 0.02j, 2.0 + 0.05j])
    cols = np.array([1, 40, system.n - 2])
    sp_out = oracle.green_columns_sparse(system, z, cols)
    off = oracle.pattern_offsets(system.row_ptr, cols)
    for k, zk in enumerate(z):
        G = g_closed(lam, Y, zk)
        for c, j in enumerate(cols):
            R = system.row_cols(int(j))
            assert np.allclose(sp_out[k, off[c] : off[c + 1]], G[R, j], rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------- chemical potential (oracle/fermi.py)
def test_fermi_level_tends_to_the_eigenvalue_occupation():
    # small eta, fine grid: the quadrature's mu tends to the mu that fills the
    # generalized eigenvalues, sum_l 2 f((lambda_l - mu) / kT) = N_e, and
    # rho to 2 sum_l f y_l y_l^T (the eigen-decomposition limit)
    from oracle import fermi as of

    system = chain_4orb(4, seed=12)  # N = 16
    H, S, lam, Y = spectral(system)
    kT, eta = 0.3, 4e-3
    eps = np.arange(lam.min() - 3.0, lam.max() + 3.0, eta / 4)
    z = eps + 1j * eta
    n_e = float(system.n)  # one electron per orbital
    # the eigenvalue occupation, by its own bisection on the spectrum
    lo, hi = lam.min() - 10, lam.max() + 10
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if 2 * of.fermi((lam - mid) / kT).sum() < n_e:
            lo = mid
        else:
            hi = mid
    mu_eig = 0.5 * (lo + hi)
    cols = np.arange(system.n)
    X = oracle.green_columns(H, S, z, cols)
    g = oracle.project_columns(system, X, cols)
    zero = np.zeros(len(z), dtype=np.complex128)
    ldos = oracle.reduce_outputs(system, g, cols, zero, zero)["ldos"]
    mu = of.fermi_level(z.real, ldos, n_e, kT)
    assert abs(mu - mu_eig) < 2e-2, (mu, mu_eig)
    c, ce = of.weights(z.real, mu, kT)
    out = oracle.reduce_outputs(system, g, cols, c, ce)
    assert abs(out["q"].sum() - n_e) < 1e-9 * n_e  # Tr[rho S] = N_e exactly at the found mu
    P = 2 * (Y * of.fermi((lam - mu_eig) / kT)) @ Y.T
    err = max(np.abs(out["rho"][out["off"][c_] : out["off"][c_ + 1]] - P[system.row_cols(j), j]).max()
              for c_, j in enumerate(cols))
    assert err < 3e-2, err


def test_fermi_level_two_site_half_filled_level_and_planted_spin():
    # 2-site case, S = I: levels e - |t| and e + |t|.  One electron (spin 2)
    # half-fills the lower level, so mu sits on it (f is antisymmetric about
    # the level and its Lorentzian is symmetric in a window centred on it; the
    # upper level's tail moves mu by ~1e-4 here)
    from oracle import fermi as of
    from synth import TBSystem

    e, t = 0.4, -1.5
    lower = e - abs(t)
    rp = np.array([0, 2, 4], np.int64)
    ci = np.array([0, 1, 0, 1], np.int32)
    sysm = TBSystem(2, rp, ci, np.array([e, t, t, e]), np.array([1.0, 0.0, 0.0, 1.0]), np.array([0, 1], np.int32))
    eps = np.linspace(lower - 4.0, lower + 4.0, 3201)
    z = eps + 1j * 0.01
    H, S = sysm.dense()
    X = oracle.green_columns(H, S, z, np.arange(2))
    g = oracle.project_columns(sysm, X, np.arange(2))
    zero = np.zeros(len(z), dtype=np.complex128)
    ldos = oracle.reduce_outputs(sysm, g, np.arange(2), zero, zero)["ldos"]
    mu = of.fermi_level(z.real, ldos, 1.0, kT=0.05)
    assert abs(mu - lower) < 2e-3, mu
    # a dropped spin factor would need the whole lower level: mu leaves it
    mu1 = of.fermi_level(z.real, ldos, 1.0, kT=0.05, spin=1.0)
    assert mu1 > lower + 0.2, mu1


# ---------------------------------------------------------------- forces (f2)
def _fd_case():
    from oracle import forces as of

    system = ppv_chain(2, seed=4)  # N = 76, 28 atoms, S diagonal at 1
    mu, kT = 0.0, 0.1
    rho, edm = of.eigen_density(system, mu, kT)
    cols = np.arange(system.n)
    from synth import model_gradients

    gh, gs = model_gradients(system)
    return system, mu, kT, of.pack(system, rho, cols), of.pack(system, edm, cols), cols, gh, gs


def test_forces_are_minus_the_gradient_of_the_grand_potential():
    # F_a = -dOmega/dR_a at fixed mu (central differences of the eigenvalue
    # grand potential with the same random matrix factors), for the exact
    # density and energy-density matrices of the eigen-decomposition
    from oracle import forces as of
    from synth import displace

    system, mu, kT, rho, edm, cols, gh, gs = _fd_case()
    F = of.forces(system, rho, edm, cols, gh, gs)
    h = 1e-5
    scale = np.abs(F).max()
    for atom in (0, 5, 11, 20):
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            wp = of.grand_potential(displace(system, atom, e), mu, kT)
            wm = of.grand_potential(displace(system, atom, -e), mu, kT)
            fd = -(wp - wm) / (2 * h)
            assert abs(F[atom, k] - fd) < 1e-6 * scale, (atom, k, F[atom, k], fd)


def test_forces_sum_to_zero_and_exert_no_torque():
    # two-center radial elements: every entry's gradients on its two atoms are
    # opposite and along the bond, so sum_a F_a = 0 and sum_a R_a x F_a = 0
    from oracle import forces as of

    system, mu, kT, rho, edm, cols, gh, gs = _fd_case()
    F = of.forces(system, rho, edm, cols, gh, gs)
    scale = np.abs(F).max()
    assert np.abs(F.sum(axis=0)).max() < 1e-11 * scale * len(F)
    assert np.abs(np.cross(system.positions, F).sum(axis=0)).max() < 1e-10 * scale * len(F)


def test_planted_dropped_energy_density_term_in_forces_is_caught():
    # with S != I the P^E dS term matters: leaving it out misses the gradient
    from oracle import forces as of
    from synth import displace

    system, mu, kT, rho, edm, cols, gh, gs = _fd_case()
    F_bad = of.forces(system, rho, np.zeros_like(edm), cols, gh, gs)
    h = 1e-5
    e = np.array([h, 0.0, 0.0])
    fd = -(of.grand_potential(displace(system, 5, e), mu, kT) - of.grand_potential(displace(system, 5, -e), mu, kT)) / (2 * h)
    assert abs(F_bad[5, 0] - fd) > 1e-3 * abs(fd)


# ---------------------------------------------------------------- pole expansion (f3)
def test_pole_expansion_reproduces_the_fermi_function():
    from oracle import fermi as of
    from synth import pole_weights

    kT, spin = 0.1, 2.0
    z, c, ce, a, b, cs = pole_weights(mu=0.3, kT=kT, n_poles=40, spin=spin)
    R = (c / (-2.0 * kT * spin * 1j)).real
    ap = z.imag / kT
    assert np.allclose(z.real, 0.3) and ap.min() > 3.14159 and ap.min() < 3.1416  # first pole at i pi kT
    x = np.linspace(-400, 400, 200001)
    fx = 0.5 + (R[None, :] * (1 / (x[:, None] - 1j * ap) + 1 / (x[:, None] + 1j * ap))).sum(1).real
    assert np.abs(fx - of.fermi(x)).max() < 1e-13


def test_pole_expansion_gives_the_finite_temperature_density_matrices():
    # rho = s f(S^-1 H) S^-1 and P^E = S^-1 H rho, exactly (eigen-decomposition),
    # from 40 resolvents far from the real axis plus the S^-1 terms
    from oracle import fermi as of
    from oracle import forces as ofo
    from synth import pole_weights

    system = ppv_chain(2, seed=4)
    mu, kT = 0.2, 0.1
    cols = np.arange(system.n)
    z, c, ce, a, b, cs = pole_weights(mu=mu, kT=kT, n_poles=40)
    out = of.outputs_with_sinv(system, z, cols, c, ce, a, b, cs)
    rho_e, edm_e = ofo.eigen_density(system, mu, kT)
    rho_p, edm_p = ofo.pack(system, rho_e, cols), ofo.pack(system, edm_e, cols)
    assert np.abs(out["rho"] - rho_p).max() < 1e-11 * np.abs(rho_p).max()
    assert np.abs(out["edm"] - edm_p).max() < 1e-11 * np.abs(edm_p).max()
    H, S = system.dense()
    assert abs(out["q"].sum() - np.trace(rho_e @ S)) < 1e-10 * system.n
    # planted: without the S^-1 H S^-1 term P^E is wrong
    si, shs = of.sinv_terms(system, cols)
    assert np.abs(out["edm"] - cs * shs - edm_p).max() > 1e-2 * np.abs(edm_p).max()


# ---------------------------------------------------------------- wavepacket (f4)
def test_wavepacket_spectral_sum_equals_the_matrix_exponential():
    import scipy.linalg as sla

    from oracle import wavepacket as ow

    system = ppv_chain(2, seed=6)
    H, S = system.dense()
    rng = np.random.default_rng(3)
    c0 = rng.standard_normal((system.n, 3)) + 1j * rng.standard_normal((system.n, 3))
    t = 1.7
    ref = sla.expm(-1j * t * np.linalg.solve(S, H)) @ c0
    got = ow.propagate(system, c0, t)
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()
    # the S-norm is conserved, and an eigenstate only turns its phase
    assert np.allclose(ow.s_norm(system, got), ow.s_norm(system, c0), rtol=1e-12)
    y, lam = ow.homo(system, system.n)
    yt = ow.propagate(system, y[:, None], t)[:, 0]
    assert np.abs(yt - np.exp(-1j * lam * t) * y).max() < 1e-12 * np.abs(y).max()


def test_wavepacket_two_site_rabi_oscillation():
    # S = I, H = [[e, v], [v, e]]: c(0) = e_1 gives exp(-i e t) (cos vt, -i sin vt)
    from oracle import wavepacket as ow

    e, v, t = 0.3, -1.1, 0.9
    sysm = two_site(e, v, 0.0)
    got = ow.propagate(sysm, np.array([[1.0], [0.0]]), t)[:, 0]
    ref = np.exp(-1j * e * t) * np.array([np.cos(v * t), -1j * np.sin(v * t)])
    assert np.abs(got - ref).max() < 1e-14
