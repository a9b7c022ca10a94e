"""Wavepacket propagation i S dc/dt = H c (gb_wavepacket) against the oracle's
generalized spectral sum: random packets and the HOMO over 40 steps of 0.1 fs,
S-norm conservation, and the HOMO's pure phase."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import wavepacket as owp
from synth import ppv_chain

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
gbg = pytest.importorskip("paper_1603_09616_gb300")

HBAR_EV_FS = 0.6582119569


def test_wavepacket_matches_spectral_sum():
    torch.cuda.set_device(0)
    system = ppv_chain(3, seed=6)  # N = 114 (padded block rows)
    H, S = system.dense()
    lam = sla.eigh(H, S, eigvals_only=True)
    span = lam.max() - lam.min()
    e_min, e_max = lam.min() - 0.01 * span, lam.max() + 0.01 * span
    rng = np.random.default_rng(11)
    c0 = rng.standard_normal((system.n, 5)) + 1j * rng.standard_normal((system.n, 5))
    y, e_homo = owp.homo(system, system.n)
    c0 = np.concatenate([c0, y[:, None]], axis=1)
    tau, steps = 0.1 / HBAR_EV_FS, 40
    mat = gbg.Matrix(system)
    psi = torch.from_numpy(np.ascontiguousarray(c0)).cuda()
    psi, nterms = gbg.wavepacket(mat, psi, steps, tau, e_min, e_max)
    got = psi.cpu().numpy()
    ref = owp.propagate(system, c0, steps * tau)
    assert nterms > 2
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()
    assert np.allclose(owp.s_norm(system, got), owp.s_norm(system, c0), rtol=1e-11)
    ph = np.exp(-1j * e_homo * steps * tau)
    assert np.abs(got[:, -1] - ph * y).max() < 1e-10 * np.abs(y).max()
    mat.close()


def test_wavepacket_rejects_bad_bounds_and_long_steps():
    torch.cuda.set_device(0)
    system = ppv_chain(2, seed=1)
    mat = gbg.Matrix(system)
    psi = torch.zeros((system.n, 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(gbg.GBError, match="EINVAL"):
        gbg.wavepacket(mat, psi, 1, 0.15, 1.0, -1.0)
    with pytest.raises(gbg.GBError, match="EINVAL"):
        gbg.wavepacket(mat, psi, 1, 100.0, -40.0, 40.0)  # a tau = 4000: too many terms
    mat.close()


def test_wavepacket_many_packets_share_teams():
    # 300 packets: more than one per SM, so teams take two columns each (the
    # panel width grows with the packet count); every packet must still match
    torch.cuda.set_device(0)
    system = ppv_chain(2, seed=2)
    H, S = system.dense()
    lam = sla.eigh(H, S, eigvals_only=True)
    span = lam.max() - lam.min()
    rng = np.random.default_rng(21)
    c0 = rng.standard_normal((system.n, 300)) + 1j * rng.standard_normal((system.n, 300))
    tau, steps = 0.1 / HBAR_EV_FS, 5
    mat = gbg.Matrix(system)
    psi = torch.from_numpy(np.ascontiguousarray(c0)).cuda()
    psi, _ = gbg.wavepacket(mat, psi, steps, tau, lam.min() - 0.01 * span, lam.max() + 0.01 * span)
    ref = owp.propagate(system, c0, steps * tau)
    assert np.abs(psi.cpu().numpy() - ref).max() < 1e-10 * np.abs(ref).max()
    mat.close()
