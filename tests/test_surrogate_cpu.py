"""Pins of the surrogate's CPU references (oracle/mlp.py, oracle/descriptors.py).

The MLP reference's backward is checked against central finite differences of
its own forward, its bfloat16 rounding against PyTorch's CPU conversion, GELU
against the normal CDF, Adam against one hand-expanded step; the descriptor
reference against rotation/translation invariance and a 2-atom hand case.
"""
import numpy as np
import pytest
import scipy.stats

from oracle import descriptors as odesc
from oracle import mlp as omlp
from synth import TBSystem, ppv_bundle


def random_net(rng, dims=(6, 5, 5, 4, 2)):
    W = [rng.normal(0, 0.6, (dims[l + 1], dims[l])).astype(np.float32) for l in range(4)]
    b = [rng.normal(0, 0.1, dims[l + 1]) for l in range(4)]
    return W, b


def test_mlp_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    W, b = random_net(rng)
    X = rng.normal(size=(7, 6))
    dY = rng.normal(size=(7, 2))
    y, cache = omlp.forward(W, b, X)
    gw, gb = omlp.backward(W, cache, dY)
    # differentiate with respect to the biases and inputs (weights enter through
    # the bf16 rounding, so they are checked through the bias path and dX chain)
    eps = 1e-6
    for l in range(4):
        for k in range(len(b[l])):
            bp = [x.copy() for x in b]
            bm = [x.copy() for x in b]
            bp[l][k] += eps
            bm[l][k] -= eps
            fd = (np.sum(omlp.forward(W, bp, X)[0] * dY) - np.sum(omlp.forward(W, bm, X)[0] * dY)) / (2 * eps)
            assert abs(fd - gb[l][k]) < 1e-6 * max(1.0, abs(fd)), (l, k)
    # weight gradients: perturb the activations' preimage through an equivalent
    # FP64 network whose weights are already bf16 values
    Wb = [omlp.bf16_round(w) for w in W]
    for l in range(4):
        for (o, i) in [(0, 0), (1, 2), (len(Wb[l]) - 1, Wb[l].shape[1] - 1)]:
            def f(delta):
                a = X
                for m in range(4):
                    Wm = Wb[m].copy()
                    if m == l:
                        Wm[o, i] += delta
                    p = a @ Wm.T + b[m]
                    a = omlp.gelu(p) if m < 3 else p
                return np.sum(a * dY)
            fd = (f(eps) - f(-eps)) / (2 * eps)
            assert abs(fd - gw[l][o, i]) < 1e-6 * max(1.0, abs(fd)), (l, o, i)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(0, 10, 1000), [1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-9, -2.5, 0.0]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(omlp.bf16_round(x), ref)


def test_gelu_and_adam_definitions():
    t = np.linspace(-5, 5, 101)
    assert np.allclose(omlp.gelu(t), t * scipy.stats.norm.cdf(t), rtol=1e-14, atol=1e-15)
    h = 1e-6
    assert np.allclose(omlp.gelu_grad(t), (omlp.gelu(t + h) - omlp.gelu(t - h)) / (2 * h), atol=1e-8)
    w, m, v = omlp.adam(np.array([1.0]), np.array([0.5]), np.zeros(1), np.zeros(1), 0.1, 0.9, 0.999, 1e-8, 1)
    # first step: m_hat = g, v_hat = g^2 -> w - lr * sign(g) (up to eps)
    assert np.allclose(w, 1.0 - 0.1 * 0.5 / (0.5 + 1e-8))


def rotation(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


def test_descriptor_rotation_translation_invariance():
    system = ppv_bundle(n_side=2, n_mono=2, seed=4)
    species = (system.atom_norb == 1).astype(int)
    d0 = odesc.descriptors(system, species)
    moved = TBSystem(system.n, system.row_ptr, system.col_idx, system.h_val, system.s_val, system.orb_atom,
                     positions=system.positions @ rotation(3).T + np.array([1.0, -2.0, 0.5]),
                     atom_norb=system.atom_norb)
    d1 = odesc.descriptors(moved, species)
    assert np.allclose(d0, d1, rtol=1e-9, atol=1e-12)
    assert d0[:, 63].min() == 1.0 and np.allclose(d0[:, 40] + d0[:, 41], 1.0)


def test_descriptor_two_atom_hand_case():
    r = 0.2
    # carbon (4 orbitals) at the origin, hydrogen (1 orbital) at distance r
    n = 5
    rows, cols = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    rp = np.arange(0, n * n + 1, n, dtype=np.int64)
    ci = cols.ravel().astype(np.int32)
    H = np.full((n, n), -0.5)
    np.fill_diagonal(H, [0.1, 0.2, 0.3, 0.4, -1.0])
    S = np.full((n, n), 0.05)
    np.fill_diagonal(S, 1.0)
    system = TBSystem(n, rp, ci, H.ravel(), S.ravel(), np.array([0, 0, 0, 0, 1], np.int32),
                      positions=np.array([[0.0, 0, 0], [0.0, 0, r]]), atom_norb=np.array([4, 1], np.int32))
    d = odesc.descriptors(system, np.array([0, 1]))
    w = 0.5 * (np.cos(np.pi * r / 0.5) + 1)
    # orbital 0 (carbon, slot 0): its only neighbour atom is the hydrogen
    mu = 0.1 + 0.4 * np.arange(16) / 15
    assert np.allclose(d[0, 16:32], w * np.exp(-(((r - mu) / 0.03) ** 2)))
    assert np.allclose(d[0, 0:16], 0.0)
    assert np.isclose(d[0, 32 + 2 * 1], w * w)  # shell 1 (0.125 <= r < 0.25), |dipole|^2
    q = np.outer([0, 0, 1], [0, 0, 1]) - np.eye(3) / 3
    assert np.isclose(d[0, 33 + 2 * 1], w * w * np.sum(q * q))
    assert d[0, 40] == 1 and d[0, 42] == 1 and d[4, 41] == 1 and d[4, 42] == 1
    assert np.isclose(d[0, 46], 0.1) and np.isclose(d[0, 47], 1.0)
    others = [1, 2, 3, 4]
    assert np.isclose(d[0, 56], 4 * 0.25)
    assert np.isclose(d[0, 59], 0.25 * sum(H[i, i] for i in others))
    assert np.isclose(d[0, 61], 0.05)


def test_adam_second_step_by_hand():
    # two steps, gradients 0.5 then -0.3 (lr 0.1, b1 0.9, b2 0.999, eps 1e-8),
    # expanded by hand: m1 = 0.05, v1 = 2.5e-4; m2 = 0.9 * 0.05 - 0.1 * 0.3 =
    # 0.015, v2 = 0.999 * 2.5e-4 + 0.001 * 0.09 = 3.3975e-4; bias corrections
    # 1 - 0.9^2 = 0.19 and 1 - 0.999^2 = 0.001999
    w1, m1, v1 = omlp.adam(np.array([1.0]), np.array([0.5]), np.zeros(1), np.zeros(1), 0.1, 0.9, 0.999, 1e-8, 1)
    w2, m2, v2 = omlp.adam(w1, np.array([-0.3]), m1, v1, 0.1, 0.9, 0.999, 1e-8, 2)
    assert np.isclose(m2[0], 0.015, rtol=1e-14) and np.isclose(v2[0], 3.3975e-4, rtol=1e-14)
    step2 = 0.1 * (0.015 / 0.19) / (np.sqrt(3.3975e-4 / 0.001999) + 1e-8)
    assert np.isclose(w2[0], w1[0] - step2, rtol=1e-14, atol=1e-16)
    assert np.isclose(step2, 0.0191498, rtol=1e-5)  # hand value: 0.1 x 0.0789474 / 0.412262


def test_descriptor_onsite_energy_bins_by_hand():
    # three 1-orbital atoms far apart (> 0.5 nm: no radial features); row 0 has
    # neighbours 1 and 2 with onsite energies placed on bin centres 3 and 6 of
    # the eight onsite-energy bins (centres -3 + 6 t / 7, width 0.75):
    # H_11 = -3/7, H_22 = 15/7.  Neighbour couplings H_01 = -0.5, H_02 = 0.2,
    # S_01 = 0.1, S_02 = -0.05.  By hand, with (centre spacing 6/7) / 0.75 = 8/7:
    #   f[48 + t] = 0.25 exp(-(8 (t - 3) / 7)^2) + 0.04 exp(-(8 (t - 6) / 7)^2)
    #   f[57] = 0.1^2 + 0.05^2 = 0.0125      f[58] = -0.05 - 0.01 = -0.06
    #   f[60] = 0.5 + 0.2 = 0.7             f[62] = 0.1 (-3/7) - 0.05 (15/7) = -0.15
    #   f[56] = 0.29                        f[59] = 0.25 (-3/7) + 0.04 (15/7) = -0.15 / 7
    n = 3
    rp = np.array([0, 3, 6, 9], np.int64)
    ci = np.tile(np.arange(3, dtype=np.int32), 3)
    H = np.array([[0.7, -0.5, 0.2], [-0.5, -3.0 / 7.0, 0.3], [0.2, 0.3, 15.0 / 7.0]])
    S = np.array([[1.0, 0.1, -0.05], [0.1, 1.0, 0.02], [-0.05, 0.02, 1.0]])
    pos = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.0, 2.0, 0]])
    system = TBSystem(n, rp, ci, H.ravel(), S.ravel(), np.arange(3, dtype=np.int32), positions=pos,
                      atom_norb=np.ones(3, np.int32))
    d = odesc.descriptors(system, np.ones(3, int))[0]
    t = np.arange(8)
    bins = 0.25 * np.exp(-((8 * (t - 3) / 7) ** 2)) + 0.04 * np.exp(-((8 * (t - 6) / 7) ** 2))
    assert np.allclose(d[48:56], bins, rtol=1e-13, atol=0)
    assert np.argmax(d[48:56]) == 3 and d[54] > 0.04 and d[54] < 0.0401
    assert np.isclose(d[56], 0.29) and np.isclose(d[57], 0.0125) and np.isclose(d[58], -0.06)
    assert np.isclose(d[59], -0.15 / 7) and np.isclose(d[60], 0.7) and np.isclose(d[62], -0.15)
    assert np.isclose(d[46], 0.7) and np.isclose(d[47], 1.0) and np.isclose(d[61], 0.03)
    assert not d[0:40].any()  # every neighbour atom is beyond the 0.5 nm cutoff
