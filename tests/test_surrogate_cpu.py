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
