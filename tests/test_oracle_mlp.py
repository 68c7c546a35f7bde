"""Pins of the FP64 oracle of the score surrogate (oracle/mlp.py) against
things other than itself: central finite differences, a zero-weight closed
form, the Gaussian minimiser of the denoising score-matching loss, the Adam
closed form of the first step, and training to the Gaussian score."""
import numpy as np
import pytest

from oracle import mlp
from paper_2603_12550_gb300 import inputs


def test_silu_and_derivative():
    z = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(mlp.silu(z), z * (1 / (1 + np.exp(-z))), rtol=1e-15)
    fd = (mlp.silu(z + 1e-6) - mlp.silu(z - 1e-6)) / 2e-6
    np.testing.assert_allclose(mlp.silu_grad(z), fd, rtol=1e-7, atol=1e-9)


def test_backprop_matches_finite_differences():
    layers = mlp.as64(inputs.mlp_init((9, 16, 16, 16, 9), seed=3))
    rng = np.random.default_rng(1)
    layers = [(W, rng.standard_normal(b.shape) * 0.1) for W, b in layers]
    x = rng.standard_normal((32, 9))
    eps = rng.standard_normal((32, 9))
    sigma = 0.7
    _, grads = mlp.dsm_grad(layers, x, eps, sigma)
    for l in range(4):
        for which in (0, 1):
            P = layers[l][which]
            for _ in range(3):
                idx = tuple(rng.integers(0, n) for n in P.shape)
                up = [(W.copy(), b.copy()) for W, b in layers]
                dn = [(W.copy(), b.copy()) for W, b in layers]
                up[l][which][idx] += 1e-6
                dn[l][which][idx] -= 1e-6
                fd = (mlp.dsm_loss(up, x, eps, sigma) - mlp.dsm_loss(dn, x, eps, sigma)) / 2e-6
                g = grads[l][which][idx]
                assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (l, which, idx, fd, g)


def test_zero_weights_closed_form():
    # all weights and hidden biases zero: s = b4 for every input,
    # L = mean |b4 + eps/sigma|^2, dL/db4 = 2 mean(b4 + eps/sigma), all else 0.
    layers = [(np.zeros((8, 9)), np.zeros(8)), (np.zeros((8, 8)), np.zeros(8)),
              (np.zeros((9, 8)), np.array([0.3, -0.2, 0.1, 0, 0.5, 0, 0, -1, 2.0]))]
    rng = np.random.default_rng(2)
    x, eps, sigma = rng.standard_normal((50, 9)), rng.standard_normal((50, 9)), 0.5
    loss, grads = mlp.dsm_grad(layers, x, eps, sigma)
    b4 = layers[-1][1]
    assert loss == pytest.approx(np.mean(np.sum((b4 + eps / sigma) ** 2, axis=1)), rel=1e-14)
    np.testing.assert_allclose(grads[-1][1], 2 * np.mean(b4 + eps / sigma, axis=0), rtol=1e-13)
    for l in range(2):
        assert np.all(grads[l][0] == 0) and np.all(grads[l][1] == 0)
    assert np.all(grads[-1][0] == 0)


def test_dsm_loss_is_minimised_by_smoothed_gaussian_score():
    # data N(0, s0^2 I): the DSM minimiser among s = a x is a = -1/(s0^2 + sigma^2)
    rng = np.random.default_rng(4)
    s0, sigma = 1.3, 0.6
    x = rng.standard_normal((200000, 9)) * s0
    eps = rng.standard_normal(x.shape)
    a_star = -1 / (s0 ** 2 + sigma ** 2)
    la = [mlp.dsm_loss_of_score(lambda z, a=a: a * z, x, eps, sigma)
          for a in (a_star * 0.9, a_star, a_star * 1.1)]
    assert la[1] < la[0] and la[1] < la[2]


def test_adam_first_step_closed_form():
    layers = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    grads = [(np.array([[0.3, -0.04]]), np.array([2.0]))]
    m, v = mlp.adam_init(layers)
    out, _, _ = mlp.adam_step(layers, grads, m, v, 1, lr=0.1, eps=1e-8)
    # first step: m_hat = g, v_hat = g^2 -> p - lr g / (|g| + eps)
    np.testing.assert_allclose(out[0][0], layers[0][0] - 0.1 * grads[0][0] / (np.abs(grads[0][0]) + 1e-8))
    np.testing.assert_allclose(out[0][1], layers[0][1] - 0.1 * grads[0][1] / (np.abs(grads[0][1]) + 1e-8))


def test_training_reaches_gaussian_score():
    # a small network trained by the oracle's DSM + Adam learns
    # s(x) = -x / (s0^2 + sigma^2) on Gaussian data
    s0, sigma = 1.0, 0.5
    rng = np.random.default_rng(5)
    data = (rng.standard_normal((20000, 3)) * s0).astype(np.float32)
    layers = mlp.as64(inputs.mlp_init((3, 32, 32, 3), seed=0))
    m, v = mlp.adam_init(layers)
    for t in range(1, 1201):
        x, eps = inputs.dsm_batch(data, 256, seed=t)
        _, g = mlp.dsm_grad(layers, x, eps, sigma)
        layers, m, v = mlp.adam_step(layers, g, m, v, t, lr=3e-3)
    z = rng.standard_normal((500, 3)) * 0.8
    s, _ = mlp.forward(layers, z)
    target = -z / (s0 ** 2 + sigma ** 2)
    assert np.linalg.norm(s - target) / np.linalg.norm(target) < 0.15


def test_fit_gradient_matches_finite_differences():
    layers = mlp.as64(inputs.mlp_init((4, 8, 8, 4), seed=2))
    rng = np.random.default_rng(3)
    x, t = rng.standard_normal((20, 4)), rng.standard_normal((20, 4))
    loss, grads = mlp.fit_grad(layers, x, t)
    s, _ = mlp.forward(layers, x)
    assert loss == pytest.approx(np.mean(np.sum((s - t) ** 2, axis=1)), rel=1e-14)
    for l in range(3):
        idx = (1, 2)
        up = [(W.copy(), b.copy()) for W, b in layers]
        dn = [(W.copy(), b.copy()) for W, b in layers]
        up[l][0][idx] += 1e-6
        dn[l][0][idx] -= 1e-6
        fd = (mlp.fit_grad(up, x, t)[0] - mlp.fit_grad(dn, x, t)[0]) / 2e-6
        assert abs(fd - grads[l][0][idx]) <= 1e-6 * max(1.0, abs(fd))


# ------------------------------------------------ score_rhs (mode iii RHS)
# Pins of the oracle's reduced right-hand side with the learned score in
# place of the entropy gradient, each against the Galerkin RHS (mode i),
# whose parts are pinned separately (closed forms of the spring and flow
# terms, the linear kBT = 0 steps):
#   * kBT = 0: the score drops out, so the two RHS agree for any network;
#   * a constant network (zero weights, nonzero output bias) has mean-centred
#     score exactly zero, so at kBT = 1 it agrees with the kBT = 0 Galerkin RHS;
#   * a network realising s(x) = -x + c on a zero-mean lifted cloud makes the
#     entropic term kBT s = -(q~) (after centring), which is the force of a
#     Hookean spring of stiffness -kBT: at kBT = 1 with no springs it agrees
#     with the kBT = 0 Galerkin RHS with H = -1.  A sign error on the kBT
#     term, a transposed Rouse coupling or a dropped centring fails one of them.

def _zero_mean_basis(N, s, r, seed):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((N, s, r))
    Y -= Y.mean(axis=0, keepdims=True)
    Q, _ = np.linalg.qr(Y.reshape(N * s, r))
    return Q


def _affine_net(D, a, c, B=40.0):
    # SiLU(z) = z sigma(z) equals z to within |z| e^{-z} for large z, so three
    # SiLU layers fed x + B pass it through; the last layer maps to a x + c
    I = np.eye(D)
    return [(I.copy(), np.full(D, B)), (I.copy(), np.zeros(D)), (I.copy(), np.zeros(D)),
            (a * I, c - a * B * np.ones(D))]


@pytest.mark.parametrize("nb,s", [(1, 2), (3, 3)])
def test_score_rhs_without_temperature_is_galerkin(orc, nb, s):
    N, r = 300, 5
    Phi = _zero_mean_basis(N, s, r, seed=nb)
    Phi[:, 0] += 0.05  # a nonzero-mean cloud: the score must not matter at kBT = 0
    Phi, _ = np.linalg.qr(Phi)
    P = np.random.default_rng(4).standard_normal((r, nb)) * 3.0
    kap = inputs.shear_kappa(s, 1.3)
    p = orc.params(nb, s, H=[1.0 + k for k in range(nb)], kBT=0.0, zeta=4.0, h=0.5, kappa=kap)
    layers = mlp.as64(inputs.mlp_init((nb * s, 32, 32, 32, nb * s), seed=2))
    np.testing.assert_allclose(orc.score_rhs(P, Phi, p, layers), orc.galerkin_rhs(P, Phi, p),
                               rtol=1e-12, atol=1e-12)


def test_score_rhs_of_a_constant_network_drops_the_entropy(orc):
    nb, s, N, r = 3, 3, 400, 6
    Phi, _ = np.linalg.qr(np.random.default_rng(8).standard_normal((N * s, r)))
    P = np.random.default_rng(9).standard_normal((r, nb)) * 4.0
    kap = inputs.shear_kappa(s, 1.0)
    layers = [(np.zeros((16, 9)), np.zeros(16)), (np.zeros((16, 16)), np.zeros(16)),
              (np.zeros((16, 16)), np.zeros(16)),
              (np.zeros((9, 16)), np.linspace(-2.0, 3.0, 9))]
    p1 = orc.params(nb, s, H=1.0, kBT=1.0, zeta=4.0, h=0.5, kappa=kap)
    p0 = orc.params(nb, s, H=1.0, kBT=0.0, zeta=4.0, h=0.5, kappa=kap)
    np.testing.assert_allclose(orc.score_rhs(P, Phi, p1, layers), orc.galerkin_rhs(P, Phi, p0),
                               rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("nb,s,kBT", [(1, 3, 1.0), (3, 3, 1.0), (3, 3, 2.5)])
def test_score_rhs_of_a_linear_score_is_a_negative_spring(orc, nb, s, kBT):
    N, r, D = 500, 7, nb * s
    Phi = _zero_mean_basis(N, s, r, seed=10 + nb)
    P = np.random.default_rng(11).standard_normal((r, nb)) * 5.0
    kap = inputs.shear_kappa(s, 0.7)
    # s(x) = -x / kBT + c  =>  kBT (s - mean s) = -(q~ - mean q~) = -q~
    layers = _affine_net(D, -1.0 / kBT, np.linspace(0.5, 1.5, D))
    p_score = orc.params(nb, s, H=0.0, kBT=kBT, zeta=4.0, h=0.5, kappa=kap)
    p_spring = orc.params(nb, s, H=-1.0, kBT=0.0, zeta=4.0, h=0.5, kappa=kap)
    got = orc.score_rhs(P, Phi, p_score, layers)
    want = orc.galerkin_rhs(P, Phi, p_spring)
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-10 * np.abs(want).max())
    # and the entropic part pushes outwards: with kBT > 0 the reduced state
    # grows faster than without the score (the score of a centred cloud
    # points inwards, the entropy force against it)
    p_flow = orc.params(nb, s, H=0.0, kBT=0.0, zeta=4.0, h=0.5, kappa=kap)
    assert np.sum(P * (got - orc.galerkin_rhs(P, Phi, p_flow))) > 0
