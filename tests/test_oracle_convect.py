"""Pins of the oracle's convection step (the u . grad_x term of Eq.
model_DymRepPar and Eq. model_DymReduced, first-order upwind on a grid of
nodes) against properties that fix the scheme, not its formula:
  * no flow leaves the field unchanged;
  * at Courant number 1 along one axis the periodic upwind step is an exact
    shift by one node, downstream for either sign of u;
  * with uniform u and periodic nodes the sum over the grid is conserved;
  * a constant field stays constant under zero-gradient boundaries and any u;
  * a smooth periodic profile is carried at speed u with first-order error:
    halving dx (at fixed Courant number) halves the error;
  * the three axes are the same scheme: a field varying along y (or z)
    transported along y (or z) equals the x case transposed.
"""
import numpy as np
import pytest


def _rand(G, M, seed):
    return np.random.default_rng(seed).standard_normal((G, M))


def test_no_flow_is_identity(orc):
    Q = _rand(4 * 3 * 2, 7, 0)
    out = orc.convect_upwind(Q, np.zeros((24, 3)), (4, 3, 2), (0.1, 0.2, 0.3), 0.05)
    np.testing.assert_array_equal(out, Q)


@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_unit_courant_is_a_shift(orc, sign, axis):
    shape = (5, 4, 3)
    G = 60
    dx = (0.5, 0.25, 2.0)
    u = np.zeros((G, 3))
    u[:, axis] = sign * 2.0
    dt = dx[axis] / 2.0  # Courant number 1
    Q = _rand(G, 6, axis)
    out = orc.convect_upwind(Q, u, shape, dx, dt)
    F = Q.reshape(3, 4, 5, 6)
    want = np.roll(F, int(sign), axis=2 - axis).reshape(G, 6)
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-14)


def test_periodic_uniform_flow_conserves_the_sum(orc):
    shape, G = (6, 5, 4), 120
    u = np.tile([0.7, -0.4, 0.3], (G, 1))
    Q = _rand(G, 11, 3)
    out = orc.convect_upwind(Q, u, shape, (0.3, 0.2, 0.5), 0.05)
    np.testing.assert_allclose(out.sum(axis=0), Q.sum(axis=0), rtol=1e-12, atol=1e-12)
    assert np.abs(out - Q).max() > 1e-3


def test_constant_field_under_zero_gradient(orc):
    shape, G = (4, 4, 3), 48
    u = np.random.default_rng(1).uniform(-1, 1, (G, 3))
    Q = np.full((G, 5), 2.5)
    out = orc.convect_upwind(Q, u, shape, (0.3, 0.3, 0.3), 0.1, bc=1)
    np.testing.assert_allclose(out, Q, rtol=0, atol=1e-14)


def test_smooth_profile_first_order(orc):
    errs = []
    for n in (64, 128, 256):
        dx = 1.0 / n
        x = (np.arange(n) + 0.5) * dx
        Q = np.sin(2 * np.pi * x)[:, None]
        u = np.tile([1.0, 0.0, 0.0], (n, 1))
        dt = 0.5 * dx
        T = 0.25
        for _ in range(int(round(T / dt))):
            Q = orc.convect_upwind(Q, u, (n, 1, 1), (dx, 1.0, 1.0), dt)
        exact = np.sin(2 * np.pi * (x - T))
        errs.append(np.sqrt(np.mean((Q[:, 0] - exact) ** 2)))
    for a, b in zip(errs, errs[1:]):
        assert 0.4 < b / a < 0.6, errs


def test_axes_are_the_same_scheme(orc):
    rng = np.random.default_rng(5)
    n, M = 7, 4
    prof = rng.standard_normal((n, M))
    ux = np.tile([0.8, 0.0, 0.0], (n, 1))
    ref = orc.convect_upwind(prof, ux, (n, 1, 1), (0.2, 1.0, 1.0), 0.1)
    for axis, shape in ((1, (1, n, 1)), (2, (1, 1, n))):
        u = np.zeros((n, 3))
        u[:, axis] = 0.8
        dx = [1.0, 1.0, 1.0]
        dx[axis] = 0.2
        np.testing.assert_allclose(orc.convect_upwind(prof, u, shape, dx, 0.1), ref, rtol=1e-15, atol=1e-15)
