"""Pins of the oracle's density, entropy gradient and energy (Sec. 2.2,
Eq. model_DeteParAppr, Eq. model_DymRepPar) against quantities other than
themselves: a library Gaussian pdf, closed forms at N=1 and N=2, invariants,
and central finite differences of the energy."""
import numpy as np
import pytest
from scipy.stats import multivariate_normal

from paper_2603_12550_gb300 import inputs


def _cloud(N, nb, s, seed):
    return inputs.equilibrium_cloud(N, nb, s, seed=seed).astype(np.float64)


@pytest.mark.parametrize("N,nb,s,h", [(40, 1, 2, 0.3), (33, 3, 3, 0.9), (17, 2, 3, 0.5)])
def test_density_matches_library_gaussian_kde(orc, N, nb, s, h):
    # f_h(q_I) = (1/N) sum_J N(q_I; q_J, h^2 I) = (2 pi h^2)^{-D/2} rho_I / N.
    q = _cloud(N, nb, s, seed=N)
    D = nb * s
    f = np.zeros(N)
    for J in range(N):
        f += multivariate_normal(mean=q[J], cov=h * h * np.eye(D)).pdf(q)
    f /= N
    rho = orc.density(q, h)
    np.testing.assert_allclose(rho, f * N * (2 * np.pi * h * h) ** (D / 2), rtol=1e-12)
    assert np.all(rho >= 1.0) and np.all(rho <= N)


def test_single_particle(orc):
    q = np.array([[0.3, -1.2, 0.7]])
    assert orc.density(q, 0.5)[0] == 1.0
    assert np.all(orc.entropy_grad(q, 0.5) == 0.0)


def test_two_particles_closed_form(orc):
    # rho_1 = rho_2 = 1 + k;  S_1 = -(2/h^2) k (q_1 - q_2) / (1 + k).
    rng = np.random.default_rng(3)
    q = rng.standard_normal((2, 5))
    h = 0.7
    k = np.exp(-np.sum((q[0] - q[1]) ** 2) / (2 * h * h))
    S = orc.entropy_grad(q, h)
    np.testing.assert_allclose(S[0], -(2 / h ** 2) * k * (q[0] - q[1]) / (1 + k), rtol=1e-13)
    np.testing.assert_allclose(S[1], -S[0], rtol=1e-13)


@pytest.mark.parametrize("nb,s", [(1, 2), (3, 3)])
def test_entropy_gradient_invariants(orc, nb, s):
    N, h = 50, 0.6
    q = _cloud(N, nb, s, seed=11)
    D = nb * s
    S = orc.entropy_grad(q, h)
    scale = np.abs(S).max()
    # antisymmetric kernel gradient times a symmetric weight sums to zero
    assert np.abs(S.sum(0)).max() < 1e-12 * scale * N
    # translation invariance
    c = np.random.default_rng(1).standard_normal(D)
    np.testing.assert_allclose(orc.entropy_grad(q + c, h), S, atol=1e-12 * scale)
    # rotation equivariance S(q R^T) = S(q) R^T
    R, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((D, D)))
    np.testing.assert_allclose(orc.entropy_grad(q @ R.T, h), S @ R.T, atol=1e-12 * scale)
    # permutation equivariance
    perm = np.random.default_rng(4).permutation(N)
    np.testing.assert_allclose(orc.entropy_grad(q[perm], h), S[perm], atol=1e-13 * scale)


@pytest.mark.parametrize("spring,kBT", [(0, 1.0), (1, 1.0), (0, 0.7)])
def test_gradient_is_scaled_energy_derivative(orc, spring, kBT):
    # g_I = N dE/dq_I, checked by central differences of the energy alone.
    N, nb, s = 24, 3, 3
    q = _cloud(N, nb, s, seed=5)
    if spring == 1:
        q *= 0.5
    p = orc.params(nb, s, H=[1.0, 2.0, 1.5], kBT=kBT, h=0.8, spring=spring, b=20.0)
    E, g, _ = orc.energy_grad(q, p)
    eps = 1e-6
    rng = np.random.default_rng(9)
    for _ in range(12):
        I, c = rng.integers(N), rng.integers(nb * s)
        qp, qm = q.copy(), q.copy()
        qp[I, c] += eps
        qm[I, c] -= eps
        fd = N * (orc.energy(qp, p) - orc.energy(qm, p)) / (2 * eps)
        assert abs(fd - g[I, c]) <= 1e-6 * max(1.0, abs(g[I, c]))


def test_energy_normalisation(orc):
    # E at kBT=1 with no spring: mean of ln f_h, f_h from the library pdf.
    N, h = 20, 0.4
    q = _cloud(N, 1, 3, seed=8)
    p = orc.params(1, 3, H=[0.0], kBT=1.0, h=h)
    f = np.zeros(N)
    for J in range(N):
        f += multivariate_normal(mean=q[J], cov=h * h * np.eye(3)).pdf(q)
    f /= N
    assert abs(orc.energy(q, p) - np.mean(np.log(f))) < 1e-12


def test_fene_domain(orc):
    q = np.array([[3.0, 0.0, 0.0], [0.1, 0.2, 0.3]])
    p = orc.params(1, 3, spring=1, b=4.0, h=0.5)
    with pytest.raises(orc.OracleError) as ei:
        orc.energy_grad(q, p)
    assert ei.value.code == orc.OR_EDOMAIN
    # inside the domain, FENE gradient = H q / (1 - |q|^2/b)
    q = np.array([[1.0, 0.5, 0.0]])
    p = orc.params(1, 3, spring=1, b=4.0, h=0.5, H=[2.0], kBT=0.0)
    _, g, _ = orc.energy_grad(q, p)
    np.testing.assert_allclose(g[0], 2.0 * q[0] / (1 - 1.25 / 4.0), rtol=1e-14)


def test_density_rows_are_the_density(orc):
    q = inputs.equilibrium_cloud(300, 3, 3, seed=4).astype(np.float64)
    rows = np.array([0, 7, 299, 150])
    np.testing.assert_array_equal(orc.density_rows(q, 0.8, rows), orc.density(q, 0.8)[rows])


@pytest.mark.parametrize("N,nb,s,h,M", [(30, 1, 2, 0.4, 13), (21, 3, 3, 0.8, 7)])
def test_density_at_matches_library_gaussian_mixture(orc, N, nb, s, h, M):
    # f(y) = (1/N) sum_I N(y; q_I, h^2 I): the library pdf at arbitrary points
    q = _cloud(N, nb, s, seed=N + 1)
    D = nb * s
    y = np.random.default_rng(M).standard_normal((M, D)) * 1.5
    f = np.zeros(M)
    for I in range(N):
        f += multivariate_normal(mean=q[I], cov=h * h * np.eye(D)).pdf(y)
    np.testing.assert_allclose(orc.density_at(q, h, y), f / N, rtol=1e-12)


def test_density_at_the_particles_is_the_pair_density(orc):
    # at the particles themselves the estimate is rho_I (1/N)(2 pi h^2)^{-D/2},
    # rho from the C oracle's pair sum
    q = _cloud(64, 3, 3, seed=5)
    h = 0.7
    f = orc.density_at(q, h, q)
    np.testing.assert_allclose(f, orc.density(q, h) / 64 * (2 * np.pi * h * h) ** (-4.5), rtol=1e-13)


def test_density_at_integrates_to_one():
    # a probability density: its integral over the plane is 1 (2D cloud,
    # midpoint rule on a grid covering the support)
    import oracle
    q = _cloud(25, 1, 2, seed=8)
    h = 0.5
    g = np.linspace(-8, 8, 321)
    dx = g[1] - g[0]
    X, Y = np.meshgrid(g, g, indexing="ij")
    f = oracle.density_at(q, h, np.stack([X.ravel(), Y.ravel()], axis=1), chunk=4096)
    assert abs(f.sum() * dx * dx - 1.0) < 1e-9


def test_grid_points_and_density_error():
    import oracle
    G = oracle.grid_points(2)
    assert G.shape == (9, 2)
    assert np.array_equal(G[1], [-2.0, 0.0]) and np.array_equal(G[-1], [2.0, 2.0])
    assert oracle.grid_points(9).shape == (3 ** 9, 9)
    e2, einf = oracle.density_error([1.0, 2.0, 2.0], [1.0, 2.0, 4.0])
    assert np.isclose(e2, 2.0 / np.sqrt(21.0)) and np.isclose(einf, 0.5)


@pytest.mark.parametrize("spring", [0, 1])
def test_sampled_rows_agree_with_the_full_gradient(orc, spring):
    # The full-size GPU tests compare sampled rows with entropy_grad_rows +
    # spring_grad; both must give exactly the rows of the full g = kBT S +
    # grad Psi at kBT = 1, whose derivative property is pinned above.
    N, nb, s = 300, 3, 3
    q = _cloud(N, nb, s, seed=12)
    if spring == 1:
        q *= 0.5
    p = orc.params(nb, s, H=[1.0, 2.0, 1.5], kBT=1.0, h=0.7, spring=spring, b=20.0)
    _, g, rho = orc.energy_grad(q, p)
    rows = np.array([0, 7, 150, N - 1])
    g_rows = orc.entropy_grad_rows(q, 0.7, rho, rows) + orc.spring_grad(q[rows], p)
    np.testing.assert_allclose(g_rows, g[rows], rtol=1e-12, atol=1e-12 * np.max(np.abs(g)))
