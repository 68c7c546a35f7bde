"""Pins of the oracle's bandwidth rules, POD (Sec. 2.3, Sec. 3.1), the
linearised reduced step (Sec. 2.4, Eq. model_DymReduced) and the batched work
queue, against library routines, textbook identities and algebraic identities
of the method."""
import numpy as np
import pytest
from scipy.spatial.distance import pdist

from paper_2603_12550_gb300 import inputs


# ---------------------------------------------------------------- bandwidth

@pytest.mark.parametrize("N,D", [(57, 9), (64, 2), (101, 6)])
def test_median_pair_distance_is_lower_median(orc, N, D):
    q = np.random.default_rng(N).standard_normal((N, D))
    d = np.sort(pdist(q))
    M = N * (N - 1) // 2
    assert orc.median_pairdist(q) == d[(M - 1) // 2]
    assert orc.median_bandwidth(q) == pytest.approx(d[(M - 1) // 2] / np.sqrt(2 * np.log(N)), rel=1e-15)


@pytest.mark.parametrize("N,D,dup", [(57, 9, False), (64, 2, False), (200, 3, True), (2, 4, False)])
def test_median_by_counting_equals_sorted_median(orc, N, D, dup):
    # the bisection on pair counts must land on the very order statistic that
    # sorting all pair distances (scipy pdist) gives, ties included
    q = np.random.default_rng(N + 11).standard_normal((N, D))
    if dup:
        q[N // 2:] = q[:N - N // 2]
    d = np.sort(pdist(q))
    M = N * (N - 1) // 2
    assert orc.median_pairdist_count(q) == d[(M - 1) // 2]
    assert orc.median_bandwidth_count(q) == orc.median_bandwidth(q)


def test_pair_counts_bracket_the_order_statistic(orc):
    q = np.random.default_rng(5).standard_normal((300, 9))
    med = orc.median_pairdist(q)
    M = 300 * 299 // 2
    # med is sqrt of the selected squared distance; bracket its square by 1 ulp-ish
    lt, _ = orc.count_pairs(q, med * med * (1 - 1e-12))
    _, le = orc.count_pairs(q, med * med * (1 + 1e-12))
    assert lt <= (M - 1) // 2 < le
    q32 = q.astype(np.float32)
    lt32, le32 = orc.count_pairs_f32(q32, np.float32(med * med))
    assert abs(lt32 - lt) <= 2 and abs(le32 - le) <= 2


def test_silverman_reduces_to_textbook_1d(orc):
    # D = 1: h = sigma (4 / (3 N))^(1/5) = 1.0592 sigma N^(-1/5)
    x = np.random.default_rng(3).standard_normal((5000, 1)) * 2.5
    h = orc.silverman_bandwidth(x)
    assert h == pytest.approx(1.0592238410488122 * np.std(x, ddof=1) * 5000 ** -0.2, rel=1e-12)


# ---------------------------------------------------------------------- POD

def _X(n_rows=300, n_cols=40, rank=40, seed=0, decay=0.7, noise=0.0):
    return inputs.snapshot_matrix(n_rows, n_cols, rank, seed=seed, decay=decay, noise=noise).astype(np.float64)


def test_pod_spectrum_matches_svd_and_frobenius(orc):
    X = _X()
    out = orc.pod_build(X, r_fixed=12)
    sv = np.linalg.svd(X, compute_uv=False)
    np.testing.assert_allclose(out["lam"], sv ** 2, rtol=1e-9, atol=1e-9 * sv[0] ** 2)
    assert out["lam"].sum() == pytest.approx(np.sum(X * X), rel=1e-12)
    Phi = out["Phi"]
    np.testing.assert_allclose(Phi.T @ Phi, np.eye(12), atol=1e-12)
    # columns are the leading left singular vectors up to sign
    U, _, _ = np.linalg.svd(X, full_matrices=False)
    np.testing.assert_allclose(np.abs(np.sum(U[:, :12] * Phi, 0)), 1.0, atol=1e-9)


def test_pod_sign_convention(orc):
    out = orc.pod_build(_X(seed=2), r_fixed=6)
    Phi = out["Phi"]
    for t in range(6):
        i = np.argmax(np.abs(Phi[:, t]))
        assert Phi[i, t] > 0


def test_pod_recovers_low_rank_data(orc):
    X = _X(n_rows=240, n_cols=30, rank=5, seed=4)
    out = orc.pod_build(X, energy=1 - 1e-9, r_max=64)
    assert out["r"] == 5
    Phi = out["Phi"]
    # X was rounded to FP32, so it is rank 5 only up to that rounding
    np.testing.assert_allclose(Phi @ (Phi.T @ X), X, atol=1e-6 * np.abs(X).max())
    assert np.all(np.abs(out["lam"][5:]) < 1e-9 * out["lam"][0])


def test_rank_rule(orc):
    lam = np.array([50.0, 30.0, 15.0, 4.0, 0.9, 0.1])
    assert orc.select_rank(lam, 0.5, 64) == 1
    assert orc.select_rank(lam, 0.80, 64) == 2
    assert orc.select_rank(lam, 0.95, 64) == 3
    assert orc.select_rank(lam, 0.99, 64) == 4
    assert orc.select_rank(lam, 0.999, 64) == 5
    assert orc.select_rank(lam, 0.999, 3) == 3


def test_project_lift_identities(orc):
    nb, s, N = 3, 3, 100
    states = [inputs.equilibrium_cloud(N, nb, s, seed=k).astype(np.float64) for k in range(6)]
    X = orc.snapshots_from_states(states, s, nb)
    assert X.shape == (N * s, 6 * nb)
    np.testing.assert_array_equal(X[:, 4], states[1][:, 3:6].reshape(-1))
    Phi = orc.pod_build(X, r_fixed=10)["Phi"]
    P = np.random.default_rng(1).standard_normal((10, nb))
    np.testing.assert_allclose(orc.project(Phi, orc.lift(Phi, P, s, nb), s, nb), P, atol=1e-12)
    q = states[3]
    q1 = orc.lift(Phi, orc.project(Phi, q, s, nb), s, nb)
    q2 = orc.lift(Phi, orc.project(Phi, q1, s, nb), s, nb)
    np.testing.assert_allclose(q2, q1, atol=1e-12)
    # snapshots lie in the span of a full-rank basis
    Phi_all = orc.pod_build(X, r_fixed=6 * nb)["Phi"]
    np.testing.assert_allclose(orc.lift(Phi_all, orc.project(Phi_all, q, s, nb), s, nb), q, atol=1e-9)


def test_xh_special_cases(orc):
    s = 3
    Phi = orc.pod_build(_X(n_rows=90, n_cols=20, seed=7), r_fixed=8)["Phi"]
    np.testing.assert_allclose(orc.x_h(Phi, np.zeros((s, s)), s), 0.0)
    np.testing.assert_allclose(orc.x_h(Phi, np.eye(s), s), np.eye(8), atol=1e-12)
    # X^H = Phi^T (I_N (x) kappa) Phi written as a dense product
    kap = np.random.default_rng(3).standard_normal((s, s))
    G = np.kron(np.eye(30), kap)
    np.testing.assert_allclose(orc.x_h(Phi, kap, s), Phi.T @ G @ Phi, atol=1e-12)


def _reduced_setup(orc, N=60, nb=3, s=3, r=12, seed=0):
    states = [inputs.equilibrium_cloud(N, nb, s, seed=seed + k).astype(np.float64) * (1 + 0.1 * k)
              for k in range(8)]
    X = orc.snapshots_from_states(states, s, nb)
    Phi = orc.pod_build(X, r_fixed=r)["Phi"]
    kap = inputs.shear_kappa(s, 1.0)
    p = orc.params(nb, s, H=[1.0, 1.0, 1.0], kBT=1.0, h=0.8, dt=0.005, kappa=kap)
    P0 = orc.project(Phi, states[0], s, nb)
    return Phi, p, P0, kap


def test_frozen_rhs_equals_galerkin_rhs_at_refresh(orc):
    # Sec. 2.4: the linearisations of the Brownian terms are exact when the
    # state lies in the span of U, so at a refresh instant Eq. model_DymReduced
    # and the Galerkin projection Eq. model_DymRepParPod give the same Pdot.
    Phi, p, P0, kap = _reduced_setup(orc)
    q = orc.lift(Phi, P0, p.s, p.nb)
    B1, B2, _ = orc.x_b(Phi, q, p.h, p.s)
    XH = orc.x_h(Phi, kap, p.s)
    r_ii = orc.reduced_rhs(P0, XH, B1 + B2, p)
    r_i = orc.galerkin_rhs(P0, Phi, p)
    np.testing.assert_allclose(r_ii, r_i, rtol=1e-10, atol=1e-10 * np.abs(r_i).max())


def test_reduced_run_with_refresh_every_step_is_galerkin(orc):
    Phi, p, P0, _ = _reduced_setup(orc, N=40, r=8, seed=3)
    P_ii = orc.reduced_run(P0, Phi, p, 5, refresh_every=1)
    P = P0.copy()
    for _ in range(5):
        P = P + p.dt * orc.galerkin_rhs(P, Phi, p)
    np.testing.assert_allclose(P_ii, P, rtol=1e-10, atol=1e-12)


def test_full_basis_galerkin_is_full_order(orc):
    # With U square orthogonal the reduced model is the full model.
    N, nb, s = 20, 2, 3
    states = [inputs.equilibrium_cloud(N, nb, s, seed=k).astype(np.float64) for k in range(30)]
    X = orc.snapshots_from_states(states, s, nb)
    Phi = orc.pod_build(X, r_fixed=N * s)["Phi"]
    p = orc.params(nb, s, kBT=1.0, h=0.7, dt=0.01, kappa=inputs.shear_kappa(s, 1.0))
    q0 = states[0]
    P = orc.project(Phi, q0, s, nb)
    P = P + p.dt * orc.galerkin_rhs(P, Phi, p)
    np.testing.assert_allclose(orc.lift(Phi, P, s, nb), orc.explicit_steps(q0, p, 1), atol=1e-10)


def test_err_mor(orc):
    a = np.ones((4, 3))
    assert orc.err_mor(a, a) == 0.0
    assert orc.err_mor(1.1 * a, a) == pytest.approx(0.1)


# ------------------------------------------------------------- work queue

def test_work_queue_order(orc):
    sizes = np.array([1000, 3000, 1000, 70, 5000])
    items = orc.work_queue(sizes, 512)
    expect_count = sum((n + 511) // 512 for n in sizes)
    assert len(items) == expect_count
    assert len({tuple(x) for x in items}) == expect_count
    cost = sizes[items[:, 0]]
    assert np.all(np.diff(cost) <= 0)
    # ties: ensemble ascending, tile ascending
    assert items[0].tolist() == [4, 0] and items[9].tolist() == [4, 9]
    same = items[cost == 1000]
    assert same[:2].tolist() == [[0, 0], [0, 1]] and same[2:].tolist() == [[2, 0], [2, 1]]
