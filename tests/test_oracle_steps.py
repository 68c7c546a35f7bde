"""Pins of the oracle's time stepping and stress (Eq. model_DymRepPar,
Appendix A explicit/implicit schemes, polymer stress of Sec. 2.1) against
linear special cases solved by numpy, the implicit equation itself, energy
monotonicity, closed-form stresses and Oldroyd-B moments."""
import numpy as np
import pytest

from paper_2603_12550_gb300 import inputs


def _linear_operator(nb, s, H, kappa, zeta):
    # kBT = 0, Hookean: v_k = kappa q_k - (1/zeta) sum_j A_kj H_j q_j
    A = 2 * np.eye(nb) - np.eye(nb, k=1) - np.eye(nb, k=-1)
    return np.kron(np.eye(nb), kappa) - np.kron(A @ np.diag(H), np.eye(s)) / zeta


def test_rouse_matrices(orc):
    for nb in (1, 2, 3, 5):
        A = orc.rouse(nb)
        np.testing.assert_array_equal(A, 2 * np.eye(nb) - np.eye(nb, k=1) - np.eye(nb, k=-1))
        np.testing.assert_allclose(orc.rouse_inv(nb) @ A, np.eye(nb), atol=1e-14)


def test_explicit_linear_limit_is_matrix_power(orc):
    nb, s, N = 3, 3, 16
    H = np.array([1.0, 2.0, 3.0])
    kap = inputs.shear_kappa(s, 1.0)
    q0 = inputs.equilibrium_cloud(N, nb, s, seed=2).astype(np.float64)
    p = orc.params(nb, s, H=H, kBT=0.0, h=0.5, dt=0.01, kappa=kap)
    q = orc.explicit_steps(q0, p, 25)
    M = np.linalg.matrix_power(np.eye(nb * s) + 0.01 * _linear_operator(nb, s, H, kap, 4.0), 25)
    np.testing.assert_allclose(q, q0 @ M.T, rtol=1e-12, atol=1e-13)


def test_implicit_linear_limit_is_linear_solve(orc):
    nb, s, N = 2, 3, 10
    H = np.array([1.0, 1.5])
    kap = inputs.shear_kappa(s, 2.0)
    q0 = inputs.equilibrium_cloud(N, nb, s, seed=3).astype(np.float64)
    p = orc.params(nb, s, H=H, kBT=0.0, h=0.5, dt=0.02, kappa=kap, tol=1e-13)
    q1, it, _ = orc.implicit_steps(q0, p, 1)
    A = 2 * np.eye(nb) - np.eye(nb, k=1) - np.eye(nb, k=-1)
    lhs = np.eye(nb * s) + 0.02 / 4.0 * np.kron(A @ np.diag(H), np.eye(s))
    rhs = q0 @ (np.eye(nb * s) + 0.02 * np.kron(np.eye(nb), kap)).T
    np.testing.assert_allclose(q1, np.linalg.solve(lhs, rhs.T).T, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("nb,s,spring", [(1, 2, 0), (3, 3, 0), (3, 3, 1)])
def test_implicit_step_solves_the_implicit_equation(orc, nb, s, spring):
    N = 48
    # FENE: keep every bond well inside |q|^2 < b so the step is not stiff
    q0 = inputs.equilibrium_cloud(N, nb, s, seed=4, fene_b=5.0 if spring else None).astype(np.float64)
    kap = inputs.shear_kappa(s, 1.0)
    dt, zeta = 0.01, 4.0
    p = orc.params(nb, s, H=1.0, kBT=1.0, h=0.6, dt=dt, kappa=kap, spring=spring, b=10.0, tol=1e-12)
    q1, it, _ = orc.implicit_steps(q0, p, 1)
    # residual of q+ = q + dt kappa q - (dt/zeta)(A (x) I) g(q+)
    _, g, _ = orc.energy_grad(q1, p)
    A = orc.rouse(nb)
    qs = q0 + dt * np.einsum("ab,Ikb->Ika", kap, q0.reshape(N, nb, s)).reshape(N, -1)
    res = q1 - qs + (dt / zeta) * np.einsum("kj,Ija->Ika", A, g.reshape(N, nb, s)).reshape(N, -1)
    assert np.abs(res).max() < 1e-9
    assert 1 <= it[0] < 50


def test_energy_decreases_without_flow(orc):
    nb, s, N = 3, 3, 40
    q = inputs.equilibrium_cloud(N, nb, s, seed=6).astype(np.float64) * 1.5
    p = orc.params(nb, s, kBT=1.0, h=0.7, dt=0.02, tol=1e-11)
    E = [orc.energy(q, p)]
    for _ in range(4):
        q, _, _ = orc.implicit_steps(q, p, 1)
        E.append(orc.energy(q, p))
    assert all(b <= a + 1e-14 for a, b in zip(E, E[1:]))
    pe = orc.params(nb, s, kBT=1.0, h=0.7, dt=1e-3)
    qe = inputs.equilibrium_cloud(N, nb, s, seed=6).astype(np.float64) * 1.5
    Ee = [orc.energy(qe, pe)]
    for _ in range(4):
        qe = orc.explicit_steps(qe, pe, 1)
        Ee.append(orc.energy(qe, pe))
    assert all(b < a for a, b in zip(Ee, Ee[1:]))


def test_explicit_and_implicit_agree_to_first_order(orc):
    nb, s, N = 2, 3, 30
    q0 = inputs.equilibrium_cloud(N, nb, s, seed=7).astype(np.float64)
    kap = inputs.shear_kappa(s, 1.0)
    diffs = []
    for dt in (4e-3, 2e-3, 1e-3):
        p = orc.params(nb, s, kBT=1.0, h=0.6, dt=dt, kappa=kap, tol=1e-13)
        qe = orc.explicit_steps(q0, p, 1)
        qi, _, _ = orc.implicit_steps(q0, p, 1)
        diffs.append(np.abs(qe - qi).max())
    # one-step difference is O(dt^2)
    assert 3.0 < diffs[0] / diffs[1] < 5.0 and 3.0 < diffs[1] / diffs[2] < 5.0


def test_stress_closed_forms(orc):
    nb, s, N = 3, 3, 200
    H = np.array([1.0, 2.0, 3.0])
    q = inputs.equilibrium_cloud(N, nb, s, H=H, seed=9).astype(np.float64)
    p = orc.params(nb, s, H=H, h=0.5)
    tau, qq = orc.stress(q, p)
    # Hookean: tau_ab = sum_k H_k <q_ka q_kb>
    expect = sum(H[k] * qq[s * k:s * k + s, s * k:s * k + s] for k in range(nb))
    np.testing.assert_allclose(tau, expect, rtol=1e-13)
    np.testing.assert_allclose(qq, q.T @ q / N, rtol=1e-13)
    # FENE stress uses H q / (1 - |q|^2/b)
    pf = orc.params(nb, s, H=H, h=0.5, spring=1, b=50.0)
    tf, _ = orc.stress(q, pf)
    qb = q.reshape(N, nb, s)
    fac = H[None, :] / (1 - (qb ** 2).sum(-1) / 50.0)
    np.testing.assert_allclose(tf, np.einsum("Ika,Ik,Ikb->ab", qb, fac, qb) / N, rtol=1e-13)


def test_equilibrium_stress_statistics(orc):
    # tau = n (N-1) kBT Id at equilibrium (Eq. experiments_equilibriumStress)
    nb, s, N = 3, 3, 20000
    q = inputs.equilibrium_cloud(N, nb, s, seed=10).astype(np.float64)
    p = orc.params(nb, s, h=0.5)
    tau, _ = orc.stress(q, p)
    # each diagonal entry: sum of nb chi^2 means; std ~ sqrt(2 nb / N)
    np.testing.assert_allclose(np.diag(tau), nb * np.ones(s), atol=5 * np.sqrt(2 * nb / N))
    np.testing.assert_allclose(orc.kramers(tau, p), tau - nb * np.eye(s))


def _golden():
    import json, os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")) as f:
        return json.load(f)


def test_equilibrium_stress_underestimate_matches_paper(orc):
    # Sec. 3.2: a 2-bead cloud at thermal equilibrium, P = 1000, median-rule h,
    # relaxes to a diagonal stress about 8 % below n (N-1) kBT.
    gold = _golden()["equilibrium_stress_underestimate_2bead_P1000"]
    N = 1000
    q = inputs.equilibrium_cloud(N, 1, 3, seed=12).astype(np.float64)
    p = orc.params(1, 3, h=orc.median_bandwidth(q), dt=0.01)
    q = orc.explicit_steps(q, p, 300)
    tau, _ = orc.stress(q, p)
    under = 1.0 - np.mean(np.diag(tau))
    assert abs(under - gold["value"]) < gold["abs_tol"], under


def test_dumbbell_shear_moments_near_oldroyd_b(orc):
    # Exact Fokker-Planck dumbbell steady state (lambda = zeta / 4H):
    # <q1q1> = kBT/H (1 + 2 (lambda g)^2), <q1q2> = kBT/H lambda g,
    # <q2q2> = <q3q3> = kBT/H.  VDS replaces f by its kernel smoothing and so
    # undershoots by the same ~10 % as at equilibrium: the check is loose.
    N, gdot = 1000, 1.0
    q = inputs.equilibrium_cloud(N, 1, 3, seed=12).astype(np.float64)
    p = orc.params(1, 3, h=orc.median_bandwidth(q), dt=0.02, kappa=inputs.shear_kappa(3, gdot))
    q = orc.explicit_steps(q, p, 300)
    _, qq = orc.stress(q, p)
    lam = 4.0 / 4.0
    exact = np.array([[1 + 2 * (lam * gdot) ** 2, lam * gdot, 0], [lam * gdot, 1, 0], [0, 0, 1]])
    assert np.all(np.abs(qq - exact) <= 0.2 * np.abs(exact) + 0.01), qq
    assert np.all(qq[[0, 0, 1, 2], [0, 1, 1, 2]] < exact[[0, 0, 1, 2], [0, 1, 1, 2]])


def test_dumbbell_moment_equation_reaches_oldroyd_b():
    # the steady state of the exact moment equation is the Oldroyd-B closed
    # form (lambda = zeta / 4H = 1), and at t = 0 it is the equilibrium start
    from closed_forms import dumbbell_cov_exact
    for rate in (0.1, 1.0, 10.0):
        C = dumbbell_cov_exact(rate, 200.0)
        ex = np.array([[1 + 2 * rate ** 2, rate, 0], [rate, 1, 0], [0, 0, 1]])
        np.testing.assert_allclose(C, ex, rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(dumbbell_cov_exact(rate, 0.0), np.eye(3), atol=1e-15)


# ------------------------------------------------ row-restricted explicit step
# explicit_step_rows (the per-rank piece of a row-sharded step) pinned to the
# whole-cloud step: the same particles' update for any row subset, the linear
# (kBT = 0) limit as one factor of the matrix power, and rows from ranks
# stacked in order equal to the whole step.

@pytest.mark.parametrize("spring", [0, 1])
def test_explicit_step_rows_equals_the_whole_step(orc, spring):
    nb, s, N = 3, 3, 257
    b = 50.0 if spring else 0.0
    q = inputs.equilibrium_cloud(N, nb, s, seed=9, fene_b=b if spring else None).astype(np.float64)
    p = orc.params(nb, s, H=[1.0, 2.0, 1.5], h=0.8, dt=0.004, kappa=inputs.shear_kappa(s, 1.3),
                   spring=spring, b=b)
    whole = orc.explicit_steps(q, p, 1)
    rho = orc.density(q, p.h)
    parts = [orc.explicit_step_rows(q, p, rho, np.arange(a, min(N, a + 100))) for a in range(0, N, 100)]
    np.testing.assert_allclose(np.concatenate(parts), whole, rtol=1e-13, atol=1e-14)
    rows = np.array([5, 0, 256, 77])
    np.testing.assert_allclose(orc.explicit_step_rows(q, p, rho, rows), whole[rows], rtol=1e-13, atol=1e-14)


def test_explicit_step_rows_linear_limit(orc):
    nb, s, N = 3, 3, 40
    H = np.array([1.0, 2.0, 3.0])
    kap = inputs.shear_kappa(s, 1.0)
    q0 = inputs.equilibrium_cloud(N, nb, s, seed=4).astype(np.float64)
    p = orc.params(nb, s, H=H, kBT=0.0, h=0.5, dt=0.01, kappa=kap)
    M = np.eye(nb * s) + 0.01 * _linear_operator(nb, s, H, kap, 4.0)
    rows = np.arange(3, 29)
    np.testing.assert_allclose(orc.explicit_step_rows(q0, p, orc.density(q0, 0.5), rows), q0[rows] @ M.T,
                               rtol=1e-13, atol=1e-14)
