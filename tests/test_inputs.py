"""The seeded input recipe (Sec. 3.1 initial condition; batched and snapshot
generators): deterministic per seed, the stated distributions, the FENE
domain respected."""
import numpy as np

from paper_2603_12550_gb300 import inputs


def test_equilibrium_cloud_is_seeded_and_fp32():
    a = inputs.equilibrium_cloud(1000, 3, 3, seed=4)
    b = inputs.equilibrium_cloud(1000, 3, 3, seed=4)
    c = inputs.equilibrium_cloud(1000, 3, 3, seed=5)
    assert a.dtype == np.float32 and a.shape == (1000, 9)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_equilibrium_cloud_has_the_boltzmann_variances():
    # bond k, every component ~ N(0, kBT / H_k): sample variances within a few
    # standard errors (relative standard error sqrt(2 / n))
    N, nb, s, kBT = 200000, 3, 3, 0.7
    H = [1.0, 2.0, 3.0]
    q = inputs.equilibrium_cloud(N, nb, s, H=H, kBT=kBT, seed=1).astype(np.float64)
    var = q.var(axis=0).reshape(nb, s)
    want = np.array([[kBT / h] * s for h in H])
    assert np.max(np.abs(var / want - 1)) <= 5 * np.sqrt(2.0 / N)
    assert np.max(np.abs(q.mean(axis=0))) <= 5 * np.sqrt(kBT / min(H) / N)


def test_fene_clouds_stay_inside_the_domain():
    b = 3.0
    q = inputs.equilibrium_cloud(5000, 3, 3, seed=2, fene_b=b).astype(np.float64)
    assert np.all((q.reshape(5000, 3, 3) ** 2).sum(-1) < b)


def test_shear_kappa():
    k = inputs.shear_kappa(3, 1.5)
    assert k.shape == (3, 3) and k[0, 1] == 1.5 and np.count_nonzero(k) == 1


def test_ensemble_sizes_ranges():
    sizes, rates = inputs.ensemble_sizes(512, seed=0)
    assert sizes.min() >= 1024 and sizes.max() <= 16384
    assert rates.min() >= 0.1 and rates.max() <= 10.0
    s2, r2 = inputs.ensemble_sizes(512, seed=0)
    assert np.array_equal(sizes, s2) and np.array_equal(rates, r2)


def test_snapshot_matrix_has_the_prescribed_spectrum():
    # geometric singular values sqrt(n_rows) 0.5^k, up to the FP32 rounding
    # of the entries
    X = inputs.snapshot_matrix(400, 60, rank=8, seed=3)
    sv = np.linalg.svd(X.astype(np.float64), compute_uv=False)
    want = 0.5 ** np.arange(8) * np.sqrt(400)
    np.testing.assert_allclose(sv[:8], want, rtol=1e-5)
    assert sv[8] <= 1e-5 * sv[0]
