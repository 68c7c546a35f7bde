"""The density estimate at query points (Eq. model_DeteParAppr; Appendix A
evaluates it on the grid {-2, 0, 2}^D) through the C ABI, against the FP64
oracle:

- ragged query and particle counts for several D (one query, fewer queries
  than one tile, several tiles);
- at the particles themselves it equals the pair pass's density rho_I times
  (1/N)(2 pi h^2)^(-D/2) (the same kernel and sums);
- the full 4-bead workload (N = 65536, D = 9) on Appendix A's grid of 3^9
  points: sampled points against the oracle;
- bad arguments are rejected.

Tolerance 1e-5 relative, as for the density pass (FP32 pair sums of positive
terms, compensated across tiles, FP64 across segments)."""
import numpy as np
import pytest

from paper_2603_12550_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12550_gb300 import build
    build.build()
    from paper_2603_12550_gb300 import vds as v
    return v


@pytest.fixture(scope="module")
def ctx(vds):
    c = vds.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("N,M,nb,s,h", [(301, 1, 1, 2, 0.3), (301, 77, 1, 3, 0.5), (2048, 1000, 2, 3, 0.7),
                                        (1000, 4099, 3, 3, 0.9), (700, 300, 8, 2, 1.2)])
def test_density_at_matches_oracle(orc, vds, ctx, N, M, nb, s, h):
    D = nb * s
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=N + D)
    y32 = (np.random.default_rng(M).standard_normal((M, D)) * 1.3).astype(np.float32)
    f = torch.full((M + 5,), -1.0, device="cuda")
    ctx.vds_density_at(_dev(q32), vds.params(nb, s, h=h), _dev(y32), f[:M])
    got = f.cpu().numpy()
    assert np.all(got[M:] == -1.0)
    ref = orc.density_at(q32.astype(np.float64), h, y32.astype(np.float64))
    assert np.max(np.abs(got[:M] - ref) / ref) <= 1e-5


def test_density_at_the_particles_equals_the_pair_density(vds, ctx):
    N, nb, s, h = 5000, 3, 3, 0.8
    D = nb * s
    q = _dev(inputs.equilibrium_cloud(N, nb, s, seed=2))
    p = vds.params(nb, s, h=h)
    rho = torch.empty(N, device="cuda")
    ctx.vds_energy_grad(q, p, g=torch.empty_like(q), rho=rho, want_energy=False)
    f = torch.empty(N, device="cuda")
    ctx.vds_density_at(q, p, q, f)
    scale = (2 * np.pi * h * h) ** (-D / 2) / N
    np.testing.assert_allclose(f.cpu().numpy(), rho.cpu().numpy().astype(np.float64) * scale, rtol=1e-6)


def test_full_size_grid_of_appendix_a(orc, vds, ctx):
    wl = inputs.WORKLOADS["chain4_n65536_d9"]
    N, nb, s = wl["N"], wl["nb"], wl["s"]
    h = 0.87
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=wl["seed"])
    G = orc.grid_points(nb * s)
    f = torch.empty(G.shape[0], device="cuda")
    ctx.vds_density_at(_dev(q32), vds.params(nb, s, h=h), _dev(G), f)
    got = f.cpu().numpy()
    assert np.all(got > 0.0)
    rows = np.random.default_rng(4).choice(G.shape[0], 48, replace=False)
    rows[:2] = [0, G.shape[0] // 2]          # a corner and the origin
    ref = orc.density_at(q32.astype(np.float64), h, G[rows])
    assert np.max(np.abs(got[rows] - ref) / ref) <= 1e-5


def test_bad_arguments_are_rejected(vds, ctx):
    q = _dev(inputs.equilibrium_cloud(10, 1, 3, seed=1))
    y = torch.zeros((4, 3), device="cuda")
    f = torch.empty(4, device="cuda")
    with pytest.raises(vds.VdsError) as ei:
        ctx.vds_density_at(q, vds.params(1, 3, h=0.5), y[:0], f)
    assert ei.value.code == vds.VDS_EARG
    with pytest.raises(vds.VdsError):
        ctx.vds_density_at(q, vds.params(1, 3, h=-1.0), y, f)
    ctx.vds_density_at(q, vds.params(1, 3, h=0.5), y, f)
    assert torch.all(f > 0)
