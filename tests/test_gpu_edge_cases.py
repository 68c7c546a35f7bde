"""Edge cases and sizes of the pair passes through the C ABI, against the FP64
oracle or exact values:

- every instantiated D (2..16, s = 2 and 3) on a ragged particle count;
- degenerate clouds with exact answers: all particles at one point
  (rho_I = N, S = 0), a bandwidth far below the spacing (rho_I = 1, S = 0),
  a bandwidth far above the cloud (oracle comparison);
- empty input (N = 0) and an empty ensemble are rejected, not run;
- the largest workload size, N = 262144 at D = 9 (the surrogate workload):
  sampled densities against the oracle's rows and sum_I S_I = 0.
"""
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


@pytest.mark.parametrize("nb,s", [(2, 2), (3, 2), (5, 2), (4, 3), (7, 2), (8, 2)])
def test_remaining_dimensions_match_oracle(orc, vds, ctx, nb, s):
    # D = 4, 6 (s = 2), 10, 12, 14, 16; the other D are in test_gpu_pair.py
    N, h = 301, 0.6 * np.sqrt(nb)
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=40 + nb * s)
    po, pg = orc.params(nb, s, h=h), vds.params(nb, s, h=h)
    E_o, g_o, rho_o = orc.energy_grad(q32.astype(np.float64), po)
    q = _dev(q32)
    g = torch.empty_like(q)
    rho = torch.empty(N, device="cuda")
    E = ctx.vds_energy_grad(q, pg, g=g, rho=rho)
    assert np.max(np.abs(rho.cpu().numpy() - rho_o) / rho_o) <= 1e-5
    assert abs(E - E_o) <= 1e-5 * (1 + abs(E_o))
    assert np.max(np.abs(g.cpu().numpy() - g_o)) <= 1e-5 * np.max(np.abs(g_o))


def test_coincident_particles(orc, vds, ctx):
    # every kernel value is exp2(0) = 1: rho_I = N exactly and S = 0 exactly,
    # so g is the spring force alone
    N, nb, s = 257, 3, 3
    q32 = np.tile(np.array([[0.3, -0.2, 0.1, 0.5, 0.0, -0.4, 0.2, 0.2, 0.1]], dtype=np.float32), (N, 1))
    pg = vds.params(nb, s, h=0.7, kBT=1.0)
    q = _dev(q32)
    g = torch.empty_like(q)
    rho = torch.empty(N, device="cuda")
    ctx.vds_energy_grad(q, pg, g=g, rho=rho)
    assert torch.all(rho == float(N))
    np.testing.assert_allclose(g.cpu().numpy(), orc.spring_grad(q32.astype(np.float64), orc.params(nb, s)),
                               rtol=1e-6, atol=0)


def test_bandwidth_far_below_spacing(vds, ctx):
    # h = 1e-3 against O(1) spacings: only the self term survives
    N, nb, s = 500, 2, 3
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=9)
    pg = vds.params(nb, s, h=1e-3, H=[0.0, 0.0], kBT=1.0)
    q = _dev(q32)
    g = torch.empty_like(q)
    rho = torch.empty(N, device="cuda")
    ctx.vds_energy_grad(q, pg, g=g, rho=rho)
    assert torch.all(rho == 1.0)
    assert torch.all(g == 0.0)


def test_bandwidth_far_above_cloud(orc, vds, ctx):
    N, nb, s, h = 700, 3, 3, 200.0
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=10)
    po, pg = orc.params(nb, s, h=h), vds.params(nb, s, h=h)
    E_o, g_o, rho_o = orc.energy_grad(q32.astype(np.float64), po)
    q = _dev(q32)
    g = torch.empty_like(q)
    rho = torch.empty(N, device="cuda")
    E = ctx.vds_energy_grad(q, pg, g=g, rho=rho)
    assert np.max(np.abs(rho.cpu().numpy() - rho_o) / rho_o) <= 1e-5
    assert abs(E - E_o) <= 1e-5 * (1 + abs(E_o))
    assert np.max(np.abs(g.cpu().numpy() - g_o)) <= 1e-5 * np.max(np.abs(g_o))


def test_empty_inputs_are_rejected(vds, ctx):
    q = torch.empty((0, 9), device="cuda")
    p = vds.params(3, 3, h=0.9, dt=0.005)
    for call in (lambda: ctx.vds_energy_grad(q, p, g=torch.empty_like(q)),
                 lambda: ctx.vds_step(q, p, 1),
                 lambda: ctx.vds_stress(q, p),
                 lambda: ctx.vds_bandwidth(q, 0)):
        with pytest.raises(vds.VdsError) as ei:
            call()
        assert ei.value.code == vds.VDS_EARG
    with pytest.raises(vds.VdsError):
        vds.Batch(ctx, [10, 0, 5], 6, vds.params(2, 3), [0.5, 0.5, 0.5], np.zeros((3, 3, 3)))
    # the context stays usable
    q1 = _dev(inputs.equilibrium_cloud(33, 3, 3, seed=1))
    ctx.vds_energy_grad(q1, p, g=torch.empty_like(q1))


def test_largest_workload_size(orc, vds, ctx):
    # N = 262144, D = 9: densities of 128 sampled particles against the
    # oracle's rows; with springs off and kBT = 1, g = S and sum_I S_I = 0
    # (antisymmetric kernel gradient times a symmetric weight)
    N, nb, s, h = 262144, 3, 3, 0.8
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=5)
    pg = vds.params(nb, s, h=h, H=[0.0] * nb, kBT=1.0)
    q = _dev(q32)
    g = torch.empty_like(q)
    rho = torch.empty(N, device="cuda")
    ctx.vds_energy_grad(q, pg, g=g, rho=rho)
    rows = np.random.default_rng(3).choice(N, 128, replace=False)
    rows[:2] = [0, N - 1]
    rho_o = orc.density_rows(q32.astype(np.float64), h, rows)
    assert np.max(np.abs(rho.cpu().numpy()[rows] - rho_o) / rho_o) <= 1e-5
    G = g.double()
    assert float(torch.linalg.norm(G.sum(0))) <= 1e-5 * float(G.abs().sum(0).max())
