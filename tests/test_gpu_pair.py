"""GPU parity of the pair passes, time steps and stress against the FP64
oracle, through the C ABI.

Tolerances (FP32 pair sums with compensated accumulation vs FP64):
  rho   elementwise relative          <= 1e-5
  E     |dE| <= 1e-5 (1 + |E|)
  g     max_I |dg_I| <= 1e-5 max_I |g_I|   (relative per evaluation)
  q     after steps: max |dq| <= 1e-5 max |q|
  tau   relative (Frobenius) <= 1e-6 at the same state
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


def _both_params(orc, vds, **kw):
    okw = dict(kw)
    okw.pop("scheme", None)
    okw.pop("jfloor", None)
    gkw = dict(kw)
    if "tol" in okw:
        okw["tol"] = 1e-10
    return orc.params(**okw), vds.params(**gkw)


CASES = [
    # N, nb, s, h, spring, b
    (512, 1, 2, 0.3, 0, 0.0),     # 2D dumbbell, several tiles
    (1, 1, 3, 0.5, 0, 0.0),       # single particle
    (2, 3, 3, 0.9, 0, 0.0),
    (129, 1, 3, 0.4, 0, 0.0),     # ragged tail
    (700, 2, 3, 0.7, 0, 0.0),     # D = 6, ragged
    (1000, 3, 3, 0.9, 0, 0.0),    # 4-bead D = 9, ragged
    (1500, 3, 3, 0.9, 1, 50.0),   # FENE b = 50
    (640, 4, 2, 0.8, 0, 0.0),     # D = 8
    (300, 5, 3, 1.2, 0, 0.0),     # D = 15
]


@pytest.mark.parametrize("N,nb,s,h,spring,b", CASES)
def test_energy_grad_matches_oracle(orc, vds, ctx, N, nb, s, h, spring, b):
    D = nb * s
    H = [1.0 + 0.5 * k for k in range(nb)]
    q32 = inputs.equilibrium_cloud(N, nb, s, H=H, seed=N + D, fene_b=b if spring else None)
    po, pg = _both_params(orc, vds, nb=nb, s=s, H=H, h=h, spring=spring, b=b, kBT=1.0)
    E_o, g_o, rho_o = orc.energy_grad(q32.astype(np.float64), po)
    q = _dev(q32)
    g = torch.empty_like(q)
    rho = torch.empty(N, device="cuda")
    E = ctx.vds_energy_grad(q, pg, g=g, rho=rho)
    torch.cuda.synchronize()
    rho_g = rho.cpu().numpy().astype(np.float64)
    g_g = g.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(rho_g - rho_o) / rho_o) <= 1e-5
    assert abs(E - E_o) <= 1e-5 * (1 + abs(E_o))
    assert np.max(np.abs(g_g - g_o)) <= 1e-5 * max(np.max(np.abs(g_o)), 1e-30)


def test_implicit_objective_matches_oracle(orc, vds, ctx):
    # J and G with q_star (the objective of the implicit step)
    N, nb, s, h, dt = 400, 3, 3, 0.9, 0.005
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=3)
    qs32 = (q32 * 1.01 + 0.003).astype(np.float32)
    po, pg = _both_params(orc, vds, nb=nb, s=s, h=h, dt=dt)
    q64, qs64 = q32.astype(np.float64), qs32.astype(np.float64)
    E_o, g_o, _ = orc.energy_grad(q64, po)
    Ainv = orc.rouse_inv(nb)
    d = (q64 - qs64).reshape(N, nb, s)
    quad = np.einsum("Ija,jk,Ika->", d, Ainv, d) / N
    J_o = E_o + 4.0 / (2 * dt) * quad
    G_o = g_o + (4.0 / dt) * np.einsum("kj,Ija->Ika", Ainv, d).reshape(N, -1)
    q, qs = _dev(q32), _dev(qs32)
    G = torch.empty_like(q)
    J = ctx.vds_energy_grad(q, pg, g=G, q_star=qs)
    assert abs(J - J_o) <= 1e-5 * (1 + abs(J_o))
    assert np.max(np.abs(G.cpu().numpy() - G_o)) <= 1e-5 * np.max(np.abs(G_o))


@pytest.mark.parametrize("N,nb,s,h,rate", [(512, 1, 2, 0.3, 1.0), (1000, 3, 3, 0.9, 1.0),
                                           (333, 2, 3, 0.6, 2.0)])
def test_explicit_steps_match_oracle(orc, vds, ctx, N, nb, s, h, rate):
    kap = inputs.shear_kappa(s, rate)
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=7)
    po, pg = _both_params(orc, vds, nb=nb, s=s, h=h, dt=0.005, kappa=kap, scheme=0)
    q_o = orc.explicit_steps(q32.astype(np.float64), po, 5)
    q = _dev(q32)
    ctx.vds_step(q, pg, 5)
    q_g = q.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(q_g - q_o)) <= 1e-5 * np.max(np.abs(q_o))


@pytest.mark.parametrize("N,nb,s,h,dt", [(512, 1, 2, 0.3, 0.01), (600, 3, 3, 0.9, 0.005)])
def test_implicit_steps_match_oracle(orc, vds, ctx, N, nb, s, h, dt):
    kap = inputs.shear_kappa(s, 1.0)
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=11)
    po, pg = _both_params(orc, vds, nb=nb, s=s, h=h, dt=dt, kappa=kap, scheme=1, tol=1e-6,
                          jfloor=1e-9)
    q_o, it_o, _ = orc.implicit_steps(q32.astype(np.float64), po, 2)
    q = _dev(q32)
    its = ctx.vds_step(q, pg, 2, want_iters=True)
    q_g = q.cpu().numpy().astype(np.float64)
    assert all(1 <= k <= 50 for k in its)
    assert np.max(np.abs(q_g - q_o)) <= 1e-5 * np.max(np.abs(q_o))


@pytest.mark.parametrize("nb,s,spring", [(1, 2, 0), (3, 3, 0), (3, 3, 1)])
def test_stress_matches_oracle(orc, vds, ctx, nb, s, spring):
    N = 3000
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=5, fene_b=50.0 if spring else None)
    H = [1.0 + k for k in range(nb)]
    po, pg = _both_params(orc, vds, nb=nb, s=s, H=H, spring=spring, b=50.0, h=0.5)
    tau_o, qq_o = orc.stress(q32.astype(np.float64), po)
    tau, qq = ctx.vds_stress(_dev(q32), pg)
    assert np.linalg.norm(tau - tau_o) <= 1e-6 * np.linalg.norm(tau_o)
    assert np.linalg.norm(qq - qq_o) <= 1e-6 * np.linalg.norm(qq_o)


def test_fene_domain_error_is_reported(vds, ctx):
    q32 = np.array([[8.0, 0.0, 0.0], [0.1, 0.2, 0.3]], dtype=np.float32)
    pg = vds.params(nb=1, s=3, h=0.5, spring=1, b=50.0)
    with pytest.raises(vds.VdsError) as ei:
        ctx.vds_energy_grad(_dev(q32), pg)
    assert ei.value.code == vds.VDS_EDOMAIN
    # the context stays usable
    ok = np.array([[1.0, 0.0, 0.0], [0.1, 0.2, 0.3]], dtype=np.float32)
    ctx.vds_energy_grad(_dev(ok), pg)


def test_bad_arguments_are_rejected(vds, ctx):
    q = _dev(np.zeros((4, 9), dtype=np.float32))
    with pytest.raises(vds.VdsError):
        ctx.vds_energy_grad(q, vds.params(nb=2, s=3, h=0.5))  # D mismatch
    with pytest.raises(vds.VdsError):
        ctx.vds_energy_grad(q, vds.params(nb=3, s=3, h=0.0))  # h = 0


def test_full_size_chain4_sampled_rows(orc, vds, ctx):
    # Full 4-bead workload (N = 65536, D = 9) in the bench's launch
    # configuration; the oracle computes the full density (O(N^2) FP64) and
    # the gradient of 192 sampled particles.
    N, nb, s = 65536, 3, 3
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=0)
    q64 = q32.astype(np.float64)
    h = 0.9
    po, pg = _both_params(orc, vds, nb=nb, s=s, h=h)
    q = _dev(q32)
    g = torch.empty_like(q)
    rho = torch.empty(N, device="cuda")
    E = ctx.vds_energy_grad(q, pg, g=g, rho=rho)
    rho_o = orc.density(q64, h)
    assert np.max(np.abs(rho.cpu().numpy() - rho_o) / rho_o) <= 1e-5
    lnorm = -np.log(N) - 0.5 * 9 * np.log(2 * np.pi * h * h)
    E_o = np.mean(np.log(rho_o) + lnorm + 0.5 * (q64 ** 2).sum(1))
    assert abs(E - E_o) <= 1e-5 * (1 + abs(E_o))
    rows = np.random.default_rng(0).choice(N, 192, replace=False)
    rows[:3] = [0, N - 1, N // 2]
    g_o = orc.entropy_grad_rows(q64, h, rho_o, rows) + orc.spring_grad(q64[rows], po)
    g_g = g.cpu().numpy()[rows].astype(np.float64)
    assert np.max(np.abs(g_g - g_o)) <= 1e-5 * np.max(np.abs(g_o))


@pytest.mark.parametrize("N", [3001, 10000, 20001])
def test_chain4_every_pass_shape_matches_oracle(orc, vds, ctx, N):
    # The pair passes pick their shape from the number of (i-tile, j-chunk)
    # items: 128 threads of one particle and 64-record chunks for small clouds
    # (N = 3001), the large shapes with 64-record chunks in between (N =
    # 10000 for both passes, N = 20001 for the density pass), and with
    # 256-record chunks above (the gradient pass at N = 20001).  Full density
    # and sampled gradient rows against the oracle at ragged N.
    nb, s = 3, 3
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=N)
    q64 = q32.astype(np.float64)
    h = 0.9
    po, pg = _both_params(orc, vds, nb=nb, s=s, h=h)
    q = _dev(q32)
    g = torch.empty_like(q)
    rho = torch.empty(N, device="cuda")
    ctx.vds_energy_grad(q, pg, g=g, rho=rho)
    rho_o = orc.density(q64, h)
    assert np.max(np.abs(rho.cpu().numpy() - rho_o) / rho_o) <= 1e-5
    rows = np.random.default_rng(N).choice(N, 96, replace=False)
    rows[:3] = [0, N - 1, N // 2]
    g_o = orc.entropy_grad_rows(q64, h, rho_o, rows) + orc.spring_grad(q64[rows], po)
    g_g = g.cpu().numpy()[rows].astype(np.float64)
    assert np.max(np.abs(g_g - g_o)) <= 1e-5 * np.max(np.abs(g_o))


@pytest.mark.parametrize("N,nb,s", [(1000, 3, 3), (512, 1, 2), (20001, 3, 3)])
def test_explicit_graph_replay_is_bit_identical(orc, vds, ctx, N, nb, s):
    # vds_step replays a captured graph of one explicit step after the first;
    # with phase timing on it launches every step directly.  Same kernels,
    # same arguments: the states after 7 steps agree bit for bit.
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=5)
    _, pg = _both_params(orc, vds, nb=nb, s=s, h=0.7, dt=1e-3, kappa=inputs.shear_kappa(s, 1.0))
    qa, qb = _dev(q32), _dev(q32)
    ctx.vds_step(qa, pg, 7)
    ctx.vds_timing(True)
    ctx.vds_step(qb, pg, 7)
    ctx.vds_timing(False)
    assert torch.equal(qa, qb)
    assert not torch.equal(qa, _dev(q32))
