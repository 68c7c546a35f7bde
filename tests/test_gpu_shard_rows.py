"""The library's row-range passes (vds_density_rows, vds_grad_rows), the
per-rank work of a row-sharded evaluation, on one GPU: the ranks of a 2-, 3-
and 8-way split are run one after another (their pieces need no waiting on
each other: the all-gathers are replaced by assembling the pieces on the
host), and the assembled density, gradient and explicit steps match the FP64
oracle within the library's FP32 tolerances (1e-5 relative per evaluation,
the gradient against max |g|), and the whole-cloud GPU path.

The split of a row's sums over CTAs depends on the rows evaluated together,
so the row passes agree with vds_energy_grad to rounding, not bit for bit."""
import numpy as np
import pytest

from paper_2603_12550_gb300 import inputs
from paper_2603_12550_gb300.shard import GpuRows, RowShardedStepper, partition

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


@pytest.mark.parametrize("N,nb,s,world", [(3001, 3, 3, 2), (1000, 1, 2, 3), (20001, 3, 3, 8), (65536, 3, 3, 2)])
def test_row_pieces_assemble_the_evaluation(orc, vds, ctx, N, nb, s, world):
    h = 0.87 if nb == 3 else 0.3
    D = nb * s
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=world)
    q = torch.from_numpy(q32).cuda()
    p = vds.params(nb, s, h=h)
    ranges, _ = partition(N, world)
    rho = torch.empty(N, device="cuda")
    g = torch.empty((N, D), device="cuda")
    for a, n in ranges:
        if n:
            ctx.vds_density_rows(q, p, a, n, rho[a:a + n])
    for a, n in ranges:
        if n:
            ctx.vds_grad_rows(q, p, rho, a, n, g[a:a + n], mode=0)
    torch.cuda.synchronize()
    q64 = q32.astype(np.float64)
    if N <= 20001:
        _, g_o, rho_o = orc.energy_grad(q64, orc.params(nb, s, h=h))
        rows = np.arange(N)
    else:
        # full size: every 97th row against the oracle's row sums
        rows = np.arange(0, N, 97)
        rho_full = orc.density(q64, h)
        rho_o = rho_full
        g_o = np.zeros((N, D))
        g_o[rows] = orc.entropy_grad_rows(q64, h, rho_full, rows) + orc.spring_grad(q64[rows], orc.params(nb, s, h=h))
    r = rho.cpu().numpy()
    assert np.max(np.abs(r[rows] - rho_o[rows]) / rho_o[rows]) <= 1e-5
    gg = g.cpu().numpy()
    assert np.max(np.abs(gg[rows] - g_o[rows])) <= 1e-5 * np.max(np.abs(g_o[rows]))
    # against the whole-cloud GPU evaluation
    g_ref, rho_ref = torch.empty_like(g), torch.empty_like(rho)
    ctx.vds_energy_grad(q, p, g=g_ref, rho=rho_ref, want_energy=False)
    assert torch.max(torch.abs(rho - rho_ref) / rho_ref).item() <= 2e-6
    assert torch.max(torch.abs(g - g_ref)).item() <= 2e-6 * torch.max(torch.abs(g_ref)).item()


@pytest.mark.parametrize("world", [1, 3])
def test_row_sharded_steps_match_oracle(orc, vds, ctx, world):
    # the stepper's own loop with world = 1, and three ranks emulated one
    # after another (pieces assembled on the device by slicing)
    N, nb, s, h, dt, nsteps = 2500, 3, 3, 0.87, 0.005, 4
    kap = inputs.shear_kappa(s, 1.0)
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=11)
    p = vds.params(nb, s, h=h, dt=dt, kappa=kap, scheme=0)
    be = GpuRows(ctx, p)
    if world == 1:
        st = RowShardedStepper(be, N, nb * s, device="cuda")
        st.load(torch.from_numpy(q32).cuda())
        q = st.step(nsteps)
    else:
        ranges, _ = partition(N, world)
        q = torch.from_numpy(q32).cuda()
        rho = torch.empty(N, device="cuda")
        q_new = torch.empty_like(q)
        for _ in range(nsteps):
            for a, n in ranges:
                be.density_rows(q, a, n, rho[a:a + n])
            for a, n in ranges:
                be.step_rows(q, rho, a, n, q_new[a:a + n])
            q.copy_(q_new)
    q_o = orc.explicit_steps(q32.astype(np.float64), orc.params(nb, s, h=h, dt=dt, kappa=kap), nsteps)
    assert np.max(np.abs(q.cpu().numpy() - q_o)) <= 1e-5 * np.max(np.abs(q_o))


def test_row_passes_reject_bad_ranges(vds, ctx):
    q = torch.zeros((100, 9), device="cuda")
    rho = torch.ones(100, device="cuda")
    out = torch.empty((100, 9), device="cuda")
    p = vds.params(3, 3, h=0.9, dt=0.01)
    for a, n in [(-1, 10), (95, 10), (0, 0)]:
        with pytest.raises(vds.VdsError) as e:
            ctx.vds_density_rows(q, p, a, n, rho)
        assert e.value.code == vds.VDS_EARG
    with pytest.raises(vds.VdsError) as e:
        ctx.vds_grad_rows(q, p, rho, 0, 10, out, mode=2)
    assert e.value.code == vds.VDS_EARG
