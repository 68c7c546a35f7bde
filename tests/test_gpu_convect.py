"""vds_convect (the u . grad_x term of Eq. model_DymRepPar on a grid of
ensembles) against the oracle's upwind step, element by element (FP32 on the
GPU against FP64: 1e-6 of the field's scale), on 1-, 2- and 3-D grids, both
boundary rules, ragged value counts; then one operator-split micro-macro step
(convection, then every ensemble's explicit VDS step with the velocity
gradient of its node through the batched path) against the oracle doing the
same two steps."""
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


@pytest.mark.parametrize("shape,M,bc", [((37, 1, 1), 5, 0), ((6, 5, 1), 4663, 1), ((4, 3, 5), 1024, 0),
                                        ((3, 4, 2), 9, 1), ((1, 1, 1), 100, 0), ((2, 7, 3), 2049, 0)])
def test_convect_matches_oracle(orc, vds, ctx, shape, M, bc):
    G = shape[0] * shape[1] * shape[2]
    rng = np.random.default_rng(M + G)
    Q = rng.standard_normal((G, M)).astype(np.float32)
    u = rng.uniform(-1.5, 1.5, (G, 3)).astype(np.float32)
    dx, dt = (0.4, 0.3, 0.5), 0.06
    q_in = torch.from_numpy(Q).cuda()
    q_out = torch.full_like(q_in, float("nan"))
    ctx.vds_convect(q_in, q_out, shape, torch.from_numpy(u).cuda(), dx, dt, bc)
    want = orc.convect_upwind(Q.astype(np.float64), u.astype(np.float64), shape, dx, dt, bc)
    got = q_out.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - want)) <= 1e-6 * np.max(np.abs(Q))


def test_operator_split_micro_macro_step(orc, vds, ctx):
    # 12 ensembles of the 3-bead chain (D = 6) on a 4 x 3 grid, equal N: the
    # flow u(x) carries the particle fields between nodes, then each node's
    # ensemble takes an explicit step in the shear of its node
    nx, ny, N, nb, s = 4, 3, 400, 2, 3
    G, D = nx * ny, nb * s
    rng = np.random.default_rng(2)
    rates = rng.uniform(0.2, 2.0, G)
    kap = np.stack([inputs.shear_kappa(s, r) for r in rates])
    hs = np.full(G, 0.8)
    q0 = np.concatenate([inputs.equilibrium_cloud(N, nb, s, seed=50 + g) for g in range(G)])
    u = np.zeros((G, 3), dtype=np.float32)
    u[:, 0] = rng.uniform(-1, 1, G)
    u[:, 1] = rng.uniform(-1, 1, G)
    dx, dt = (0.5, 0.5, 1.0), 0.01
    p = vds.params(nb, s, dt=dt, scheme=0)
    b = vds.Batch(ctx, [N] * G, D, p, hs, kap)
    q = torch.from_numpy(q0).cuda()
    q2 = torch.empty_like(q)
    ctx.vds_convect(q, q2, (nx, ny, 1), torch.from_numpy(u).cuda(), dx, dt, 1)
    b.step(q2, 1)
    Qo = orc.convect_upwind(q0.reshape(G, N * D).astype(np.float64), u.astype(np.float64), (nx, ny, 1), dx, dt, 1)
    got = q2.cpu().numpy().reshape(G, N, D)
    for g in range(G):
        po = orc.params(nb, s, h=hs[g], dt=dt, kappa=kap[g])
        # the oracle steps the convected FP64 field; the GPU its FP32 rounding
        want = orc.explicit_steps(Qo[g].reshape(N, D), po, 1)
        assert np.max(np.abs(got[g] - want)) <= 1e-5 * np.max(np.abs(want)), g
    b.free()


def test_convect_rejects_bad_arguments(vds, ctx):
    q = torch.zeros((6, 10), device="cuda")
    u = torch.zeros((6, 3), device="cuda")
    for args in [((q, q, (6, 1, 1), u, (1, 1, 1), 0.1, 0)),          # in place
                 ((q, q.view(-1)[5:], (6, 1, 1), u, (1, 1, 1), 0.1, 0)),  # overlapping
                 ((q, torch.empty_like(q), (6, 1, 1), u, (0, 1, 1), 0.1, 0)),
                 ((q, torch.empty_like(q), (6, 1, 1), u, (1, 1, 1), -0.1, 0)),
                 ((q, torch.empty_like(q), (6, 1, 1), u, (1, 1, 1), 0.1, 2))]:
        with pytest.raises(vds.VdsError) as e:
            ctx.vds_convect(*args)
        assert e.value.code == vds.VDS_EARG
