"""GPU parity of the reduced-order steps (Sec. 2.3-2.4): the frozen Brownian
matrices X^B1, X^B2, mode 1 (Galerkin, Eq. model_DymRepParPod) and mode 2
(Eq. model_DymReduced with periodic refresh) against the FP64 oracle.

Both sides start from the same reduced state P0 (the oracle's projection of an
oracle trajectory state) and use the same basis: the oracle's POD basis of an
oracle trajectory, rounded to FP32, loaded on the GPU with pod_load (the GPU's
own pod_build is checked against the oracle in test_gpu_pod.py; its TF32 Gram
moves basis columns with small eigenvalue gaps by up to about 1e-9 / gap,
which these trajectory snapshots have).  Tolerances: X^B within 1e-4 relative
(Frobenius; FP32 pair sums with O(1) cancellation in Phi - W/rho), P within
1e-4 relative after the steps.
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


@pytest.fixture(scope="module")
def setup(orc, vds, ctx):
    N, nb, s, r = 500, 3, 3, 10
    kap = inputs.shear_kappa(s, 1.0)
    q = inputs.equilibrium_cloud(N, nb, s, seed=21).astype(np.float64)
    po = orc.params(nb, s, h=0.9, dt=0.005, kappa=kap)
    states = [q]
    for _ in range(9):
        q = orc.explicit_steps(q, po, 5)
        states.append(q)
    X = orc.snapshots_from_states([x.astype(np.float32).astype(np.float64) for x in states], s, nb)
    X32 = X.astype(np.float32)
    o = orc.pod_build(X32.astype(np.float64), r_fixed=r)
    Phi32 = o["Phi"].astype(np.float32)
    basis = ctx.pod_load(torch.from_numpy(np.ascontiguousarray(Phi32)).cuda(), s, kappa=kap)
    Phi = Phi32.astype(np.float64)
    P0 = orc.project(Phi, states[0], s, nb)
    pg = vds.params(nb, s, h=0.9, dt=0.005, kappa=kap)
    return dict(N=N, nb=nb, s=s, r=r, kap=kap, po=po, pg=pg, Phi=Phi, basis=basis, P0=P0)


def test_pod_load_keeps_the_basis(orc, vds, ctx, setup):
    S = setup
    Phi = S["basis"].phi().cpu().numpy().astype(np.float64)
    assert np.array_equal(Phi, S["Phi"])
    XH_o = orc.x_h(S["Phi"], S["kap"], S["s"])
    assert np.abs(S["basis"].xh() - XH_o).max() <= 1e-5 * max(1.0, np.abs(XH_o).max())


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_brownian_matrices_match_oracle(orc, vds, ctx, setup):
    S = setup
    P = torch.from_numpy(S["P0"].astype(np.float32)).cuda()
    B1, B2 = ctx.pod_brownian(S["basis"], P, S["N"], S["nb"] * S["s"], S["pg"])
    q = orc.lift(S["Phi"], S["P0"].astype(np.float32).astype(np.float64), S["s"], S["nb"])
    B1o, B2o, _ = orc.x_b(S["Phi"], q, 0.9, S["s"])
    assert _rel(B1, B1o) <= 1e-4
    assert _rel(B2, B2o) <= 1e-4


def test_mode2_frozen_steps_match_oracle(orc, vds, ctx, setup):
    S = setup
    P = torch.from_numpy(S["P0"].astype(np.float32)).cuda()
    ctx.pod_step(S["basis"], P, S["N"], S["nb"] * S["s"], S["pg"], nsteps=12, refresh_every=5, mode=2)
    P_o = orc.reduced_run(S["P0"].astype(np.float32).astype(np.float64), S["Phi"], S["po"], 12, 5)
    assert _rel(P.cpu().numpy(), P_o) <= 1e-4


def test_mode1_galerkin_steps_match_oracle(orc, vds, ctx, setup):
    S = setup
    P = torch.from_numpy(S["P0"].astype(np.float32)).cuda()
    ctx.pod_step(S["basis"], P, S["N"], S["nb"] * S["s"], S["pg"], nsteps=3, mode=1)
    Po = S["P0"].astype(np.float32).astype(np.float64)
    for _ in range(3):
        Po = Po + S["po"].dt * orc.galerkin_rhs(Po, S["Phi"], S["po"])
    assert _rel(P.cpu().numpy(), Po) <= 1e-4


def test_mode2_with_refresh_every_step_is_galerkin(vds, ctx, setup):
    # Sec. 2.4: the frozen terms are exact at a refresh instant, so refreshing
    # every step reproduces the Galerkin trajectory (here: GPU against GPU).
    S = setup
    P1 = torch.from_numpy(S["P0"].astype(np.float32)).cuda()
    P2 = P1.clone()
    D = S["nb"] * S["s"]
    ctx.pod_step(S["basis"], P1, S["N"], D, S["pg"], nsteps=4, refresh_every=1, mode=2)
    ctx.pod_step(S["basis"], P2, S["N"], D, S["pg"], nsteps=4, mode=1)
    assert _rel(P1.cpu().numpy(), P2.cpu().numpy()) <= 1e-4


def test_mode2_rejects_fene(vds, ctx, setup):
    S = setup
    P = torch.from_numpy(S["P0"].astype(np.float32)).cuda()
    pf = vds.params(S["nb"], S["s"], h=0.9, dt=0.005, spring=1, b=50.0)
    with pytest.raises(vds.VdsError):
        ctx.pod_step(S["basis"], P, S["N"], S["nb"] * S["s"], pf, nsteps=1, mode=2)


def _score_net(vds, ctx, seed=11):
    from paper_2603_12550_gb300 import inputs as inp
    layers = inp.mlp_init((9, 256, 256, 256, 9), seed=seed, scale=0.5)
    return layers, vds.Score(ctx, 9, layers)


def test_score_mode_matches_oracle(orc, vds, ctx, setup):
    # the surrogate reduced step (no checks) against the FP64 oracle with the
    # same network weights; BF16 network: 1e-2 relative on P
    S = setup
    layers, net = _score_net(vds, ctx)
    P = torch.from_numpy(S["P0"].astype(np.float32)).cuda()
    D = S["nb"] * S["s"]
    ctx.pod_step_score(S["basis"], net, P, S["N"], D, S["pg"], nsteps=3, check_every=0)
    Po = S["P0"].astype(np.float32).astype(np.float64)
    for _ in range(3):
        Po = Po + S["po"].dt * orc.score_rhs(Po, S["Phi"], S["po"], layers)
    assert _rel(P.cpu().numpy(), Po) <= 1e-2


def test_score_steps_replayed_as_a_graph_equal_uncaptured_steps(vds, ctx, setup):
    # the steps between checks replay one captured CUDA graph; a call in which
    # every step is a check step (with a tolerance no error exceeds, so no
    # fallback) launches the same update kernels one by one, uncaptured: the
    # reduced coordinates come out bit-identical, with and without checks in
    # between
    S = setup
    _, net = _score_net(vds, ctx)
    D = S["nb"] * S["s"]
    P0 = torch.from_numpy(S["P0"].astype(np.float32)).cuda()
    runs = {}
    for name, every in (("graph", 0), ("graph_between_checks", 3), ("uncaptured", 1)):
        P = P0.clone()
        ctx.pod_step_score(S["basis"], net, P, S["N"], D, S["pg"], nsteps=7, check_every=every, check_n=100,
                           check_tol=1e9)
        runs[name] = P
    assert torch.equal(runs["graph"], runs["uncaptured"])
    assert torch.equal(runs["graph_between_checks"], runs["uncaptured"])


def test_score_check_falls_back_to_exact(vds, ctx, setup):
    # with a zero tolerance every checked step uses the exact entropy gradient,
    # which is the Galerkin step
    S = setup
    _, net = _score_net(vds, ctx)
    D = S["nb"] * S["s"]
    P1 = torch.from_numpy(S["P0"].astype(np.float32)).cuda()
    P2 = P1.clone()
    err, nf = ctx.pod_step_score(S["basis"], net, P1, S["N"], D, S["pg"], nsteps=3, check_every=1,
                                 check_n=100, check_tol=0.0)
    assert nf == 3 and err > 0.0
    ctx.pod_step(S["basis"], P2, S["N"], D, S["pg"], nsteps=3, mode=1)
    assert _rel(P1.cpu().numpy(), P2.cpu().numpy()) <= 1e-5


@pytest.mark.parametrize("N,nb,s,r", [(1000, 3, 3, 5), (1000, 3, 3, 20), (777, 2, 3, 42), (1300, 3, 3, 64),
                                      (2000, 4, 2, 30), (129, 1, 3, 3), (300, 2, 3, 16), (300, 2, 3, 17),
                                      (300, 2, 3, 32), (300, 2, 3, 33), (600, 2, 3, 10), (3000, 2, 3, 4),
                                      (100, 3, 3, 3), (5000, 3, 3, 10)])
def test_brownian_matrices_every_column_chunk_shape(orc, vds, ctx, N, nb, s, r):
    # the refresh pass for every width of its B slice (2 s r + 1 columns padded
    # to 32, 64, 128 or 256; r = 64 with s = 3 takes two column chunks), ragged
    # N, and a segment count that is not a multiple of the flush schedule;
    # r = 16/17 and 32/33 straddle the corner sizes (16, 32, 64) of the r x r
    # contractions Phi^T U; D = 6 and 9 with 2 s r + 1 <= 64 take the kernel
    # values' dot products on the tensor cores (one to many passes per CTA):
    # X^B1 and X^B2 at the lifted state against the oracle
    D = nb * s
    rng = np.random.default_rng(N + r)
    Phi, _ = np.linalg.qr(rng.standard_normal((N * s, r)))
    Phi32 = np.ascontiguousarray(Phi.astype(np.float32))
    basis = ctx.pod_load(torch.from_numpy(Phi32).cuda(), s)
    q0 = inputs.equilibrium_cloud(N, nb, s, seed=N).astype(np.float64)
    P = orc.project(Phi32.astype(np.float64), q0, s, nb)
    qt = orc.lift(Phi32.astype(np.float64), P.astype(np.float32).astype(np.float64), s, nb)
    h = 0.8
    B1o, B2o, _ = orc.x_b(Phi32.astype(np.float64), qt, h, s)
    B1, B2 = ctx.pod_brownian(basis, torch.from_numpy(np.ascontiguousarray(P.astype(np.float32))).cuda(), N, D,
                              vds.params(nb, s, h=h))
    assert _rel(B1, B1o) <= 1e-4, _rel(B1, B1o)
    assert _rel(B2, B2o) <= 1e-4, _rel(B2, B2o)
    basis.free()
