"""What the trained score network gains over the method without it.

The reduced-order step with the exact O(N^2) entropy gradient (mode i,
Galerkin projection of Eq. model_DymRepPar) is the method without the
network; the surrogate step replaces that gradient by the network's O(N)
output.  On the 4-bead chain (D = 9) at N = 32768, a network fitted on the GPU
to the exact VDS entropy gradient of full-order snapshots at shear rates 0.5,
1 and 2 runs the reduced step at the held-out rate 1.5:

- it is at least twice as fast per step as the exact reduced step;
- its stress after 100 steps stays within max(3 x, 0.08) of the exact reduced
  step's error against the full-order run (the same training reaches about
  3 % at N = 65536 in the benchmark, against 2 % for the exact step);
- the same network untrained (its initial weights) is far worse: training is
  what makes the substitution usable.
"""
import time

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


N, NB, S, H = 32768, 3, 3, 0.9
D = NB * S
DT = 0.005


def _timed(fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, out


def test_trained_surrogate_beats_the_exact_reduced_step(vds, ctx):
    # training pool: full-order snapshots over t in [0, 0.5] at three rates
    pool = []
    for k, rate in enumerate((0.5, 1.0, 2.0)):
        q = torch.from_numpy(inputs.equilibrium_cloud(N, NB, S, seed=200 + k)).cuda()
        p = vds.params(NB, S, h=H, dt=DT, kappa=inputs.shear_kappa(S, rate))
        for _ in range(11):
            pool.append(q.clone())
            ctx.vds_step(q, p, 10)
    pool = torch.cat(pool)
    # targets: the exact entropy gradient S (kBT = 1, no springs)
    pS = vds.params(NB, S, H=[0.0] * NB, kBT=1.0, h=H)
    target = torch.empty_like(pool)
    for k in range(pool.shape[0] // N):
        ctx.vds_energy_grad(pool[k * N:(k + 1) * N], pS, g=target[k * N:(k + 1) * N], want_energy=False)
    layers0 = inputs.mlp_init((D, 256, 256, 256, D), seed=0)
    net = vds.Score(ctx, D, layers0)
    for t in range(1, 501):
        rows, _ = inputs.dsm_rows(pool.shape[0], 8192, D, seed=t)
        net.fit_step(pool, target, 1e-3 if t < 400 else 3e-4, rows=torch.from_numpy(rows).cuda(),
                     want_loss=False)
    untrained = vds.Score(ctx, D, layers0)

    # held-out rate 1.5: full-order run with snapshots every 5 steps
    rate, K = 1.5, 100
    kap = inputs.shear_kappa(S, rate)
    p = vds.params(NB, S, h=H, dt=DT, kappa=kap)
    q0 = torch.from_numpy(inputs.equilibrium_cloud(N, NB, S, seed=7)).cuda()
    q = q0.clone()
    X = torch.empty(((K // 5) * NB, N * S), device="cuda")
    for l in range(K // 5):
        qv = q.view(N, NB, S)
        for k in range(NB):
            X[l * NB + k].copy_(qv[:, k, :].reshape(-1))
        ctx.vds_step(q, p, 5)
    basis, r = ctx.pod_build(X, N * S, X.shape[0], S, energy=0.9999, r_max=64, kappa=kap)
    tau_ref, _ = ctx.vds_stress(q, p)
    P0 = torch.empty((r, NB), device="cuda")
    ctx.pod_project(basis, q0, P0)
    qt = torch.empty_like(q0)

    def stress_err(P):
        ctx.pod_lift(basis, P, qt)
        tau, _ = ctx.vds_stress(qt, p)
        return float(np.linalg.norm(tau - tau_ref) / np.linalg.norm(tau_ref))

    # warm both paths once (graph / workspace set-up), then time K steps
    Pw = P0.clone()
    ctx.pod_step(basis, Pw, N, D, p, nsteps=2, mode=1)
    ctx.pod_step_score(basis, net, Pw, N, D, p, nsteps=2, check_every=0)
    P = P0.clone()
    t_exact, _ = _timed(lambda: ctx.pod_step(basis, P, N, D, p, nsteps=K, mode=1))
    e_exact = stress_err(P)
    P = P0.clone()
    t_sur, _ = _timed(lambda: ctx.pod_step_score(basis, net, P, N, D, p, nsteps=K, check_every=0))
    e_sur = stress_err(P)
    P = P0.clone()
    ctx.pod_step_score(basis, untrained, P, N, D, p, nsteps=K, check_every=0)
    e_untrained = stress_err(P)

    assert t_sur < 0.5 * t_exact, (t_sur, t_exact)
    assert e_sur <= max(3.0 * e_exact, 0.08), (e_sur, e_exact)
    assert e_untrained > 2.0 * e_sur, (e_untrained, e_sur)
    basis.free()
    net.free()
    untrained.free()
