"""The 4-bead chain in shear at its full size (N = 65536, D = 9; Sec. 3.3's
set-up, Appendix A's schemes) against the FP64 oracle, in the launch
configurations the benchmark times:

- final-time stress: explicit runs compared, at every stored checkpoint, with
  the oracle's trajectories written by tests/golden/make_chain4_trajectories.py
  (N = 16384 over t in [0, 5], i.e. 1000 steps, and N = 65536 over 100 steps,
  Hookean and FENE b = 50; and the 3D dumbbell, N = 16384, shear rates 0.1, 1
  and 10 over t in [0, 5]): the paper's stress tau and the second moments
  within 1e-3 relative (Frobenius), and every 256th particle's connectors
  (not for the dumbbell at rate 10, whose particle paths separate);
  the bandwidth (median rule of Eq. model_bandwidth, or Silverman for the
  dumbbell) against the oracle's;
- the reduced path (Sec. 2.4) at N = 65536, r = 10: X^B1 and X^B2 at a lifted
  state within 1e-4 relative, and 61 frozen-term steps refreshed every 60
  (so the run crosses one refresh) within 1e-4 relative on P;
- implicit steps (Appendix A, solved by iteration) at N = 65536: two steps in
  one call, the first from q*, the second from the previous step's correction
  (warm start) -- the same minimiser as the oracle's within the solver
  tolerance.

The oracle computes its side here on the host cores (seconds to a minute at
N = 65536) except the long explicit runs, read from the JSON fixtures.
"""
import json
import os

import numpy as np
import pytest

from paper_2603_12550_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
N_FULL, NB, S = 65536, 3, 3


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


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


# ------------------------------------------------------- final-time stress

# Runs whose individual particle paths separate from the oracle's: in the
# dumbbell at shear rate 10 the flow stretches the cloud to |q| ~ 30 while the
# kernel keeps h = 0.24, and the FP32/FP64 rounding differences grow along
# the paths to O(1) by T = 5 (measured: up to 1.4 against max |q| = 29), while
# the stress and second moments, the quantities compared above, still agree
# within about 3e-5.  Their rows are not compared.
PATHS_SEPARATE = {"dumbbell3d_n16384_rate10_T5"}


@pytest.mark.parametrize("name", ["chain4_n16384_hookean_T5", "chain4_n65536_hookean_s100",
                                  "chain4_n65536_fene50_s100", "dumbbell3d_n16384_rate0.1_T5",
                                  "dumbbell3d_n16384_rate1_T5", "dumbbell3d_n16384_rate10_T5"])
def test_final_time_stress_matches_oracle_trajectory(vds, ctx, name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        gold = json.load(f)
    N, nb, s = gold["N"], gold["nb"], gold["s"]
    fene = gold["spring"] == 1
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=gold["seed"], fene_b=gold["b"] if fene else None)
    q = _dev(q32)
    # the GPU's bandwidth rule (median over FP32 pair distances, or Silverman)
    # against the oracle's FP64 one
    rule = 1 if gold.get("bandwidth") == "silverman" else 0
    assert ctx.vds_bandwidth(q, rule=rule) == pytest.approx(gold["h"], rel=1e-6)
    p = vds.params(nb, s, H=gold["H"], kBT=gold["kBT"], zeta=gold["zeta"], h=gold["h"], dt=gold["dt"],
                   kappa=inputs.shear_kappa(s, gold["rate"]), spring=gold["spring"], b=gold["b"],
                   scheme=0)
    done = 0
    for ck in gold["checkpoints"]:
        ctx.vds_step(q, p, ck["step"] - done)
        done = ck["step"]
        tau, qq = ctx.vds_stress(q, p)
        assert _rel(tau, ck["tau"]) <= 1e-3, (done, tau, ck["tau"])
        assert _rel(qq, ck["qq"]) <= 1e-3, (done, qq, ck["qq"])
    if name in PATHS_SEPARATE:
        return
    rows = q.cpu().numpy()[gold["rows"]].astype(np.float64)
    ref = np.asarray(gold["q_rows"])
    assert np.max(np.abs(rows - ref)) <= 1e-4 * np.max(np.abs(ref))


# ------------------------------------------------------- reduced path

@pytest.fixture(scope="module")
def reduced(orc, vds, ctx):
    # a basis whose span holds the bonds of the equilibrium cloud itself (so
    # that the lifted state is that cloud, not a collapsed one), completed by
    # bonds of other seeded clouds: the columns of 4 clouds x 3 bonds,
    # orthonormalised, the first r = 10 kept
    r, h = 10, 0.87
    cols = []
    for seed in (0, 1, 2, 3):
        c = inputs.equilibrium_cloud(N_FULL, NB, S, seed=seed).astype(np.float64)
        cols += [c[:, S * k:S * k + S].reshape(-1) for k in range(NB)]
    Phi, _ = np.linalg.qr(np.stack(cols, axis=1)[:, :r])
    Phi32 = np.ascontiguousarray(Phi.astype(np.float32))
    Phi = Phi32.astype(np.float64)
    kap = inputs.shear_kappa(S, 1.0)
    basis = ctx.pod_load(torch.from_numpy(Phi32).cuda(), S, kappa=kap)
    q0 = inputs.equilibrium_cloud(N_FULL, NB, S, seed=0).astype(np.float64)
    P0 = orc.project(Phi, q0, S, NB).astype(np.float32).astype(np.float64)
    yield dict(Phi=Phi, basis=basis, P0=P0, h=h, kap=kap, r=r)
    basis.free()


def test_brownian_matrices_at_full_size(orc, vds, ctx, reduced):
    R = reduced
    q = orc.lift(R["Phi"], R["P0"], S, NB)
    B1o, B2o, _ = orc.x_b(R["Phi"], q, R["h"], S)
    B1, B2 = ctx.pod_brownian(R["basis"], _dev(R["P0"]), N_FULL, NB * S, vds.params(NB, S, h=R["h"]))
    assert _rel(B1, B1o) <= 1e-4, _rel(B1, B1o)
    assert _rel(B2, B2o) <= 1e-4, _rel(B2, B2o)


def test_mode2_across_a_refresh_at_full_size(orc, vds, ctx, reduced):
    R = reduced
    steps, every = 61, 60
    po = orc.params(NB, S, h=R["h"], dt=0.005, kappa=R["kap"])
    pg = vds.params(NB, S, h=R["h"], dt=0.005, kappa=R["kap"])
    P = _dev(R["P0"])
    ctx.pod_step(R["basis"], P, N_FULL, NB * S, pg, nsteps=steps, refresh_every=every, mode=2)
    P_o = orc.reduced_run(R["P0"], R["Phi"], po, steps, every)
    assert _rel(P.cpu().numpy(), P_o) <= 1e-4, _rel(P.cpu().numpy(), P_o)


# ------------------------------------------------------- implicit steps

def test_implicit_steps_at_full_size(orc, vds, ctx):
    # two steps in one call: the first from q*, the second warm-started
    nsteps = 2
    h, dt = 0.87, 0.005
    kap = inputs.shear_kappa(S, 1.0)
    q32 = inputs.equilibrium_cloud(N_FULL, NB, S, seed=0)
    q = _dev(q32)
    pg = vds.params(NB, S, h=h, dt=dt, kappa=kap, scheme=1, tol=1e-6, jfloor=1e-9)
    its = ctx.vds_step(q, pg, nsteps, want_iters=True)
    q_o, its_o, _ = orc.implicit_steps(q32.astype(np.float64), orc.params(NB, S, h=h, dt=dt, kappa=kap),
                                       nsteps)
    assert np.max(np.abs(q.cpu().numpy() - q_o)) <= 1e-5 * np.max(np.abs(q_o)), (its, its_o)
    tau_o, qq_o = orc.stress(q_o, orc.params(NB, S, h=h, dt=dt, kappa=kap))
    tau, qq = ctx.vds_stress(q, pg)
    assert _rel(tau, tau_o) <= 1e-4 and _rel(qq, qq_o) <= 1e-4
