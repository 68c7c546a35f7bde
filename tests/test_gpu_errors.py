"""Error statuses raised on the device and read by the host, triggered from
the host side only (no fault, trap or endless wait on the GPU):

- a NaN planted in the connector array q makes every density sum non-finite:
  vds_energy_grad and vds_step (explicit) report VDS_ENAN, and so does
  vds_bandwidth when the median pair distance itself is not finite;
- an implicit step allowed one minimiser iteration with a tolerance it cannot
  meet reports VDS_ENOCONV (Appendix A's implicit scheme solved by
  iteration: the solve did not finish);
- the bounded-wait pattern of every device-side wait, run on an mbarrier
  phase and a flag that nothing completes with a 50 ms limit, gives up and
  reports VDS_ETIMEOUT (vds_wait_selftest);

and after each, the same context evaluates a clean cloud exactly as the FP64
oracle does, i.e. the error left no stale flag or state behind.
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


def _clean_matches_oracle(orc, vds, ctx, N=1000, seed=3):
    nb, s, h = 3, 3, 0.9
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=seed)
    q = _dev(q32)
    g = torch.empty_like(q)
    p = vds.params(nb, s, h=h)
    E = ctx.vds_energy_grad(q, p, g=g)
    E_o, g_o, _ = orc.energy_grad(q32.astype(np.float64), orc.params(nb, s, h=h))
    assert abs(E - E_o) <= 1e-5 * (1 + abs(E_o))
    assert np.max(np.abs(g.cpu().numpy() - g_o)) <= 1e-5 * np.max(np.abs(g_o))


@pytest.mark.parametrize("N,row", [(1000, 17), (20001, 20000)])
def test_nan_in_q_is_reported_and_the_context_survives(orc, vds, ctx, N, row):
    nb, s = 3, 3
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=4)
    q32[row, 4] = np.nan
    q = _dev(q32)
    p = vds.params(nb, s, h=0.9, dt=0.005, kappa=inputs.shear_kappa(s, 1.0))
    with pytest.raises(vds.VdsError) as e:
        ctx.vds_energy_grad(q, p, g=torch.empty_like(q))
    assert e.value.code == vds.VDS_ENAN
    with pytest.raises(vds.VdsError) as e:
        ctx.vds_step(q, p, 3)
    assert e.value.code == vds.VDS_ENAN
    _clean_matches_oracle(orc, vds, ctx)


def test_nonfinite_median_is_reported(orc, vds, ctx):
    # one NaN row leaves most pair distances finite and the median with them;
    # with 40 % of the rows NaN, 64 % of the pairs are, and the median is not
    N, nb, s = 2000, 3, 3
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=8)
    q32[::5, 0] = np.nan
    q32[1::5, 3] = np.nan
    with pytest.raises(vds.VdsError) as e:
        ctx.vds_bandwidth(_dev(q32), rule=0)
    assert e.value.code == vds.VDS_ENAN
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=8)
    h = ctx.vds_bandwidth(_dev(q32), rule=0)
    assert h == pytest.approx(orc.median_bandwidth(q32.astype(np.float64)), rel=1e-6)


def test_minimiser_out_of_iterations_is_reported_and_the_context_survives(orc, vds, ctx):
    N, nb, s, h, dt = 600, 3, 3, 0.9, 0.01
    kap = inputs.shear_kappa(s, 1.0)
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=6)
    q = _dev(q32)
    p = vds.params(nb, s, h=h, dt=dt, kappa=kap, scheme=1, tol=1e-12, max_iter=1)
    with pytest.raises(vds.VdsError) as e:
        ctx.vds_step(q, p, 1)
    assert e.value.code == vds.VDS_ENOCONV
    # a normal implicit step from the same start still reaches the oracle's
    # minimiser
    q = _dev(q32)
    ctx.vds_step(q, vds.params(nb, s, h=h, dt=dt, kappa=kap, scheme=1, tol=1e-6), 1)
    q_o, _, _ = orc.implicit_steps(q32.astype(np.float64), orc.params(nb, s, h=h, dt=dt, kappa=kap), 1)
    assert np.max(np.abs(q.cpu().numpy() - q_o)) <= 1e-5 * np.max(np.abs(q_o))
    _clean_matches_oracle(orc, vds, ctx)


def test_bounded_waits_give_up_and_the_context_survives(orc, vds, ctx):
    import time
    t0 = time.perf_counter()
    assert ctx.vds_wait_selftest(0.05) == vds.VDS_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert ctx.vds_wait_selftest(0.01) == vds.VDS_ETIMEOUT
    _clean_matches_oracle(orc, vds, ctx)
