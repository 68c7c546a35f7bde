"""vds_density_tc (the kernel density of every particle, Sec. 2.2, with the
pair dot products on the tensor cores) against the FP64 oracle, element by
element: within 1e-4 relative everywhere and 1e-5 for the median particle on
equilibrium clouds of 1 to 20001 particles (one to many 128-row and
256-column tiles, ragged last tiles, several column splits), D = 6 and 9, and
at the full size N = 65536 against the library's exact FP32 pass; within
1e-3 (1e-4 median) on a cloud stretched five-fold, where the error of the
expanded form grows with |q|^2 / h^2.  The library uses it for the density at
the lifted state of the refresh (X^B, a sum over all particles, is tested
against the oracle at 1e-4 in test_gpu_reduced.py and at full size) and for
the density of the surrogate's subset check.
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


def _rel(got, want):
    return np.abs(got.astype(np.float64) - want) / want


@pytest.mark.parametrize("N,nb,h", [(1, 3, 0.9), (100, 3, 0.9), (129, 2, 0.7), (255, 3, 0.9), (257, 3, 0.8),
                                    (1000, 2, 0.6), (4097, 3, 0.9), (20001, 3, 0.85)])
def test_density_tc_matches_oracle(orc, vds, ctx, N, nb, h):
    q = inputs.equilibrium_cloud(N, nb, 3, seed=N)
    rho = torch.empty(N, device="cuda")
    ctx.vds_density_tc(torch.from_numpy(q).cuda(), vds.params(nb, 3, h=h), rho)
    want = orc.density(q.astype(np.float64), h)
    rel = _rel(rho.cpu().numpy(), want)
    assert rel.max() <= 1e-4, rel.max()
    assert np.median(rel) <= 1e-5, np.median(rel)


def test_density_tc_on_a_stretched_cloud(orc, vds, ctx):
    # a cloud stretched five-fold along one axis (as shear stretches it):
    # |q|^2 / h^2 up to several hundred, where the error of the expanded form
    # grows (measured: 3.4e-4 at the worst particle, a few 1e-5 typically)
    N = 3000
    q = inputs.equilibrium_cloud(N, 3, 3, seed=5)
    q[:, 0::3] *= 5.0
    h = 0.7
    rho = torch.empty(N, device="cuda")
    ctx.vds_density_tc(torch.from_numpy(q).cuda(), vds.params(3, 3, h=h), rho)
    want = orc.density(q.astype(np.float64), h)
    rel = _rel(rho.cpu().numpy(), want)
    assert rel.max() <= 1e-3 and np.median(rel) <= 1e-4, (rel.max(), np.median(rel))


def test_density_tc_at_full_size(vds, ctx):
    # N = 65536, D = 9: against the exact FP32 pass of vds_energy_grad
    N = 65536
    q = torch.from_numpy(inputs.equilibrium_cloud(N, 3, 3, seed=0)).cuda()
    p = vds.params(3, 3, h=0.868)
    rho = torch.empty(N, device="cuda")
    ctx.vds_density_tc(q, p, rho)
    g, rho_ref = torch.empty_like(q), torch.empty(N, device="cuda")
    ctx.vds_energy_grad(q, p, g=g, rho=rho_ref)
    rel = (torch.abs(rho.double() - rho_ref.double()) / rho_ref.double()).cpu().numpy()
    assert rel.max() <= 1e-4 and np.median(rel) <= 1e-5, (rel.max(), np.median(rel))


def test_density_tc_rejects_other_dimensions(vds, ctx):
    q = torch.zeros((64, 3), device="cuda")
    rho = torch.empty(64, device="cuda")
    with pytest.raises(vds.VdsError) as e:
        ctx.vds_density_tc(q, vds.params(1, 3, h=0.5), rho)
    assert e.value.code == vds.VDS_EARG
