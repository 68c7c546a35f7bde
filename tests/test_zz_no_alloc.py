"""The allocation-free entry point vds_energy_grad_noalloc, for callers that
cannot allocate device memory when they evaluate the density and gradient
(e.g. a solver that reserves its whole device-memory budget up front), gives
the same energy, gradient and density as vds_energy_grad, on two calls in a
row through the C ABI, and rejects sizes beyond its fixed scratch.

Kept in a file that pytest collects last, so that a run stopping at its first
failure has already run every other test.
"""
import ctypes

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


def _call_noalloc(vds, q, p, g, rho):
    N, D = q.shape
    E = ctypes.c_double()
    st = vds.lib.vds_energy_grad_noalloc(q.data_ptr(), N, D, ctypes.byref(p), ctypes.byref(E),
                                         g.data_ptr(), rho.data_ptr(),
                                         torch.cuda.current_stream().cuda_stream)
    return st, E.value


def test_noalloc_matches_energy_grad_on_two_calls(vds):
    ctx = vds.Context(0)
    # two different problems back to back: the second call must not see the
    # first call's leftovers in the shared scratch
    for N, nb, s, h, seed in [(3000, 3, 3, 0.9, 1), (777, 1, 2, 0.3, 2)]:
        D = nb * s
        q = torch.from_numpy(inputs.equilibrium_cloud(N, nb, s, seed=seed)).cuda()
        p = vds.params(nb, s, h=h)
        g_ref, rho_ref = torch.empty_like(q), torch.empty(N, device="cuda")
        E_ref = ctx.vds_energy_grad(q, p, g=g_ref, rho=rho_ref)
        g, rho = torch.empty_like(q), torch.empty(N, device="cuda")
        st, E = _call_noalloc(vds, q, p, g, rho)
        assert st == vds.VDS_OK, vds.strerror(st)
        assert abs(E - E_ref) <= 1e-5 * (1 + abs(E_ref))
        assert torch.max(torch.abs(rho - rho_ref) / rho_ref).item() <= 1e-5
        assert torch.max(torch.abs(g - g_ref)).item() <= 1e-5 * torch.max(torch.abs(g_ref)).item()
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(vds):
    N = vds.VDS_NOALLOC_MAX_N + 1
    q = torch.zeros((N, 9), device="cuda")
    g, rho = torch.empty_like(q), torch.empty(N, device="cuda")
    st, _ = _call_noalloc(vds, q, vds.params(3, 3, h=0.9), g, rho)
    assert st == vds.VDS_ESIZE
    assert "fixed-size" in vds.strerror(st)
