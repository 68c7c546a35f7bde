"""The allocation-free entry point vds_energy_grad_noalloc, for callers that
cannot allocate device memory when they evaluate the density and gradient
(e.g. a solver that reserves its whole device-memory budget up front), gives
the same energy, gradient and density as vds_energy_grad and as the FP64
oracle, on two calls in a row through the C ABI, also at its largest size
(where its gradient pass runs on a cut-down grid so that the partial sums fit
the fixed scratch), rejects sizes beyond its fixed scratch, and refuses a
stream that is being captured.

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


def _check_against_oracle(orc, q, p_o, E, g, rho):
    E_o, g_o, rho_o = orc.energy_grad(q.cpu().numpy().astype(np.float64), p_o)
    assert abs(E - E_o) <= 1e-5 * (1 + abs(E_o)), (E, E_o)
    assert np.max(np.abs(rho.cpu().numpy() - rho_o) / rho_o) <= 1e-5
    assert np.max(np.abs(g.cpu().numpy() - g_o)) <= 1e-5 * np.max(np.abs(g_o))


def test_noalloc_matches_energy_grad_on_two_calls(vds, orc):
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
        _check_against_oracle(orc, q, orc.params(nb, s, h=h), E, g, rho)
    ctx.close()


# gradient-pass i-tile sizes (threads x particles per thread) of the pair
# kernel at D = 9 and D = 16, and the fixed partial-sum buffer (4 MiB)
_GRAD_TI = {9: 384 * 3, 16: 256 * 2}
_PART_BYTES = 4 << 20


@pytest.mark.parametrize("nb,s", [(3, 3), (8, 2)])
def test_noalloc_at_its_largest_size(vds, orc, nb, s):
    N, D = vds.VDS_NOALLOC_MAX_N, nb * s
    # with one CTA per SM or more, some i-tile is split over at least
    # ceil(G / n_itiles) CTAs, each writing its own FP64 partial of TI x D:
    # more than the buffer holds, so the grid-cutting loop must run
    n_itiles = -(-N // _GRAD_TI[D])
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    need = n_itiles * (-(-sms // n_itiles)) * _GRAD_TI[D] * D * 8
    assert need > _PART_BYTES, need
    q = torch.from_numpy(inputs.equilibrium_cloud(N, nb, s, seed=5)).cuda()
    p = vds.params(nb, s, h=0.8)
    ctx = vds.Context(0)
    g_ref, rho_ref = torch.empty_like(q), torch.empty(N, device="cuda")
    E_ref = ctx.vds_energy_grad(q, p, g=g_ref, rho=rho_ref)
    ctx.close()
    for _ in range(2):
        g, rho = torch.full_like(q, float("nan")), torch.full((N,), float("nan"), device="cuda")
        st, E = _call_noalloc(vds, q, p, g, rho)
        assert st == vds.VDS_OK, vds.strerror(st)
        assert abs(E - E_ref) <= 1e-5 * (1 + abs(E_ref))
        assert torch.max(torch.abs(rho - rho_ref) / rho_ref).item() <= 1e-5
        assert torch.max(torch.abs(g - g_ref)).item() <= 1e-5 * torch.max(torch.abs(g_ref)).item()
    _check_against_oracle(orc, q, orc.params(nb, s, h=0.8), E, g, rho)


def test_noalloc_rejects_sizes_beyond_its_scratch(vds):
    N = vds.VDS_NOALLOC_MAX_N + 1
    q = torch.zeros((N, 9), device="cuda")
    g, rho = torch.empty_like(q), torch.empty(N, device="cuda")
    st, _ = _call_noalloc(vds, q, vds.params(3, 3, h=0.9), g, rho)
    assert st == vds.VDS_ESIZE
    assert "fixed-size" in vds.strerror(st)


def test_noalloc_refuses_stream_capture(vds):
    # a call on a stream being captured returns VDS_EARG before it enqueues
    # anything (it would copy to the host and synchronise), the capture stays
    # valid, and the entry point works again afterwards
    N = 256
    q = torch.from_numpy(inputs.equilibrium_cloud(N, 3, 3, seed=3)).cuda()
    g, rho = torch.empty_like(q), torch.empty(N, device="cuda")
    p = vds.params(3, 3, h=0.8)
    st, _ = _call_noalloc(vds, q, p, g, rho)  # the device's one-time set-up, outside any capture
    assert st == vds.VDS_OK
    g_ref = g.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        st_cap, _ = _call_noalloc(vds, q, p, g, rho)
        g.mul_(2.0)
    assert st_cap == vds.VDS_EARG
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(g, 2.0 * g_ref)
    st, _ = _call_noalloc(vds, q, p, g, rho)
    assert st == vds.VDS_OK
    assert torch.equal(g, g_ref)
