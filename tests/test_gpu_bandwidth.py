"""GPU parity of the bandwidth rules (Sec. 2.2, Eq. model_bandwidth) against
the FP64 oracle.  The median rule selects exactly on FP32 squared distances,
so the selected distance may differ from the FP64 one only by FP32 rounding
of the squared distances (<= ~2.4e-7 relative): tolerance 1e-6 relative."""
import numpy as np
import pytest

from paper_2603_12550_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12550_gb300 import build
    build.build()
    from paper_2603_12550_gb300 import vds
    c = vds.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("N,nb,s", [(2, 1, 2), (3, 1, 3), (64, 3, 3), (1000, 3, 3), (2048, 1, 2),
                                    (333, 2, 3), (777, 5, 3)])
def test_median_bandwidth_matches_oracle(orc, ctx, N, nb, s):
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=N)
    h = ctx.vds_bandwidth(torch.from_numpy(q32).cuda(), 0)
    h_o = orc.median_bandwidth(q32.astype(np.float64))
    assert abs(h / h_o - 1) <= 1e-6


def test_median_with_duplicates(orc, ctx):
    # many coincident particles: zero distances, ties at the median
    q32 = np.repeat(inputs.equilibrium_cloud(40, 3, 3, seed=2), 5, axis=0)
    h = ctx.vds_bandwidth(torch.from_numpy(q32).cuda(), 0)
    h_o = orc.median_bandwidth(q32.astype(np.float64))
    assert abs(h - h_o) <= 1e-6 * max(h_o, 1e-30)


@pytest.mark.parametrize("N,nb,s", [(5000, 1, 3), (1000, 3, 3), (16384, 1, 2)])
def test_silverman_matches_oracle(orc, ctx, N, nb, s):
    q32 = inputs.equilibrium_cloud(N, nb, s, seed=3)
    h = ctx.vds_bandwidth(torch.from_numpy(q32).cuda(), 1)
    assert abs(h / orc.silverman_bandwidth(q32.astype(np.float64)) - 1) <= 1e-9


def test_full_size_chain4_median_brackets_rank(orc, ctx):
    # N = 65536, D = 9: the exact FP64 order statistic lies within 1e-6 of the
    # selected distance (pair counts by the oracle, O(N^2) on the host).
    N = 65536
    q32 = inputs.equilibrium_cloud(N, 3, 3, seed=0)
    h = ctx.vds_bandwidth(torch.from_numpy(q32).cuda(), 0)
    med = h * np.sqrt(2 * np.log(N))
    M = N * (N - 1) // 2
    k = (M - 1) // 2
    q64 = q32.astype(np.float64)
    lt, _ = orc.count_pairs(q64, (med * (1 - 1e-6)) ** 2)
    _, le = orc.count_pairs(q64, (med * (1 + 1e-6)) ** 2)
    assert lt <= k < le
