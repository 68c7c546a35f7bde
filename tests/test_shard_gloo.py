"""The row-sharded explicit step (paper_2603_12550_gb300/shard.py) on CPU
ranks: the partition covers every particle row once, and two or three gloo
ranks (127.0.0.1), each evaluating only its own rows, end a run of steps with
exactly the state that one rank computing every row reaches -- bit for bit,
because each row's arithmetic does not depend on the split -- and that state
is the FP64 oracle's whole-cloud explicit steps (Appendix A).

The per-rank pair work here is the oracle's row-restricted step, so the test
checks the partition, the two all-gathers and the step order, not the GPU
kernels (tests/test_gpu_shard_rows.py runs the library's row passes)."""
import os
import socket

import numpy as np
import pytest

from paper_2603_12550_gb300 import inputs
from paper_2603_12550_gb300.shard import RowShardedStepper, partition

torch = pytest.importorskip("torch")

NB, S, H_BW, DT = 3, 3, 0.8, 0.005


class OracleRows:
    """The oracle's row-restricted passes on CPU float64 tensors."""

    def __init__(self, p):
        import oracle
        oracle.build()
        self.o, self.p = oracle, p

    def density_rows(self, q_all, row0, nrows, rho_out):
        rows = np.arange(row0, row0 + nrows)
        rho_out.copy_(torch.from_numpy(self.o.density_rows(q_all.numpy(), self.p.h, rows)))

    def step_rows(self, q_all, rho_all, row0, nrows, q_out):
        rows = np.arange(row0, row0 + nrows)
        q_out.copy_(torch.from_numpy(self.o.explicit_step_rows(q_all.numpy(), self.p, rho_all.numpy(), rows)))


def _params():
    import oracle
    return oracle.params(NB, S, h=H_BW, dt=DT, kappa=inputs.shear_kappa(S, 1.0))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, N, nsteps, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q0 = torch.from_numpy(inputs.equilibrium_cloud(N, NB, S, seed=3).astype(np.float64))
        st = RowShardedStepper(OracleRows(_params()), N, NB * S, rank, world, dist=dist, dtype=torch.float64)
        st.load(q0)
        st.step(nsteps)
        out[rank] = st.q.numpy().copy()
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_partition_covers_every_row_once():
    for N, world in [(301, 2), (301, 3), (5, 4), (8, 8), (65536, 8), (7, 1)]:
        ranges, C = partition(N, world)
        assert len(ranges) == world and C == -(-N // world)
        rows = np.concatenate([np.arange(a, a + n) for a, n in ranges])
        np.testing.assert_array_equal(rows, np.arange(N))
        assert all(n <= C for _, n in ranges)
    assert partition(5, 4)[0] == [(0, 2), (2, 2), (4, 1), (5, 0)]


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_steps_equal_one_rank_bit_for_bit(world):
    import torch.multiprocessing as mp
    N, nsteps = 301, 3
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), N, nsteps, out), nprocs=world, join=True,
                       start_method="spawn")
    q0 = torch.from_numpy(inputs.equilibrium_cloud(N, NB, S, seed=3).astype(np.float64))
    one = RowShardedStepper(OracleRows(_params()), N, NB * S, dtype=torch.float64)
    one.load(q0)
    ref = one.step(nsteps).numpy()
    for rank in range(world):
        np.testing.assert_array_equal(out[rank], ref)
    import oracle
    whole = oracle.explicit_steps(q0.numpy(), _params(), nsteps)
    np.testing.assert_allclose(ref, whole, rtol=1e-12, atol=1e-13)
