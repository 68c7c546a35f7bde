"""Row-sharded explicit VDS steps over ranks.

The cost of a VDS step is its two O(N^2) pair sums (Sec. 1.2, The VDS Scheme
and its Limitation).  Here G ranks split them by particle rows: rank k owns
the contiguous rows [k C, k C + n_k), C = ceil(N / G), and evaluates those
rows against all N particles.  One explicit step (Appendix A) is then

  1. the density of the own rows               (library: vds_density_rows)
  2. all-gather of rho                          (N FP32)
  3. the gradient pass and Euler update of the own rows, with every rho
                                                (library: vds_grad_rows, mode 1)
  4. all-gather of the updated rows into q      (N x D FP32)

so every rank holds the whole state after each step, and the only exchange
is those two all-gathers.  The pair arithmetic runs in the CUDA library; this
module only partitions, allocates and calls the collectives (any
torch.distributed backend: NCCL between GPUs, gloo for the CPU tests).
"""
from __future__ import annotations


def partition(N: int, world: int):
    """Row ranges (row0, nrows) of every rank and the per-rank chunk C: rank k
    owns rows [k C, min(N, (k + 1) C)); trailing ranks may own none."""
    if N < 1 or world < 1:
        raise ValueError("N and world must be positive")
    C = -(-N // world)
    ranges = []
    for k in range(world):
        a = min(N, k * C)
        ranges.append((a, min(N, a + C) - a))
    return ranges, C


class GpuRows:
    """The per-rank pair work through the C ABI (device tensors)."""

    def __init__(self, ctx, p):
        self.ctx, self.p = ctx, p

    def density_rows(self, q_all, row0, nrows, rho_out):
        self.ctx.vds_density_rows(q_all, self.p, row0, nrows, rho_out)

    def step_rows(self, q_all, rho_all, row0, nrows, q_out):
        self.ctx.vds_grad_rows(q_all, self.p, rho_all, row0, nrows, q_out, mode=1)


class RowShardedStepper:
    """Explicit steps of one cloud of N particles (D coordinates each) split by
    rows over the ranks of `group` (torch.distributed; None with world = 1)."""

    def __init__(self, backend, N, D, rank=0, world=1, dist=None, group=None, device="cpu", dtype=None):
        import torch
        self.torch = torch
        self.backend, self.N, self.D = backend, int(N), int(D)
        self.rank, self.world, self.dist, self.group = int(rank), int(world), dist, group
        if self.world > 1 and dist is None:
            raise ValueError("world > 1 needs torch.distributed")
        self.ranges, self.C = partition(self.N, self.world)
        self.row0, self.nrows = self.ranges[self.rank]
        dt = dtype or torch.float32
        # the whole state lives in the gather buffer: its first N rows are q
        self.q_buf = torch.zeros((self.world * self.C, self.D), dtype=dt, device=device)
        self.rho_buf = torch.ones(self.world * self.C, dtype=dt, device=device)
        self.q_loc = torch.zeros((self.C, self.D), dtype=dt, device=device)
        self.rho_loc = torch.ones(self.C, dtype=dt, device=device)

    @property
    def q(self):
        return self.q_buf[:self.N]

    def load(self, q0):
        self.q_buf[:self.N].copy_(q0)

    def _gather(self, out, inp):
        if self.world == 1:
            out.copy_(inp)
            return
        if hasattr(self.dist, "all_gather_into_tensor"):
            try:
                self.dist.all_gather_into_tensor(out, inp, group=self.group)
                return
            except (RuntimeError, NotImplementedError):
                pass
        self.dist.all_gather(list(out.chunk(self.world)), inp, group=self.group)

    def step(self, nsteps=1):
        q_all, rho_all = self.q_buf[:self.N], self.rho_buf[:self.N]
        for _ in range(int(nsteps)):
            if self.nrows > 0:
                self.backend.density_rows(q_all, self.row0, self.nrows, self.rho_loc[:self.nrows])
            self._gather(self.rho_buf, self.rho_loc)
            if self.nrows > 0:
                self.backend.step_rows(q_all, rho_all, self.row0, self.nrows, self.q_loc[:self.nrows])
            self._gather(self.q_buf, self.q_loc)
        return self.q
