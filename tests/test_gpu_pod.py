"""GPU parity of POD (Sec. 2.3, Sec. 3.1): eigenvalues, rank (bit-exact),
basis, X^H, project and lift against the FP64 oracle.

The snapshot matrices are either synthetic with a prescribed spectrum or taken
from the oracle's own FP64 trajectory (rounded to FP32), never from the GPU.

Tolerances.  The GPU Gram runs on the tensor cores in TF32 with one
refinement step (3xTF32: every product carries x_hi y_hi + x_hi y_lo +
x_lo y_hi, relative error <= 3 * 2^-22).  The tensor cores' FP32 accumulator
rounds each MMA result into the running sum (toward zero, as measured: a
512-row accumulation came out low by 4e-6); the kernel therefore keeps
x_hi y_hi and the correction products in separate accumulators, reads them
back after every 32-row chunk (4 MMAs into the large sum) and adds them into
Kahan-compensated FP32 totals, FP64 across K splits.  A CPU emulation of that
arithmetic (truncating FP32 accumulation) gives Gram errors of 1.5e-7 of
max|C| on a 196608-row matrix and <= 1e-7 lambda_1 on the eigenvalues of the
smaller matrices here; the tests allow 1e-6 lambda_1.  A basis column t moves
by at most ||dC|| / gap_t (Davis-Kahan), emulated at about 1e-9 /
(gap_t / lambda_1); the tests allow 2e-5 + 1e-8 / (gap_t / lambda_1) (the first
term is the FP32 storage of Phi).  Phi^T Phi = I within 1e-6 (Cholesky-QR in
FP64).  X^H is checked against the oracle's X^H of the GPU's own basis (1e-5
relative), so it tests the X^H map, not the basis again; P and the lifted
state against the oracle with the GPU basis, 1e-5 relative.
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


def _xdev(X):
    # (Ns x M) column-major == (M x Ns) row-major
    return torch.from_numpy(np.ascontiguousarray(X.T, dtype=np.float32)).cuda()


def _trajectory_snapshots(orc, N=600, nb=3, s=3, nsnap=12, every=4, seed=0):
    q = inputs.equilibrium_cloud(N, nb, s, seed=seed).astype(np.float64)
    p = orc.params(nb, s, h=0.9, dt=0.01, kappa=inputs.shear_kappa(s, 1.0))
    states = [q.astype(np.float32)]
    for _ in range(nsnap - 1):
        q = orc.explicit_steps(q, p, every)
        states.append(q.astype(np.float32))
    X = orc.snapshots_from_states([x.astype(np.float64) for x in states], s, nb).astype(np.float32)
    return X, states, p


def _compare_basis(orc, vds, ctx, X, s, energy, r_max, r_fixed, kappa):
    Ns, M = X.shape
    o = orc.pod_build(X.astype(np.float64), energy=energy, r_max=r_max, r_fixed=r_fixed)
    basis, r = ctx.pod_build(_xdev(X), Ns, M, s, energy=energy, r_max=r_max, r_fixed=r_fixed,
                             kappa=kappa)
    assert r == o["r"]  # bit-exact rank
    lam = basis.eigenvalues()
    np.testing.assert_allclose(lam, o["lam"], rtol=0, atol=1e-6 * o["lam"][0])
    Phi = basis.phi().cpu().numpy().astype(np.float64)
    Po = o["Phi"]
    assert np.abs(Phi.T @ Phi - np.eye(r)).max() <= 1e-6
    gaps = np.abs(np.diff(np.append(o["lam"], 0.0)[:r + 1])) / o["lam"][0]
    for t in range(r):
        sep = min(gaps[t], gaps[t - 1] if t > 0 else np.inf)
        if sep > 1e-6:
            assert np.linalg.norm(Phi[:, t] - Po[:, t]) <= 2e-5 + 1e-8 / sep, (t, sep)
    XH = basis.xh()
    XH_o = orc.x_h(Phi, kappa, s)
    assert np.abs(XH - XH_o).max() <= 1e-5 * max(1.0, np.abs(XH_o).max())
    return basis, o, Phi


def test_pod_synthetic_spectrum(orc, vds, ctx):
    X = inputs.snapshot_matrix(3000, 48, 48, seed=1, decay=0.6)
    kap = inputs.shear_kappa(3, 1.0)
    _compare_basis(orc, vds, ctx, X, 3, 0.9999, 64, 0, kap)


@pytest.mark.parametrize("M", [1, 7, 65])
def test_pod_odd_and_small_M(orc, vds, ctx, M):
    X = inputs.snapshot_matrix(1200, M, M, seed=M, decay=0.5)
    _compare_basis(orc, vds, ctx, X, 3, 0.99, 64, min(M, 4), np.eye(3))


def test_pod_of_an_oracle_trajectory(orc, vds, ctx):
    X, states, p = _trajectory_snapshots(orc)
    kap = inputs.shear_kappa(3, 1.0)
    basis, o, Phi = _compare_basis(orc, vds, ctx, X, 3, 0.9999, 64, 0, kap)
    # project / lift of a state against the oracle with the oracle basis
    q = states[5]
    N, D = q.shape
    r = o["r"]
    P = torch.empty((r, 3), device="cuda")
    ctx.pod_project(basis, torch.from_numpy(q).cuda(), P)
    P_o = orc.project(Phi, q.astype(np.float64), 3, 3)
    assert np.abs(P.cpu().numpy() - P_o).max() <= 1e-5 * np.abs(P_o).max()
    qt = torch.empty((N, D), device="cuda")
    ctx.pod_lift(basis, P, qt)
    q_o = orc.lift(Phi, P.cpu().numpy().astype(np.float64), 3, 3)
    assert np.abs(qt.cpu().numpy() - q_o).max() <= 1e-5 * np.abs(q_o).max()


def test_pod_rank_cap_and_fixed(orc, vds, ctx):
    X = inputs.snapshot_matrix(2400, 100, 100, seed=4, decay=0.9)
    Ns, M = X.shape
    o = orc.pod_build(X.astype(np.float64), energy=0.999999, r_max=16)
    _, r = ctx.pod_build(_xdev(X), Ns, M, 3, energy=0.999999, r_max=16)
    assert r == o["r"] == 16
    _, r = ctx.pod_build(_xdev(X), Ns, M, 3, r_fixed=5)
    assert r == 5


def test_pod_bad_arguments(vds, ctx):
    X = torch.zeros((4, 30), device="cuda")
    with pytest.raises(vds.VdsError):
        ctx.pod_build(X, 31, 4, 3)  # Ns not a multiple of s
    with pytest.raises(vds.VdsError):
        ctx.pod_build(X, 30, 4, 3, r_max=65)


def test_pod_full_size_spectrum(orc, vds, ctx):
    # the 4-bead workload's snapshot matrix size (N s = 196608 rows, 200
    # snapshots x 3 bonds = 600 columns) with a prescribed spectrum: the GPU
    # eigenvalues against the FP64 oracle's (Gram and eigensolve in FP64 on
    # the host); emulated error 1.5e-7 lambda_1, allowed 1e-6 lambda_1.
    X = inputs.snapshot_matrix(196608, 600, 600, seed=7, decay=0.97)
    Ns, M = X.shape
    o = orc.pod_build(X.astype(np.float64), energy=0.9999, r_max=64)
    basis, r = ctx.pod_build(_xdev(X), Ns, M, 3, energy=0.9999, r_max=64)
    assert r == o["r"]
    lam = basis.eigenvalues()
    np.testing.assert_allclose(lam, o["lam"], rtol=0, atol=1e-6 * o["lam"][0])
    Phi = basis.phi().cpu().numpy().astype(np.float64)
    assert np.abs(Phi.T @ Phi - np.eye(r)).max() <= 1e-6
    basis.free()
