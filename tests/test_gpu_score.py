"""GPU parity of the score surrogate's tensor-core (tcgen05, BF16 operands,
FP32 accumulation) forward and backward passes against the FP64 oracle
(oracle/mlp.py), and end-to-end training on the GPU to the Gaussian score.

Tolerances derived from BF16 rounding (2^-9 relative per rounding, four
layers): outputs 2e-2 relative (Frobenius), loss 2e-2, per-layer gradients
5e-2 relative (Frobenius)."""
import numpy as np
import pytest

from oracle import mlp
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


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def _layers(seed, D=9):
    layers = inputs.mlp_init((D, 256, 256, 256, D), seed=seed)
    rng = np.random.default_rng(seed + 1)
    return [(W, (rng.standard_normal(b.shape) * 0.1).astype(np.float32)) for W, b in layers]


@pytest.mark.parametrize("N", [1000, 128, 1])
def test_forward_matches_oracle(vds, ctx, N):
    layers = _layers(0)
    net = vds.Score(ctx, 9, layers)
    x = np.random.default_rng(N).standard_normal((N, 9)).astype(np.float32)
    out = torch.empty((N, 9), device="cuda")
    net.eval(torch.from_numpy(x).cuda(), out)
    s_o, _ = mlp.forward(mlp.as64(layers), x.astype(np.float64))
    assert _rel(out.cpu().numpy(), s_o) <= 2e-2


def _bf16(a):
    """Round to the nearest BF16 (ties to even) through FP32, as the kernels
    round their FP32 values; returned as float64."""
    f = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    f = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16
    return f.astype(np.uint32).view(np.float32).astype(np.float64)


def _forward_bf16_points(layers, x):
    """The oracle's forward with BF16 rounding applied where the inference
    kernel rounds (input, weights, hidden activations); FP64 otherwise."""
    lo = mlp.as64(layers)
    h = _bf16(x)
    for i, (W, b) in enumerate(lo):
        z = h @ _bf16(W).T + b
        h = _bf16(mlp.silu(z)) if i < len(lo) - 1 else z
    return h


@pytest.mark.parametrize("N", [1, 127, 129, 19457, 100003])
def test_fused_inference_per_tile(vds, ctx, N):
    # one persistent launch covers every 128-row tile; with 100003 rows each
    # CTA takes 5 or 6 tiles (three rounds of the two in-flight slots, the
    # last one half empty on some CTAs).  Every tile is checked on its own
    # against the FP64 forward with the kernel's BF16 rounding points, and
    # the rows past N are left untouched.
    layers = _layers(11)
    net = vds.Score(ctx, 9, layers)
    x = np.random.default_rng(N + 5).standard_normal((N, 9)).astype(np.float32)
    buf = torch.full((N + 64, 9), 12345.0, device="cuda")
    net.eval(torch.from_numpy(x).cuda(), buf[:N])
    got = buf.cpu().numpy()
    assert np.all(got[N:] == 12345.0)
    got = got[:N]
    ref = _forward_bf16_points(layers, x)
    worst = 0.0
    for t0 in range(0, N, 128):
        worst = max(worst, _rel(got[t0:t0 + 128], ref[t0:t0 + 128]))
    assert worst <= 6e-3, worst
    s_o, _ = mlp.forward(mlp.as64(layers), x.astype(np.float64))
    assert _rel(got, s_o) <= 2e-2


@pytest.mark.parametrize("D", [2, 6, 16])
def test_fused_inference_other_dimensions(vds, ctx, D):
    # the input block holds D <= 16 coordinates in its first two 8-column
    # groups and the output layer stores the first D of its 16 columns
    layers = _layers(21 + D, D=D)
    net = vds.Score(ctx, D, layers)
    N = 3 * 128 + 5
    x = np.random.default_rng(D).standard_normal((N, D)).astype(np.float32)
    out = torch.empty((N, D), device="cuda")
    net.eval(torch.from_numpy(x).cuda(), out)
    got = out.cpu().numpy()
    ref = _forward_bf16_points(layers, x)
    for t0 in range(0, N, 128):
        assert _rel(got[t0:t0 + 128], ref[t0:t0 + 128]) <= 6e-3


def test_inference_follows_parameter_updates(vds, ctx):
    # the packed weight stream of the inference kernel is rebuilt after a
    # training step and after set_params
    layers = _layers(12)
    net = vds.Score(ctx, 9, layers)
    x = np.random.default_rng(13).standard_normal((3000, 9)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    out = torch.empty((3000, 9), device="cuda")
    net.eval(xd, out)
    xb, eps = inputs.dsm_batch(x, 512, seed=14)
    net.train_step(torch.from_numpy(xb).cuda(), torch.from_numpy(eps).cuda(), 0.8, 1e-2)
    net.eval(xd, out)
    assert _rel(out.cpu().numpy(), _forward_bf16_points(net.params(), x)) <= 6e-3
    layers2 = _layers(15)
    net.set_params(layers2)
    net.eval(xd, out)
    assert _rel(out.cpu().numpy(), _forward_bf16_points(layers2, x)) <= 6e-3


def test_loss_and_gradients_match_oracle(vds, ctx):
    layers = _layers(1)
    net = vds.Score(ctx, 9, layers)
    x, eps = inputs.dsm_batch(np.random.default_rng(2).standard_normal((5000, 9)).astype(np.float32), 512, seed=3)
    sigma = 0.8
    loss, grads = net.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(eps).cuda(), sigma)
    loss_o, grads_o = mlp.dsm_grad(mlp.as64(layers), x, eps, sigma)
    assert abs(loss - loss_o) <= 2e-2 * loss_o
    for (gW, gb), (oW, ob) in zip(grads, grads_o):
        assert _rel(gW, oW) <= 5e-2
        assert _rel(gb, ob) <= 5e-2


def test_adam_steps_follow_oracle(vds, ctx):
    layers = _layers(4)
    net = vds.Score(ctx, 9, layers)
    data = np.random.default_rng(5).standard_normal((5000, 9)).astype(np.float32)
    lo = mlp.as64(layers)
    m, v = mlp.adam_init(lo)
    for t in range(1, 4):
        x, eps = inputs.dsm_batch(data, 256, seed=10 + t)
        net.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(eps).cuda(), 0.8, 1e-3)
        _, g = mlp.dsm_grad(lo, x, eps, 0.8)
        lo, m, v = mlp.adam_step(lo, g, m, v, t, lr=1e-3)
    got = net.params()
    for (W0, b0), (Wg, bg), (Wo, bo) in zip(layers, got, lo):
        # the updates agree; Adam normalises the step so BF16 gradient noise
        # matters only where a gradient component is near zero
        assert _rel(Wg - W0, Wo - W0) <= 0.15


def test_gpu_training_learns_the_gaussian_score(vds, ctx):
    s0, sigma = 1.0, 0.5
    data = (np.random.default_rng(6).standard_normal((50000, 9)) * s0).astype(np.float32)
    net = vds.Score(ctx, 9, inputs.mlp_init((9, 256, 256, 256, 9), seed=7))
    for t in range(1, 601):
        x, eps = inputs.dsm_batch(data, 1024, seed=1000 + t)
        net.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(eps).cuda(), sigma, 1e-3, want_loss=False)
    z = (np.random.default_rng(8).standard_normal((2000, 9)) * 0.8).astype(np.float32)
    out = torch.empty((2000, 9), device="cuda")
    net.eval(torch.from_numpy(z).cuda(), out)
    target = -z / (s0 ** 2 + sigma ** 2)
    assert _rel(out.cpu().numpy(), target) < 0.15


def test_row_gather_equals_gathered_batch(vds, ctx):
    # training batches drawn as rows of a device pool give the same loss and
    # gradients as the gathered rows passed directly
    layers = _layers(9)
    net = vds.Score(ctx, 9, layers)
    pool = np.random.default_rng(9).standard_normal((3000, 9)).astype(np.float32)
    rows, eps = inputs.dsm_rows(3000, 256, 9, seed=1)
    l1, g1 = net.loss_grad(torch.from_numpy(pool).cuda(), torch.from_numpy(eps).cuda(), 0.7,
                           rows=torch.from_numpy(rows).cuda())
    l2, g2 = net.loss_grad(torch.from_numpy(pool[rows]).cuda(), torch.from_numpy(eps).cuda(), 0.7)
    assert l1 == l2
    for (a, b), (c, d) in zip(g1, g2):
        assert np.array_equal(a, c) and np.array_equal(b, d)


def test_fit_gradients_match_oracle(vds, ctx):
    layers = _layers(12)
    net = vds.Score(ctx, 9, layers)
    rng = np.random.default_rng(13)
    pool = rng.standard_normal((2000, 9)).astype(np.float32)
    tgt = (-0.6 * pool + 0.1 * rng.standard_normal(pool.shape)).astype(np.float32)
    rows = rng.integers(0, 2000, 384).astype(np.int32)
    loss, grads = net.fit_step(torch.from_numpy(pool).cuda(), torch.from_numpy(tgt).cuda(), 0.0,
                               rows=torch.from_numpy(rows).cuda(), want_grads=True)
    loss_o, grads_o = mlp.fit_grad(mlp.as64(layers), pool[rows], tgt[rows])
    assert abs(loss - loss_o) <= 2e-2 * loss_o
    for (gW, gb), (oW, ob) in zip(grads, grads_o):
        assert _rel(gW, oW) <= 5e-2
        assert _rel(gb, ob) <= 5e-2
