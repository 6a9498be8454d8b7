"""The surrogate network's CUDA kernels against the FP64 oracle MLP: forward outputs,
loss and every gradient component (FP32 tolerances), one Adam step against numpy Adam on
the oracle gradients, bitwise-reproducible training."""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu

WIDTHS = [5, 256, 256, 256, 4]


@pytest.fixture(scope="module")
def kd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2307_01571_gb300 import _build
    _build.build()
    from paper_2307_01571_gb300 import kd as mod
    return mod


def _data(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, WIDTHS[0])).astype(np.float32), rng.standard_normal((n, WIDTHS[-1])).astype(np.float32)


@pytest.mark.parametrize("batch", [1, 37, 300])
def test_forward_and_gradients_match_oracle(kd, batch):
    net = kd.MLP(WIDTHS)
    p = mlp.init_params(WIDTHS, 7)
    net.set_params(p)
    x, t = _data(batch, batch)
    y = net.forward(x)
    yr, _, _ = mlp.forward(p.astype(np.float64), WIDTHS, x.astype(np.float64))
    assert np.max(np.abs(y - yr)) <= 2e-5 * max(1.0, np.max(np.abs(yr)))
    loss, g = net.gradients(x, t)
    lr_, gr = mlp.loss_and_grad(p.astype(np.float64), WIDTHS, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - lr_) <= 2e-5 * max(1.0, lr_)
    assert np.max(np.abs(g - gr)) <= 1e-4 * max(1e-3, np.max(np.abs(gr)))
    assert np.array_equal(net.get_params(), p)
    net.close()


def test_adam_step_and_determinism(kd):
    import torch
    x, t = _data(128, 3)
    p0 = mlp.init_params(WIDTHS, 11)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    runs = []
    for _ in range(2):
        net = kd.MLP(WIDTHS)
        net.set_params(p0)
        for _ in range(5):
            net.train_step(xd.data_ptr(), td.data_ptr(), 128, 1e-3)
        torch.cuda.synchronize()
        runs.append(net.get_params())
        net.close()
    assert np.array_equal(runs[0], runs[1])
    # one step against numpy Adam on the oracle gradient
    net = kd.MLP(WIDTHS)
    net.set_params(p0)
    net.train_step(xd.data_ptr(), td.data_ptr(), 128, 1e-3)
    torch.cuda.synchronize()
    _, g = mlp.loss_and_grad(p0.astype(np.float64), WIDTHS, x.astype(np.float64), t.astype(np.float64))
    m = 0.1 * g
    v = 0.001 * g * g
    ref = p0 - 1e-3 * (m / 0.1) / (np.sqrt(v / 0.001) + 1e-8)
    got = net.get_params()
    big = np.abs(g) > 1e-4
    assert np.max(np.abs(got - ref)[big]) <= 1e-5
    net.close()


def test_training_reduces_loss(kd):
    import torch
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (512, 5)).astype(np.float32)
    t = np.stack([np.sin(2 * x[:, 0]) * x[:, 1], x[:, 2] ** 2, np.cos(x[:, 3] + x[:, 4]), x.sum(1) / 5], 1).astype(np.float32)
    net = kd.MLP(WIDTHS)
    net.set_params(mlp.init_params(WIDTHS, 2))
    l0, _ = net.gradients(x, t)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    for _ in range(400):
        net.train_step(xd.data_ptr(), td.data_ptr(), 512, 2e-3)
    torch.cuda.synchronize()
    l1, _ = net.gradients(x, t)
    assert l1 < 0.02 * l0, (l0, l1)
    net.close()


def test_gathered_minibatch_step_equals_plain_step(kd):
    """kd_mlp_train_step_gather selects the minibatch rows with the library's own gather
    kernel; the update equals kd_mlp_train_step on the same rows gathered on the host, bit
    for bit, and an index outside the sample range selects a row of zeros."""
    import torch
    x, t = _data(300, 9)
    p0 = mlp.init_params(WIDTHS, 4)
    rng = np.random.default_rng(1)
    steps = [rng.integers(0, 300, 64).astype(np.int32) for _ in range(4)]
    steps[-1][5] = 300                      # outside [0, n): a zero row
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    a = kd.MLP(WIDTHS)
    a.set_params(p0)
    for idx in steps:
        idev = torch.from_numpy(idx).cuda()
        a.train_step_gather(xd.data_ptr(), td.data_ptr(), 300, idev.data_ptr(), 64, 1e-3)
        torch.cuda.synchronize()
    b = kd.MLP(WIDTHS)
    b.set_params(p0)
    for idx in steps:
        ok = idx < 300
        xb = np.where(ok[:, None], x[np.minimum(idx, 299)], 0.0).astype(np.float32)
        tb = np.where(ok[:, None], t[np.minimum(idx, 299)], 0.0).astype(np.float32)
        xbd, tbd = torch.from_numpy(xb).cuda(), torch.from_numpy(tb).cuda()
        b.train_step(xbd.data_ptr(), tbd.data_ptr(), 64, 1e-3)
        torch.cuda.synchronize()
    assert np.array_equal(a.get_params(), b.get_params())
    a.close()
    b.close()


# BF16 products on the tensor cores: every operand rounded to 8 significand bits (relative
# 2^-9), sums over K in FP32; outputs within a few 2^-9 of the FP64 oracle's scale
BF16_TOL = 2e-2


@pytest.mark.parametrize("batch", [1, 37, 300])
def test_bf16_tensor_core_forward_and_gradients_match_oracle(kd, batch):
    net = kd.MLP(WIDTHS)
    net.set_precision(kd.KD_MLP_BF16)
    p = mlp.init_params(WIDTHS, 7)
    net.set_params(p)
    x, t = _data(batch, batch)
    y = net.forward(x)
    yr, _, _ = mlp.forward(p.astype(np.float64), WIDTHS, x.astype(np.float64))
    assert np.max(np.abs(y - yr)) <= BF16_TOL * max(1.0, np.max(np.abs(yr)))
    loss, g = net.gradients(x, t)
    lr_, gr = mlp.loss_and_grad(p.astype(np.float64), WIDTHS, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - lr_) <= BF16_TOL * max(1.0, lr_)
    assert np.max(np.abs(g - gr)) <= BF16_TOL * np.max(np.abs(gr))
    # the BF16 result is not the FP32 one (the tensor-core path really ran)
    net32 = kd.MLP(WIDTHS)
    net32.set_params(p)
    assert not np.array_equal(net32.forward(x), y)
    net.close()
    net32.close()


def test_bf16_training_reduces_loss_and_is_deterministic(kd):
    import torch
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (512, 5)).astype(np.float32)
    t = np.stack([np.sin(2 * x[:, 0]) * x[:, 1], x[:, 2] ** 2, np.cos(x[:, 3] + x[:, 4]), x.sum(1) / 5], 1).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    finals = []
    for _ in range(2):
        net = kd.MLP(WIDTHS)
        net.set_precision(kd.KD_MLP_BF16)
        net.set_params(mlp.init_params(WIDTHS, 2))
        l0, _ = net.gradients(x, t)
        for _ in range(400):
            net.train_step(xd.data_ptr(), td.data_ptr(), 512, 2e-3)
        torch.cuda.synchronize()
        l1, _ = net.gradients(x, t)
        assert l1 < 0.1 * l0, (l0, l1)
        finals.append(net.get_params())
        net.close()
    assert np.array_equal(finals[0], finals[1])
