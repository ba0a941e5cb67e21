"""The surrogate network's kernels (lb_mlp) against the numpy reference of
tests/mlp_reference.py: forward pass, gradients, the Adam step, and that
training fits a smooth field."""
import numpy as np
import pytest

from gpu_helpers import lib
from mlp_reference import adam_step, forward, grads, unpack

pytestmark = pytest.mark.gpu

# (n_fourier, width, depth, plain inputs): a small net, ragged against the
# 64-wide tiles of the products; and the surrogate's own shape (5 layers of
# 256, six plain inputs), which spans several tiles in every dimension
SHAPES = {"small": (3, 40, 4, 2), "surrogate": (4, 256, 5, 6)}


@pytest.fixture(params=list(SHAPES), ids=list(SHAPES))
def shape(request):
    return SHAPES[request.param]


def _net(shape, max_batch=300, seed=7):
    L = lib()
    nf, w, d, npl = shape
    return L.LBMlp(n_fourier=nf, width=w, depth=d, max_batch=max_batch, seed=seed, n_plain=npl)


def _inputs(n, seed, n_plain=2):
    rng = np.random.default_rng(seed)
    cols = [rng.uniform(0.2, 0.8, n)] + [rng.uniform(0, 1, n) for _ in range(n_plain)]
    x = np.stack(cols, axis=1)          # (De-like, ..., r-like, z)
    a, r, z = x[:, 0], x[:, n_plain - 1], x[:, n_plain]
    y = np.stack([1 + 0.01 * np.sin(2 * np.pi * z), a * np.sin(np.pi * r),
                  r * (1 - r), 0.1 * np.cos(2 * np.pi * z) * a], axis=1)
    return x.astype(np.float32), y.astype(np.float32)


def test_forward_matches_reference(shape):
    import torch
    NF, W, D, NP = shape
    net = _net(shape)
    rng = np.random.default_rng(3)
    p = rng.normal(0, 0.3 * (40 / W) ** 0.5, net.param_count()).astype(np.float32)
    net.set_params(p)
    mean, std = np.array([1.0, 0.1, 0.2, 0.0], np.float32), np.array([0.5, 2.0, 1.0, 0.25], np.float32)
    net.set_output_scale(mean, std)
    x, _ = _inputs(257, 1, NP)
    y = net.predict(torch.from_numpy(x).cuda()).cpu().numpy()
    Y, _ = forward(p.astype(np.float64), x, NF, W, D)
    ref = Y * std + mean
    assert np.abs(y - ref).max() <= 2e-5 * np.abs(ref).max()
    net.close()


def test_gradients_and_adam_step_match_reference(shape):
    import torch
    NF, W, D, NP = shape
    net = _net(shape)
    p0 = net.get_params()
    assert np.all(np.concatenate([b for _, b in unpack(p0, NF, W, D, NP)]) == 0)   # zero biases
    mean, std = np.array([1.0, 0.0, 0.1, 0.0], np.float32), np.array([0.01, 0.5, 0.1, 0.05], np.float32)
    net.set_output_scale(mean, std)
    x, y = _inputs(300, 2, NP)
    loss = net.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), 1e-3)
    g = net.get_grads()
    loss_ref, g_ref = grads(p0.astype(np.float64), x, y, mean, std, NF, W, D)
    assert loss == pytest.approx(loss_ref, rel=1e-4)
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    p1 = net.get_params()
    p_ref, _, _ = adam_step(p0.astype(np.float64), g.astype(np.float64), 0.0, 0.0, 1, 1e-3)
    assert np.abs(p1 - p_ref).max() <= 1e-6
    net.close()


def test_training_fits_a_smooth_field(shape):
    import torch
    net = _net(shape, max_batch=4096, seed=11)
    x, y = _inputs(4096, 5, shape[3])
    net.set_output_scale(y.mean(axis=0), y.std(axis=0))
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    first = net.train_step(xd, yd, 3e-3)
    for _ in range(600):
        last = net.train_step(xd, yd, 3e-3, want_loss=False)
    last = net.train_step(xd, yd, 1e-3)
    assert last < 0.02 * first, (first, last)
    net.close()


def test_argument_errors():
    import torch
    L = lib()
    with pytest.raises(L.LBError) as e:
        L.LBMlp(n_fourier=2, width=2, depth=5)
    assert e.value.status == L.LB_ERR_ARG
    net = _net(SHAPES["small"], max_batch=16)
    x = torch.zeros((17, 3), device="cuda")
    with pytest.raises(L.LBError) as e:
        net.predict(x)
    assert e.value.status == L.LB_ERR_ARG
    with pytest.raises(L.LBError):
        net.set_output_scale([0, 0, 0, 0], [1, 0, 1, 1])
    net.close()
