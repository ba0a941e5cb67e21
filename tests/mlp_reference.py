"""Plain numpy reference of the surrogate network of include/lbgm.h (lb_mlp):
features, forward pass, mean-squared-error gradients and one Adam step, in
FP64 with the weights rounded to BF16 as the library uses them in every
product. Test code only."""
import numpy as np

NOUT = 4


def bf16(a):
    """Round float32 values to the nearest BF16 (ties to even), as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    r = ((b >> 16) & 1) + 0x7FFF
    return ((b + r) & 0xFFFF0000).astype(np.uint32).view(np.float32)


def layer_shapes(n_fourier, width, depth, n_plain=2):
    nin = n_plain + 2 * n_fourier
    fi = [nin] + [width] * (depth - 1)
    fo = [width] * (depth - 1) + [NOUT]
    return list(zip(fo, fi))


def unpack(params, n_fourier, width, depth, n_plain=2):
    out, k = [], 0
    for fo, fi in layer_shapes(n_fourier, width, depth, n_plain):
        W = params[k:k + fo * fi].reshape(fo, fi)
        k += fo * fi
        b = params[k:k + fo]
        k += fo
        out.append((W, b))
    assert k == len(params)
    return out


def features(x, n_fourier):
    """Rows (p_1 .. p_P, z): the plain inputs, then sin, cos(2 pi k z)."""
    z = x[:, -1]
    cols = [x[:, j] for j in range(x.shape[1] - 1)]
    for k in range(1, n_fourier + 1):
        cols += [np.sin(2 * np.pi * k * z), np.cos(2 * np.pi * k * z)]
    return np.stack(cols, axis=1).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def forward(params, x, n_fourier, width, depth):
    """Normalised outputs and the per-layer (input, pre-activation) cache."""
    h = features(np.asarray(x, np.float64), n_fourier)
    cache = []
    layers = unpack(params, n_fourier, width, depth, np.shape(x)[1] - 1)
    for l, (W, b) in enumerate(layers):
        z = h @ bf16(W).astype(np.float64).T + b
        cache.append((h, z))
        h = z if l == len(layers) - 1 else silu(z)
    return h, cache


def grads(params, x, y, mean, std, n_fourier, width, depth):
    """(loss, gradient vector) of the mean squared error of normalised outputs."""
    Y, cache = forward(params, x, n_fourier, width, depth)
    T = (np.asarray(y, np.float64) - mean) / std
    n = len(x)
    loss = ((Y - T) ** 2).mean()
    dz = 2.0 * (Y - T) / (n * NOUT)
    layers = unpack(params, n_fourier, width, depth, np.shape(x)[1] - 1)
    g = []
    for l in range(len(layers) - 1, -1, -1):
        h, z = cache[l]
        W, _ = layers[l]
        g.append((dz.T @ h, dz.sum(axis=0)))
        if l == 0:
            break
        dh = dz @ bf16(W).astype(np.float64)
        zp = cache[l - 1][1]
        s = 1.0 / (1.0 + np.exp(-zp))
        dz = dh * s * (1.0 + zp * (1.0 - s))
    flat = []
    for dW, db in reversed(g):
        flat += [dW.ravel(), db]
    return loss, np.concatenate(flat)


def adam_step(params, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    p = params - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return p, m, v
