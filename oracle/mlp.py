"""FP64 reference of the learned initialiser of the multipole fit.

The network proposes the parameters of Eq. modelf for N_p = 2 from a curve
Sigma^c(i w_j) on 24 nodes. Layout (readings of an unspecified design): input
x = (Re y_j / s, Im y_j / s)_j with s = max_j |y_j| (48 values); two hidden layers of
128 with SiLU; 8 outputs o read as a_p = s (o_{4p} + i o_{4p+1}),
w_p = o_{4p+2} + i o_{4p+3}. Training loss per curve: the imaginary-axis fit residual
of the proposed parameters, L = (1/n_w) sum_j |f(i w_j) - y_j|^2 / s^2, averaged over
the batch; Adam (Kingma & Ba 2015) updates.

Weights are stored row-major: W1 [128][48], W2 [128][128], W3 [8][128]; the packed
vector is W1, b1, W2, b2, W3, b3 in that order.

Inference in BF16 storage arithmetic (forward_bf16): the input, weights, biases and
both hidden activations are rounded to BF16 (round to nearest, ties to even), sums are
exact (FP64) and SiLU is FP64; a reference for a BF16 inference kernel, not a claim
about rounding inside its sums.

This module is test infrastructure: only the tests and the benchmark's CPU baseline use it.
"""
import numpy as np

SIZES = (48, 128, 128, 8)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def pack(p):
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in ORDER])


def unpack(v):
    v = np.asarray(v, dtype=np.float64)
    shapes = {"W1": (128, 48), "b1": (128,), "W2": (128, 128), "b2": (128,), "W3": (8, 128),
              "b3": (8,)}
    p, o = {}, 0
    for k in ORDER:
        n = int(np.prod(shapes[k]))
        p[k] = v[o:o + n].reshape(shapes[k])
        o += n
    assert o == len(v)
    return p


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), via the FP32 bit pattern."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(p, x):
    q = {k: bf16_round(v) for k, v in p.items()}
    h1 = bf16_round(silu(bf16_round(x) @ q["W1"].T + q["b1"]))
    h2 = bf16_round(silu(h1 @ q["W2"].T + q["b2"]))
    return h2 @ q["W3"].T + q["b3"]


def init_params(seed):
    rng = np.random.default_rng(seed)
    p = {}
    for l, (n_in, n_out) in enumerate(zip(SIZES[:-1], SIZES[1:]), start=1):
        lim = np.sqrt(6.0 / (n_in + n_out))
        p[f"W{l}"] = rng.uniform(-lim, lim, size=(n_out, n_in))
        p[f"b{l}"] = np.zeros(n_out)
    return p


def features(y):
    """x [B][48] and scale s [B] from curves y [B][24] (complex)."""
    y = np.asarray(y, dtype=np.complex128)
    s = np.max(np.abs(y), axis=1)
    s = np.where(s > 0, s, 1.0)
    x = np.concatenate([y.real / s[:, None], y.imag / s[:, None]], axis=1)
    # interleave as (Re y_0, Im y_0, Re y_1, ...)
    xi = np.empty_like(x)
    n = y.shape[1]
    xi[:, 0::2] = x[:, :n]
    xi[:, 1::2] = x[:, n:]
    return xi, s


def forward(p, x):
    z1 = x @ p["W1"].T + p["b1"]
    h1 = silu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(z2)
    o = h2 @ p["W3"].T + p["b3"]
    return o, (x, z1, h1, z2, h2)


def decode(o, s):
    o = np.asarray(o).reshape(o.shape[0], -1, 4)
    a = s[:, None] * (o[:, :, 0] + 1j * o[:, :, 1])
    wp = o[:, :, 2] + 1j * o[:, :, 3]
    return a, wp


def loss_and_grad_outputs(o, s, omega, y):
    """Batch-mean loss and dL/do."""
    B = o.shape[0]
    nw = len(omega)
    a, wp = decode(o, s)
    z = 1j * np.asarray(omega)[None, :, None]
    phi = 1.0 / (z - wp[:, None, :])                       # [B][nw][P]
    f = (a[:, None, :] * phi).sum(axis=2)
    r = f - y
    L = np.mean(np.sum(np.abs(r) ** 2, axis=1) / (nw * s ** 2))
    coef = 2.0 / (nw * s ** 2 * B)                          # d mean / d |r|^2 terms
    rc = np.conj(r)[:, :, None]
    dfa = s[:, None, None] * phi                            # d f / d Re a-output
    dfw = a[:, None, :] * phi * phi                         # d f / d Re w_p
    g = np.empty_like(o).reshape(B, -1, 4)
    g[:, :, 0] = coef[:, None] * np.sum((rc * dfa).real, axis=1)
    g[:, :, 1] = coef[:, None] * np.sum((rc * 1j * dfa).real, axis=1)
    g[:, :, 2] = coef[:, None] * np.sum((rc * dfw).real, axis=1)
    g[:, :, 3] = coef[:, None] * np.sum((rc * 1j * dfw).real, axis=1)
    return L, g.reshape(B, -1)


def backward(p, cache, go):
    x, z1, h1, z2, h2 = cache
    grads = {}
    grads["W3"] = go.T @ h2
    grads["b3"] = go.sum(axis=0)
    gh2 = go @ p["W3"]
    gz2 = gh2 * dsilu(z2)
    grads["W2"] = gz2.T @ h1
    grads["b2"] = gz2.sum(axis=0)
    gh1 = gz2 @ p["W2"]
    gz1 = gh1 * dsilu(z1)
    grads["W1"] = gz1.T @ x
    grads["b1"] = gz1.sum(axis=0)
    return grads


def loss_and_grads(p, omega, y):
    x, s = features(y)
    o, cache = forward(p, x)
    L, go = loss_and_grad_outputs(o, s, omega, y)
    return L, backward(p, cache, go)


def adam_step(p, grads, state, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = b1 * m + (1 - b1) * grads[k]
        v[...] = b2 * v + (1 - b2) * grads[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p
