"""FP64 reference of the learned interpolation correction (oracle; test only).

The paper has no learned component; this follows the problem statement's network: one shared
multilayer perceptron evaluated per (point, field f in {u, v, w, dphi/dt}):
  input  x = [stencil_f / s_f (64 values of the time-blended 4x4x4 stencil, x fastest, then y,
              then z), dx, dy, dz (in-cell offsets in [0, 1])],  s_f = max |stencil_f| + 1e-30;
  layers 67 -> 64 -> 64 -> 4 with GELU (tanh form, Hendrycks & Gimpel 2016) on the hidden
         layers; output y (4 values), of which y[f] is used;
  correction  f = lagrange_f + s_f * y[f];  pressure recomputed from the corrected fields.
Training minimises the mean of (y[f] - target)^2 with target = (exact_f - lagrange_f) / s_f, by
Adam (Kingma & Ba 2015) on FP32 master weights.
"""
import numpy as np

N_IN, N_HID, N_OUT = 67, 64, 4
_C = np.sqrt(2.0 / np.pi)


def gelu(x):
    """0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))."""
    return 0.5 * x * (1.0 + np.tanh(_C * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    t = np.tanh(_C * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * _C * (1.0 + 3 * 0.044715 * x * x)


def init_params(seed=0, scale=1.0):
    """Seeded initialisation: W ~ N(0, 1/fan_in) (scaled), biases 0. W_l has shape [out][in]."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, (o, i) in (("1", (N_HID, N_IN)), ("2", (N_HID, N_HID)), ("3", (N_OUT, N_HID))):
        p["W" + name] = rng.standard_normal((o, i)) * scale / np.sqrt(i)
        p["b" + name] = np.zeros(o)
    return p


def features(stencil, offsets):
    """stencil [n][64], offsets [n][3] -> (x [n][67], s [n])."""
    stencil = np.asarray(stencil, np.float64)
    s = np.max(np.abs(stencil), axis=1) + 1e-30
    return np.concatenate([stencil / s[:, None], np.asarray(offsets, np.float64)], 1), s


def forward(p, x):
    z1 = x @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (x, z1, h1, z2, h2)


def loss_and_grad(p, x, field, target):
    """Mean squared error of y[field] against target, and its gradient w.r.t. every parameter."""
    y, (x, z1, h1, z2, h2) = forward(p, x)
    n = len(x)
    rows = np.arange(n)
    r = y[rows, field] - target
    loss = np.mean(r * r)
    dy = np.zeros_like(y)
    dy[rows, field] = 2.0 * r / n
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    dz2 = (dy @ p["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    return loss, g


def adam_init(p):
    return {"t": 0, "m": {k: np.zeros_like(v) for k, v in p.items()},
            "v": {k: np.zeros_like(v) for k, v in p.items()}}


def adam_step(p, g, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected moments), in place on p and state."""
    state["t"] += 1
    t = state["t"]
    for k in p:
        state["m"][k] = beta1 * state["m"][k] + (1 - beta1) * g[k]
        state["v"][k] = beta2 * state["v"][k] + (1 - beta2) * g[k] * g[k]
        mh = state["m"][k] / (1 - beta1 ** t)
        vh = state["v"][k] / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p
