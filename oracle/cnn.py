"""FP64 oracle of the learned warm start: a small CNN that predicts a band's
Z0 from its bicubic upsampling and the PAN. TEST INFRASTRUCTURE ONLY (see
the package docstring).

Architecture (the paper has no network; this is the project's extension of
the CG warm start): six 3 x 3 convolutions on the torus (circular padding,
the scenes' boundary model), widths 2 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1,
bias and ReLU after every layer but the last, and a residual output:
    x = (bicubic(X_b) / s, Y / s)           (2 channels, s = 255)
    z = s (x_0 + f(x))
Convolutions are cross-correlations, out[o](y, x) = b[o] +
sum_{i, dy, dx} w[o, i, dy + 1, dx + 1] in[i]((y + dy) mod H, (x + dx) mod W).
Loss: mean squared error of z / s against the target / s over all pixels.
The backward pass is the chain rule written out layer by layer.
"""
from __future__ import annotations

import numpy as np

WIDTHS = (2, 32, 32, 32, 32, 32, 1)
SCALE = 255.0


def n_layers() -> int:
    return len(WIDTHS) - 1


def init_params(seed: int = 0):
    """He-normal weights, zero biases. Returns a list of (w, b) per layer,
    w of shape (out, in, 3, 3)."""
    rng = np.random.default_rng(seed)
    params = []
    for l in range(n_layers()):
        ci, co = WIDTHS[l], WIDTHS[l + 1]
        std = np.sqrt(2.0 / (9 * ci))
        if l == n_layers() - 1:
            std *= 0.1          # the last layer starts near zero: z ~ bicubic
        params.append((rng.standard_normal((co, ci, 3, 3)) * std, np.zeros(co)))
    return params


def conv3x3(x, w, b=None):
    """Circular 3 x 3 cross-correlation: x (in, H, W), w (out, in, 3, 3)."""
    x, w = np.asarray(x, np.float64), np.asarray(w, np.float64)
    out = np.zeros((w.shape[0],) + x.shape[1:])
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            xs = np.roll(x, (-dy, -dx), axis=(1, 2))      # xs(y, x) = x(y + dy, x + dx)
            out += np.einsum("oi,ihw->ohw", w[:, :, dy + 1, dx + 1], xs)
    if b is not None:
        out += np.asarray(b, np.float64)[:, None, None]
    return out


def conv3x3_adjoint(g, w):
    """Adjoint of conv3x3 in its input: g (out, H, W) -> (in, H, W)."""
    g, w = np.asarray(g, np.float64), np.asarray(w, np.float64)
    out = np.zeros((w.shape[1],) + g.shape[1:])
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            t = np.einsum("oi,ohw->ihw", w[:, :, dy + 1, dx + 1], g)
            out += np.roll(t, (dy, dx), axis=(1, 2))      # back to (y + dy, x + dx)
    return out


def conv3x3_weight_grad(x, g):
    """d<g, conv3x3(x, w)>/dw: x (in, H, W), g (out, H, W) -> (out, in, 3, 3)."""
    x, g = np.asarray(x, np.float64), np.asarray(g, np.float64)
    dw = np.zeros((g.shape[0], x.shape[0], 3, 3))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            xs = np.roll(x, (-dy, -dx), axis=(1, 2))
            dw[:, :, dy + 1, dx + 1] = np.einsum("ohw,ihw->oi", g, xs)
    return dw


def make_input(up, pan):
    """The two input channels of one band: bicubic upsampling and PAN, / s."""
    return np.stack([np.asarray(up, np.float64), np.asarray(pan, np.float64)]) / SCALE


def forward(params, x, round_act=None):
    """Returns (z, cache): z (H, W) on the intensity scale, cache of the
    pre-activations and activations for the backward pass. round_act, if
    given, is applied to every hidden activation (to model a storage
    precision); None keeps plain FP64."""
    acts = [np.asarray(x, np.float64)]
    pre = []
    a = acts[0]
    for l, (w, b) in enumerate(params):
        p = conv3x3(a, w, b)
        pre.append(p)
        a = np.maximum(p, 0.0) if l < len(params) - 1 else p
        if round_act is not None and l < len(params) - 1:
            a = round_act(a)
        acts.append(a)
    z = SCALE * (acts[0][0] + acts[-1][0])
    return z, {"acts": acts, "pre": pre}


def loss(z, target, weight=None) -> float:
    """Mean over pixels of weight * ((z - target) / s)^2 (weight 1 if None)."""
    d = (np.asarray(z, np.float64) - np.asarray(target, np.float64)) / SCALE
    w = 1.0 if weight is None else np.asarray(weight, np.float64)
    return float(np.mean(w * d * d))


def backward(params, cache, z, target, round_grad=None, weight=None):
    """Gradients of loss(z, target, weight) with respect to every (w, b).
    round_grad, if given, is applied to the gradient passed between hidden
    layers."""
    acts, pre = cache["acts"], cache["pre"]
    H, W = z.shape
    d = (np.asarray(z, np.float64) - np.asarray(target, np.float64)) / SCALE
    if weight is not None:
        d = d * np.asarray(weight, np.float64)
    # dL/dz_scaled = 2 w d / (H W), z_scaled = x_0 + f(x): dL/df = that
    g = (2.0 / (H * W)) * d[None]
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        w, _ = params[l]
        if l < len(params) - 1:
            g = g * (acts[l + 1] > 0.0)            # ReLU (its output is > 0 where it passes)
            if round_grad is not None:
                g = round_grad(g)
        grads[l] = (conv3x3_weight_grad(acts[l], g), g.sum(axis=(1, 2)))
        if l > 0:
            g = conv3x3_adjoint(g, w)
    return grads


def adam_step(params, grads, state, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma & Ba 2015, Alg. 1) of every tensor, in place in
    a copy; state = {"t": int, "m": [...], "v": [...]} (created if empty)."""
    if not state:
        state["t"] = 0
        state["m"] = [np.zeros_like(a) for wb in params for a in wb]
        state["v"] = [np.zeros_like(a) for wb in params for a in wb]
    state["t"] += 1
    t = state["t"]
    flat_p = [a for wb in params for a in wb]
    flat_g = [a for wb in grads for a in wb]
    out = []
    for i, (p, g) in enumerate(zip(flat_p, flat_g)):
        state["m"][i] = beta1 * state["m"][i] + (1 - beta1) * g
        state["v"][i] = beta2 * state["v"][i] + (1 - beta2) * g * g
        mh = state["m"][i] / (1 - beta1 ** t)
        vh = state["v"][i] / (1 - beta2 ** t)
        out.append(p - lr * mh / (np.sqrt(vh) + eps))
    return [(out[2 * l], out[2 * l + 1]) for l in range(len(params))]


# ----------------------------------------------------------------------------
# Learned diagonal preconditioner (an extension of the Z0 CG; the paper runs
# plain CG). A second network of the same architecture, with its own
# parameters, reads (bicubic, PAN); its learned part c = f(x) = z / s - x_0
# gives the diagonal s_d = max(c, floor) > 0 of P^{-1} = diag(s_d).
# Training fits one preconditioned correction step from the warm start z_w,
# z_w + kappa c r_0 ~ z*, with r_0 = b - A z_w and e = z* - z_w: the squared
# error sum (kappa c r_0 - e)^2 equals, pixel by pixel,
# kappa^2 r_0^2 (c - e / (kappa r_0))^2, i.e. the weighted loss above with
# target z_t = s (x_0 + e / (kappa r_0)) and weight kappa^2 r_0^2. kappa is
# a fixed scale (the least-squares constant step over the training pixels)
# so that c is of order one; PCG is invariant under a constant scaling of
# s_d, so kappa does not reach the solver.
# ----------------------------------------------------------------------------
DIAG_FLOOR = 1.0 / 64.0


def diag_head(z, up, floor: float = DIAG_FLOOR):
    """s_d = max(z / s - up / s, floor): the learned part of the diagonal
    network's output, kept positive (a non-finite value gives the floor)."""
    c = (np.asarray(z, np.float64) - np.asarray(up, np.float64)) / SCALE
    return np.fmax(c, floor)


def diag_fit(up, z_w, z_star, r0, kappa: float):
    """(target, weight) of the weighted loss whose minimiser over the network's
    learned part c is the one-step fit kappa c r_0 ~ z* - z_w (pixels with
    r_0 = 0 get weight 0)."""
    up, z_w, z_star, r0 = (np.asarray(a, np.float64) for a in (up, z_w, z_star, r0))
    e = z_star - z_w
    live = r0 != 0.0
    q = np.where(live, e / np.where(live, kappa * r0, 1.0), 0.0)
    target = up + SCALE * q
    weight = (kappa * r0) ** 2
    return target, weight

