"""FP64 CPU oracle of the learned inlet-profile initialiser (test infrastructure only).

The paper proposes, as future work (section 3 closing remarks and section 4), a network that maps
an observed flow field to a first guess of the unknown boundary condition, so that the gradient
inversion starts close to the answer.  This module states that network from definitions, in plain
numpy FP64 with explicit loops over the few kernel taps, forward and backward:

  input   x[b, h, w, c]  (NHWC): u_x / s, u_y / s, obstacle mask, zero channels up to C0
  level l (l = 0..3): two 3x3 convolutions (zero padding 1, cross-correlation) + ReLU; between
          encoder levels a 2x2 max-pool; channels c_l = base * 2^l
  decoder (l = 2..0): 2x2 stride-2 transposed convolution c_{l+1} -> c_l, concatenation
          [upsampled, skip] along channels, two 3x3 convolutions + ReLU
  head    1x1 convolution c_0 -> 1, then the mean over x: one value per row y (the inlet profile,
          in units of 1e-3 of density)
  loss    L = mean over batch and rows of (out - target)^2
  Adam    on FP32 master weights (beta 0.9 / 0.999, eps 1e-8)

Only tests/ (and the benchmark's CPU leg) may import this module; the GPU path shares no code
with it.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------- layers


def conv3x3(x, w, b):
    """y[b,h,w,o] = sum_{dy,dx,c} x[b,h+dy-1,w+dx-1,c] w[dy,dx,c,o] + b[o] (zero padding)."""
    B, H, W, C = x.shape
    xp = np.zeros((B, H + 2, W + 2, C))
    xp[:, 1:-1, 1:-1, :] = x
    y = np.zeros((B, H, W, w.shape[3])) + b
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("bhwc,co->bhwo", xp[:, dy:dy + H, dx:dx + W, :], w[dy, dx])
    return y


def conv3x3_backward(x, w, gy):
    """Gradients of conv3x3 with respect to x, w and b, given dL/dy."""
    B, H, W, C = x.shape
    xp = np.zeros((B, H + 2, W + 2, C))
    xp[:, 1:-1, 1:-1, :] = x
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            gw[dy, dx] = np.einsum("bhwc,bhwo->co", xp[:, dy:dy + H, dx:dx + W, :], gy)
            gxp[:, dy:dy + H, dx:dx + W, :] += np.einsum("bhwo,co->bhwc", gy, w[dy, dx])
    return gxp[:, 1:-1, 1:-1, :], gw, gy.sum(axis=(0, 1, 2))


def relu(x):
    return np.maximum(x, 0.0)


def relu_backward(y, gy):
    """Gradient through ReLU from its output y (y > 0 exactly where the input was > 0)."""
    return gy * (y > 0)


def maxpool2(x):
    """2x2 max-pool, stride 2; returns the output and the winning tap (first maximum in the
    order (0,0), (0,1), (1,0), (1,1))."""
    B, H, W, C = x.shape
    taps = np.stack([x[:, dy::2, dx::2, :] for dy in range(2) for dx in range(2)], axis=0)
    arg = np.argmax(taps, axis=0)
    return np.max(taps, axis=0), arg


def maxpool2_backward(arg, gy, shape):
    gx = np.zeros(shape)
    for t in range(4):
        dy, dx = divmod(t, 2)
        gx[:, dy::2, dx::2, :] += gy * (arg == t)
    return gx


def upconv2(x, w, b):
    """2x2 stride-2 transposed convolution: y[b,2h+dy,2w+dx,o] = sum_c x[b,h,w,c] w[dy,dx,c,o] + b[o]."""
    B, H, W, C = x.shape
    y = np.zeros((B, 2 * H, 2 * W, w.shape[3]))
    for dy in range(2):
        for dx in range(2):
            y[:, dy::2, dx::2, :] = np.einsum("bhwc,co->bhwo", x, w[dy, dx]) + b
    return y


def upconv2_backward(x, w, gy):
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for dy in range(2):
        for dx in range(2):
            g = gy[:, dy::2, dx::2, :]
            gx += np.einsum("bhwo,co->bhwc", g, w[dy, dx])
            gw[dy, dx] = np.einsum("bhwc,bhwo->co", x, g)
    return gx, gw, gy.sum(axis=(0, 1, 2))


def head(x, w, b):
    """1x1 convolution to one channel, then the mean over x: out[b, h]."""
    z = np.einsum("bhwc,c->bhw", x, w) + b
    return z.mean(axis=2)


def head_backward(x, w, gout):
    W = x.shape[2]
    gz = np.repeat(gout[:, :, None], W, axis=2) / W
    return np.einsum("bhw,c->bhwc", gz, w), np.einsum("bhwc,bhw->c", x, gz), gz.sum()


def mse(out, target):
    d = out - target
    return float(np.mean(d * d)), 2.0 * d / d.size


# ---------------------------------------------------------------- network

def param_shapes(base: int, c_in: int):
    """Names and shapes of the parameters, in the order the GPU path stores them."""
    c = [base * 2 ** l for l in range(4)]
    s = []
    prev = c_in
    for l in range(4):
        s += [(f"enc{l}a.w", (3, 3, prev, c[l])), (f"enc{l}a.b", (c[l],)),
              (f"enc{l}b.w", (3, 3, c[l], c[l])), (f"enc{l}b.b", (c[l],))]
        prev = c[l]
    for l in (2, 1, 0):
        s += [(f"up{l}.w", (2, 2, c[l + 1], c[l])), (f"up{l}.b", (c[l],)),
              (f"dec{l}a.w", (3, 3, 2 * c[l], c[l])), (f"dec{l}a.b", (c[l],)),
              (f"dec{l}b.w", (3, 3, c[l], c[l])), (f"dec{l}b.b", (c[l],))]
    s += [("head.w", (c[0],)), ("head.b", (1,))]
    return s


def init_params(base: int, c_in: int, seed: int):
    """He-normal weights, zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = {}
    for name, shape in param_shapes(base, c_in):
        if name.endswith(".b"):
            p[name] = np.zeros(shape)
        else:
            fan_in = int(np.prod(shape[:-1])) if len(shape) > 1 else shape[0]
            p[name] = rng.normal(0.0, np.sqrt(2.0 / fan_in), shape)
    return p


def keep(a):
    return a


def forward(p, x, store=keep):
    """Network output [b, h] and the activations the backward pass needs.
    `store` models the precision in which an implementation keeps each
    activation (identity: exact FP64; a rounding function: e.g. BF16 storage);
    it is applied to every stored layer output."""
    a = {"x": x}
    h = x
    for l in range(4):
        h = store(relu(conv3x3(h, p[f"enc{l}a.w"], p[f"enc{l}a.b"])))
        a[f"enc{l}a"] = h
        h = store(relu(conv3x3(h, p[f"enc{l}b.w"], p[f"enc{l}b.b"])))
        a[f"enc{l}b"] = h
        if l < 3:
            h, arg = maxpool2(h)
            a[f"pool{l}"], a[f"arg{l}"] = h, arg
    for l in (2, 1, 0):
        u = store(upconv2(h, p[f"up{l}.w"], p[f"up{l}.b"]))
        a[f"up{l}"] = u
        cat = np.concatenate([u, a[f"enc{l}b"]], axis=3)
        a[f"cat{l}"] = cat
        h = store(relu(conv3x3(cat, p[f"dec{l}a.w"], p[f"dec{l}a.b"])))
        a[f"dec{l}a"] = h
        h = store(relu(conv3x3(h, p[f"dec{l}b.w"], p[f"dec{l}b.b"])))
        a[f"dec{l}b"] = h
    out = head(h, p["head.w"], p["head.b"])
    return out, a


def backward(p, a, gout, store=keep):
    """dL/dparams given dL/dout, through the activations of forward(); `store`
    is applied to every stored activation gradient (see forward)."""
    g = {}
    gh, g["head.w"], gb = head_backward(a["dec0b"], p["head.w"], gout)
    gh = store(gh)
    g["head.b"] = np.array([gb])
    skips = {}
    for l in (0, 1, 2):
        gh = relu_backward(a[f"dec{l}b"], gh)
        gh, g[f"dec{l}b.w"], g[f"dec{l}b.b"] = conv3x3_backward(a[f"dec{l}a"], p[f"dec{l}b.w"], gh)
        gh = relu_backward(a[f"dec{l}a"], store(gh))
        gcat, g[f"dec{l}a.w"], g[f"dec{l}a.b"] = conv3x3_backward(a[f"cat{l}"], p[f"dec{l}a.w"], gh)
        gcat = store(gcat)
        cu = a[f"up{l}"].shape[3]
        skips[l] = gcat[..., cu:]
        below = a["enc3b"] if l == 2 else a[f"dec{l + 1}b"]
        gh, g[f"up{l}.w"], g[f"up{l}.b"] = upconv2_backward(below, p[f"up{l}.w"], gcat[..., :cu])
        gh = store(gh)
    for l in (3, 2, 1, 0):
        if l < 3:
            gh = store(maxpool2_backward(a[f"arg{l}"], gh, a[f"enc{l}b"].shape) + skips[l])
        gh = relu_backward(a[f"enc{l}b"], gh)
        gh, g[f"enc{l}b.w"], g[f"enc{l}b.b"] = conv3x3_backward(a[f"enc{l}a"], p[f"enc{l}b.w"], gh)
        gh = relu_backward(a[f"enc{l}a"], store(gh))
        inp = a["x"] if l == 0 else a[f"pool{l - 1}"]
        gh, g[f"enc{l}a.w"], g[f"enc{l}a.b"] = conv3x3_backward(inp, p[f"enc{l}a.w"], gh)
        gh = store(gh)
    return g


def loss_and_grad(p, x, target, store=keep):
    out, a = forward(p, x, store)
    L, gout = mse(out, target)
    return L, backward(p, a, gout, store), out


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step on every parameter (t is 1-based)."""
    for k in p:
        m[k] = b1 * m[k] + (1 - b1) * g[k]
        v[k] = b2 * v[k] + (1 - b2) * g[k] * g[k]
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p, m, v
