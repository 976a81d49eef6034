"""FP64 NumPy oracle of the learned initialiser's network (TEST INFRASTRUCTURE ONLY).

A multilayer perceptron x -> SiLU(x W_0 + b_0) -> ... -> y = h W_L + b_L, mean squared error
loss, Adam.  With bf16=True every matrix product first rounds both operands to bfloat16
(round to nearest even), as the GPU does, and then multiplies in double precision.

Parity pins (tests/test_oracle_mlp.py): the bfloat16 rounding against torch's conversion; the
backward pass against central finite differences of the forward pass and against torch
autograd in double precision; Adam against its closed form after one step.
"""
import numpy as np


def bf16(x):
    """Round float64 values to bfloat16 (via float32, round to nearest even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def split(params, dims):
    """Flat parameter vector -> [(W [in, out], b [out])] in the library's layout."""
    out, o = [], 0
    for a, b in zip(dims[:-1], dims[1:]):
        W = params[o:o + a * b].reshape(a, b); o += a * b
        bb = params[o:o + b]; o += b
        out.append((W, bb))
    return out


def forward(params, dims, x, bf16_ops=True):
    q = bf16 if bf16_ops else (lambda v: np.asarray(v, np.float64))
    layers = split(np.asarray(params, np.float64), dims)
    h = np.asarray(x, np.float64)
    zs, hs = [], [h]
    for l, (W, b) in enumerate(layers):
        z = q(h) @ q(W) + b
        if l + 1 < len(layers):
            zs.append(z)
            h = silu(z)
            hs.append(h)
        else:
            h = z
    return h, zs, hs


def loss_and_grad(params, dims, x, t, bf16_ops=True):
    """Mean squared error mean((net(x) - t)^2) and its gradient (flat, library layout)."""
    q = bf16 if bf16_ops else (lambda v: np.asarray(v, np.float64))
    layers = split(np.asarray(params, np.float64), dims)
    y, zs, hs = forward(params, dims, x, bf16_ops)
    d = y - t
    loss = np.mean(d * d)
    dz = 2.0 * d / d.size
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, b = layers[l]
        gW = q(hs[l]).T @ q(dz)
        gb = dz.sum(axis=0)
        grads.append((gW, gb))
        if l > 0:
            dz = (q(dz) @ q(W).T) * dsilu(zs[l - 1])
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def magnitude_sums(params, dims, x, t, bf16_ops=True):
    """Element-wise scales for comparing a computed network with this oracle: for every element of
    the forward output and of the gradient, the sum of the absolute values of the terms of the
    product that forms it (|q(h)| @ |q(W)| + |b| for the output, |q(h)|^T @ |q(dz)| and
    sum |dz| for the gradient).  Rounding one operand of a product to the other side of a
    bfloat16 boundary, or accumulating it in float32, moves an element by a fraction of its
    scale.  Returns (output scale [B, n_out], flat gradient scale in the library's layout)."""
    q = bf16 if bf16_ops else (lambda v: np.asarray(v, np.float64))
    layers = split(np.asarray(params, np.float64), dims)
    y, zs, hs = forward(params, dims, x, bf16_ops)
    WL, bL = layers[-1]
    sy = np.abs(q(hs[-1])) @ np.abs(q(WL)) + np.abs(bL)
    d = y - t
    dz = 2.0 * d / d.size
    scales = []
    for l in range(len(layers) - 1, -1, -1):
        W, b = layers[l]
        scales.append((np.abs(q(hs[l])).T @ np.abs(q(dz)), np.abs(dz).sum(axis=0)))
        if l > 0:
            dz = (q(dz) @ q(W).T) * dsilu(zs[l - 1])
    scales.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in scales])
    return sy, flat


def initial_profiles(params, dims, feats, x_mu, x_sd, y_mu, y_sd, n_layers, fallback, T_min=50.0, T_max=8000.0):
    """Start profiles from the learned initialiser: features standardised in float32 (the precision
    in which the inputs' bfloat16 rounding is then decided), the network in FP64 on bfloat16-rounded
    operands, de-standardised, and interpolated linearly (numpy.interp) from the outputs' evenly
    spaced normalised log-P positions to each atmosphere's evenly spaced layer centres; an invalid
    profile (non-finite, or outside (T_min, T_max)) is replaced by the fallback.  Returns
    (profiles, used, network outputs in K at the output positions)."""
    f32 = np.float32
    xs = ((np.asarray(feats, f32) - np.asarray(x_mu, f32)) / np.asarray(x_sd, f32)).astype(np.float64)
    y, _, _ = forward(params, dims, xs, bf16_ops=True)
    t = y * np.asarray(x_sd_like(y_sd), np.float64) + np.asarray(y_mu, f32).astype(np.float64)
    s_out = np.linspace(0.0, 1.0, dims[-1])
    profiles, used = [], []
    for i, n in enumerate(n_layers):
        T = np.interp(np.linspace(0.0, 1.0, n), s_out, t[i])
        ok = bool(np.all(np.isfinite(T)) and T.min() > T_min and T.max() < T_max)
        profiles.append(T if ok else np.asarray(fallback[i], np.float64))
        used.append(ok)
    return profiles, np.array(used), t


def x_sd_like(sd):
    """The float32 statistics widened to float64 (the library stores them in float32)."""
    return np.asarray(sd, np.float32).astype(np.float64)


def adam(params, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (bias-corrected), returns new (params, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
