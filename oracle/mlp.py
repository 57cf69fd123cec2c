"""FP64 oracle of the learned proposal network (not part of the SGTP paper).

TEST INFRASTRUCTURE ONLY: imported by the test-suite alone; the product
library shares no code with it.

The network maps the 64 features of a best response to a Gaussian over its
control sequence: x -> 256 -> 256 -> 256 -> 4T with ReLU hidden layers.
Output row: [mu_a (T), mu_delta (T), logsig_a (T), logsig_delta (T)], in
units of the plain sampler's sigma per channel.  Parameters are one flat
vector, per layer W [out][in] (row-major) followed by b [out].

Loss: Gaussian negative log-likelihood of the target (the residual of the
selected controls U* around the nominal controls U-bar, divided by sigma_a,
sigma_delta) under N(mu, diag exp(2 logsig)), logsig
clamped to [-5, 2], constant term dropped, mean over batch x 2T elements.

With ``bf16=True`` the arithmetic is FP64 on BF16-rounded tensors, rounded
at the points where a BF16 network stores them: the input, the weights, each
hidden activation (after bias and ReLU), and each back-propagated dZ before
its products; biases and bias gradients stay unrounded.  With ``bf16=False``
everything is plain FP64 (for the finite-difference check).

Parity status: pinned -- the gradient by central finite differences in
FP64, the loss by its closed form at special points, BF16 rounding by the
round-to-nearest-even definition on exact binary values, Adam by its
first-step closed form.
"""
from __future__ import annotations

import numpy as np

IN = 64
HIDDEN = 256


def dims_for(T: int):
    """Layer widths of the network for horizon T."""
    return [IN, HIDDEN, HIDDEN, HIDDEN, 4 * T]


def param_count(dims) -> int:
    return int(sum(dims[l + 1] * dims[l] + dims[l + 1] for l in range(len(dims) - 1)))


def unpack(w, dims):
    """Views (W [out][in], b [out]) of every layer of the flat vector w."""
    out, o = [], 0
    for l in range(len(dims) - 1):
        n_in, n_out = dims[l], dims[l + 1]
        W = w[o:o + n_out * n_in].reshape(n_out, n_in)
        o += n_out * n_in
        b = w[o:o + n_out]
        o += n_out
        out.append((W, b))
    assert o == w.size
    return out


def bf16_round(x):
    """Round to BF16 (8 significand bits) by round-to-nearest-even, from the
    float32 value (the precision the value has before it is stored)."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    bits = (bits + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def _r(x, bf16):
    return bf16_round(x) if bf16 else np.asarray(x, dtype=np.float64)


def forward(w, x, dims, bf16=True):
    """Output [B x dims[-1]] and the cache (the stored activations)."""
    layers = unpack(np.asarray(w, dtype=np.float64), dims)
    a = _r(x, bf16)
    acts = [a]
    for l, (W, b) in enumerate(layers):
        z = a @ _r(W, bf16).T + b
        if l == len(layers) - 1:
            return z, acts
        a = _r(np.maximum(z, 0.0), bf16)
        acts.append(a)
    raise AssertionError("unreachable")


def nll(out, target, T):
    """Loss and d loss / d out of the clamped Gaussian NLL."""
    out = np.asarray(out, dtype=np.float64)
    n2 = 2 * T
    mu, ls_raw = out[:, :n2], out[:, n2:2 * n2]
    ls = np.clip(ls_raw, -5.0, 2.0)
    inv_s = np.exp(-ls)
    z = (np.asarray(target, dtype=np.float64) - mu) * inv_s
    n = out.shape[0] * n2
    loss = float(np.sum(0.5 * z * z + ls) / n)
    d = np.zeros_like(out)
    d[:, :n2] = -z * inv_s / n
    inside = (ls_raw > -5.0) & (ls_raw < 2.0)
    d[:, n2:2 * n2] = np.where(inside, (1.0 - z * z) / n, 0.0)
    return loss, d


def backward(w, acts, dout, dims, bf16=True):
    """Gradient of the loss with respect to the flat parameters, by the chain
    rule through the layers in reverse order."""
    layers = unpack(np.asarray(w, dtype=np.float64), dims)
    g = np.zeros(param_count(dims))
    grads = unpack(g, dims)
    dz = np.asarray(dout, dtype=np.float64)
    for l in range(len(layers) - 1, -1, -1):
        dzr = _r(dz, bf16)
        gW, gb = grads[l]
        gW[...] = dzr.T @ acts[l]
        gb[...] = dz.sum(axis=0)
        if l == 0:
            break
        dh = dzr @ _r(layers[l][0], bf16)
        dz = np.where(acts[l] > 0.0, dh, 0.0)
    return g


def loss_and_grad(w, x, target, T, dims=None, bf16=True):
    dims = dims or dims_for(T)
    out, acts = forward(w, x, dims, bf16)
    loss, d = nll(out, target, T)
    return loss, backward(w, acts, d, dims, bf16), out


def adam(w, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, 2015) with bias correction; step is the
    1-based count after this update.  Returns (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def proposal(out_row, T, sigma_a, sigma_delta, u_nom=None):
    """Per-step Gaussian (T x 4: mean a, mean delta, sigma a, sigma delta) of
    one output row around the nominal controls u_nom (T x 2; None: zero):
    mean = u_nom + plain sigma x mu (a residual around the plain sampler's
    centre), sigma = plain sigma x exp(logsig) with logsig clamped to
    [-5, 2]."""
    o = np.asarray(out_row, dtype=np.float64)
    un = np.zeros((T, 2)) if u_nom is None else np.asarray(u_nom, dtype=np.float64).reshape(T, 2)
    la = np.clip(o[2 * T:3 * T], -5.0, 2.0)
    ld = np.clip(o[3 * T:4 * T], -5.0, 2.0)
    return np.stack([un[:, 0] + sigma_a * o[:T], un[:, 1] + sigma_delta * o[T:2 * T], sigma_a * np.exp(la),
                     sigma_delta * np.exp(ld)], axis=1)
