"""FP64 reference of the learned-preconditioner network (no counterpart in the paper).

Test infrastructure only (see ``oracle/__init__.py``).

Definition: layers l map widths[l] -> widths[l+1], y = W h + b with W stored
row-major (out x in); ReLU on hidden layers, linear output; loss = mean over
batch and outputs of (y - t)^2.  The weights and biases used in the products
are the FP32 parameters rounded to bfloat16 (round to nearest, ties to even),
as in the product.  With tf32=True (the product's network: its products run
on the tensor cores in TF32) the other operand of every product -- the layer
input h in the forward pass and in the weight gradient, the back-propagated
error dy in both gradients -- enters rounded to FP32 and then to TF32 (10
mantissa bits, nearest, ties away from zero); the bf16 weights are exact in
TF32.  Everything else is FP64 here.  tf32=False is the exact network, which
the finite-difference pin checks.
"""

import numpy as np


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    bias = 0x7FFF + ((bits >> 16) & 1)
    r = ((bits + bias) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def tf32_round(x):
    """Round to FP32, then to the nearest TF32 value (10 mantissa bits, ties away
    from zero: add half an ulp to the magnitude bits and truncate), as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    r = ((bits + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def _identity(x):
    return np.asarray(x, dtype=np.float64)


def unpack(params, widths):
    out = []
    off = 0
    for l in range(len(widths) - 1):
        i, o = widths[l], widths[l + 1]
        W = params[off:off + i * o].reshape(o, i)
        off += i * o
        b = params[off:off + o]
        off += o
        out.append((W, b))
    return out


def forward(params, widths, x, tf32=False):
    """Activations h_0 = x, ..., h_L = y with bf16-rounded parameters."""
    rnd = tf32_round if tf32 else _identity
    layers = unpack(bf16_round(params), widths)
    hs = [np.asarray(x, dtype=np.float64)]
    for l, (W, b) in enumerate(layers):
        z = rnd(hs[-1]) @ W.T + b
        hs.append(np.maximum(z, 0.0) if l + 1 < len(layers) else z)
    return hs


def loss(params, widths, x, t, tf32=False):
    y = forward(params, widths, x, tf32)[-1]
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def loss_grad(params, widths, x, t, tf32=False):
    """Loss and its gradient w.r.t. the (bf16-rounded) flat parameters by backpropagation."""
    rnd = tf32_round if tf32 else _identity
    layers = unpack(bf16_round(params), widths)
    hs = forward(params, widths, x, tf32)
    y = hs[-1]
    t = np.asarray(t, dtype=np.float64)
    n = y.size
    dy = 2.0 * (y - t) / n
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        dyr = rnd(dy)
        dW = dyr.T @ rnd(hs[l])
        db = dyr.sum(axis=0)
        grads.append((dW, db))
        if l > 0:
            dy = (dyr @ W) * (hs[l] > 0.0)
    grads.reverse()
    flat = np.concatenate([np.concatenate([dW.reshape(-1), db]) for dW, db in grads])
    return float(np.mean((y - t) ** 2)), flat


def init_params(widths, seed=0):
    """He-scaled normal weights, zero biases, as float32."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(len(widths) - 1):
        i, o = widths[l], widths[l + 1]
        parts.append(rng.standard_normal(i * o) * np.sqrt(2.0 / i))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)
