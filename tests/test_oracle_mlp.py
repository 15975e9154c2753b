"""Pins of the FP64 network reference: bf16 rounding and backpropagated gradients."""
import numpy as np

from oracle import mlp as OM


def test_bf16_rounding_ties_to_even():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: rounds to the even mantissa (1.0)
    x = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -2.5, 0.0], dtype=np.float32)
    r = OM.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0 + 2.0 ** -6 and r[2] == 1.0 and r[3] == -2.5 and r[4] == 0.0
    # rounding error within half an ulp of bf16 (8 mantissa bits)
    y = np.random.default_rng(0).standard_normal(1000).astype(np.float32)
    assert np.all(np.abs(OM.bf16_round(y) - y) <= np.abs(y) * 2.0 ** -8)


def test_gradient_matches_finite_differences():
    widths = [5, 7, 6, 2]
    rng = np.random.default_rng(1)
    p = OM.bf16_round(OM.init_params(widths, 2) + 0.01 * rng.standard_normal(
        sum(widths[i] * widths[i + 1] + widths[i + 1] for i in range(3))).astype(np.float32))
    x = rng.standard_normal((4, 5))
    t = rng.standard_normal((4, 2))
    _, g = OM.loss_grad(p, widths, x, t)

    def f(q):
        # loss as a function of the already-rounded parameters (no re-rounding)
        hs = [x]
        off = 0
        for l in range(3):
            i, o = widths[l], widths[l + 1]
            W = q[off:off + i * o].reshape(o, i)
            off += i * o
            b = q[off:off + o]
            off += o
            z = hs[-1] @ W.T + b
            hs.append(np.maximum(z, 0.0) if l < 2 else z)
        return np.mean((hs[-1] - t) ** 2)

    h = 1e-6
    for j in rng.choice(len(p), 40, replace=False):
        e = np.zeros(len(p))
        e[j] = h
        fd = (f(p + e) - f(p - e)) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(1.0, abs(fd))


def test_tf32_rounding_ties_away():
    # 1 + 2^-11 is a tie between 1 and 1 + 2^-10: rounds away from zero
    x = np.array([1.0 + 2.0 ** -11, -(1.0 + 2.0 ** -11), 1.0 + 2.0 ** -12, 1.0 + 3 * 2.0 ** -11, 0.0])
    r = OM.tf32_round(x)
    assert r[0] == 1.0 + 2.0 ** -10 and r[1] == -(1.0 + 2.0 ** -10) and r[2] == 1.0
    assert r[3] == 1.0 + 2.0 ** -9 and r[4] == 0.0
    # bf16 values are TF32 values; the error is within half a TF32 ulp
    y = np.random.default_rng(0).standard_normal(1000).astype(np.float32)
    assert np.array_equal(OM.tf32_round(OM.bf16_round(y)), OM.bf16_round(y))
    assert np.all(np.abs(OM.tf32_round(y) - y) <= np.abs(y) * 2.0 ** -11)


def test_tf32_network_is_the_exact_one_on_tf32_data():
    """With inputs, errors and activations already TF32 values the rounded
    network is the exact one: here every product operand is a small dyadic
    number (exact in TF32), so both give the same loss and gradient."""
    widths = [4, 3, 2]
    x = np.array([[0.5, -1.0, 0.25, 2.0], [1.0, 0.0, -0.5, 0.75]])
    p = np.zeros(4 * 3 + 3 + 3 * 2 + 2, dtype=np.float32)
    p[:12] = np.array([1, 0, -1, 0.5, 0.25, 1, 0, 0, -0.5, 0, 1, 2], dtype=np.float32)
    p[15:21] = np.array([1, -1, 0.5, 0, 0.25, 1], dtype=np.float32)
    t = np.array([[0.25, -0.5], [1.0, 0.0]])
    l0, g0 = OM.loss_grad(p, widths, x, t, tf32=False)
    l1, g1 = OM.loss_grad(p, widths, x, t, tf32=True)
    assert l0 == l1 and np.array_equal(g0, g1)
