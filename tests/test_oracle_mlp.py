"""Pins of the float64 MLP reference (CPU only): finite differences, closed forms."""
import numpy as np

from oracle import mlp


def small_net(rng, dims):
    return [(rng.normal(size=(a, b)) * 0.5, rng.normal(size=b) * 0.1) for a, b in zip(dims[:-1], dims[1:])]


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    dims = [5, 7, 6, 3]
    layers = small_net(rng, dims)
    x = rng.normal(size=(9, 5))
    y = rng.normal(size=(9, 3))
    for tau in (0.99, 0.5, 0.1):
        loss, grads = mlp.loss_and_grads(layers, x, y, tau)
        flat = mlp.flatten(layers)
        g = mlp.flatten(grads)
        h = 1e-6
        num = np.zeros_like(flat)
        for i in range(flat.size):
            fp, fm = flat.copy(), flat.copy()
            fp[i] += h
            fm[i] -= h
            lp = mlp.loss_and_grads(mlp.unflatten(fp, dims), x, y, tau)[0]
            lm = mlp.loss_and_grads(mlp.unflatten(fm, dims), x, y, tau)[0]
            num[i] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-8)


def test_forward_by_hand():
    # 2 -> 2 -> 1 with hand-picked weights: y = relu(x W1 + b1) W2 + b2
    W1 = np.array([[1.0, -1.0], [2.0, 0.5]]); b1 = np.array([0.0, -1.0])
    W2 = np.array([[3.0], [-2.0]]); b2 = np.array([0.25])
    x = np.array([[1.0, 1.0], [-1.0, 0.0]])
    # row 0: z1 = (3, -1.5) -> (3, 0) -> 9.25 ; row 1: z1 = (-1, 0) -> (0, 0) -> 0.25
    y = mlp.forward([(W1, b1), (W2, b2)], x)[-1]
    np.testing.assert_allclose(y, [[9.25], [0.25]])


def test_pinball_special_cases():
    yhat = np.array([[0.0], [1.0], [3.0]])
    y = np.array([[1.0], [1.0], [1.0]])
    loss, d = mlp.pinball(yhat, y, 0.5)
    assert np.isclose(loss, 0.5 * np.mean(np.abs(y - yhat)))
    loss, d = mlp.pinball(yhat, y, 0.99)
    assert np.isclose(loss, (0.99 * 1.0 + 0.0 + 0.01 * 2.0) / 3)
    np.testing.assert_allclose(d.ravel(), np.array([-0.99, 0.01, 0.01]) / 3)


def test_adam_first_step_closed_form():
    p = np.array([1.0, -2.0, 0.5]); g = np.array([0.3, -4.0, 1e-3])
    p1, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> p - lr * g / (|g| + eps)
    np.testing.assert_allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8))


def test_capacity_rounding():
    yhat = np.log(np.array([[100.0, 5.0], [1e9, 1.0]]))
    cap = mlp.capacity(yhat, 0.1, 128, np.array([[4096, 4096], [4096, 4096]]), np.array([[10, 200], [0, 0]]))
    assert cap.tolist() == [[128, 256], [4096, 128]]


def test_features_by_hand():
    """The twelve inputs of the capacity network, computed by hand for three
    models: log1p of the side and of the two initial populations, each rule
    parameter over its nominal value with both read as unsigned 32-bit words
    (thresholds of 2^31 and above are stored as negative int32), and the
    horizon over 500."""
    T_s, T_w, T_g = 171798691, 214748364, 2**31  # floor(0.04 2^32), floor(0.05 2^32), 0.5
    as_i32 = lambda v: v - 2**32 if v >= 2**31 else v  # noqa: E731
    nominal = [4, 20, T_s, T_w, 30, 1, 1, as_i32(T_g)]
    table = np.array([
        # side, n0 sheep, n0 wolves, 8 params, horizon
        [16, 100, 25, 4, 20, T_s, T_w, 30, 1, 1, as_i32(T_g), 200],
        [256, 0, 13106, 5, 15, as_i32(0xC0000000), T_w // 2, 38, 1, 1, as_i32(0xFFFFFFFF), 500],
        [40, 1, 2, 3, 25, 0, 2**31 - 1, 22, 2, 1, 0, 1],
    ], dtype=np.int64)
    x = mlp.features(table.astype(np.int32), np.array(nominal, dtype=np.int32))
    want = np.array([
        [np.log(17.0), np.log(101.0), np.log(26.0), 1, 1, 1, 1, 1, 1, 1, 1, 0.4],
        # 0xC0000000 / T_s: T_s * 18.75 = 3221225456.25, so 18.75 + 15.75 / T_s;
        # T_w // 2 / T_w = 107374182 / 214748364 = 0.5; 0xFFFFFFFF / 2^31 = 2 - 2^-31
        [np.log(257.0), 0.0, np.log(13107.0), 1.25, 0.75, 18.75 + 15.75 / T_s, 0.5, 38 / 30, 1, 1,
         2.0 - 2.0**-31, 1.0],
        # (2^31 - 1) / T_w = 10 + 7 / T_w  (T_w * 10 = 2147483640)
        [np.log(41.0), np.log(2.0), np.log(3.0), 0.75, 1.25, 0.0, 10 + 7 / T_w, 22 / 30, 2, 1, 0.0, 0.002],
    ])
    assert x.shape == (3, 12)
    np.testing.assert_allclose(x, want, rtol=1e-14, atol=0)
