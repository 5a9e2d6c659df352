"""Pins of the surrogate's CPU statement: gradients against central finite
differences, Adam against its closed-form first step, feature symmetry."""
import numpy as np

from oracle import mlp_oracle as M


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    params = M.init_params(1)
    X = rng.standard_normal((17, 5))
    y = rng.standard_normal(17)
    out, _ = M.forward(params, X)
    et = np.log(np.abs(out[:, 0] - y) + M.ERR_FLOOR)   # stop-gradient target, frozen
    loss, grads = M.loss_and_grads(params, X, y, lam=0.3, err_target=et)
    h = 1e-6
    for k, (W, b) in enumerate(params):
        for (arr, g) in ((W, grads[k][0]), (b, grads[k][1])):
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp, _ = M.loss_and_grads(params, X, y, lam=0.3, err_target=et)
                flat[idx] = old - h
                lm, _ = M.loss_and_grads(params, X, y, lam=0.3, err_target=et)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx)


def test_adam_first_step_is_signed_lr():
    """After one step from zero moments, Adam moves every parameter by
    lr * g / (|g| + eps) (bias corrections cancel)."""
    params = [(np.array([[1.0, -2.0]]), np.array([0.5, 0.0]))]
    grads = [(np.array([[0.3, -4.0]]), np.array([1e-3, -2.0]))]
    st = M.adam_init(params)
    new, _ = M.adam_step(params, grads, st, lr=0.01)
    for (p, g), q in zip(((params[0][0], grads[0][0]), (params[0][1], grads[0][1])), new[0]):
        np.testing.assert_allclose(q, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_features_symmetric_and_scale_free():
    f1 = M.features([100.0, 900.0], [900.0, 100.0], [0.01, 0.01], 1.0, 20.0)
    np.testing.assert_array_equal(f1[0], f1[1])
    # doubling every length leaves the first three features unchanged
    f2 = M.features([200.0], [1800.0], [0.01], 1.0, 40.0)
    np.testing.assert_allclose(f2[0, :3], f1[0, :3], rtol=1e-14)
