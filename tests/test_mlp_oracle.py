"""Pins of the surrogate's CPU statement: gradients against central finite
differences, the pinball loss against its quantile property, Adam against its
closed-form first step, feature symmetry."""
import numpy as np
import pytest

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


def test_error_head_loss_is_minimised_at_the_quantile():
    """For a constant error head the pinball term is minimised at the
    ERR_QUANTILE empirical quantile of the log errors (Koenker & Bassett 1978);
    a plain squared loss would put it at the mean instead."""
    rng = np.random.default_rng(4)
    et = rng.standard_normal(4001)
    # one-parameter model: the network's error output is a constant c
    grid = np.linspace(-3, 3, 6001)
    vals = []
    for cst in grid:
        u = et - cst
        vals.append(np.mean(u * np.where(u > 0, M.ERR_QUANTILE, M.ERR_QUANTILE - 1.0)))
    best = grid[int(np.argmin(vals))]
    assert abs(best - np.quantile(et, M.ERR_QUANTILE)) < 2e-3
    # and the oracle's loss gives that term for the error head
    params = [(np.zeros((5, 64)), np.zeros(64)), (np.zeros((64, 64)), np.zeros(64)),
              (np.zeros((64, 64)), np.zeros(64)), (np.zeros((64, 2)), np.array([0.0, 0.7]))]
    X = np.zeros((len(et), 5))
    y = np.zeros(len(et))
    loss, _ = M.loss_and_grads(params, X, y, lam=1.0, err_target=et)
    u = et - 0.7
    assert loss == pytest.approx(np.mean(u * np.where(u > 0, 0.95, -0.05)), rel=1e-12)


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
    # doubling every length leaves the geometric features unchanged
    f2 = M.features([200.0], [1800.0], [0.01], 1.0, 40.0)
    np.testing.assert_allclose(f2[0, :3], f1[0, :3], rtol=1e-14)
    # transverse offset at the geometric-mean distance, along-sightline offset
    f3 = M.features([400.0], [900.0], [0.02], 1.0, 20.0)[0]
    assert f3[1] == pytest.approx(500.0 / 60.0) and f3[2] == pytest.approx(0.02 * 600.0 / 60.0)
