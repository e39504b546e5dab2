"""Pins of the oracle's surrogate network (learned proposal; not in the paper).

Gradients are pinned by central finite differences of the oracle's own loss
and output in FP64; bfloat16 rounding by its definition (nearest of the 8-bit
mantissa grid, ties to even); Adam by its closed form on a quadratic."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def rand_params(D, H, seed):
    rng = np.random.default_rng(seed)
    P = O.mlp_nparams(D, H)
    p = rng.standard_normal(P) * 0.3
    return p


@pytest.mark.parametrize("D,H", [(3, 8), (4, 64)])
def test_loss_gradient_matches_finite_differences(D, H):
    rng = np.random.default_rng(D * H)
    p = rand_params(D, H, 1)
    x = rng.standard_normal((17, D))
    y = rng.standard_normal(17)
    loss, g = O.mlp_loss_grad(p, x, y, H=H)
    idx = rng.choice(len(p), size=min(len(p), 40), replace=False)
    for q in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[q] += h
        pm[q] -= h
        fd = (O.mlp_loss_grad(pp, x, y, H=H)[0] - O.mlp_loss_grad(pm, x, y, H=H)[0]) / (2 * h)
        assert g[q] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    assert loss == pytest.approx(np.mean((O.mlp_forward(p, x, H=H) - y) ** 2), rel=1e-14)


@pytest.mark.parametrize("D,H", [(3, 8), (4, 64)])
def test_input_gradient_matches_finite_differences(D, H):
    rng = np.random.default_rng(7)
    p = rand_params(D, H, 2)
    x = rng.standard_normal((5, D))
    s, dx = O.mlp_input_grad(p, x, H=H)
    np.testing.assert_allclose(s, O.mlp_forward(p, x, H=H), rtol=1e-14)
    for r in range(5):
        for d in range(D):
            h = 1e-6
            xp, xm = x.copy(), x.copy()
            xp[r, d] += h
            xm[r, d] -= h
            fd = (O.mlp_forward(p, xp, H=H)[r] - O.mlp_forward(p, xm, H=H)[r]) / (2 * h)
            assert dx[r, d] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_bf16_rounding():
    assert O.bf16(1.0) == 1.0
    assert O.bf16(1.0 + 2 ** -8) == 1.0              # tie: to even (fraction 0)
    assert O.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6  # tie: to even (fraction 2)
    assert O.bf16(1.0 + 2 ** -7) == 1.0 + 2 ** -7      # exact
    assert O.bf16(1.0 + 2 ** -7 + 2 ** -9) == 1.0 + 2 ** -7
    assert O.bf16(-3.14159265) == -3.140625
    rng = np.random.default_rng(3)
    for v in rng.standard_normal(200) * 10:
        r = O.bf16(v)
        assert abs(r - v) <= abs(v) * 2 ** -8 + 1e-300
        m, e = math.frexp(r)
        assert (m * 256) == int(m * 256)               # 8 significant bits


def test_adam_closed_form():
    # first step of Adam moves each parameter by lr * sign(g) (bias-corrected moments)
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    O.adam_step(p, g, m, v, 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(p, [0.99, -1.99, 0.49], rtol=1e-12)
    # on f(p) = p^2 / 2 Adam converges to the minimum
    p = np.array([3.0])
    m, v = np.zeros(1), np.zeros(1)
    for t in range(1, 3001):
        O.adam_step(p, p.copy(), m, v, t, lr=0.01)
    assert abs(p[0]) < 1e-2
