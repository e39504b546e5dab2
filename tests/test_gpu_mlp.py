"""Tensor-core surrogate network against the oracle (learned proposal).

The oracle evaluates the same network in FP64, rounding to bfloat16 at the
points where the kernels feed a tensor-core product (x, h1, h2, dz2, dz1);
parameters are bfloat16-exact.  The remaining differences are the FP32
accumulation of the products (relative 2^-24 per term, 64 terms) and tanhf,
which move a rounding decision to the neighbouring bfloat16 (relative step
2^-8) in a small fraction of the activations."""
import numpy as np
import pytest
import torch

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2311_12973_gb300 import smc2
    return smc2


def bf16_params(D, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(O.mlp_nparams(D)) * scale
    return np.array([O.bf16(v) for v in p])


@pytest.mark.parametrize("D,R", [(4, 256), (3, 100), (4, 1000), (8, 64)])
def test_loss_gradient_against_oracle(S, D, R):
    rng = np.random.default_rng(D + R)
    p = bf16_params(D, R)
    x = rng.standard_normal((R, D))
    y = rng.standard_normal(R)
    loss_o, g_o = O.mlp_loss_grad(p, x, y, bf16_points=True)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    loss_g, g_g = S.mlp_loss_grad(t(p), t(x), t(y))
    loss_g, g_g = float(loss_g.item()), g_g.cpu().numpy().astype(np.float64)
    rel_norm = np.linalg.norm(g_g - g_o) / np.linalg.norm(g_o)
    rel_elem = np.max(np.abs(g_g - g_o) / (np.abs(g_o) + 1e-2 * np.max(np.abs(g_o))))
    print(f"D={D} R={R} loss {loss_g:.8g} vs {loss_o:.8g}  grad rel norm {rel_norm:.3g}  elem {rel_elem:.3g}")
    # measured on GB300: loss 4e-6, norm <= 2.4e-5, element <= 1e-3 (one bf16 step of
    # an activation is 2^-8 = 4e-3 of its contribution; a few flips per R rows)
    assert abs(loss_g - loss_o) <= 1e-4 * abs(loss_o)
    assert rel_norm < 2e-4
    assert rel_elem < 5e-3


@pytest.mark.parametrize("D,R", [(4, 300), (3, 64)])
def test_input_gradient_against_oracle(S, D, R):
    rng = np.random.default_rng(5 * D + R)
    p = bf16_params(D, 9)
    x = rng.standard_normal((R, D))
    s_o, dx_o = O.mlp_input_grad(p, x, bf16_points=True)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    s_g, dx_g = S.mlp_input_grad(t(p), t(x))
    s_g, dx_g = s_g.cpu().numpy(), dx_g.cpu().numpy()
    es = np.max(np.abs(s_g - s_o)) / np.max(np.abs(s_o))
    ed = np.linalg.norm(dx_g - dx_o) / np.linalg.norm(dx_o)
    print(f"D={D} R={R} s err {es:.3g}  dx rel norm {ed:.3g}")
    assert es < 2e-3   # one bf16 step of an h2 value moves s by up to |w3| 2^-8
    assert ed < 1e-3


def weights_bf16(p, D, H=64):
    """W1 [D][H], W2 [H][H] and w3 [H] rounded to bfloat16; b1, b2, b3 unchanged."""
    q = np.array(p, dtype=np.float64)
    blocks = [(0, D * H), (D * H + H, D * H + H + H * H), (D * H + 2 * H + H * H, D * H + 3 * H + H * H)]
    for a, b in blocks:
        q[a:b] = [O.bf16(v) for v in q[a:b]]
    return q


@pytest.mark.parametrize("D,R", [(4, 300), (3, 1000)])
def test_adam_step_against_oracle(S, D, R):
    """Three training steps as the sampler takes them.  Each step is checked
    stage-wise from the device's own state: the loss and the moments m, v (both
    linear in the gradient) against the oracle's bf16-point gradient at the
    device parameters, then the parameter update against Adam's formula
    evaluated in FP64 from the device moments."""
    rng = np.random.default_rng(7 * D + R)
    x = rng.standard_normal((R, D))
    y = rng.standard_normal(R)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    params, xs, ys = t(bf16_params(D, R)), t(x), t(y)
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    lr = 1e-2
    b1, b2, eps = (float(np.float32(c)) for c in (0.9, 0.999, 1e-8))  # as the FP32 kernel holds them
    for it in range(1, 4):
        p0, m0, v0 = (a.cpu().numpy().astype(np.float64) for a in (params, m, v))
        loss = float(S.mlp_adam_step(params, m, v, step, xs, ys, lr).item())
        assert int(step.item()) == it
        # the kernels use the weights W1, W2, w3 rounded to bfloat16 and the biases as they are
        loss_o, g_o = O.mlp_loss_grad(weights_bf16(p0, D), x, y, bf16_points=True)
        p1, m1, v1 = (a.cpu().numpy().astype(np.float64) for a in (params, m, v))
        scale = np.max(np.abs(g_o))
        # moments: the gradient bar of the test above (5e-3 of the largest element)
        assert abs(loss - loss_o) <= 1e-4 * abs(loss_o)
        m_g, v_g = m0.copy(), v0.copy()   # the oracle's moments after its step on g_o
        O.adam_step(p0.copy(), g_o, m_g, v_g, it, lr, b1, b2, eps)
        assert np.max(np.abs(m1 - m_g)) <= (1 - b1) * 5e-3 * scale
        assert np.max(np.abs(v1 - v_g)) <= (1 - b2) * 1e-2 * scale * scale
        # the update: the oracle's Adam on the gradient the device used (read from its first
        # moment), from the device's moments: FP32 arithmetic, relative 1e-5 of a step of size lr
        g_dev = (m1 - b1 * m0) / (1 - b1)
        p_o, m_o, v_o = p0.copy(), m0.copy(), v0.copy()
        O.adam_step(p_o, g_dev, m_o, v_o, it, lr, b1, b2, eps)
        assert np.max(np.abs(v1 - v_o)) <= 1e-5 * np.max(v_o) + 1e-30
        assert np.max(np.abs(p1 - p_o)) <= 1e-5 * lr + 4e-7 * np.max(np.abs(p0))
