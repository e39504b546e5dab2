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
