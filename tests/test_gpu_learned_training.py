"""The learned proposal's training call on the device against the oracle
(choice L2's training set and L1's Adam steps; not in the paper).

Stage-wise on identical inputs: the standardisation of a ring of (theta, log
pi^) rows; each Adam step from the device's own state (the gradient through
the moments, the update through the oracle's Adam); a many-step call equal to
the same number of single steps bit for bit; and the oracle's own training
call from the same start, compared on the trained network's outputs.  In the
sampler: each in-run call equals the training call on the read-back ring and
state, and its result is published for the iteration after next."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2311_12973_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LR = 5e-3
# Adam's constants as the FP32 kernel holds them (0.999 in float is 0.99900001287, so
# 1 - beta2 differs from 1e-3 by 1.3e-5 relative)
B1, B2, EPS = (float(np.float32(c)) for c in (0.9, 0.999, 1e-8))


@pytest.fixture(scope="module")
def S():
    from paper_2311_12973_gb300 import smc2
    return smc2


def _ring(rng, R, D, n_low=30, n_inf=7):
    """Rows around a Gaussian target in float32: some far below the clip, some -inf."""
    mu = rng.standard_normal(D)
    sc = np.linspace(0.3, 1.2, D)
    th = (mu + rng.standard_normal((R, D)) * sc).astype(np.float32)
    lp = (-0.5 * np.sum(((th - mu) / sc) ** 2, axis=1) - 55.0).astype(np.float32)
    lp[:n_low] -= 500.0
    lp[n_low:n_low + n_inf] = -np.inf
    return th, lp


def _xavier(rng, D, H=64):
    lim = np.concatenate([np.full(D * H, math.sqrt(6 / (D + H))), np.zeros(H), np.full(H * H, math.sqrt(6 / (2 * H))),
                          np.zeros(H), np.full(H, math.sqrt(6 / (H + 1))), np.zeros(1)])
    return ((rng.random(len(lim)) * 2 - 1) * lim).astype(np.float32)


def _dev(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _host(t):
    return t.cpu().numpy().astype(np.float64)


def _check_standardisation(sd, x, y, th, lp):
    """Device training set (FP32 moments) against the oracle's FP64 one from the same rows."""
    x_o, y_o, nm = O.mlp_standardise(th.astype(np.float64), lp.astype(np.float64))
    D = th.shape[1]
    assert sd["tau"] == nm["tau"] and sd["var_y"] == nm["var_y"]
    assert sd["ymax"] == nm["ymax"]                 # the largest float row, exactly
    assert np.allclose(sd["mu"], nm["mu"], rtol=0, atol=2e-6 * (np.abs(nm["mu"]) + nm["sd"]))
    assert np.allclose(sd["sd"], nm["sd"], rtol=2e-5)
    assert abs(sd["zmean"] - nm["zmean"]) <= 2e-5 * (1 + abs(nm["zmean"]))
    assert abs(sd["zsd"] - nm["zsd"]) <= 2e-5 * nm["zsd"]
    assert np.max(np.abs(_host(x) - x_o) / (1 + np.abs(x_o))) <= 2e-5
    assert np.max(np.abs(_host(y) - y_o) / (1 + np.abs(y_o))) <= 2e-5
    return x_o, y_o, nm


def _outputs(params, x):
    """The trained network's outputs as the kernels evaluate it (bf16 points)."""
    return O.mlp_forward(O.mlp_weights_bf16(params, x.shape[1]), x, bf16_points=True)


@pytest.mark.parametrize("D,R", [(4, 1000), (3, 4096), (2, 300)])
def test_training_call_stagewise_against_oracle(S, D, R):
    rng = np.random.default_rng(100 * D + R)
    th, lp = _ring(rng, R, D)
    p_init = _xavier(rng, D)
    params, m, v = _dev(p_init), _dev(np.zeros_like(p_init)), _dev(np.zeros_like(p_init))
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    th_d, lp_d = _dev(th), _dev(lp)

    # standardisation only (no step)
    x, y, sd = S.mlp_train_ring(params, m, v, step, th_d, lp_d, 0, LR)
    assert int(step.item()) == 0 and np.array_equal(params.cpu().numpy(), p_init)
    _check_standardisation(sd, x, y, th, lp)
    xd, yd = _host(x), _host(y)

    # sixteen single steps, each stage-wise from the device's own state
    for it in range(1, 17):
        p0, m0, v0 = _host(params), _host(m), _host(v)
        x, y, sd = S.mlp_train_ring(params, m, v, step, th_d, lp_d, 1, LR)
        assert int(step.item()) == it
        p1, m1, v1 = _host(params), _host(m), _host(v)
        # the gradient the device used, from its first moment, against the oracle's at its inputs
        loss_o, g_o = O.mlp_loss_grad(O.mlp_weights_bf16(p0, D), xd, yd, bf16_points=True)
        g_dev = (m1 - B1 * m0) / (1 - B1)
        scale = np.max(np.abs(g_o))
        assert abs(sd["loss"] - loss_o) <= 1e-4 * loss_o, (it, sd["loss"], loss_o)
        assert np.max(np.abs(g_dev - g_o)) <= 5e-3 * scale, (it, np.max(np.abs(g_dev - g_o)) / scale)
        # the update: the oracle's Adam on that gradient, from the device's moments
        p_o, m_o, v_o = p0.copy(), m0.copy(), v0.copy()
        O.adam_step(p_o, g_dev, m_o, v_o, it, LR, B1, B2, EPS)
        assert np.max(np.abs(v1 - v_o)) <= 1e-5 * np.max(v_o) + 1e-30
        assert np.max(np.abs(p1 - p_o)) <= 1e-5 * LR + 4e-7 * np.max(np.abs(p0))
    p16 = params.cpu().numpy().copy()

    # one sixteen-step call from the same start: the same parameters, bit for bit
    params2, m2, v2 = _dev(p_init), _dev(np.zeros_like(p_init)), _dev(np.zeros_like(p_init))
    step2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    _, _, sd16 = S.mlp_train_ring(params2, m2, v2, step2, th_d, lp_d, 16, LR)
    assert int(step2.item()) == 16 and np.array_equal(params2.cpu().numpy(), p16)
    assert np.array_equal(m2.cpu().numpy(), m.cpu().numpy()) and np.array_equal(v2.cpu().numpy(), v.cpu().numpy())

    # the oracle's own sixteen-step call from the same start, on the trained network's outputs
    z = np.zeros(len(p_init))
    p_or, _, _, t_or, loss_or, nm, x_o, y_o = O.mlp_train(p_init.astype(np.float64), z, z, 0, th, lp, 16, LR)
    assert t_or == 16
    s_dev, s_or = _outputs(p16.astype(np.float64), x_o), _outputs(p_or, x_o)
    ds = np.max(np.abs(s_dev - s_or))
    print(f"D={D} R={R}: loss dev {sd16['loss']:.5f} oracle {loss_or:.5f}; max |s_dev - s_oracle| {ds:.3g}")
    assert abs(sd16["loss"] - loss_or) <= 0.02 * loss_or
    assert ds <= 0.02


def test_training_call_edge_rows(S):
    """Fewer than 2 D + 2 rows above the clip (moments over every finite row),
    and constant targets (target variance 0)."""
    D, R = 3, 64
    rng = np.random.default_rng(7)
    th = rng.standard_normal((R, D)).astype(np.float32)
    lp = np.full(R, -1e4, dtype=np.float32)
    lp[:3] = [0.0, -1.0, -2.5]
    lp[50:] = -np.inf
    p = _dev(_xavier(rng, D))
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    x, y, sd = S.mlp_train_ring(p, m, v, step, _dev(th), _dev(lp), 0, LR)
    _, _, nm = _check_standardisation(sd, x, y, th, lp)
    assert nm["rows_moments"] == 50
    x, y, sd = S.mlp_train_ring(p, m, v, step, _dev(th), _dev(np.full(R, -7.0, dtype=np.float32)), 0, LR)
    assert sd["var_y"] == 0.0 and sd["zsd"] == 1.0 and np.all(y.cpu().numpy() == 0.0)


def test_in_run_training_is_the_training_call_and_is_published_two_iterations_later(S):
    """Choice L5's schedule: the call after iteration k continues the previous
    call's state on the ring holding iterations k - W + 1 .. k; the proposal of
    iteration k + 2 reads its result."""
    w = I.workload("seir_t100_n1024_mlp", N=256, M=128, T=40, K=9, precision=I.PREC_FP64)
    ctx = S.SMC2(S.make_config(w), w.y)
    W, N, D = 4, w.N, w.D
    steps = 16
    ctx.run(1)
    prev = ctx.learned_training()
    worst = 0.0
    for k in range(2, w.K + 1):
        ctx.run(1)
        cur = ctx.learned_training()
        pub = ctx.learned_state()
        # the ring: iteration k's proposals in rows ((k - 1) mod W) N ...
        assert cur["ring_rows"] == min(k, W) * N
        th_k, _ = ctx.proposals()
        r0 = ((k - 1) % W) * N
        assert np.array_equal(cur["ring_th"][r0:r0 + N], th_k.astype(np.float32))
        # the in-run call = the training call on that ring from the previous call's state
        p, m, v = _dev(prev["params"]), _dev(prev["m"]), _dev(prev["v"])
        step = torch.tensor([prev["step"]], dtype=torch.int32, device="cuda")
        _, _, sd = S.mlp_train_ring(p, m, v, step, _dev(cur["ring_th"]), _dev(cur["ring_lp"]), steps, LR)
        assert int(step.item()) == cur["step"] == prev["step"] + steps
        assert np.array_equal(p.cpu().numpy(), cur["params"]) and np.array_equal(m.cpu().numpy(), cur["m"])
        assert sd["loss"] == cur["loss"] and np.array_equal(sd["mu"], cur["mu"])
        # published after iteration k: the state trained after iteration k - 1
        assert np.array_equal(pub["params"], prev["params"]) and pub["loss"] == prev["loss"]
        assert np.array_equal(pub["mu"], prev["mu"]) and pub["zsd"] == prev["zsd"]
        # the oracle's training call from the same state on the same ring, on the network's outputs
        p_or, _, _, t_or, loss_or, nm, x_o, _ = O.mlp_train(prev["params"].astype(np.float64),
                                                              prev["m"].astype(np.float64),
                                                              prev["v"].astype(np.float64), prev["step"],
                                                              cur["ring_th"], cur["ring_lp"], steps, LR)
        ds = np.max(np.abs(_outputs(cur["params"].astype(np.float64), x_o) - _outputs(p_or, x_o)))
        worst = max(worst, ds)
        assert t_or == cur["step"]
        assert abs(cur["loss"] - loss_or) <= 0.02 * loss_or + 1e-4, (k, cur["loss"], loss_or)
        assert ds <= 0.02, (k, ds)
        prev = cur
    print(f"largest |s_dev - s_oracle| over the in-run calls: {worst:.3g}")
    ctx.close()
