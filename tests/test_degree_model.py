"""Learned filter degree: training-data assembly (CPU) and the CUDA perceptron (GPU):
forward and gradients against a NumPy float64 restatement, training, the untrained model
reproducing the closed-form rule, and a solve with a trained model."""
import math

import numpy as np
import pytest
import torch

import oracle.chfsi_oracle as O
from paper_1206_3768_gb300 import degree_model as dm
from paper_1206_3768_gb300 import inputs

DEV = "cuda"


def test_mlp_struct_layout_matches_the_parameter_count():
    import ctypes

    from paper_1206_3768_gb300 import binding as cb

    assert cb.MLP_NPARAM == 4 * 64 + 64 + 64 * 64 + 64 + 64 + 1
    assert ctypes.sizeof(cb.chfsi_mlp) == 4 * (cb.MLP_NPARAM + 2 * cb.MLP_IN)
    assert cb.chfsi_mlp.b3.offset == 4 * (cb.MLP_NPARAM - 1)


def _rec(p, k, g, i, m, th, r, tau, d, c, e, gap):
    return [p, k, g, i, m, th, r, tau, d, c, e, gap]


def test_training_pairs_recover_planted_rate():
    """A vector whose residual falls by exactly rho^(2d) per loop gives z = ln 2."""
    c, e, tau = 1.0, 0.5, 1e-10
    th = -0.5                        # t = (th - c)/e = -3
    t = 3.0
    lrho = math.log(t + math.sqrt(t * t - 1))
    d, r0 = 7, 1e-2
    r1 = r0 * math.exp(-2 * lrho * d)
    log = np.array([_rec(0, 3, 5, 2, 10, th, r0, tau, d, c, e, 0.1),
                    _rec(0, 4, 5, 1, 9, th, r1, tau, d, c, e, 0.1),
                    _rec(1, 4, 5, 1, 9, th, r1, tau, d, c, e, 0.1)])   # other problem: no pair
    X, z = dm.training_pairs(log)
    assert X.shape == (1, 4)
    assert abs(z[0] - math.log(2.0)) < 1e-6
    assert abs(X[0, 0] - lrho) < 1e-6 and abs(X[0, 1] - 8.0) < 1e-6
    assert abs(X[0, 2] - 0.2) < 1e-7 and abs(X[0, 3] - math.log10(0.2)) < 1e-6


def test_training_pairs_skip_converged_and_inside_interval():
    c, e, tau = 1.0, 0.5, 1e-10
    log = np.array([_rec(0, 0, 0, 0, 4, 1.2, 1e-3, tau, 5, c, e, 0.1),   # |t| <= 1
                    _rec(0, 1, 0, 0, 4, 1.2, 1e-4, tau, 5, c, e, 0.1),
                    _rec(0, 0, 1, 1, 4, -1.0, 1e-12, tau, 5, c, e, 0.1),  # r <= tau
                    _rec(0, 1, 1, 1, 4, -1.0, 1e-13, tau, 5, c, e, 0.1)])
    X, z = dm.training_pairs(log)
    assert X.shape[0] == 0


# ------------------------------------------------------------------------------ GPU
def _np_model(m):
    p = m.params().astype(np.float64)
    H, I = 64, 4
    w1 = p[:H * I].reshape(H, I); b1 = p[H * I:H * I + H]
    o = H * I + H
    w2 = p[o:o + H * H].reshape(H, H); b2 = p[o + H * H:o + H * H + H]
    o += H * H + H
    w3 = p[o:o + H]; b3 = p[o + H]
    mean = np.array(m.mean, np.float64); scale = np.array(m.scale, np.float64)
    return w1, b1, w2, b2, w3, b3, mean, scale


def _np_forward_grad(m, X, z):
    w1, b1, w2, b2, w3, b3, mean, scale = _np_model(m)
    xh = (X.astype(np.float64) - mean) * scale
    h1 = np.tanh(xh @ w1.T + b1)
    h2 = np.tanh(h1 @ w2.T + b2)
    y = h2 @ w3 + b3
    n = len(z)
    dy = (y - z) / n
    loss = 0.5 * np.mean((y - z) ** 2)
    gw3 = h2.T @ dy; gb3 = dy.sum()
    da2 = np.outer(dy, w3) * (1 - h2 ** 2)
    gw2 = da2.T @ h1; gb2 = da2.sum(0)
    da1 = (da2 @ w2) * (1 - h1 ** 2)
    gw1 = da1.T @ xh; gb1 = da1.sum(0)
    g = np.concatenate([gw1.ravel(), gb1, gw2.ravel(), gb2, gw3, [gb3]])
    return y, g, loss


def _random_model(cb, seed):
    m = cb.chfsi_mlp_init(seed)
    rng = np.random.default_rng(seed)
    for i in range(64):
        m.w3[i] = float(rng.normal(0, 0.3))
        m.b1[i] = float(rng.normal(0, 0.1))
        m.b2[i] = float(rng.normal(0, 0.1))
    m.b3 = 0.05
    for f in range(4):
        m.mean[f] = float(rng.normal(0, 0.5))
        m.scale[f] = float(rng.uniform(0.5, 2.0))
    return m


@pytest.mark.gpu
def test_mlp_forward_and_gradient_match_numpy():
    from paper_1206_3768_gb300 import binding as cb

    rng = np.random.default_rng(3)
    X = rng.normal(size=(300, 4)).astype(np.float32)
    z = rng.normal(size=300).astype(np.float32)
    m = _random_model(cb, 11)
    with cb.Solver(64, 8) as s:
        y = cb.chfsi_mlp_predict(s.ctx, m, X)
        g, loss = cb.chfsi_mlp_gradient(s.ctx, m, X, z)
    y_ref, g_ref, loss_ref = _np_forward_grad(m, X, z)
    assert np.max(np.abs(y - y_ref)) < 1e-5 * (1 + np.max(np.abs(y_ref)))
    assert abs(loss - loss_ref) < 1e-5 * loss_ref
    assert np.max(np.abs(g - g_ref)) < 1e-4 * np.max(np.abs(g_ref))


@pytest.mark.gpu
def test_mlp_training_fits_a_smooth_target():
    from paper_1206_3768_gb300 import binding as cb

    rng = np.random.default_rng(4)
    X = rng.normal(size=(4000, 4)).astype(np.float32)
    z = (0.5 * np.tanh(X[:, 0]) - 0.3 * X[:, 1] + 0.2 * X[:, 2] * X[:, 3]).astype(np.float32)
    m = cb.chfsi_mlp_init(5)
    with cb.Solver(64, 8) as s:
        _, loss0 = cb.chfsi_mlp_gradient(s.ctx, m, X, z)
        loss = cb.chfsi_mlp_train(s.ctx, m, X, z, epochs=60, batch=256, lr=3e-3, seed=7)
        _, loss1 = cb.chfsi_mlp_gradient(s.ctx, m, X, z)
    assert loss1 < 0.05 * loss0, (loss0, loss1, loss)


@pytest.mark.gpu
def test_untrained_model_reproduces_the_closed_form_degrees():
    from paper_1206_3768_gb300 import binding as cb

    rng = np.random.default_rng(6)
    m_act = 40
    theta = np.sort(rng.uniform(-1.0, 0.5, m_act))
    r = 10.0 ** rng.uniform(-11, -2, m_act)
    a, b, tau = 0.5, 3.0, 1e-10
    with cb.Solver(64, 64) as s:
        d0 = cb.chfsi_degrees(s.ctx, torch.tensor(theta, device=DEV), torch.tensor(r, device=DEV),
                              a, b, tau, 4, 40, 30)
        cb.chfsi_set_degree_model(s.ctx, cb.chfsi_mlp_init(9))
        d1 = cb.chfsi_degrees(s.ctx, torch.tensor(theta, device=DEV), torch.tensor(r, device=DEV),
                              a, b, tau, 4, 40, 30)
    ref = O.adaptive_degrees(theta, r, a, b, tau, 4, 40, 30)
    assert list(d0.cpu().numpy()) == list(ref)
    assert list(d1.cpu().numpy()) == list(ref)


@pytest.mark.gpu
def test_solve_with_a_model_trained_on_degree_logs():
    """Log degrees on a training sequence, train, install, and solve another sequence: the
    eigenpairs meet the same bar as with the closed form."""
    from paper_1206_3768_gb300 import binding as cb

    train = inputs.planted_sequence("c2", n=520, N=3, nev=20, blk=26, device=DEV, seed_offset=7)
    test = inputs.planted_sequence("c2", n=520, N=3, nev=20, blk=26, device=DEV)
    with cb.Solver(520, 26, deg_min=4, deg_max=40) as s:
        cb.chfsi_degree_log_start(s.ctx, 100000)
        cb.chfsi_reset_warm_state(s.ctx)
        _, _, st = cb.chfsi_solve_sequence(s.ctx, [p.A for p in train.problems], [p.B for p in train.problems],
                                           20, 26, 0, 1e-10)
        log = cb.chfsi_degree_log_read(s.ctx)
        assert log.shape[0] > 0
        X, z = dm.training_pairs(log)
        assert X.shape[0] > 50
        model = cb.chfsi_mlp_init(3)
        cb.chfsi_mlp_train(s.ctx, model, X, z, epochs=40, batch=128, lr=2e-3, seed=1)
        cb.chfsi_degree_log_start(s.ctx, 0)
        cb.chfsi_set_degree_model(s.ctx, model)
        cb.chfsi_reset_warm_state(s.ctx)
        ev, X_out, st = cb.chfsi_solve_sequence(s.ctx, [p.A for p in test.problems], [p.B for p in test.problems],
                                                20, 26, 0, 1e-10)
    scale = max(float(np.max(np.abs(p.lam))) for p in test.problems)
    for ell, p in enumerate(test.problems):
        assert np.max(np.abs(ev[ell].numpy() - p.lam[:20])) <= 1e-10 * scale
        assert st[ell]["max_resid"] <= 1e-10
