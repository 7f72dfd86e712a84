"""Pins of the policy oracle (oracle/policy.py): gradients by central finite differences,
softmax cross-entropy on a hand-worked case, Lanczos Ritz values against exact
eigenvalues, and features against their definitions on matrices with known answers."""
import numpy as np
import pytest

from oracle import policy
from synth import dominant_spd, gram_spd, seed_for


def test_parameter_count():
    assert policy.NPARAM == 5512


def test_loss_hand_worked():
    # zero weights: every logit 0, softmax uniform over 8 classes, loss = log 8
    p = np.zeros(policy.NPARAM)
    X = np.random.default_rng(0).standard_normal((5, 12))
    loss, g = policy.loss_and_grad(p, X, np.array([0, 1, 2, 3, 7]))
    assert abs(loss - np.log(8.0)) < 1e-15
    # only b3 gets a gradient: mean of (1/8 - onehot)
    W1, b1, W2, b2, W3, b3 = policy.unpack(g)
    exp_b3 = np.full(8, 1 / 8.0) - np.bincount([0, 1, 2, 3, 7], minlength=8) / 5.0
    assert np.allclose(b3, exp_b3, atol=1e-15) and np.all(W1 == 0) and np.all(W3 == 0)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    p = rng.standard_normal(policy.NPARAM) * 0.3
    X = rng.standard_normal((7, 12))
    y = rng.integers(0, 8, size=7)
    _, g = policy.loss_and_grad(p, X, y)
    idx = rng.choice(policy.NPARAM, size=60, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = 1e-6
        fd = (policy.loss_and_grad(p + e, X, y)[0] - policy.loss_and_grad(p - e, X, y)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_lanczos_exact_on_small_and_diagonal():
    d = np.array([0.5, 2.0, 3.0, 7.5, 11.0])
    a, b = policy.lanczos(np.diag(d), 5)
    lo, hi = policy.ritz_extremes(a, b)
    assert abs(lo - 0.5) < 1e-12 and abs(hi - 11.0) < 1e-12
    A = dominant_spd(40, 1.2, seed_for(5, 1))
    ev = np.linalg.eigvalsh(A)
    lo, hi = policy.ritz_extremes(*policy.lanczos(A, 40))
    assert abs(lo - ev[0]) < 1e-9 * ev[-1] and abs(hi - ev[-1]) < 1e-9 * ev[-1]


def test_features_on_known_matrices():
    n = 64
    A = np.diag(np.arange(1.0, n + 1))
    f = policy.features(A, k=n)
    assert f[0] == 6.0 and f[1] == 1e6 and f[3] == 1.0
    assert abs(f[5] - np.log10(n)) < 1e-12 and abs(f[6]) < 1e-12
    assert abs(f[8] - np.log10(n)) < 1e-9 and abs(f[9]) < 1e-9
    assert abs(f[10] - np.log10(n)) < 1e-9
    A = dominant_spd(200, 2.0, seed_for(5, 2))
    f = policy.features(A)
    assert abs(f[1] - 2.0) < 1e-12 and abs(f[2] - 2.0) < 1e-12 and f[3] == 1.0
    G = gram_spd(128, 1e-2, seed_for(5, 3))
    f = policy.features(G)
    assert f[10] > 2.0                    # rank-deficient Gram + small shift: ill-conditioned


def test_order_gate_takes_the_smallest_order_from_which_the_policy_always_wins():
    import numpy as np

    from paper_2601_08082_gb300.train_policy import order_gate
    ns = np.array([1024] * 3 + [2048] * 3 + [4096] * 3 + [8192] * 3)
    t_feat = np.full(12, 1.0)
    t_fb = np.array([3.0] * 3 + [6.0] * 3 + [20.0] * 3 + [60.0] * 3)
    # the policy saves 0.5, 2, 5, 10 ms: it pays for the 1 ms pass from 2048 on
    t_pick = t_fb - np.repeat([0.5, 2.0, 5.0, 10.0], 3)
    gate, wins = order_gate(ns, t_feat, t_pick, t_fb)
    assert gate == 2048 and wins == {1024: False, 2048: True, 4096: True, 8192: True}
    # a loss at a larger order moves the gate above it
    t_pick2 = t_pick.copy()
    t_pick2[6:9] = t_fb[6:9]
    assert order_gate(ns, t_feat, t_pick2, t_fb)[0] == 8192
    # never wins: no order qualifies
    assert order_gate(ns, t_feat, t_fb.copy(), t_fb)[0] == 1 << 30
