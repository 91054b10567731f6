"""Pins of the oracle CNN: gradients against central finite differences of the
loss (FP64), the conv against a direct sum, and Adam against its first-step form."""
import numpy as np
import pytest

from oracle import cnn as oc


def _data(B, L, seed):
    rng = np.random.default_rng(seed)
    snr = rng.normal(size=(B, L))
    harm = [rng.normal(size=(B, L)) for _ in range(oc.IN_CH - 2)]
    x0 = np.stack([snr, (rng.uniform(size=(B, L)) > 0.2)] + harm, axis=-1).astype(np.float64)
    labels = np.zeros((B, L))
    labels[:, L // 3] = 1.0
    return x0, labels


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 11, 3))
    W = rng.normal(size=(9, 4, 3))
    b = rng.normal(size=4)
    y = oc.conv(x, W, b)
    for bb in range(2):
        for l in range(11):
            for co in range(4):
                s = b[co]
                for k in range(9):
                    ll = l + k - 4
                    if 0 <= ll < 11:
                        s += W[k, co] @ x[bb, ll]
                assert y[bb, l, co] == pytest.approx(s, abs=1e-12)


def test_gradients_match_finite_differences():
    x0, labels = _data(1, 24, 3)
    params = oc.init_params(5) * 0.5
    params[-1] = -1.0
    loss, grads = oc.backward(params, x0, labels, 20.0)
    rng = np.random.default_rng(9)
    idx = np.concatenate([rng.choice(oc.N_PARAMS, 40, replace=False), [oc.N_PARAMS - 1, 0, 1216]])
    for i in idx:
        e = 1e-6
        pp, pm = params.copy(), params.copy()
        pp[i] += e
        pm[i] -= e
        lp = oc.bce(oc.forward(pp, x0)[0], labels, 20.0)[0]
        lm = oc.bce(oc.forward(pm, x0)[0], labels, 20.0)[0]
        fd = (lp - lm) / (2 * e)
        assert grads[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i


def test_adam_first_step_is_signed_lr():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 4.0])
    p1, m, v = oc.adam(p, g, np.zeros(3), np.zeros(3), 1, 0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> step = lr g / (|g| + eps)
    np.testing.assert_allclose(p1, p - 0.01 * np.sign(g), rtol=1e-6)


def test_round_bf16_values():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: to even (1); 1 + 3*2^-9 rounds up
    assert oc.round_bf16(1.0 + 2 ** -8) == 1.0
    assert oc.round_bf16(1.0 + 3 * 2 ** -9) == 1.0 + 2 ** -7
    assert oc.round_bf16(-3.140625) == -3.140625
    x = np.random.default_rng(0).normal(size=1000)
    r = oc.round_bf16(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8)


def test_bf16_mode_equals_fp64_mode_on_representable_data():
    # with BF16-exact weights and inputs the rounding points only round activations:
    # gradients agree to the BF16 precision
    x0, labels = _data(1, 32, 4)
    params = oc.round_bf16(oc.init_params(6) * 0.5)
    l64, g64 = oc.backward(params, x0, labels, 10.0)
    l16, g16 = oc.backward(params, x0, labels, 10.0, bf16=True)
    assert l16 == pytest.approx(l64, rel=2e-2)
    assert np.dot(g16, g64) / (np.linalg.norm(g16) * np.linalg.norm(g64)) > 0.99
