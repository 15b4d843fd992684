"""Pins of the oracle's surrogate network: a closed form with zeroed
layers, SiLU identities, and central finite differences of the loss on
every kind of parameter."""
import math

import numpy as np
import pytest


def _params(H, seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(2 * H * H + 7 * H + 1) * scale).astype(np.float32)


def _slices(H):
    sizes = [3 * H, H, H * H, H, H * H, H, H, 1]
    names = ["W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"]
    out, o = {}, 0
    for n, sz in zip(names, sizes):
        out[n] = slice(o, o + sz)
        o += sz
    return out


def test_closed_form_with_zeroed_layers(orc):
    """W1 = b1 = W2 = b2 = W3 = 0: f = w4 . s(b3) + b4; with b3 = ln 3,
    s(ln 3) = ln 3 / (1 + 1/3) = 0.75 ln 3."""
    H = 4
    sl = _slices(H)
    p = np.zeros(2 * H * H + 7 * H + 1, np.float32)
    p[sl["b3"]] = np.float32(math.log(3.0))
    p[sl["w4"]] = np.array([1.0, -2.0, 0.5, 0.25], np.float32)
    p[sl["b4"]] = 0.125
    x = np.random.default_rng(0).normal(size=(5, 3)).astype(np.float32)
    f = orc.mlp_forward(p, x, H)
    b3 = float(np.float32(math.log(3.0)))
    want = (1.0 - 2.0 + 0.5 + 0.25) * (b3 / (1.0 + math.exp(-b3))) + 0.125
    assert np.allclose(f, want, rtol=0, atol=1e-12)
    assert abs(b3 / (1 + math.exp(-b3)) - 0.75 * b3) < 1e-7


def test_silu_identities_through_the_net(orc):
    """With one unit per layer and identity-like weights the net composes
    s three times: check s(-z) = s(z) - z on the first layer's output."""
    H = 1
    sl = _slices(H)
    p = np.zeros(2 + 7 + 1, np.float32)
    p[sl["W1"]] = [1.0, 0.0, 0.0]
    p[sl["W2"]] = 1.0
    p[sl["W3"]] = 1.0
    p[sl["w4"]] = 1.0
    s = lambda z: z / (1 + math.exp(-z))
    for z in (-3.0, -0.5, 0.0, 0.75, 4.0):  # float32-exact inputs
        x = np.array([[z, 9.0, -9.0]], np.float32)
        assert orc.mlp_forward(p, x, H)[0] == pytest.approx(s(s(s(z))), abs=1e-14)
        assert s(-z) == pytest.approx(s(z) - z, abs=1e-14)


@pytest.mark.parametrize("H,ow", [(3, 1.0), (8, 1.0), (8, 4.0)])
def test_gradients_match_finite_differences(orc, H, ow):
    rng = np.random.default_rng(H)
    p = _params(H, H)
    x = rng.uniform(-0.8, 0.8, (6, 3)).astype(np.float32)
    # targets on both sides of the network's output
    y = (orc.mlp_forward(p, x, H) + np.array([0.3, -0.2, 0.25, -0.3, 0.1, -0.15])).astype(np.float32)
    loss, g = orc.mlp_grads(p, x, y, H, over_weight=ow)
    r = orc.mlp_forward(p, x, H) - y
    assert (r > 0).any() and (r < 0).any()
    assert loss == pytest.approx(np.mean(np.where(r > 0, ow, 1.0) * r ** 2), rel=1e-12)
    h = 2.0 ** -14  # parameters are float32: the step actually taken is used below
    for name, sl in _slices(H).items():
        idx = np.arange(sl.start, sl.stop)
        for i in rng.choice(idx, min(6, idx.size), replace=False):
            pp, pm = p.copy(), p.copy()
            pp[i] += np.float32(h)
            pm[i] -= np.float32(h)
            dh = float(pp[i]) - float(pm[i])
            fd = (orc.mlp_grads(pp, x, y, H, over_weight=ow)[0]
                  - orc.mlp_grads(pm, x, y, H, over_weight=ow)[0]) / dh
            assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9), (name, i)


def test_bf16_activation_rounding_points(orc):
    """One unit per layer: the bfloat16 variant rounds s(z1) and s(z2) (via
    float32, ties to even, as torch's bfloat16 cast does) and nothing else."""
    import torch
    H = 1
    sl = _slices(H)
    p = np.zeros(10, np.float32)
    p[sl["W1"]] = [1.0, 0.0, 0.0]
    p[sl["W2"]] = 1.0
    p[sl["W3"]] = 1.0
    p[sl["w4"]] = 1.0
    s = lambda z: z / (1 + math.exp(-z))
    bf = lambda v: float(torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).double())
    for z in (-3.0, -0.5, 0.0, 0.75, 4.0, 1.3125):
        x = np.array([[z, 0.0, 0.0]], np.float32)
        want = s(bf(s(bf(s(z)))))
        assert orc.mlp_forward(p, x, H, bf16_activations=True)[0] == pytest.approx(want, abs=1e-15)


def test_bf16_variant_equals_plain_when_hidden_layers_are_off(orc):
    """W3 = 0: the output depends on b3 only, so rounding a1 and a2 changes nothing."""
    H = 8
    p = _params(H, 3)
    sl = _slices(H)
    p[sl["W3"]] = 0.0
    x = np.random.default_rng(1).uniform(-1, 1, (16, 3)).astype(np.float32)
    assert np.array_equal(orc.mlp_forward(p, x, H), orc.mlp_forward(p, x, H, bf16_activations=True))
