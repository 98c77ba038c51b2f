"""Pins for the surrogate's FP64 reference (CPU only): finite-difference gradients,
numpy forward pass, torch's bfloat16 conversion, and Adam's closed form."""
import numpy as np
import torch


def _params(rng, din=6, h=5, dout=2, scale=0.5):
    return {"W1": rng.standard_normal((h, din)) * scale, "b1": rng.standard_normal(h) * 0.1,
            "W2": rng.standard_normal((h, h)) * scale, "b2": rng.standard_normal(h) * 0.1,
            "W3": rng.standard_normal((dout, h)) * scale, "b3": rng.standard_normal(dout) * 0.1}


def test_forward_matches_numpy(orc):
    from scipy.special import erf
    rng = np.random.default_rng(0)
    P = _params(rng)
    X = rng.standard_normal((9, 6))
    g = lambda z: 0.5 * z * (1 + erf(z / np.sqrt(2)))
    a1 = g(X @ P["W1"].T + P["b1"])
    a2 = g(a1 @ P["W2"].T + P["b2"])
    Y = a2 @ P["W3"].T + P["b3"]
    np.testing.assert_allclose(orc.mlp_forward(X, P, bf16=False), Y, rtol=1e-12, atol=1e-13)


def test_gradients_match_finite_differences(orc):
    rng = np.random.default_rng(1)
    P = _params(rng)
    X = rng.standard_normal((7, 6))
    T = rng.standard_normal((7, 2))
    loss, G, _ = orc.mlp_loss_backward(X, T, P, bf16=False)
    eps = 1e-6
    for k, a in P.items():
        flat = a.reshape(-1)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + eps
            lp, _, _ = orc.mlp_loss_backward(X, T, P, bf16=False)
            flat[i] = old - eps
            lm, _, _ = orc.mlp_loss_backward(X, T, P, bf16=False)
            flat[i] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - G[k].reshape(-1)[i]) < 1e-6 * max(1.0, abs(fd)), (k, i)


def test_bf16_rounding_matches_torch(orc):
    rng = np.random.default_rng(2)
    bits = rng.integers(0, 2**32, 20000, dtype=np.uint64).astype(np.uint32)
    bits[:4] = [0x3F808000, 0x3F818000, 0x3F80C000, 0x3F817FFF]   # ties to even both ways
    f = bits.view(np.float32)
    f = f[np.isfinite(f)]
    want = torch.from_numpy(f.copy()).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([orc.bf16_round(float(x)) for x in f])
    assert np.array_equal(got, want)


def test_bf16_mode_rounds_activations(orc):
    rng = np.random.default_rng(3)
    P = _params(rng, din=8, h=16)
    X = rng.standard_normal((4, 8))
    y32 = orc.mlp_forward(X, P, bf16=False)
    y16 = orc.mlp_forward(X, P, bf16=True)
    assert not np.array_equal(y32, y16)
    assert np.abs(y32 - y16).max() < 0.05 * np.abs(y32).max()


def test_adam_constant_gradient(orc):
    # With a constant gradient the bias-corrected moments equal g and g^2, so each step moves
    # every weight by lr * g / (|g| + eps).
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m = np.zeros(3); v = np.zeros(3)
    for t in range(1, 11):
        orc.adam_update(w, g, m, v, t, lr=1e-2)
    np.testing.assert_allclose(w, np.array([1.0, -2.0, 0.5]) - 10 * 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)
