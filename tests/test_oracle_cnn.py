"""Pins for the oracle's CNN scorer: normalisation, forward, backward, Adam.

The forward is checked against an FFT circular cross-correlation and against
PyTorch's CPU float64 modules (circular Conv1d, MaxPool1d, Linear); the backward
against central finite differences and PyTorch autograd; Adam against torch.optim.
"""
import numpy as np
import pytest
import torch

import lcsynth
import oracle


def torch_model(weights):
    m = torch.nn.Sequential(
        torch.nn.Conv1d(1, 16, 5, padding=2, padding_mode="circular"), torch.nn.ReLU(), torch.nn.MaxPool1d(2),
        torch.nn.Conv1d(16, 32, 5, padding=2, padding_mode="circular"), torch.nn.ReLU(), torch.nn.MaxPool1d(2),
        torch.nn.Conv1d(32, 64, 5, padding=2, padding_mode="circular"), torch.nn.ReLU(), torch.nn.MaxPool1d(2),
        torch.nn.Flatten(), torch.nn.Linear(2048, 256), torch.nn.ReLU(), torch.nn.Linear(256, 1),
    ).double()
    layers = [m[0], m[3], m[6], m[10], m[12]]
    names = ["conv1", "conv2", "conv3", "fc1", "fc2"]
    with torch.no_grad():
        for l, n in zip(layers, names):
            l.weight.copy_(torch.from_numpy(np.asarray(weights[n + ".w"], np.float64)))
            l.bias.copy_(torch.from_numpy(np.asarray(weights[n + ".b"], np.float64)))
    return m, layers, names


def weights(seed=5):
    return lcsynth.cnn_init(seed, bias_scale=0.05)


def test_normalisation_keeps_mean_and_unit_std():
    rng = np.random.default_rng(0)
    v = (1.0 + rng.normal(0, 3e-4, (3, 256))).astype(np.float32)
    counts = rng.integers(0, 5, (3, 256)).astype(np.int32)
    x = oracle.cnn_normalise(v, counts)
    for k in range(3):
        ne = counts[k] > 0
        m = v[k][ne].astype(np.float64).mean()
        assert x[k][ne].mean() == pytest.approx(m, rel=1e-14)
        assert np.std(x[k][ne]) == pytest.approx(1.0, rel=1e-12)
        assert np.all(x[k][~ne] == pytest.approx(m, rel=1e-15))
    # NaN marks empty bins when no counts are given
    v2 = v[0].copy()
    v2[::7] = np.nan
    x2 = oracle.cnn_normalise(v2[None])
    ne = ~np.isnan(v2)
    assert np.std(x2[0][ne]) == pytest.approx(1.0, rel=1e-12)
    # constant profile stays constant
    x3 = oracle.cnn_normalise(np.full((1, 256), 0.999, np.float32))
    assert np.all(x3 == np.float64(np.float32(0.999)))


def test_first_conv_is_circular_cross_correlation_by_fft():
    w = weights()
    rng = np.random.default_rng(1)
    x = rng.normal(0, 1, (1, 256))
    # isolate conv1 channel 0: zero everything after it except a probe path is hard;
    # instead compare torch's conv1 (library) against an FFT cross-correlation, then
    # the whole oracle forward against torch below.
    k = np.asarray(w["conv1.w"], np.float64)[0, 0]
    kern = np.zeros(256)
    for j in range(5):
        kern[(j - 2) % 256] = k[j]
    # y[l] = sum_j k[j] x[l + j - 2]  ==  ifft(fft(x) * conj(fft(kern)))
    y_fft = np.real(np.fft.ifft(np.fft.fft(x[0]) * np.conj(np.fft.fft(kern))))
    m, layers, _ = torch_model(w)
    with torch.no_grad():
        y_t = layers[0](torch.from_numpy(x)[None])[0, 0].numpy() - float(w["conv1.b"][0])
    np.testing.assert_allclose(y_t, y_fft, atol=1e-12)


def test_forward_matches_torch_float64():
    w = weights()
    rng = np.random.default_rng(2)
    x = rng.normal(0, 1, (8, 256)) + 1.0
    z = oracle.cnn_forward(w, x)
    m, _, _ = torch_model(w)
    with torch.no_grad():
        zt = m(torch.from_numpy(x)[:, None, :])[:, 0].numpy()
    np.testing.assert_allclose(z, zt, rtol=1e-11, atol=1e-12)


def test_score_is_sigmoid_of_forward_of_normalised():
    w = weights()
    prof, _ = lcsynth.profiles_mixed(6, seed=3)
    z, s = oracle.cnn_score(w, prof)
    x = oracle.cnn_normalise(prof)
    np.testing.assert_allclose(z, oracle.cnn_forward(w, x), rtol=0, atol=0)
    np.testing.assert_allclose(s, 1 / (1 + np.exp(-z)), rtol=1e-15)


def test_backward_matches_torch_autograd():
    w = weights()
    rng = np.random.default_rng(4)
    x = rng.normal(0, 1, (6, 256))
    y = np.array([1, 0, 1, 1, 0, 0], np.float32)
    loss, grads, dx = oracle.cnn_loss_backward(w, x, y, want_dx=True)
    m, layers, names = torch_model(w)
    xt = torch.from_numpy(x)[:, None, :].clone().requires_grad_(True)
    zt = m(xt)[:, 0]
    lt = torch.nn.functional.binary_cross_entropy_with_logits(zt, torch.from_numpy(y.astype(np.float64)))
    lt.backward()
    assert loss == pytest.approx(lt.item(), rel=1e-12)
    for l, n in zip(layers, names):
        np.testing.assert_allclose(grads[n + ".w"], l.weight.grad.numpy(), rtol=1e-9, atol=1e-13)
        np.testing.assert_allclose(grads[n + ".b"], l.bias.grad.numpy(), rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(dx, xt.grad[:, 0].numpy(), rtol=1e-9, atol=1e-13)


def test_backward_matches_central_differences():
    w = {k: np.asarray(v, np.float64) for k, v in weights(8).items()}
    rng = np.random.default_rng(6)
    x = rng.normal(0, 1, (4, 256))
    y = np.array([1, 0, 0, 1], np.float32)
    _, grads, _ = oracle.cnn_loss_backward(w, x, y)
    h = 1e-6
    for name in oracle.CNN_NAMES:
        flat = w[name].reshape(-1)
        picks = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for j in picks:
            old = flat[j]
            flat[j] = old + h
            lp, _, _ = oracle.cnn_loss_backward(w, x, y)
            flat[j] = old - h
            lm, _, _ = oracle.cnn_loss_backward(w, x, y)
            flat[j] = old
            fd = (lp - lm) / (2 * h)
            g = grads[name].reshape(-1)[j]
            assert abs(fd - g) <= 1e-6 * max(1e-3, abs(g)) + 1e-9, (name, j, fd, g)


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(7)
    p0 = rng.normal(0, 1, 50)
    pt = torch.nn.Parameter(torch.from_numpy(p0.copy()))
    opt = torch.optim.Adam([pt], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 6):
        g = rng.normal(0, 1, 50)
        pt.grad = torch.from_numpy(g.copy())
        opt.step()
        p, m, v = oracle.adam_step(p, g, m, v, t)
    np.testing.assert_allclose(p, pt.detach().numpy(), rtol=1e-12, atol=1e-15)
