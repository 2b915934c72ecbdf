"""Pins of the float64 decoder MLP and Adam against torch (an independent library,
float64 autograd and optimizer) and against central finite differences.  CPU only."""
import numpy as np
import pytest
import torch

from oracle import filters, mlp, neural, textures

rng = np.random.default_rng(7)


def _params():
    return {k: rng.normal(0, 0.4, s) for k, s in mlp.shapes().items()}


def test_forward_and_backward_match_torch_autograd():
    P = _params()
    X = rng.normal(0, 1, (33, 8))
    T = rng.normal(0, 1, (33, 7))
    Y, cache = mlp.forward(X, P)
    g = mlp.backward(cache, P, Y, T)
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in P.items()}
    tx = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    h = torch.relu(tx @ tp["W1"] + tp["b1"])
    h = torch.relu(h @ tp["W2"] + tp["b2"])
    ty = h @ tp["W3"] + tp["b3"]
    tl = ((ty - torch.tensor(T)) ** 2).sum() / 33
    tl.backward()
    assert np.allclose(Y, ty.detach().numpy(), rtol=1e-12, atol=1e-12)
    assert abs(mlp.loss(Y, T) - tl.item()) < 1e-12
    for k in mlp.NAMES:
        assert np.allclose(g[k], tp[k].grad.numpy(), rtol=1e-10, atol=1e-12), k
    assert np.allclose(g["X"], tx.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_backward_matches_central_differences():
    P = _params()
    X = rng.normal(0, 1, (5, 8))
    T = rng.normal(0, 1, (5, 7))
    Y, cache = mlp.forward(X, P)
    g = mlp.backward(cache, P, Y, T)
    h = 1e-6
    for k in ("W1", "b2", "W3"):
        for idx in [tuple(rng.integers(0, s) for s in P[k].shape) for _ in range(5)]:
            Pp = {a: b.copy() for a, b in P.items()}
            Pm = {a: b.copy() for a, b in P.items()}
            Pp[k][idx] += h
            Pm[k][idx] -= h
            num = (mlp.loss(mlp.forward(X, Pp)[0], T) - mlp.loss(mlp.forward(X, Pm)[0], T)) / (2 * h)
            assert abs(num - g[k][idx]) <= 1e-6 * max(1.0, abs(num)), (k, idx)
    Xp, Xm = X.copy(), X.copy()
    Xp[2, 3] += h
    Xm[2, 3] -= h
    num = (mlp.loss(mlp.forward(Xp, P)[0], T) - mlp.loss(mlp.forward(Xm, P)[0], T)) / (2 * h)
    assert abs(num - g["X"][2, 3]) <= 1e-6 * max(1.0, abs(num))


def test_flat_order_round_trip():
    P = _params()
    flat = mlp.flatten(P)
    assert flat.size == 8 * 64 + 64 + 64 * 64 + 64 + 64 * 7 + 7
    Q = mlp.unflatten(flat)
    assert all(np.array_equal(P[k], Q[k]) for k in mlp.NAMES)


def test_adam_matches_torch_optimizer():
    p0 = rng.normal(0, 1, 20)
    tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=0.01, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(20), np.zeros(20)
    for t in range(1, 8):
        g = np.sin(p * t) + 0.1 * p
        tp.grad = torch.tensor(g)
        opt.step()
        p, m, v = mlp.adam(p, g, m, v, t, 0.01)
        assert np.allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def _identity_decoder():
    """ReLU network that returns the first 7 of its 8 inputs exactly:
    H1 = [relu(z), relu(-z), 0], H2 = H1, Y_c = relu(z_c) - relu(-z_c) = z_c."""
    P = {k: np.zeros(s) for k, s in mlp.shapes().items()}
    for j in range(8):
        P["W1"][j, j], P["W1"][j, 8 + j] = 1.0, -1.0
    P["W2"][:] = np.eye(64)
    for c in range(7):
        P["W3"][c, c], P["W3"][8 + c, c] = 1.0, -1.0
    return P


@pytest.mark.parametrize("filt", ["linear", "bspline3", "catmull_rom"])
def test_neural_lookup_with_identity_decoder_equals_plain_lookup(filt):
    lat = [rng.normal(0, 1, (16 >> L, 16 >> L, 8)) for L in range(3)]
    fb = [rng.normal(0, 1, (16 >> L, 16 >> L, 7)) for L in range(3, 5)]
    nt = neural.NeuralTexture2D(lat, _identity_decoder(), fb)
    plain = textures.Texture2D([l[..., :7] for l in lat] + fb)
    uv = rng.uniform(0, 1, (400, 2)).astype(np.float32)
    lod = rng.uniform(0, 5, 400).astype(np.float32)
    for sto in (True, False):
        a, ta, _ = filters.lookup_2d(nt, uv, lod, filt, stochastic_form=sto, seed=4)
        b, tb, _ = filters.lookup_2d(plain, uv, lod, filt, stochastic_form=sto, seed=4)
        assert np.allclose(a, b, rtol=0, atol=1e-12)
        if sto:
            assert np.array_equal(ta, tb)
