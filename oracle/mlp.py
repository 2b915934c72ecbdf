"""Float64 forward and backward of the neural-texture decoder, and Adam
(test infrastructure only).

The paper motivates stochastic filtering for expensive decoders, neural texture
representations included (Section 1; Section 5.2 "Texture compression"), without
fixing an architecture.  The decoder here maps one 8-channel latent texel to one
7-channel texel (RGB albedo, normal xyz, roughness):

    H1 = relu(X W1 + b1)      X: (N, 8)   W1: (8, 64)
    H2 = relu(H1 W2 + b2)     W2: (64, 64)
    Y  = H2 W3 + b3           W3: (64, 7)

Training loss: L = (1/N) sum_n sum_c (Y - T)^2 over a batch of N texels.
Adam (Kingma and Ba, ICLR 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
"""
import numpy as np

NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def shapes(din=8, hidden=64, dout=7):
    """Parameter shapes of the decoder (W1, b1, W2, b2, W3, b3), in flattening order."""
    return {"W1": (din, hidden), "b1": (hidden,), "W2": (hidden, hidden), "b2": (hidden,),
            "W3": (hidden, dout), "b3": (dout,)}


def flatten(P):
    """Parameters in the library's flat order: W1, b1, W2, b2, W3, b3, row-major."""
    return np.concatenate([np.asarray(P[k], dtype=np.float64).reshape(-1) for k in NAMES])


def unflatten(flat, din=8, hidden=64, dout=7):
    """Inverse of `flatten`: a flat parameter vector to the named arrays."""
    out, o = {}, 0
    for k in NAMES:
        shp = shapes(din, hidden, dout)[k]
        size = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + size], dtype=np.float64).reshape(shp)
        o += size
    return out


def forward(X, P):
    """Decoder forward pass H1 = relu(X W1 + b1), H2 = relu(H1 W2 + b2),
    Y = H2 W3 + b3; returns (Y, cache of the activations for `backward`)."""
    X = np.asarray(X, dtype=np.float64)
    A1 = X @ P["W1"] + P["b1"]
    H1 = np.maximum(A1, 0.0)
    A2 = H1 @ P["W2"] + P["b2"]
    H2 = np.maximum(A2, 0.0)
    Y = H2 @ P["W3"] + P["b3"]
    return Y, (X, A1, H1, A2, H2)


def loss(Y, T):
    """Mean squared error over every output value."""
    d = np.asarray(Y) - np.asarray(T, dtype=np.float64)
    return float(np.sum(d * d) / Y.shape[0])


def backward(cache, P, Y, T):
    """Gradients of the batch loss with respect to every parameter and to X."""
    X, A1, H1, A2, H2 = cache
    N = X.shape[0]
    dY = 2.0 * (Y - np.asarray(T, dtype=np.float64)) / N
    g = {"W3": H2.T @ dY, "b3": dY.sum(axis=0)}
    dA2 = (dY @ P["W3"].T) * (A2 > 0)
    g["W2"] = H1.T @ dA2
    g["b2"] = dA2.sum(axis=0)
    dA1 = (dA2 @ P["W2"].T) * (A1 > 0)
    g["W1"] = X.T @ dA1
    g["b1"] = dA1.sum(axis=0)
    g["X"] = dA1 @ P["W1"].T
    return g


def adam(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t >= 1); returns new (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
