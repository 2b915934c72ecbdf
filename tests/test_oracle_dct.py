"""Pins of the DCT-texture and triplanar oracle (`oracle/dct.py`) against scipy's
DCT, closed forms of the quantiser, brute-force enumeration and Monte Carlo."""
import numpy as np
import pytest
from scipy import fft

from oracle import dct, filters, textures

rng = np.random.default_rng(77)


def test_kept_coefficients_match_scipy_dct():
    """The six coefficients equal scipy's orthonormal 2D DCT-II entries (v, u) of the
    block (array axes y, x); the basis is orthonormal."""
    blk = rng.uniform(0, 1, (8, 8, 3))
    co = dct.forward(blk)
    ref = fft.dctn(blk, type=2, norm="ortho", axes=(0, 1))
    for k, (u, v) in enumerate(dct.KEPT):
        assert np.allclose(co[k], ref[v, u], atol=1e-13)
    c = dct.basis_1d()
    assert np.allclose(c @ c.T, np.eye(3), atol=1e-14)


def test_reconstruction_equals_scipy_inverse_of_kept_coefficients():
    """Decoding a texel is the inverse DCT of the dequantised six coefficients with
    every other coefficient zero (scipy idctn)."""
    lv = rng.uniform(0, 1, (16, 24, 2))
    T = dct.DCTTexture2D([lv])
    for by in range(2):
        for bx in range(3):
            F = dct.dequantise(T.codes[0][by, bx], T.R)          # (6, C)
            full = np.zeros((8, 8, 2))
            for k, (u, v) in enumerate(dct.KEPT):
                full[v, u] = F[k]
            rec = fft.idctn(full, type=2, norm="ortho", axes=(0, 1))
            ys, xs = np.mgrid[0:8, 0:8]
            got = T.fetch(0, (bx * 8 + xs).ravel(), (by * 8 + ys).ravel()).reshape(8, 8, 2)
            assert np.allclose(got, rec, atol=1e-12)


def test_quantiser_closed_forms():
    """A constant block of value c decodes to the DC code's value: the nearest multiple
    of 1/127 of c (DC = 8c); AC codes are 0.  The block with the channel's largest |AC|
    carries code +-15 for it; packing round-trips every code."""
    for c in (0.0, 0.25, 0.5, 1.0, 63.4 / 127):
        T = dct.DCTTexture2D([np.full((8, 8, 1), c)])
        q = dct.unpack(T.codes[0][0, 0, 0])
        assert q[0] == np.floor(c * 127 + 0.5) and np.all(q[1:] == 0)
        assert np.allclose(T.fetch(0, np.arange(8), np.arange(8)), q[0] / 127, atol=1e-15)
    lv = rng.uniform(0, 1, (32, 32, 1))
    T = dct.DCTTexture2D([lv])
    q = dct.unpack(T.codes[0][..., 0])                             # (6, 4, 4)
    assert np.max(np.abs(q[1:])) == 15
    codes = rng.integers(-15, 16, (5, 1000))
    dc = rng.integers(0, 128, 1000)
    w = dc.astype(np.uint64)
    for j in range(5):
        w |= (codes[j].astype(np.int64) & 31).astype(np.uint64) << np.uint64(7 + 5 * j)
    back = dct.unpack(w.astype(np.uint32))
    assert np.array_equal(back[0], dc) and np.array_equal(back[1:], codes)


def test_quantisation_error_bound():
    """|decoded - truncated reconstruction| <= half a DC step times a(0)^2 plus half an
    AC step times the sum of the AC basis maxima."""
    lv = rng.uniform(0, 1, (32, 40, 3))
    T = dct.DCTTexture2D([lv])
    co = dct.coefficients([lv])[0]
    c = dct.basis_1d()
    ys, xs = np.mgrid[0:32, 0:40]
    got = T.fetch(0, xs.ravel(), ys.ravel()).reshape(32, 40, 3)
    trunc = np.zeros_like(got)
    for k, (u, v) in enumerate(dct.KEPT):
        trunc += co[ys >> 3, xs >> 3, k, :] * (c[u, xs & 7] * c[v, ys & 7])[..., None]
    bound = 0.5 * 8 / 127 / 8 + 0.5 * (T.R / 15) * sum(np.max(np.abs(c[u])) * np.max(np.abs(c[v]))
                                                         for (u, v) in dct.KEPT[1:])
    assert np.all(np.abs(got - trunc) <= bound + 1e-12)


def test_edge_blocks_repeat_edge_texels():
    lv = rng.uniform(0, 1, (5, 11, 1))
    T = dct.DCTTexture2D([lv])
    assert T.codes[0].shape == (1, 2, 1)
    padded = lv[np.minimum(np.arange(8), 4)][:, np.minimum(np.arange(16), 10)]
    co = dct.forward(padded[:, 8:16])
    F = dct.dequantise(T.codes[0][0, 1], T.R)
    assert np.allclose(F[0], np.clip(np.floor(co[0] * 127 / 8 + 0.5), 0, 127) * 8 / 127)


def test_plane_choice_frequencies():
    n = 1 << 18
    u = np.arange(n) / n
    a = np.array([0.2, 0.5, 0.3], dtype=np.float32)
    k, _ = dct.choose_plane(np.repeat(a[:, None], n, axis=1), u)
    assert np.allclose(np.bincount(k, minlength=3) / n, a / a.sum(), atol=2.0 ** -17)


def test_triplanar_monte_carlo_matches_deterministic():
    """Stochastic plane + stochastic bilinear tap on a DCT texture: 2048-sample means
    against the blend of the three deterministic bilinear lookups."""
    base = rng.uniform(0, 1, (32, 32, 2))
    tex = dct.DCTTexture2D(textures.Texture2D.box_pyramid(base, 1).levels)
    N = 48
    p = rng.uniform(0.05, 0.95, (N, 3)).astype(np.float32)
    nrm = rng.standard_normal((N, 3))
    nrm = (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32)
    S = 2048
    acc = np.zeros((N, 2))
    acc2 = np.zeros((N, 2))
    qid = np.arange(N, dtype=np.uint64)
    for s in range(S):
        v, _, _ = dct.lookup_triplanar(tex, p, nrm, 1.0, None, "linear", stochastic_form=True,
                                       sample_index=s, seed=9, qid=qid)
        acc += v
        acc2 += v * v
    mean = acc / S
    var = np.maximum(acc2 / S - mean ** 2, 1e-12)
    ref, _, _ = dct.lookup_triplanar(tex, p, nrm, 1.0, None, "linear", stochastic_form=False)
    z = (mean - ref) / np.sqrt(var / S)
    assert np.mean(np.abs(z) > 3.5) <= 2 / (2 * N)
    assert abs(np.sum(mean - ref) / np.sqrt(np.sum(var) / S)) < 4
