"""Pins of the filter-importance-sampling oracle (Section 4.4, "Filter Importance
Sampling") against facts that do not come from the oracle itself: exhaustive and
lattice enumeration of the variates against the B-spline kernels of
`oracle.kernels`, closed-form Gaussian moments, numerical integration of the
normal density over each texel's box, and Monte Carlo agreement of the full lookup
with its deterministic twin."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import filters, fis, kernels, textures

rng = np.random.default_rng(1234)


def _xs():
    # fractions across [0, 1), negative coordinates, a fraction below 2^-24, integers
    return np.array([0.0, 0.25, 0.5, 0.999, 3.3, -0.7, -2.125, 7 + 2.0 ** -20,
                     2.0 ** -30, -(2.0 ** -30), 100.75], dtype=np.float32)


def test_linear_fis_exhaustive_over_all_variates():
    """n = 1 (uniform jitter): over all 2^24 variates the upper tap's frequency is the
    tent weight f, to the 2^-24 resolution of the variates (Hofmann et al.'s
    stochastic trilinear, Section 4.4)."""
    u = np.arange(1 << 24, dtype=np.float64) * 2.0 ** -24
    for x in _xs():
        idx, _ = fis.bspline_nearest(np.full(u.shape, x, dtype=np.float32), [u])
        i0 = math.floor(float(x))
        f = float(x) - i0
        assert set(np.unique(idx)) <= {i0, i0 + 1}
        p1 = np.mean(idx == i0 + 1)
        assert abs(p1 - f) <= 2.0 ** -24, (x, p1, f)
        # the tent kernel of the deterministic filter at the same fraction
        assert abs(p1 - kernels.k1_tent(np.array([1.0 - f]))[0]) <= 2.0 ** -24


@pytest.mark.parametrize("n,kernel,offsets", [
    (3, kernels.k_bspline3, (-1, 0, 1, 2)),
    (2, None, (-1, 0, 1, 2)),
])
def test_bspline_fis_lattice_frequencies(n, kernel, offsets):
    """Summing n uniforms and taking the nearest texel applies the degree-n B-spline:
    tap frequencies over a midpoint lattice of M points per variate match the kernel
    within the lattice's O(1/M) discretisation error (bounded here by 1 / M; a
    half-texel shift or a wrong number of uniforms misses by more than 0.05).  The
    quadratic B-spline (n = 2) is written here from its piecewise definition:
    3/4 - t^2 for |t| < 1/2, (3/2 - |t|)^2 / 2 for |t| < 3/2."""
    if kernel is None:
        def kernel(t):
            a = np.abs(t)
            return np.where(a < 0.5, 0.75 - a * a, np.where(a < 1.5, 0.5 * (1.5 - a) ** 2, 0.0))
    M = 128 if n == 3 else 512
    g = (np.arange(M) + 0.5) / M
    grids = np.meshgrid(*([g] * n), indexing="ij")
    us = [q.ravel() for q in grids]
    # keep the variates on the 2^-24 lattice the sampler assumes
    us = [np.floor(u * 2.0 ** 24) * 2.0 ** -24 for u in us]
    for x in _xs()[:9]:
        idx, _ = fis.bspline_nearest(np.full(us[0].shape, x, dtype=np.float32), us)
        i0 = math.floor(float(x))
        f = float(x) - i0
        for o in offsets:
            p = np.mean(idx == i0 + o)
            assert abs(p - float(kernel(np.array([f - o]))[0])) <= 1.0 / M, (n, x, o, p)
        assert set(np.unique(idx - i0)) <= set(offsets)


def test_box_muller_moments():
    """Offsets over a midpoint lattice of (u0, u1): mean 0, variance sigma^2, fourth
    moment 3 sigma^4, uncorrelated x and y (standard normal moments)."""
    M = 2048
    g = (np.arange(M) + 0.5) / M
    u0, u1 = [q.ravel() for q in np.meshgrid(g, g, indexing="ij")]
    for sigma in (0.5, 1.0, 2.5):
        ox, oy = fis.box_muller(u0, u1, sigma)
        for o in (ox, oy):
            assert abs(np.mean(o)) < 1e-3 * sigma
            assert abs(np.mean(o ** 2) / sigma ** 2 - 1.0) < 2e-3
            assert abs(np.mean(o ** 4) / sigma ** 4 - 3.0) < 3e-2
        assert abs(np.mean(ox * oy)) < 1e-3 * sigma ** 2


def test_gaussian_tap_weight_is_box_integral_of_normal_density():
    """Tap weight i = integral of the N(x, sigma^2) density over [i - 1/2, i + 1/2)
    (numerical quadrature), and the weights of the reachable window sum to 1."""
    for sigma in (0.3, 1.0, 3.0):
        for x in (0.0, 0.4, -1.3, 5.5):
            lo, hi = fis.gaussian_window(np.array([x], dtype=np.float32), sigma)
            tot = 0.0
            for i in range(int(lo[0]), int(hi[0]) + 1):
                w = float(fis.gaussian_tap_weight(i, x, sigma))
                q, _ = integrate.quad(lambda s: math.exp(-0.5 * ((s - x) / sigma) ** 2)
                                      / (sigma * math.sqrt(2 * math.pi)), i - 0.5, i + 0.5)
                assert abs(w - q) < 1e-12
                tot += w
            assert abs(tot - 1.0) < 2e-8


def test_gaussian_fis_tap_frequencies():
    """Nearest taps of x + Box-Muller offsets over a (u0, u1) lattice have the
    box-convolved Gaussian's tap weights; the reach bounds every tap."""
    M = 2048
    g = (np.arange(M) + 0.5) / M
    u0, u1 = [q.ravel() for q in np.meshgrid(g, g, indexing="ij")]
    for sigma in (0.4, 1.5):
        ox, _ = fis.box_muller(u0, u1, sigma)
        for x in (0.0, 0.3, -2.6):
            idx, _, _ = fis.gaussian_nearest(np.full(ox.shape, x, dtype=np.float32), ox)
            lo, hi = fis.gaussian_window(np.array([x], dtype=np.float32), sigma)
            assert idx.min() >= lo[0] and idx.max() <= hi[0]
            for i in range(int(lo[0]), int(hi[0]) + 1):
                assert abs(np.mean(idx == i) - fis.gaussian_tap_weight(i, x, sigma)) < 2e-3


def test_gaussian_deterministic_limits():
    """Constant texture -> constant; a narrow Gaussian -> the nearest texel; the
    result is symmetric under mirroring the texture and the coordinate."""
    tex = textures.Texture2D([rng.uniform(0, 1, (12, 12, 1))])
    fetch = lambda ix, iy: tex.fetch(0, ix, iy)
    const = textures.Texture2D([np.full((12, 12, 1), 0.625)])
    xs = [rng.uniform(3, 8, 50).astype(np.float32), rng.uniform(3, 8, 50).astype(np.float32)]
    v = fis.deterministic_gaussian(lambda ix, iy: const.fetch(0, ix, iy), xs, 1.2)
    assert np.allclose(v, 0.625, atol=1e-8)
    narrow = fis.deterministic_gaussian(fetch, xs, 0.02)
    ix = np.floor(xs[0].astype(np.float64) + 0.5).astype(np.int64)
    iy = np.floor(xs[1].astype(np.float64) + 0.5).astype(np.int64)
    far = (np.abs(xs[0] - np.round(xs[0])) < 0.3) & (np.abs(xs[1] - np.round(xs[1])) < 0.3)
    assert np.allclose(narrow[far], fetch(ix, iy)[far], atol=1e-9)
    mir = textures.Texture2D([tex.levels[0][::-1, ::-1]])
    m = fis.deterministic_gaussian(lambda ix, iy: mir.fetch(0, ix, iy),
                                   [(11 - xs[0]).astype(np.float32), (11 - xs[1]).astype(np.float32)], 0.9)
    assert np.allclose(m, fis.deterministic_gaussian(fetch, xs, 0.9), atol=1e-12)


@pytest.mark.parametrize("filt,width", [("fis_linear", None), ("fis_bspline3", None),
                                        ("fis_gaussian", 0.8)])
def test_fis_lookup_monte_carlo_matches_twin(filt, width):
    """Full 2D lookups with the Philox variates: the mean of 4096 samples per query
    agrees with the deterministic twin (z-test against the sample variance)."""
    tex = textures.Texture2D([rng.uniform(0, 1, (16, 16, 1))])
    uv = rng.uniform(0.1, 0.9, (64, 2)).astype(np.float32)
    S = 4096
    acc = np.zeros((64, 1))
    acc2 = np.zeros((64, 1))
    qid = np.arange(64, dtype=np.uint64)
    for s in range(S):
        v, _, _ = filters.lookup_2d(tex, uv, None, filt, stochastic_form=True, qid=qid,
                                    sample_index=s, seed=77, width=width)
        acc += v
        acc2 += v * v
    mean = acc / S
    var = acc2 / S - mean ** 2
    ref, _, _ = filters.lookup_2d(tex, uv, None, filt, stochastic_form=False, width=width)
    z = (mean - ref) / np.sqrt(np.maximum(var, 1e-30) / S)
    assert np.mean(np.abs(z) > 3.5) <= 2 / 64
    assert abs(np.sum(mean - ref) / np.sqrt(np.sum(var) / S)) < 4


def test_fis_3d_streams_and_twin():
    """3D: B-spline FIS draws its three uniforms of axis a from word a of streams 0, 1
    and 2; Gaussian FIS uses the pairs (w0, w1) and (w2, w3) of stream 0."""
    g = textures.Dense3D(rng.uniform(0, 1, (6, 7, 8)))
    p = rng.uniform(1, 5, (200, 3)).astype(np.float32)
    qid = np.arange(200, dtype=np.uint64)
    v, taps, _ = filters.lookup_3d(g, p, "fis_bspline3", stochastic_form=True, qid=qid, seed=3)
    from oracle.philox import query_variates
    st = [query_variates(qid, 0, 3, stream=j) for j in range(3)]
    for a in range(3):
        i = np.floor(p[:, a].astype(np.float64) + st[0][a] + st[1][a] + st[2][a] - 1.0)
        assert np.array_equal(taps[:, a], i.astype(np.int64))
    v, taps, ex = filters.lookup_3d(g, p, "fis_gaussian", stochastic_form=True, qid=qid, seed=3,
                                    width=1.1)
    r2 = 1.1 * np.sqrt(-2 * np.log(1 - st[0][2]))
    z = np.floor(p[:, 2].astype(np.float64) + r2 * np.cos(2 * np.pi * st[0][3]) + 0.5)
    assert np.array_equal(taps[~ex, 2], z.astype(np.int64)[~ex])
    d, _, _ = filters.lookup_3d(g, p[:20], "fis_gaussian", stochastic_form=False, width=0.6)
    assert d.shape == (20, 1) and np.all(np.isfinite(d))
