"""Pins of the anisotropic-LOD and EWA oracle (`oracle/ewa.py`) against closed
forms, an independent linear-algebra evaluation of the ellipse, and brute force."""
import math

import numpy as np
import pytest

from oracle import ewa, textures

rng = np.random.default_rng(99)


def _jac(d0, d1):
    return np.array([[d0[0], d1[0]], [d0[1], d1[1]]], dtype=np.float64)


@pytest.mark.parametrize("d0,d1", [((3.0, 0.0), (0.0, 0.5)), ((2.0, 2.0), (-0.3, 0.3)),
                                   ((0.1, -7.0), (1.5, 0.2)), ((0.0, 0.0), (0.0, 0.0))])
def test_ellipse_is_inverse_covariance(d0, d1):
    """(A, B, C) of the normalised quadratic form equal the entries of
    (J J^T + I)^-1 (numpy linear algebra in float64), and the bounding-box half
    extents are the ellipse's exact extents sqrt(Sigma_ss), sqrt(Sigma_tt)."""
    d0 = [float(np.float32(v)) for v in d0]       # the float32 axes the oracle is given
    d1 = [float(np.float32(v)) for v in d1]
    A, B, C, hs, ht = (x[0] for x in ewa.ellipse(d0[0], d0[1], d1[0], d1[1]))
    J = _jac(d0, d1)
    Sigma = J @ J.T + np.eye(2)
    M = np.linalg.inv(Sigma)
    assert np.allclose([A, B, C], [M[0, 0], 2 * M[0, 1], M[1, 1]], rtol=1e-12, atol=1e-15)
    assert math.isclose(hs, math.sqrt(Sigma[0, 0]), rel_tol=1e-12)
    assert math.isclose(ht, math.sqrt(Sigma[1, 1]), rel_tol=1e-12)
    # points of the ellipse boundary Q = 1 (Sigma^(1/2) applied to the unit circle)
    ev, V = np.linalg.eigh(Sigma)
    th = np.linspace(0, 2 * np.pi, 721)
    pts = (V @ np.diag(np.sqrt(ev)) @ np.stack([np.cos(th), np.sin(th)])).T
    q = A * pts[:, 0] ** 2 + B * pts[:, 0] * pts[:, 1] + C * pts[:, 1] ** 2
    assert np.allclose(q, 1.0, rtol=1e-10)
    assert np.max(np.abs(pts[:, 0])) <= hs * (1 + 1e-10) and np.max(np.abs(pts[:, 1])) <= ht * (1 + 1e-10)


def test_weight_table():
    lut = ewa.weight_lut()
    assert lut.shape == (128,) and lut.dtype == np.float64
    assert lut[0] == 1 - math.exp(-2) and lut[-1] == 0
    assert np.all(np.diff(lut) < 0)
    assert lut[64] == math.exp(-2 * 64 / 127) - math.exp(-2)


def test_anisotropic_lod_closed_forms():
    """Isotropic footprints of 2^k texels give lod k; an anisotropy above the limit
    lengthens the minor axis to major / limit; the longer derivative is the major
    axis whichever screen axis it belongs to."""
    W = H = 1024
    k = np.arange(-2, 9)
    g = np.stack([2.0 ** k / W, 0 * k, 0 * k, 2.0 ** k / H], axis=1).astype(np.float32)
    lod = ewa.footprint(W, H, g, 64).lod
    assert np.array_equal(lod, k.astype(np.float64))
    g = np.array([[1000 / W, 0, 0, 1 / H], [0, 1 / H, 1000 / W, 0], [0, 10 / H, 1 / W, 0]], dtype=np.float32)
    fp = ewa.footprint(W, H, g, 64)
    f32 = lambda x: float(np.float32(x))
    assert math.isclose(fp.lod[0], math.log2(f32(1000 / W) * W / 64), rel_tol=1e-12)
    assert math.isclose(fp.lod[1], math.log2(f32(1000 / W) * W / 64), rel_tol=1e-12)
    assert fp.lod[2] == 0.0                    # ratio 10 <= 64: minor = 1 texel
    assert fp.major[0][0][1] == f32(1000 / W) and fp.major[1][0][2] == f32(10 / H)
    assert math.isclose(ewa.footprint(W, H, g[:1], 8).lod[0], math.log2(f32(1000 / W) * W / 8), rel_tol=1e-12)
    assert ewa.footprint(W, H, np.zeros((1, 4), np.float32), 64).lod[0] == -np.inf


def test_selection_frequencies_over_u_lattice():
    ell = ewa.ellipse(np.float32(2.5), np.float32(1.0), np.float32(-0.4), np.float32(0.9))
    s, t, w, lo, hi = ewa.texels_and_weights(float(np.float32(10.3)), float(np.float32(7.8)), ell)
    assert np.all(lo <= w) and np.all(w <= hi)
    n = 1 << 20
    u = np.arange(n) / n
    csum = np.cumsum(w)
    ks = np.sum(csum[None, :-1] <= (u * csum[-1])[:, None], axis=1)
    freq = np.bincount(ks, minlength=len(w)) / n
    assert np.allclose(freq, w / np.sum(w), atol=2.0 ** -19)
    assert np.all(freq[w == 0] == 0)
    assert all(ewa.select(w, x)[0] == k for x, k in zip(u[::4099], ks[::4099]))


def _f32_ellipse(d, order):
    """A float32 evaluation of the ellipse coefficients and half extents, in one of two
    operation orders (1: sums grouped the other way, products reassociated)."""
    f = np.float32
    d0u, d0v, d1u, d1v = (f(x) for x in d)
    if order == 0:
        A = f(f(f(d0v * d0v) + f(d1v * d1v)) + f(1))
        B = f(f(-2) * f(f(d0u * d0v) + f(d1u * d1v)))
        C = f(f(f(d0u * d0u) + f(d1u * d1u)) + f(1))
        F = f(f(A * C) - f(f(B * B) * f(0.25)))
    else:
        A = f(f(d0v * d0v) + f(f(d1v * d1v) + f(1)))
        B = f(f(f(-2) * f(d0u * d0v)) - f(f(2) * f(d1u * d1v)))
        C = f(f(d0u * d0u) + f(f(d1u * d1u) + f(1)))
        F = f(f(A * C) - f(f(f(0.5) * B) * f(f(0.5) * B)))
    inv = f(f(1) / F)
    A, B, C = f(A * inv), f(B * inv), f(C * inv)
    det = f(f(f(4) * f(A * C)) - f(B * B))
    hs = f(f(f(2) / det) * np.sqrt(f(det * C))) if order else f(f(f(2) * f(f(1) / det)) * np.sqrt(f(det * C)))
    ht = f(f(f(2) / det) * np.sqrt(f(A * det))) if order else f(f(f(2) * f(f(1) / det)) * np.sqrt(f(A * det)))
    return A, B, C, hs, ht


@pytest.mark.parametrize("order", [0, 1])
def test_derived_float32_bounds_hold(order):
    """The oracle's bounds on a float32 evaluation (ellipse coefficients, half
    extents, Q per texel) contain two float32 evaluations of the same formulas in
    different operation orders, over random elongated and rotated footprints."""
    r = np.random.default_rng(7 + order)
    f = np.float32
    worst = 0.0
    for _ in range(300):
        a = r.uniform(0.2, 64.0)
        b = a / r.uniform(1.0, 64.0)
        th = r.uniform(0, np.pi)
        d = [a * np.cos(th), a * np.sin(th), -b * np.sin(th), b * np.cos(th)]
        d = [float(f(x)) for x in d]
        ell = ewa.ellipse(*d)
        got = _f32_ellipse(d, order)
        for (v, e), x in zip(ell, got):
            assert abs(float(x) - v) <= e, (d, v, e, x)
            worst = max(worst, abs(float(x) - v) / e)
        st_s, st_t = float(f(r.uniform(0, 64))), float(f(r.uniform(0, 64)))
        s, t, w, lo, hi = ewa.texels_and_weights(st_s, st_t, ell)
        A, B, C = (f(x) for x in got[:3])
        ss = (s.astype(np.float32) - f(st_s)).astype(np.float32)
        tt = (t.astype(np.float32) - f(st_t)).astype(np.float32)
        if order == 0:
            q32 = f(1) * ((A * ss + B * tt) * ss + C * (tt * tt))
        else:
            q32 = A * (ss * ss) + (B * (ss * tt) + C * (tt * tt))
        lut32 = ewa.weight_lut().astype(np.float32)
        w32 = np.where(q32 < 1, lut32[np.clip((q32 * f(128)).astype(np.int64), 0, 127)], 0)
        inside = (s >= np.ceil(f(f(st_s) - got[3]))) & (s <= np.floor(f(f(st_s) + got[3]))) & \
                 (t >= np.ceil(f(f(st_t) - got[4]))) & (t <= np.floor(f(f(st_t) + got[4])))
        w32 = np.where(inside, w32, 0)
        assert np.all(lo <= w32) and np.all(w32 <= hi)
    assert worst > 1e-3            # the bounds are not vacuous


def test_lod_bound_holds_for_float32_footprints():
    """lod_lo <= log2 of a float32 evaluation of the clamped minor axis <= lod_hi."""
    r = np.random.default_rng(3)
    g = (r.standard_normal((4000, 4)) * np.exp(r.uniform(-8, 3, (4000, 1)))).astype(np.float32)
    for ma in (1.0, 8.0, 64.0):
        fp = ewa.footprint(256, 128, g, ma)
        f = np.float32
        la = (g[:, 0] * f(256)) ** 2 + (g[:, 1] * f(128)) ** 2
        lb = (g[:, 2] * f(256)) ** 2 + (g[:, 3] * f(128)) ** 2
        major, minor = np.sqrt(np.maximum(la, lb)), np.sqrt(np.minimum(la, lb))
        clamp = (minor > 0) & (minor * f(ma) < major)
        minor = np.where(clamp, minor * (major / (minor * f(ma))), minor).astype(np.float32)
        with np.errstate(divide="ignore"):
            lod32 = np.log2(minor).astype(np.float64)
        ok = fp.finite
        assert np.all((fp.lod_lo[ok] <= lod32[ok]) & (lod32[ok] <= fp.lod_hi[ok]))
        assert np.mean(fp.ambiguous) < 1e-3


def test_deterministic_ewa_against_brute_force_gaussian():
    """sum w t / sum w over every texel of a small random texture with
    w = exp(-2 Q) - exp(-2) inside the ellipse, Q from the float64 inverse covariance,
    matches the table-based oracle to the table's resolution; the mirrored ellipse
    (B negated) does not."""
    tex = textures.Texture2D([rng.uniform(0, 1, (64, 64, 1))])
    n = 60
    uv = rng.uniform(0.3, 0.7, (n, 2)).astype(np.float32)
    ang = rng.uniform(0, np.pi, n)
    ratio = rng.uniform(2, 6, n)
    scale = rng.uniform(1.0, 1.8, n) / 64
    g = np.stack([scale * ratio * np.cos(ang), scale * ratio * np.sin(ang),
                  -scale * np.sin(ang), scale * np.cos(ang)], axis=1).astype(np.float32)
    # a single level: the filter runs at level 0
    v, _, _ = ewa.lookup(tex, uv, g, 64, stochastic_form=False, level_mode=0)
    ii, jj = np.meshgrid(np.arange(64), np.arange(64), indexing="xy")
    worst_ok, worst_mirror = 0.0, 0.0
    for q in range(n):
        d0 = g[q, :2].astype(np.float64) * 64
        d1 = g[q, 2:].astype(np.float64) * 64
        M = np.linalg.inv(_jac(d0, d1) @ _jac(d0, d1).T + np.eye(2))
        ds = ii - (uv[q, 0] * 64 - 0.5)
        dt = jj - (uv[q, 1] * 64 - 0.5)
        for sgn, store in ((1, "ok"), (-1, "mirror")):
            Q = M[0, 0] * ds ** 2 + sgn * 2 * M[0, 1] * ds * dt + M[1, 1] * dt ** 2
            w = np.where(Q < 1, np.exp(-2 * Q) - np.exp(-2), 0.0)
            bf = np.sum(w * tex.levels[0][:, :, 0]) / np.sum(w)
            err = abs(bf - v[q, 0])
            if store == "ok":
                worst_ok = max(worst_ok, err)
            else:
                worst_mirror = max(worst_mirror, err)
    assert worst_ok < 0.01, worst_ok
    assert worst_mirror > 0.05, worst_mirror


def test_stochastic_expectation_equals_deterministic_at_fixed_level():
    tex = textures.Texture2D.box_pyramid(rng.uniform(0, 1, (32, 32, 2)), 6)
    n = 80
    uv = rng.uniform(0, 1, (n, 2)).astype(np.float32)
    g = (rng.uniform(-1, 1, (n, 4)) * rng.uniform(0.1, 12, (n, 1)) / 32).astype(np.float32)
    e = ewa.expectation(tex, uv, g, 16, level_mode=0)
    d, _, tol = ewa.lookup(tex, uv, g, 16, stochastic_form=False, level_mode=0)
    assert np.all(np.isfinite(tol)) and np.median(tol) < 1e-5
    assert np.max(np.abs(e - d)) < 1e-12


def test_stochastic_monte_carlo_matches_trilinear_ewa():
    """Stochastic level and texel (Philox variates): the mean over 2048 samples agrees
    with the deterministic EWA blended over the two levels around lod."""
    tex = textures.Texture2D.box_pyramid(rng.uniform(0, 1, (32, 32, 1)), 6)
    n = 24
    uv = rng.uniform(0.2, 0.8, (n, 2)).astype(np.float32)
    g = (rng.uniform(-1, 1, (n, 4)) * rng.uniform(0.5, 6, (n, 1)) / 32).astype(np.float32)
    S = 2048
    acc = np.zeros((n, 1))
    acc2 = np.zeros((n, 1))
    for s in range(S):
        v, _, _ = ewa.lookup(tex, uv, g, 16, stochastic_form=True, sample_index=s, seed=3)
        acc += v
        acc2 += v * v
    mean = acc / S
    var = np.maximum(acc2 / S - mean ** 2, 1e-12)
    ref, _, _ = ewa.lookup(tex, uv, g, 16, stochastic_form=False)
    z = (mean - ref) / np.sqrt(var / S)
    assert np.mean(np.abs(z) > 3.5) <= 2 / n
    assert abs(np.sum(mean - ref) / np.sqrt(np.sum(var) / S)) < 4
