"""Pins of the float64 oracle against things other than itself: closed forms,
brute force on tiny grids, independent libraries, and Eq. 8's printed case table.
CPU only."""
import itertools
import os
from math import comb

import numpy as np
import pytest
import torch

from oracle import codecs, filters, kernels, philox, textures

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(12345)


# ------------------------------------------------------------------ generator

@pytest.mark.parametrize("ctr,key", [((0, 0, 0, 0), (0, 0)), ((5, 7, 9, 11), (123, 456)),
                                     ((2**64 - 2, 3, 2**63, 1), (2**64 - 1, 99))])
def test_philox_round_structure_matches_numpy_philox4x64(ctr, key):
    """numpy's Philox bit generator is Philox4x64-10; it increments its counter once
    before producing the first block."""
    bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    ref = [int(x) for x in bg.random_raw(4)]
    c = list(ctr)
    c[0] = (c[0] + 1) % 2**64
    if c[0] == 0:
        c[1] = (c[1] + 1) % 2**64
    assert list(philox.philox4x64(c, key)) == ref


def test_philox4x32_10_known_answers():
    """The published known answers of Philox4x32-10 (golden fixture, cited there):
    they fix the 4x32 multipliers and Weyl constants, which the 4x64 structure pin
    and the statistical pins cannot."""
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([int(w, 16) for w in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = philox.philox4x32(*r[:6])
        assert [int(x) for x in out] == r[6:]


def test_philox_weyl_constants_are_the_published_irrationals():
    """W0 = floor(2^32 (golden ratio - 1)), W1 = floor(2^32 (sqrt 3 - 1)) (Salmon et al.,
    Section 4.2), computed here with exact integer square roots."""
    from math import isqrt
    w0 = (isqrt(5 << 128) - (1 << 64)) >> 33          # 2^32 (sqrt5 - 1)/2
    w1 = isqrt(3 << 64) - (1 << 32)                   # 2^32 (sqrt3 - 1)
    assert philox.PHILOX4X32["W"] == (w0, w1)


def test_philox4x32_uniform_chi2_and_exact_variates():
    n = 1 << 20
    u = philox.query_variates(np.arange(n, dtype=np.uint64), 0, 42)
    for w in range(4):
        assert np.all(u[w] * 2**24 == np.floor(u[w] * 2**24))      # 24-bit lattice
        assert np.all(u[w].astype(np.float32).astype(np.float64) == u[w])
        counts = np.bincount((u[w] * 256).astype(int), minlength=256)
        chi2 = np.sum((counts - n / 256) ** 2 / (n / 256))
        assert 150 < chi2 < 380, chi2                                 # 255 dof, p ~ 1e-6 bounds


def test_philox4x32_independence():
    n = 1 << 18
    q = np.arange(n, dtype=np.uint64)
    u = philox.query_variates(q, 0, 7)
    for a, b in itertools.combinations(range(4), 2):
        assert abs(np.corrcoef(u[a], u[b])[0, 1]) < 5 / np.sqrt(n)
    assert abs(np.corrcoef(u[0][:-1], u[0][1:])[0, 1]) < 5 / np.sqrt(n)
    v = philox.query_variates(q, 1, 7)          # another sample index
    w = philox.query_variates(q, 0, 8)          # another seed
    assert abs(np.corrcoef(u[0], v[0])[0, 1]) < 5 / np.sqrt(n)
    assert abs(np.corrcoef(u[0], w[0])[0, 1]) < 5 / np.sqrt(n)
    big = philox.query_variates(q + np.uint64(2**32), 0, 7)   # high counter word matters
    assert not np.array_equal(big[0], u[0])


# ------------------------------------------------------------------ kernels

F = np.linspace(0, 1, 1001)[:-1]


@pytest.mark.parametrize("filt", ["linear", "bspline3", "catmull_rom"])
def test_partition_of_unity(filt):
    w = filters.axis_weights(F.astype(np.float32), filt)
    assert np.max(np.abs(w.sum(axis=0) - 1)) < 1e-14


@pytest.mark.parametrize("a", [-0.5, -0.75, -1.0])
def test_cubic_family_partition_and_interpolation(a):
    t = F
    w = sum(kernels.k3_cubic(t - o, a) for o in (-1, 0, 1, 2))
    assert np.max(np.abs(w - 1)) < 1e-14
    assert kernels.k3_cubic(np.array([0.0]), a)[0] == 1
    assert np.all(kernels.k3_cubic(np.array([-2.0, -1.0, 1.0, 2.0, 2.5]), a) == 0)


def test_bspline_matches_truncated_power_form():
    """Uniform cubic B-spline centred at 0: (1/6) sum_j (-1)^j C(4,j) (t + 2 - j)_+^3."""
    t = np.linspace(-3, 3, 6001)
    ref = sum((-1) ** j * comb(4, j) * np.maximum(t + 2 - j, 0) ** 3 for j in range(5)) / 6
    assert np.max(np.abs(kernels.k_bspline3(t) - ref)) < 1e-13
    assert abs(kernels.k_bspline3(np.array([0.0]))[0] - 2 / 3) < 1e-15   # not interpolating


def test_tent_and_box():
    assert np.allclose(kernels.k1_tent(np.array([-1.5, -0.25, 0, 0.5, 1])), [0, 0.75, 1, 0.5, 0])
    assert np.array_equal(kernels.k0_box(np.array([-0.6, -0.4, 0, 0.49, 0.5])), [0, 1, 1, 1, 0])


def test_catmull_rom_reproduces_quadratics_and_other_a_does_not():
    x = rng.uniform(10, 20, 500)
    p = lambda z: 0.3 * z * z - 2 * z + 5
    i0 = np.floor(x)
    for a, ok in ((-0.5, True), (-0.75, False)):
        s = sum(kernels.k3_cubic(x - (i0 + o), a) * p(i0 + o) for o in (-1, 0, 1, 2))
        assert (np.max(np.abs(s - p(x))) < 1e-10) == ok


@pytest.mark.parametrize("filt", ["linear", "bspline3", "catmull_rom"])
def test_filters_reproduce_affine(filt):
    x = rng.uniform(10, 20, 500)
    offs = kernels.FILTERS[filt][0]
    i0 = np.floor(x)
    s = sum(kernels.FILTERS[filt][1](x - (i0 + o)) * (2.5 * (i0 + o) - 1) for o in offs)
    assert np.max(np.abs(s - (2.5 * x - 1))) < 1e-11


# ------------------------------------------------------------------ tap selection

@pytest.mark.parametrize("filt", ["linear", "bspline3", "catmull_rom"])
@pytest.mark.parametrize("f", [0.0, 0.125, 0.37, 0.5, 0.9])
def test_selection_frequencies_equal_abs_weights(filt, f):
    n = 1 << 20
    u = np.arange(n) / n                                    # exact 20-bit lattice
    f32 = np.full(n, f, dtype=np.float32)
    w = filters.axis_weights(f32, filt)
    k, _ = filters.select_tap(u, w)
    assert np.all(np.diff(k) >= 0)                          # CDF order: low to high
    freq = np.bincount(k, minlength=w.shape[0]) / n
    p = np.abs(w[:, 0]) / np.abs(w[:, 0]).sum()
    assert np.max(np.abs(freq - p)) <= 2.0 / n + 1e-6
    assert np.all(freq[p == 0] == 0)                        # zero-weight taps never drawn


def test_bilinear_at_integer_never_takes_second_tap():
    u = np.arange(1 << 16) / (1 << 16)
    w = filters.axis_weights(np.zeros(u.size, dtype=np.float32), "linear")
    k, _ = filters.select_tap(u, w)
    assert np.all(k == 0)


def _golden_eq8():
    rows = []
    with open(os.path.join(GOLDEN, "eq8_bilerp_cases.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                xi, s, t, c = line.split()
                rows.append((float(xi), float(s), float(t), c))
    return rows


@pytest.mark.parametrize("xi,s,t,corner", _golden_eq8())
def test_eq8_case_table_with_reused_variate(xi, s, t, corner):
    """The inverse-CDF rule with taps ordered low to high and one variate carried
    through Eq. 4 reproduces Eq. 8 under the reflection u = 1 - xi."""
    tex = textures.Texture2D([np.arange(16.0).reshape(4, 4, 1)])
    x = np.array([1 + s], dtype=np.float32)
    y = np.array([1 + t], dtype=np.float32)
    u = np.array([1.0 - xi])
    _, idx, _, _ = filters.stochastic(lambda ix, iy: tex.fetch(0, ix, iy), [x, y], "linear",
                                      [u, u], reuse=True)
    assert (int(idx[0][0]) - 1, int(idx[1][0]) - 1) == (int(corner[1]), int(corner[2]))


def test_reuse_remap_is_uniform_within_each_tap():
    n = 1 << 18
    u = (np.arange(n) + 0.5) / n
    w = filters.axis_weights(np.full(n, 0.3, dtype=np.float32), "bspline3")
    k, u2 = filters.select_tap(u, w)
    for kk in range(4):
        sub = u2[k == kk]
        assert abs(sub.mean() - 0.5) < 1e-3 and sub.min() < 1e-3 and sub.max() > 1 - 1e-3


# ------------------------------------------------------------------ estimators

def _tex2d(h=9, w=11, c=3, seed=0):
    return textures.Texture2D([np.random.default_rng(seed).uniform(-1, 2, (h, w, c))])


@pytest.mark.parametrize("filt", ["linear", "bspline3", "catmull_rom"])
def test_expectation_by_enumeration_equals_deterministic_2d(filt):
    tex = _tex2d()
    x = rng.uniform(-2, 13, 400).astype(np.float32)
    y = rng.uniform(-2, 11, 400).astype(np.float32)
    fetch = lambda ix, iy: tex.fetch(0, ix, iy)
    e = filters.expectation_by_enumeration(fetch, [x, y], filt)
    d = filters.deterministic(fetch, [x, y], filt)
    assert np.max(np.abs(e - d) / (np.abs(d) + 1)) < 1e-12


@pytest.mark.parametrize("filt", ["linear", "bspline3", "catmull_rom"])
def test_expectation_by_enumeration_equals_deterministic_3d(filt):
    g = textures.Dense3D(rng.uniform(0, 1, (5, 6, 7)))
    p = [rng.uniform(-2, 8, 200).astype(np.float32) for _ in range(3)]
    e = filters.expectation_by_enumeration(g.fetch, p, filt)
    d = filters.deterministic(g.fetch, p, filt)
    assert np.max(np.abs(e - d)) < 1e-12


def test_second_moment_of_two_point_estimator():
    """Stochastic lerp (Eq. 7) is a two-point distribution: variance f(1-f)(t1-t0)^2."""
    vals = rng.uniform(-1, 1, (1, 12, 1))
    tex = textures.Texture2D([vals])
    x = rng.uniform(0, 10, 300).astype(np.float32)
    y = np.zeros(300, dtype=np.float32)
    fetch = lambda ix, iy: tex.fetch(0, ix, iy)
    m1 = filters.expectation_by_enumeration(fetch, [x, y], "linear")[:, 0]
    m2 = filters.expectation_by_enumeration(fetch, [x, y], "linear", power=2)[:, 0]
    i0 = np.floor(x.astype(np.float64)).astype(int)
    f = x.astype(np.float64) - i0
    t0, t1 = vals[0, i0, 0], vals[0, np.minimum(i0 + 1, 11), 0]
    assert np.max(np.abs((m2 - m1 ** 2) - f * (1 - f) * (t1 - t0) ** 2)) < 1e-12


def test_tap_counts_are_2n_and_4n():
    calls = []
    g = textures.Dense3D(np.ones((6, 6, 6)))

    def fetch(*idx):
        calls.append(1)
        return g.fetch(*idx) if len(idx) == 3 else np.ones((idx[0].shape[0], 1))
    pts = [np.array([2.5], dtype=np.float32)] * 3
    for filt, dims, n in (("linear", 2, 4), ("linear", 3, 8), ("bspline3", 2, 16), ("bspline3", 3, 64)):
        calls.clear()
        filters.deterministic(fetch, pts[:dims], filt)
        assert len(calls) == n


@pytest.mark.parametrize("filt", ["linear", "bspline3", "catmull_rom"])
def test_monte_carlo_mean_converges_to_deterministic(filt):
    tex = _tex2d(seed=3)
    uv = np.array([[0.31, 0.62], [0.5, 0.5], [0.05, 0.97], [0.77, 0.13]], dtype=np.float32)
    S = 4096
    qid = np.repeat(np.arange(4, dtype=np.uint64), S)
    samples = np.tile(np.arange(S), 4)
    vals = np.zeros((4 * S, 3))
    for s in range(S):                     # vary the sample index, as the GPU sweep does
        m = samples == s
        v, _, _ = filters.lookup_2d(tex, uv, None, filt, stochastic_form=True, qid=qid[m],
                                    sample_index=s, seed=9)
        vals[m] = v
    vals = vals.reshape(4, S, 3)
    det, _, _ = filters.lookup_2d(tex, uv, None, filt, stochastic_form=False)
    sd = vals.std(axis=1)
    z = (vals.mean(axis=1) - det) / (sd / np.sqrt(S) + 1e-300)
    assert np.all(np.abs(z[sd > 1e-9]) < 4.5)
    assert np.all(np.abs(vals.mean(axis=1) - det)[sd <= 1e-9] < 1e-12)   # no variance: exact


def _brute_2d(tex, x, y, K):
    """Sum over every lattice point of an extended range, no tap window."""
    h, w, _ = tex.levels[0].shape
    out = np.zeros((x.size, tex.channels))
    for j in range(-6, h + 6):
        for i in range(-6, w + 6):
            wt = K(x - i) * K(y - j)
            out += wt[:, None] * tex.levels[0][min(max(j, 0), h - 1), min(max(i, 0), w - 1)]
    return out


@pytest.mark.parametrize("filt", ["linear", "bspline3", "catmull_rom"])
def test_deterministic_equals_brute_force_continuous_filter_2d(filt):
    tex = _tex2d(4, 4, 2, seed=5)
    uv = rng.uniform(-0.3, 1.3, (300, 2)).astype(np.float32)
    d, _, _ = filters.lookup_2d(tex, uv, None, filt, stochastic_form=False)
    x = (uv[:, 0] * np.float32(4) - np.float32(0.5)).astype(np.float64)
    y = (uv[:, 1] * np.float32(4) - np.float32(0.5)).astype(np.float64)
    K = kernels.FILTERS[filt][1]
    assert np.max(np.abs(d - _brute_2d(tex, x, y, K))) < 1e-12


@pytest.mark.parametrize("filt", ["linear", "bspline3", "catmull_rom"])
def test_deterministic_equals_brute_force_continuous_filter_3d(filt):
    vals = rng.uniform(0, 1, (5, 5, 5))
    g = textures.Dense3D(vals)
    p = rng.uniform(-2, 7, (200, 3)).astype(np.float32)
    d, _, _ = filters.lookup_3d(g, p, filt, stochastic_form=False)
    K = kernels.FILTERS[filt][1]
    ref = np.zeros(200)
    pp = p.astype(np.float64)
    for z, y, x in itertools.product(range(5), repeat=3):
        ref += K(pp[:, 0] - x) * K(pp[:, 1] - y) * K(pp[:, 2] - z) * vals[z, y, x]
    assert np.max(np.abs(d[:, 0] - ref)) < 1e-12


@pytest.mark.parametrize("filt", ["linear", "bspline3", "catmull_rom"])
def test_affine_texture_interior_points_use_half_texel_offset(filt):
    W = H = 32
    j, i = np.mgrid[0:H, 0:W]
    tex = textures.Texture2D([(0.25 + 0.5 * i + 0.75 * j)[..., None].astype(np.float64)])
    uv = rng.uniform(4 / 32, 28 / 32, (300, 2)).astype(np.float32)
    d, _, _ = filters.lookup_2d(tex, uv, None, filt, stochastic_form=False)
    x = uv[:, 0].astype(np.float64) * W - 0.5
    y = uv[:, 1].astype(np.float64) * H - 0.5
    assert np.max(np.abs(d[:, 0] - (0.25 + 0.5 * x + 0.75 * y))) < 1e-10


def test_constant_texture_returned_exactly():
    tex = textures.Texture2D([np.full((8, 8, 4), 0.625)])
    uv = rng.uniform(0, 1, (500, 2)).astype(np.float32)
    for filt in ("linear", "bspline3", "catmull_rom"):
        d, _, _ = filters.lookup_2d(tex, uv, None, filt, stochastic_form=False)
        assert np.max(np.abs(d - 0.625)) < 1e-14          # float64 rounding of the weight sum
    for filt in ("linear", "bspline3"):
        s, _, _ = filters.lookup_2d(tex, uv, None, filt, stochastic_form=True, seed=3)
        assert np.all(s == 0.625)
    # Catmull-Rom, one tap per axis by |w|: each sample is +-Sx*Sy*c, exact in expectation
    s, taps, _ = filters.lookup_2d(tex, uv, None, "catmull_rom", stochastic_form=True, seed=3)
    assert np.all(np.abs(s) >= 0.625 - 1e-15)


def test_catmull_rom_at_texel_centres_returns_texel():
    tex = _tex2d(8, 8, 1, seed=7)
    i = rng.integers(2, 6, (100, 2))
    uv = ((i + 0.5) / 8).astype(np.float32)
    exact = tex.levels[0][i[:, 1], i[:, 0]]
    d, _, _ = filters.lookup_2d(tex, uv, None, "catmull_rom", stochastic_form=False)
    s, _, _ = filters.lookup_2d(tex, uv, None, "catmull_rom", stochastic_form=True, seed=1)
    assert np.max(np.abs(d - exact)) < 1e-15 and np.array_equal(s, exact)


def test_non_finite_coordinates_give_background():
    tex = _tex2d()
    uv = np.array([[np.nan, 0.5], [0.5, np.inf], [0.5, 0.5]], dtype=np.float32)
    s, taps, _ = filters.lookup_2d(tex, uv, None, "bspline3", stochastic_form=True)
    d, _, _ = filters.lookup_2d(tex, uv, None, "bspline3", stochastic_form=False)
    assert np.all(s[:2] == 0) and np.all(d[:2] == 0) and np.all(taps[:2, 3] == -1)
    assert taps[2, 3] == 0


# ------------------------------------------------------------------ MIP levels

def test_box_pyramid_is_block_mean():
    base = rng.uniform(0, 1, (8, 16, 2))
    tex = textures.Texture2D.box_pyramid(base, 5)
    for L in range(5):
        h, w = max(1, 8 >> L), max(1, 16 >> L)
        by, bx = 8 // h, 16 // w
        for y in range(h):
            for x in range(w):
                blk = base[y * by:(y + 1) * by, x * bx:(x + 1) * bx]
                assert np.allclose(tex.levels[L][y, x], blk.reshape(-1, 2).mean(axis=0), atol=1e-15)


def test_stochastic_level_probability_and_deterministic_blend():
    base = rng.uniform(0, 1, (16, 16, 1))
    tex = textures.Texture2D.box_pyramid(base, 5)
    n = 1 << 14
    lod = np.full(n, 1.3, dtype=np.float32)
    L0, _, _, _ = filters._level_choice(lod, 5, filters.LEVEL_STOCHASTIC, np.arange(n) / n, True)
    assert abs(np.mean(L0 == 2) - (np.float32(1.3) - 1)) < 2.0 / n
    assert set(np.unique(L0)) == {1, 2}
    Ln, _, _, _ = filters._level_choice(np.array([1.49, 1.5, 3.9, 9.0], dtype=np.float32), 5,
                                        filters.LEVEL_NEAREST, None, True)
    assert list(Ln) == [1, 2, 4, 4]
    # deterministic blend = expectation over the level choice of per-level filters
    uv = rng.uniform(0, 1, (50, 2)).astype(np.float32)
    lods = rng.uniform(0, 4, 50).astype(np.float32)
    d, _, _ = filters.lookup_2d(tex, uv, lods, "bspline3", stochastic_form=False)
    ref = np.zeros((50, 1))
    for L in range(5):
        a = lods.astype(np.float64) - np.floor(lods)
        p = np.where(np.floor(lods) == L, 1 - a, 0) + np.where(np.floor(lods) + 1 == L, a, 0)
        dl, _, _ = filters.lookup_2d(tex, uv, np.full(50, L, dtype=np.float32), "bspline3",
                                     stochastic_form=False, level_mode=filters.LEVEL_NEAREST)
        ref += p[:, None] * dl
    assert np.max(np.abs(d - ref)) < 1e-12


# ------------------------------------------------------------------ sparse map

def test_sparse_map_equals_dense_grid():
    vals = np.zeros((24, 24, 24))
    vals[3:11, 9:20, 0:7] = rng.uniform(0.1, 1, (8, 11, 7))
    vals[17, 2, 20] = 0.5
    dense = textures.Dense3D(vals)
    origins, leaves = [], []
    for oz, oy, ox in itertools.product(range(0, 24, 8), repeat=3):
        blk = vals[oz:oz + 8, oy:oy + 8, ox:ox + 8]
        if np.any(blk):
            origins.append((ox, oy, oz))
            leaves.append(np.transpose(blk, (2, 1, 0)))    # [x][y][z]
    sp = textures.Sparse3D(np.array(origins), np.array(leaves))
    pts = rng.integers(-5, 30, (5000, 3))
    assert np.array_equal(sp.fetch(*pts.T), dense.fetch(*pts.T))


# ------------------------------------------------------------------ codecs

def test_f16_codec_matches_numpy():
    codes = np.arange(65536)
    v = codecs.f16_decode(codes)
    ref = codes.astype(np.uint16).view(np.float16).astype(np.float64)
    assert np.array_equal(np.isnan(v), np.isnan(ref))
    assert np.array_equal(v[~np.isnan(v)], ref[~np.isnan(ref)])
    x = rng.standard_normal(200000) * np.exp2(rng.uniform(-28, 17, 200000))
    with np.errstate(over="ignore"):
        assert np.array_equal(codecs.f16_encode(x), x.astype(np.float16).view(np.uint16))
    fin = v[np.isfinite(v)]
    assert np.array_equal(codecs.f16_decode(codecs.f16_encode(fin)), fin)


def test_e4m3_codec_matches_torch_and_saturates():
    v = codecs.e4m3_decode(np.arange(256))
    ref = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).double().numpy()
    assert np.array_equal(np.isnan(v), np.isnan(ref))
    assert np.array_equal(v[~np.isnan(v)], ref[~np.isnan(ref)])
    assert np.nanmax(v) == 448
    x = rng.uniform(-448, 448, 200000) * np.exp2(rng.uniform(-14, 0, 200000))
    tref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(codecs.e4m3_encode(x), tref)
    assert list(codecs.e4m3_encode(np.array([500.0, -1e9, np.inf, np.nan]))) == [0x7E, 0xFE, 0x7E, 0x7F]
    fin = v[np.isfinite(v)]
    assert np.array_equal(codecs.e4m3_decode(codecs.e4m3_encode(fin)), fin)


def test_e4m3_leaf_quantisation_error_bound():
    leaves = rng.uniform(0.05, 1.0, (64, 512)).astype(np.float32)
    codes, scales = codecs.e4m3_leaf_quantise(leaves)
    deq = codecs.e4m3_leaf_dequantise(codes, scales)
    assert np.all(np.max(np.abs(deq), axis=1) <= 448 * scales.astype(np.float64) * (1 + 1e-7))
    rel = np.abs(deq - leaves) / leaves
    big = leaves >= scales[:, None] * 2.0 ** -6          # normal E4M3 range
    assert np.max(rel[big]) <= 2.0 ** -4 * (1 + 1e-6)


# ------------------------------------------------------------------ positivization

def _set_moments(fetch, xs32, sign):
    """W, E[t] and E[t^2] of one sign's set under the positivized sampler (exact,
    by enumeration of its blocks and taps)."""
    D = len(xs32)
    frames = [filters.axis_frame(x) for x in xs32]
    w64 = [filters.axis_weights(f, "catmull_rom") for (_, f, _) in frames]
    m = filters._block_masses(w64, D)
    blocks = filters._blocks_of_sign(D, sign)
    W = np.sum([m[b] for b in blocks], axis=0)
    e1 = e2 = 0.0
    for b in blocks:
        pb = np.where(W > 0, m[b] / np.where(W > 0, W, 1), 0)
        for combo in itertools.product((0, 1), repeat=D):
            p, idx = pb.copy(), []
            for a in range(D):
                t0, t1 = ((0, 3) if (b >> a) & 1 else (1, 2))
                tap = (t0, t1)[combo[a]]
                s = np.abs(w64[a][t0]) + np.abs(w64[a][t1])
                p = p * np.where(s > 0, np.abs(w64[a][tap]) / np.where(s > 0, s, 1), 0)
                idx.append(frames[a][0] - 1 + tap)
            t = fetch(*idx)[:, 0]
            e1 = e1 + p * t
            e2 = e2 + p * t * t
    return W, e1, e2


@pytest.mark.parametrize("dims", [2, 3])
def test_positivized_expectation_equals_deterministic(dims):
    if dims == 2:
        tex = _tex2d(9, 11, 2, seed=8)
        fetch = lambda ix, iy: tex.fetch(0, ix, iy)
        xs = [rng.uniform(-2, 13, 300).astype(np.float32), rng.uniform(-2, 11, 300).astype(np.float32)]
    else:
        g = textures.Dense3D(rng.uniform(0, 1, (5, 6, 7)))
        fetch = g.fetch
        xs = [rng.uniform(-2, 8, 200).astype(np.float32) for _ in range(3)]
    e = filters.positivized_expectation(fetch, xs)
    d = filters.deterministic(fetch, xs, "catmull_rom")
    assert np.max(np.abs(e - d)) < 1e-12


def test_positivized_block_and_tap_frequencies():
    """The block of each set is drawn with probability mass / W, the tap within it with
    probability |w| / pair sum (u-lattice frequencies)."""
    n = 1 << 16
    u = np.arange(n) / n
    f = np.float32(0.3)
    x = np.full(n, 3 + f, dtype=np.float32)
    y = np.full(n, 5 + np.float32(0.8), dtype=np.float32)
    tex = textures.Texture2D([np.arange(100.0).reshape(10, 10, 1)])
    fetch = lambda ix, iy: tex.fetch(0, ix, iy)
    const = np.full(n, 0.5)
    _, ip, ineg, _, _ = filters.positivized(fetch, [x, y], [const, const, u], [const, const, u])
    w = [filters.axis_weights(np.array([0.3]), "catmull_rom")[:, 0],
         filters.axis_weights(np.array([np.float64(np.float32(0.8))]), "catmull_rom")[:, 0]]
    ain = [abs(v[1]) + abs(v[2]) for v in w]
    aout = [abs(v[0]) + abs(v[3]) for v in w]
    m = {0: ain[0] * ain[1], 1: aout[0] * ain[1], 2: ain[0] * aout[1], 3: aout[0] * aout[1]}
    outer_x = np.isin(ip[0] - 3, [-1, 2])
    outer_y = np.isin(ip[1] - 5, [-1, 2])
    assert abs(np.mean(~outer_x & ~outer_y) - m[0] / (m[0] + m[3])) < 2.0 / n + 1e-6
    outer_x = np.isin(ineg[0] - 3, [-1, 2])
    assert abs(np.mean(outer_x) - m[1] / (m[1] + m[2])) < 2.0 / n + 1e-6
    # within a block, each axis picks its tap by |w| (variate u[a])
    _, ip, _, _, _ = filters.positivized(fetch, [x, y], [u, const, np.zeros(n)], [const, const, u])
    assert abs(np.mean(ip[0] == 3) - abs(w[0][1]) / ain[0]) < 2.0 / n + 1e-6


def test_positivized_has_lower_variance_than_single_tap():
    """Positivization (two taps) against the one-tap |w| estimator on a random
    texture: exact variances, averaged over positions (Section 2.2)."""
    tex = _tex2d(16, 16, 1, seed=11)
    fetch = lambda ix, iy: tex.fetch(0, ix, iy)
    xs = [rng.uniform(2, 13, 400).astype(np.float32), rng.uniform(2, 13, 400).astype(np.float32)]
    F = filters.deterministic(fetch, xs, "catmull_rom")[:, 0]
    Wp, p1, p2 = _set_moments(fetch, xs, 1)
    Wn, n1, n2 = _set_moments(fetch, xs, -1)
    var_pos = Wp ** 2 * (p2 - p1 ** 2) + Wn ** 2 * (n2 - n1 ** 2)
    assert np.allclose(Wp * p1 - Wn * n1, F, atol=1e-12)
    m2 = filters.expectation_by_enumeration(fetch, xs, "catmull_rom", power=2)[:, 0]
    var_abs = m2 - F ** 2
    assert np.mean(var_pos) < 0.8 * np.mean(var_abs), (np.mean(var_pos), np.mean(var_abs))


def test_positivized_at_texel_centres_returns_texel():
    tex = _tex2d(8, 8, 1, seed=7)
    i = rng.integers(2, 6, (100, 2))
    uv = ((i + 0.5) / 8).astype(np.float32)
    v, _, _ = filters.lookup_2d(tex, uv, None, "catmull_rom_positivized", stochastic_form=True, seed=2)
    assert np.array_equal(v, tex.levels[0][i[:, 1], i[:, 0]])
