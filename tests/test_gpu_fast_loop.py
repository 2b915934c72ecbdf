"""The stochastic kernels of dense, sparse and 2D textures run calls that ask for no tap
output and no binning on 32-bit indices (a loop of their own, with 32-bit voxel offsets
on dense grids); on 3D grids with 16-byte aligned coordinates and results that loop
takes four consecutive queries per thread (three 16-byte coordinate loads, one 16-byte
result store), otherwise one.  The parity tests check the general loop against the
oracle with tap output on; here the same calls without tap output must give
bit-identical results, for every filter, on inputs that include NaN, huge and
out-of-range coordinates, with a ragged tail (n mod 4 != 0) and misaligned views."""
import numpy as np
import pytest
import torch

import paper_2305_05810_gb300 as stf
import synth
from parity import dev, to_dev

pytestmark = pytest.mark.gpu

FILTERS = ["linear", "bspline3", "catmull_rom", "catmull_rom_positivized", "fis_linear",
           "fis_bspline3", "fis_gaussian"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stf.load()


def _edge(d):
    return np.array([[np.nan] * d, [1e30] * d, [-1e30] * d, [16777216.0] * d, [-16777217.0] * d,
                     [0.0] * d, [-0.5] * d, [np.inf] + [0.0] * (d - 1)], dtype=np.float32)


def _same(T, q, lod=None, **params):
    """One call with tap output (general loop), one without (fast loop): bit-equal."""
    n = q.shape[0]
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    general = T.lookup(q, lod, taps=taps, **params)
    fast = T.lookup(q, lod, **params)
    torch.cuda.synchronize()
    torch.testing.assert_close(fast, general, rtol=0, atol=0, equal_nan=True)


def _params(filt):
    return {"filter": filt, "seed": 99, "sample_index": 3, "query_offset": 12345,
            "width": 0.9 if filt == "fis_gaussian" else 0.0}


def _same_3d_views(T, q, **params):
    """Aligned (four queries per thread), misaligned by one query (one per thread) and
    the general loop with tap output: bit-equal on the common queries."""
    n = q.shape[0]
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    general = T.lookup(q, taps=taps, **params)
    quad = T.lookup(q, **params)
    p1 = dict(params, query_offset=params["query_offset"] + 1)
    out1 = torch.empty((n, 1), dtype=torch.float32, device=dev())
    stf.stf_lookup_batch(T.handle, stf.make_params(**p1), q[1:], None, n - 1, out1[1:])  # 12-byte offset
    torch.cuda.synchronize()
    assert q.shape[0] % 4 != 0 and q[1:].data_ptr() % 16 != 0
    torch.testing.assert_close(quad, general, rtol=0, atol=0, equal_nan=True)
    torch.testing.assert_close(out1[1:], general[1:], rtol=0, atol=0, equal_nan=True)


@pytest.mark.parametrize("filt", ["linear", "bspline3", "catmull_rom", "catmull_rom_positivized"])
def test_dense_and_sparse_quad_loop_views(filt):
    vals = synth.dense_density(n=40, seed=6, period=9.0)
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(40, 40, 40), fmt=stf.FMT_F16)
    q = (synth.uniform(3 * 70001, 8).reshape(-1, 3) * np.float32(48) - np.float32(4)).astype(np.float32)
    _same_3d_views(T, to_dev(np.concatenate([q, _edge(3)])), **_params(filt))
    origins, values = synth.sparse_cloud(domain=512, seed=9)
    S = stf.Texture(stf.KIND_SPARSE3D, values, fmt=stf.FMT_E4M3_SCALED, leaf_origins=origins)
    o = origins[np.arange(30001) % len(origins)].astype(np.float32)
    q = (o + synth.uniform(3 * 30001, 10).reshape(-1, 3) * np.float32(10) - np.float32(1)).astype(np.float32)
    _same_3d_views(S, to_dev(np.concatenate([q, _edge(3)])), **_params(filt))


@pytest.mark.parametrize("fmt", [stf.FMT_F32, stf.FMT_F16])
@pytest.mark.parametrize("filt", FILTERS)
def test_dense_fast_loop_equals_general_loop(filt, fmt):
    vals = synth.dense_density(n=40, seed=6, period=9.0)
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(40, 40, 40), fmt=fmt)
    q = (synth.uniform(3 * 70001, 8).reshape(-1, 3) * np.float32(48) - np.float32(4)).astype(np.float32)
    _same(T, to_dev(np.concatenate([q, _edge(3)])), **_params(filt))


def _miss_box_edges(n):
    """Coordinates on and next to the boundaries of the miss test of a grid of n voxels per
    axis (the tent's window misses for x < -1 or x >= n, the B-spline's for x < -2 or
    x >= n + 1), one axis at a time, the others inside the grid."""
    vals = []
    for b in (-2.0, -1.0, float(n), float(n + 1)):
        vals += [np.nextafter(np.float32(b), np.float32(-np.inf)), np.float32(b),
                 np.nextafter(np.float32(b), np.float32(np.inf))]
    rows = []
    for a in range(3):
        for v in vals:
            r = [np.float32(n / 2 + 0.25)] * 3
            r[a] = v
            rows.append(r)
    return np.array(rows, dtype=np.float32)


@pytest.mark.parametrize("fmt", [stf.FMT_F32, stf.FMT_F16])
@pytest.mark.parametrize("filt", FILTERS)
def test_dense_quads_mixing_live_and_dead_queries(filt, fmt):
    """Four-query groups in which some queries are dead (NaN, infinite, huge, or with a
    window outside the grid) and others live: the joint form draws for all four and
    keeps only the live results, so every query must equal the general loop's; queries
    on the miss test's boundaries check that the shortcut is exact."""
    n = 40
    vals = synth.dense_density(n=n, seed=6, period=9.0)
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(n, n, n), fmt=fmt)
    q = (synth.uniform(3 * 40003, 12).reshape(-1, 3) * np.float32(48) - np.float32(4)).astype(np.float32)
    special = np.concatenate([_edge(3), _miss_box_edges(n)])
    rng = np.random.default_rng(5)
    pos = rng.choice(q.shape[0], size=4000, replace=False)
    q[pos] = special[rng.integers(0, special.shape[0], size=pos.size)]
    q[: special.shape[0]] = special                     # and a run of them at the start
    _same(T, to_dev(q), **_params(filt))


@pytest.mark.parametrize("fmt", [stf.FMT_F32, stf.FMT_E4M3_SCALED])
@pytest.mark.parametrize("filt", FILTERS)
def test_sparse_fast_loop_equals_general_loop(filt, fmt):
    origins, values = synth.sparse_cloud(domain=512, seed=9)
    T = stf.Texture(stf.KIND_SPARSE3D, values, fmt=fmt, leaf_origins=origins)
    o = origins[np.arange(60000) % len(origins)].astype(np.float32)
    q = (o + synth.uniform(3 * 60000, 10).reshape(-1, 3) * np.float32(10) - np.float32(1)).astype(np.float32)
    # points around the active leaves' bounding box, inside and outside it (outside it the
    # fast loop returns the background without drawing)
    lo, hi = origins.min(axis=0), origins.max(axis=0) + 8
    far = (lo + (synth.uniform(3 * 20000, 11).reshape(-1, 3) * 1.6 - 0.3) * (hi - lo)).astype(np.float32)
    _same(T, to_dev(np.concatenate([q, far, _edge(3)])), **_params(filt))


@pytest.mark.parametrize("C", [1, 2, 4])
@pytest.mark.parametrize("filt", FILTERS)
def test_tex2d_fast_loop_equals_general_loop(filt, C):
    T = stf.Texture(stf.KIND_TEX2D, synth.texture2d(128, 64, C, seed=12), dims=(128, 64, 1), channels=C,
                    mip_levels=7, generate_mips=True)
    uv = np.concatenate([synth.uv_queries(50000, seed=13) * np.float32(1.4) - np.float32(0.2), _edge(2)])
    lod = synth.lods(uv.shape[0], seed=14, lo=-1, hi=7).astype(np.float32)
    lod[-3:] = [np.nan, np.inf, -np.inf]
    for level_mode in (stf.LEVEL_NEAREST, stf.LEVEL_STOCHASTIC):
        _same(T, to_dev(uv.astype(np.float32)), to_dev(lod), level_mode=level_mode, **_params(filt))


def test_dct_fast_loop_equals_general_loop():
    base = synth.texture2d(128, 64, 8, seed=15)
    T = stf.Texture(stf.KIND_TEX2D, base, dims=(128, 64, 1), channels=8, mip_levels=6,
                    generate_mips=True, fmt=stf.FMT_DCT6)
    uv = to_dev(np.concatenate([synth.uv_queries(40000, seed=16), _edge(2)]))
    lod = to_dev(synth.lods(uv.shape[0], seed=17, lo=0, hi=5).astype(np.float32))
    for filt in ("linear", "bspline3"):
        _same(T, uv, lod, **_params(filt))


@pytest.mark.parametrize("kind", ["dense", "tex2d"])
def test_calls_around_2_30_queries(kind):
    """The loop switch at 2^30 queries: a call of 2^30 queries (fast loop, 3 i + 2 just
    below 2^32) and one of 2^30 + 4097 (general 64-bit loop) end with the same values as
    a small call over their last queries with the matching query offset."""
    n_big = (1 << 30) + 4097
    d = 3 if kind == "dense" else 2
    g = torch.Generator(device=dev()).manual_seed(5)
    coords = torch.rand((n_big, d), generator=g, device=dev())
    if kind == "dense":
        T = stf.Texture(stf.KIND_DENSE3D, synth.dense_density(n=32, seed=3, period=8.0), dims=(32, 32, 32),
                        fmt=stf.FMT_F16)
        coords.mul_(36.0).sub_(2.0)
    else:
        T = stf.Texture(stf.KIND_TEX2D, synth.texture2d(64, 64, 1, seed=3), dims=(64, 64, 1), channels=1)
    out = torch.empty((n_big, 1), device=dev())
    tail = 1 << 16
    for n in (1 << 30, n_big):
        stf.stf_lookup_batch(T.handle, stf.make_params("bspline3", seed=8), coords, None, n, out)
        small = torch.empty((tail, 1), device=dev())
        stf.stf_lookup_batch(T.handle, stf.make_params("bspline3", seed=8, query_offset=n - tail),
                             coords[n - tail:n], None, tail, small)
        torch.cuda.synchronize()
        assert torch.equal(out[n - tail:n], small)
        assert torch.equal(out[:tail], T.lookup(coords[:tail], filter="bspline3", seed=8))
    del coords, out
    torch.cuda.empty_cache()
