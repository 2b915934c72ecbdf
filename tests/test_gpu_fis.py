"""GPU parity for filter importance sampling (Section 4.4, "Filter Importance
Sampling") through the C ABI against the float64 oracle (`oracle/fis.py`).

Bar: the B-spline FIS index is computed exactly on both sides (integer arithmetic
on the 2^-24 variate lattice), so taps and values must match bit for bit with no
exemption.  Gaussian FIS evaluates Box-Muller in float32 on the GPU (logf, sqrtf,
sincospif) and in float64 in the oracle, so a tap may differ only where x + s + 1/2
lies within 4e-6 (1 + |s|) of a texel boundary (oracle-reported), and then by at
most one texel.  Deterministic Gaussian: each of the two float32 erf values per tap
weight is within a few 1e-7 of the truth, so the window sum may differ from the
float64 one by at most 2e-6 |ref| + 5e-7 * taps_per_axis * D * max|t|."""
import numpy as np
import pytest
import torch

import paper_2305_05810_gb300 as stf
import synth
from oracle import codecs, filters, fis, textures
from parity import dev, quantise, to_dev

pytestmark = pytest.mark.gpu
FIS = ["fis_linear", "fis_bspline3", "fis_gaussian"]
WIDTH = {"fis_linear": 0.0, "fis_bspline3": 0.0, "fis_gaussian": 1.3}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stf.load()


def _check_fis(filt, gpu_val, gpu_taps, rv, rt, ex):
    gv = np.asarray(gpu_val, dtype=np.float64).reshape(rv.shape)
    gt = np.asarray(gpu_taps, dtype=np.int64).reshape(-1, 4)
    same = np.all(gt == rt, axis=1)
    if filt != "fis_gaussian":
        assert not np.any(ex)
    bad = ~same & ~ex
    assert not np.any(bad), "tap mismatch at %s: gpu %s ref %s" % (
        np.nonzero(bad)[0][:5], gt[bad][:5], rt[bad][:5])
    assert np.all(np.abs(gt - rt)[~same] <= 1)
    # an FIS value is the stored texel itself: exact
    assert np.array_equal(gv[same], rv[same])
    return int(np.sum(~same))


def _gauss_tol(ref_val, sigma, dims, tmax):
    taps = 2 * fis.gaussian_reach(sigma) + 2
    return 2e-6 * np.abs(ref_val) + 5e-7 * taps * dims * tmax


def _c1(n=65536):
    tex = synth.texture2d(256, 256, 4, seed=1)
    uv = synth.uv_queries(n, seed=2)
    edge = np.array([[np.nan, 0.5], [0.5, np.inf], [-0.25, 0.5], [1.3, -2.0], [0.5 / 256, 0.5 / 256],
                     [1.0, 1.0], [0.0, 0.0], [1e30, -1e30], [255.5 / 256, 3.5 / 256]], dtype=np.float32)
    return tex, np.concatenate([uv, edge])


@pytest.mark.parametrize("filt", FIS)
def test_fis_tex2d_matches_oracle(filt):
    tex, uv = _c1()
    T = stf.Texture(stf.KIND_TEX2D, tex, dims=(256, 256, 1), channels=4)
    n = uv.shape[0]
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    out = T.lookup(to_dev(uv), taps=taps, filter=filt, seed=41, sample_index=2, width=WIDTH[filt])
    ref = textures.Texture2D([tex.astype(np.float64)])
    rv, rt, ex = filters.lookup_2d(ref, uv, None, filt, stochastic_form=True, seed=41, sample_index=2,
                                   width=WIDTH[filt])
    torch.cuda.synchronize()
    _check_fis(filt, out.cpu().numpy(), taps.cpu().numpy(), rv, rt, ex)


@pytest.mark.parametrize("level_mode", [stf.LEVEL_NEAREST, stf.LEVEL_STOCHASTIC])
@pytest.mark.parametrize("filt", FIS)
def test_fis_tex2d_mip_levels(filt, level_mode):
    base = synth.texture2d(64, 32, 2, seed=11)
    T = stf.Texture(stf.KIND_TEX2D, base, dims=(64, 32, 1), channels=2, mip_levels=7, generate_mips=True)
    n = 20000
    uv = synth.uv_queries(n, seed=12)
    lod = synth.lods(n, seed=13, lo=-1.0, hi=8.0)
    ref = textures.Texture2D.box_pyramid(base.astype(np.float64), 7)
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    w = 0.6 if filt == "fis_gaussian" else 0.0
    out = T.lookup(to_dev(uv), to_dev(lod), taps=taps, filter=filt, seed=5, level_mode=level_mode, width=w)
    rv, rt, ex = filters.lookup_2d(ref, uv, lod, filt, stochastic_form=True, seed=5,
                                   level_mode=level_mode, width=w)
    torch.cuda.synchronize()
    # level choices within 1e-6 of a level boundary are exempt as for the other filters;
    # the library builds the pyramid in float32 (the oracle in float64), so texels of
    # levels above 0 agree to float32 rounding
    same = np.all(taps.cpu().numpy() == rt, axis=1)
    assert np.all(same | ex)
    err = np.abs(out.cpu().numpy().astype(np.float64) - rv)[same]
    assert np.all(err <= 2e-6 * np.abs(rv[same]))
    det = T.lookup_deterministic(to_dev(uv), to_dev(lod), filter=filt, level_mode=level_mode, width=w)
    dv, _, _ = filters.lookup_2d(ref, uv, lod, filt, stochastic_form=False, level_mode=level_mode, width=w)
    err = np.abs(det.cpu().numpy().astype(np.float64) - dv)
    lim = _gauss_tol(dv, w, 2, 1.0) if filt == "fis_gaussian" else 2e-6 * np.maximum(np.abs(dv), 1.0)
    assert np.all(err <= lim), np.max(err)


@pytest.mark.parametrize("filt", FIS)
def test_fis_deterministic_twins_tex2d(filt):
    """FIS linear / B-spline deterministic forms are the linear / B-spline filters
    (same kernel, bit for bit); the Gaussian twin matches the oracle's window sum."""
    tex, uv = _c1(8192)
    T = stf.Texture(stf.KIND_TEX2D, tex, dims=(256, 256, 1), channels=4)
    d = to_dev(uv)
    out = T.lookup_deterministic(d, filter=filt, width=WIDTH[filt])
    torch.cuda.synchronize()
    if filt != "fis_gaussian":
        twin = T.lookup_deterministic(d, filter=fis.FIS_TWIN[filt])
        assert torch.equal(out, twin)
        return
    ref = textures.Texture2D([tex.astype(np.float64)])
    rv, _, _ = filters.lookup_2d(ref, uv, None, filt, stochastic_form=False, width=WIDTH[filt])
    err = np.abs(out.cpu().numpy().astype(np.float64) - rv)
    assert np.all(err <= _gauss_tol(rv, WIDTH[filt], 2, float(np.max(tex)))), np.max(err)


@pytest.mark.parametrize("fmt", [stf.FMT_F32, stf.FMT_F16])
@pytest.mark.parametrize("filt", FIS)
def test_fis_dense(filt, fmt):
    n = 48
    vals = synth.dense_density(n=n, seed=3, period=12.0)
    pts = synth.uniform(3 * 30000, 4).reshape(-1, 3) * np.float32(n + 8) - np.float32(4)
    edge = np.array([[np.nan, 1, 1], [1, 1, -np.inf], [0, 0, 0], [n - 1, n - 1, n - 1],
                     [n - 0.5, 3.25, 7.75], [-1.5, 2, 2], [3e9, 1, 1], [-3e9, 5, 5]], dtype=np.float32)
    pts = np.concatenate([pts.astype(np.float32), edge])
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(n, n, n), fmt=fmt)
    ref = textures.Dense3D(quantise(vals, fmt))
    N = pts.shape[0]
    w = 0.9 if filt == "fis_gaussian" else 0.0
    taps = torch.empty((N, 4), dtype=torch.int32, device=dev())
    out = T.lookup(to_dev(pts), taps=taps, filter=filt, seed=123, sample_index=1, width=w)
    rv, rt, ex = filters.lookup_3d(ref, pts, filt, stochastic_form=True, seed=123, sample_index=1, width=w)
    torch.cuda.synchronize()
    _check_fis(filt, out.cpu().numpy(), taps.cpu().numpy(), rv, rt, ex)
    if filt == "fis_gaussian":
        sub = pts[:3000]
        det = T.lookup_deterministic(to_dev(sub), filter=filt, width=w)
        dv, _, _ = filters.lookup_3d(ref, sub, filt, stochastic_form=False, width=w)
        err = np.abs(det.cpu().numpy().astype(np.float64) - dv)
        assert np.all(err <= _gauss_tol(dv, w, 3, 1.0)), np.max(err)


@pytest.mark.parametrize("filt", FIS)
def test_fis_sparse(filt):
    origins, values = synth.sparse_cloud(domain=256, seed=4)
    T = stf.Texture(stf.KIND_SPARSE3D, values, fmt=stf.FMT_E4M3_SCALED, leaf_origins=origins)
    codes, scales = codecs.e4m3_leaf_quantise(values)
    ref = textures.Sparse3D(origins, codecs.e4m3_leaf_dequantise(codes, scales), 0.0)
    pts = (origins[np.arange(20000) % len(origins)]
           + synth.uniform(60000, 14).reshape(-1, 3) * np.float32(8)).astype(np.float32)
    pts = np.concatenate([pts, synth.uniform(3 * 5000, 15).reshape(-1, 3).astype(np.float32) * 272 - 8,
                          np.array([[np.nan, 1, 1], [-5000.0, -5000.0, 7.0]], dtype=np.float32)])
    N = pts.shape[0]
    w = 1.1 if filt == "fis_gaussian" else 0.0
    taps = torch.empty((N, 4), dtype=torch.int32, device=dev())
    out = T.lookup(to_dev(pts), taps=taps, filter=filt, seed=8, width=w)
    rv, rt, ex = filters.lookup_3d(ref, pts, filt, stochastic_form=True, seed=8, width=w)
    torch.cuda.synchronize()
    gv, gt = out.cpu().numpy().astype(np.float64), taps.cpu().numpy()
    same = np.all(gt == rt, axis=1)
    if filt != "fis_gaussian":
        assert not np.any(ex)
    assert np.all(same | ex)
    # E4M3 leaves: value = decoded code * float32 leaf scale, one float32 product
    assert np.all(np.abs(gv - rv)[same] <= 1e-7 * np.abs(rv[same]))
    if filt == "fis_gaussian":
        sub = pts[:1500]
        det = T.lookup_deterministic(to_dev(sub), filter=filt, width=w)
        dv, _, _ = filters.lookup_3d(ref, sub, filt, stochastic_form=False, width=w)
        err = np.abs(det.cpu().numpy().astype(np.float64) - dv)
        assert np.all(err <= _gauss_tol(dv, w, 3, float(np.max(values)))), np.max(err)
    stf.stf_synchronize(T.handle)


@pytest.mark.parametrize("filt", FIS)
def test_fis_unbiased_over_4096_samples(filt):
    """4096 samples per query: z-scores of the mean against the applied filter with
    the exact variance sum_i p_i t_i^2 - F^2 of the nearest-texel estimator."""
    tex, uv = _c1(16384)
    uv = uv[:16384]
    T = stf.Texture(stf.KIND_TEX2D, tex, dims=(256, 256, 1), channels=4)
    S = 4096
    s, _ = T.accumulate(to_dev(uv), S, filter=filt, seed=31, width=WIDTH[filt])
    mean = s.cpu().numpy() / S
    ref = textures.Texture2D([tex.astype(np.float64)])
    x = (uv[:, 0] * np.float32(256) - np.float32(0.5)).astype(np.float32)
    y = (uv[:, 1] * np.float32(256) - np.float32(0.5)).astype(np.float32)
    fetch = lambda ix, iy: ref.fetch(np.zeros_like(ix), ix, iy)
    fetch2 = lambda ix, iy: ref.fetch(np.zeros_like(ix), ix, iy) ** 2
    if filt == "fis_gaussian":
        F = fis.deterministic_gaussian(fetch, [x, y], WIDTH[filt])
        m2 = fis.deterministic_gaussian(fetch2, [x, y], WIDTH[filt])
    else:
        twin = fis.FIS_TWIN[filt]
        F = filters.expectation_by_enumeration(fetch, [x, y], twin)
        m2 = filters.expectation_by_enumeration(fetch, [x, y], twin, power=2)
    var = np.maximum(m2 - F * F, 0)
    for c in range(4):
        live = var[:, c] > 1e-18
        z = (mean[live, c] - F[live, c]) / np.sqrt(var[live, c] / S)
        assert np.mean(np.abs(z) > 3) <= 0.005, np.mean(np.abs(z) > 3)
        pooled = np.sum(mean[live, c] - F[live, c]) / np.sqrt(np.sum(var[live, c]) / S)
        assert abs(pooled) <= 3.0, pooled


@pytest.mark.parametrize("filt", FIS)
def test_fis_binned_equals_unbinned(filt):
    vals = synth.dense_density(n=64, seed=3, period=12.0)
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(64, 64, 64), fmt=stf.FMT_F16)
    q = to_dev(synth.camera_queries(W=160, H=90, steps=16, centre=(32, 32, 32), radius=96,
                                    half_span=56, seed=3))
    N = q.shape[0]
    t1 = torch.empty((N, 4), dtype=torch.int32, device=dev())
    t2 = torch.empty((N, 4), dtype=torch.int32, device=dev())
    a = T.lookup(q, taps=t1, filter=filt, seed=5, query_offset=17, width=WIDTH[filt])
    b = T.lookup(q, taps=t2, filter=filt, seed=5, query_offset=17, width=WIDTH[filt], bin_queries=True)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(t1, t2)


def test_fis_argument_checks():
    vals = synth.dense_density(n=8, seed=2, period=4.0)
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(8, 8, 8))
    d = to_dev(np.zeros((4, 3), dtype=np.float32))
    out = torch.empty((4, 1), device=dev())
    for w in (0.0, -1.0, float("nan"), stf.FIS_MAX_WIDTH * 1.01):
        with pytest.raises(stf.StfError) as e:
            stf.stf_lookup_batch(T.handle, stf.make_params("fis_gaussian", width=w), d, None, 4, out)
        assert e.value.status == 1
    stf.stf_lookup_batch(T.handle, stf.make_params("fis_gaussian", width=stf.FIS_MAX_WIDTH), d, None, 4, out)
    # the width is ignored by the other filters
    stf.stf_lookup_batch(T.handle, stf.make_params("fis_bspline3", width=-3.0), d, None, 4, out)
    torch.cuda.synchronize()


@pytest.mark.parametrize("filt,width", [("fis_linear", 0.0), ("fis_bspline3", 0.0), ("fis_gaussian", 1.0)])
def test_full_size_dense_fis_sampled(filt, width):
    """The benchmark's dense workload (256^3 FP16, 1920x1080 rays x 16 steps) with each
    FIS filter as the benchmark times it (Gaussian sigma = 1, no tap output), bit-equal
    to the call with tap output and checked on a seeded sample of outputs (2^20 for
    the B-spline, 2^18 for the others)."""
    vals = synth.dense_density(n=256, seed=3)
    q = synth.camera_queries(**synth.C2_RAYS)
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(256, 256, 256), fmt=stf.FMT_F16)
    N = q.shape[0]
    d = to_dev(q)
    fast = T.lookup(d, filter=filt, seed=2024, width=width)
    taps = torch.empty((N, 4), dtype=torch.int32, device=dev())
    out = T.lookup(d, taps=taps, filter=filt, seed=2024, width=width)
    torch.cuda.synchronize()
    torch.testing.assert_close(fast, out, rtol=0, atol=0)
    m = 1 << (20 if filt == "fis_bspline3" else 18)
    idx = np.sort(np.random.default_rng(1).choice(N, m, replace=False))
    ref = textures.Dense3D(quantise(vals, stf.FMT_F16))
    rv, rt, ex = filters.lookup_3d(ref, q[idx], filt, stochastic_form=True, seed=2024,
                                   qid=idx.astype(np.uint64), width=width or None)
    _check_fis(filt, out.cpu().numpy()[idx], taps.cpu().numpy()[idx], rv, rt, ex)


def test_fis_ignores_reuse_flag():
    """reuse_xi has no meaning for FIS (and positivization): results are the same."""
    vals = synth.dense_density(n=32, seed=3, period=8.0)
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(32, 32, 32), fmt=stf.FMT_F16)
    q = to_dev(synth.uniform(3 * 20000, 9).reshape(-1, 3) * np.float32(30))
    for filt in ("fis_linear", "fis_bspline3", "fis_gaussian", "catmull_rom_positivized"):
        w = 0.7 if filt == "fis_gaussian" else 0.0
        a = T.lookup(q, filter=filt, seed=4, width=w)
        b = T.lookup(q, filter=filt, seed=4, width=w, reuse_xi=True)
        torch.cuda.synchronize()
        assert torch.equal(a, b), filt
