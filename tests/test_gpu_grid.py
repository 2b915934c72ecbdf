"""GPU parity: 2D textures and dense 3D grids through the C ABI vs the float64 oracle."""
import numpy as np
import pytest
import torch

import paper_2305_05810_gb300 as stf
import synth
from oracle import filters, textures
from parity import (abs_weighted_sum, check_deterministic, check_stochastic, dev,
                    positivized_moments, positivized_scale, quantise, to_dev)

pytestmark = pytest.mark.gpu
FILTERS = ["linear", "bspline3", "catmull_rom"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stf.load()


def _edge_uv():
    return np.array([[np.nan, 0.5], [0.5, np.inf], [-0.25, 0.5], [1.3, -2.0], [0.5, 0.5],
                     [0.5 / 256, 0.5 / 256], [1.0, 1.0], [0.0, 0.0], [1e30, -1e30],
                     [255.5 / 256, 3.5 / 256]], dtype=np.float32)


def _c1():
    tex = synth.texture2d(256, 256, 4, seed=1)
    uv = np.concatenate([synth.uv_queries(65536, seed=2), _edge_uv()])   # ragged tail
    return tex, uv


@pytest.mark.parametrize("filt", FILTERS)
def test_tex2d_c1_stochastic_matches_oracle(filt):
    tex, uv = _c1()
    T = stf.Texture(stf.KIND_TEX2D, tex, dims=(256, 256, 1), channels=4)
    n = uv.shape[0]
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    out = T.lookup(to_dev(uv), taps=taps, filter=filt, seed=77, sample_index=3)
    ref = textures.Texture2D([tex.astype(np.float64)])
    rv, rt, ex = filters.lookup_2d(ref, uv, None, filt, stochastic_form=True, seed=77, sample_index=3)
    torch.cuda.synchronize()
    check_stochastic(out.cpu().numpy(), taps.cpu().numpy(), rv, rt, ex)
    stf.stf_synchronize(T.handle)


@pytest.mark.parametrize("filt", FILTERS)
def test_tex2d_c1_deterministic_matches_oracle(filt):
    tex, uv = _c1()
    T = stf.Texture(stf.KIND_TEX2D, tex, dims=(256, 256, 1), channels=4)
    out = T.lookup_deterministic(to_dev(uv), filter=filt)
    ref = textures.Texture2D([tex.astype(np.float64)])
    rv, _, _ = filters.lookup_2d(ref, uv, None, filt, stochastic_form=False)
    x = (uv[:, 0] * np.float32(256) - np.float32(0.5)).astype(np.float32)
    y = (uv[:, 1] * np.float32(256) - np.float32(0.5)).astype(np.float32)
    scale = abs_weighted_sum(lambda ix, iy: ref.fetch(np.zeros_like(ix), ix, iy), [x, y], filt)
    check_deterministic(out.cpu().numpy(), rv, np.nan_to_num(scale))


@pytest.mark.parametrize("level_mode", [stf.LEVEL_NEAREST, stf.LEVEL_STOCHASTIC])
@pytest.mark.parametrize("filt", FILTERS)
def test_tex2d_mip_levels(level_mode, filt):
    base = synth.texture2d(64, 32, 2, seed=11)
    T = stf.Texture(stf.KIND_TEX2D, base, dims=(64, 32, 1), channels=2, mip_levels=7,
                    generate_mips=True)
    n = 20000
    uv = synth.uv_queries(n, seed=12)
    lod = synth.lods(n, seed=13, lo=-1.0, hi=8.0)
    lod[:4] = [np.nan, 0.0, 6.0, 2.0]
    ref = textures.Texture2D.box_pyramid(base.astype(np.float64), 7)
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    out = T.lookup(to_dev(uv), to_dev(lod), taps=taps, filter=filt, seed=5, level_mode=level_mode)
    rv, rt, ex = filters.lookup_2d(ref, uv, lod, filt, stochastic_form=True, seed=5,
                                   level_mode=level_mode)
    torch.cuda.synchronize()
    check_stochastic(out.cpu().numpy(), taps.cpu().numpy(), rv, rt, ex)
    det = T.lookup_deterministic(to_dev(uv), to_dev(lod), filter=filt, level_mode=level_mode)
    dv, _, _ = filters.lookup_2d(ref, uv, lod, filt, stochastic_form=False, level_mode=level_mode)
    # float32 box averaging of the pyramid adds ~1e-7 relative per level; the
    # tolerance scale is the largest texel magnitude reached by the filter.
    check_deterministic(det.cpu().numpy(), dv, 1.5 * np.max(np.abs(base)))


@pytest.mark.parametrize("channels", [1, 2, 4, 8])
def test_tex2d_f16_channels(channels):
    img = synth.texture2d(40, 24, channels, seed=21)      # non-power-of-two, ragged
    T = stf.Texture(stf.KIND_TEX2D, img, dims=(40, 24, 1), channels=channels, fmt=stf.FMT_F16)
    uv = synth.uv_queries(5001, seed=22)
    ref = textures.Texture2D([quantise(img, stf.FMT_F16)])
    taps = torch.empty((5001, 4), dtype=torch.int32, device=dev())
    out = T.lookup(to_dev(uv), taps=taps, filter="catmull_rom", seed=3)
    rv, rt, ex = filters.lookup_2d(ref, uv, None, "catmull_rom", stochastic_form=True, seed=3)
    torch.cuda.synchronize()
    check_stochastic(out.cpu().numpy(), taps.cpu().numpy(), rv, rt, ex)
    det = T.lookup_deterministic(to_dev(uv), filter="bspline3")
    dv, _, _ = filters.lookup_2d(ref, uv, None, "bspline3", stochastic_form=False)
    check_deterministic(det.cpu().numpy(), dv, 0.0)


@pytest.mark.parametrize("filt", FILTERS)
def test_tex2d_reused_variate(filt):
    tex, uv = _c1()
    T = stf.Texture(stf.KIND_TEX2D, tex, dims=(256, 256, 1), channels=4)
    n = uv.shape[0]
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    out = T.lookup(to_dev(uv), taps=taps, filter=filt, seed=8, reuse_xi=True)
    ref = textures.Texture2D([tex.astype(np.float64)])
    rv, rt, ex = filters.lookup_2d(ref, uv, None, filt, stochastic_form=True, seed=8, reuse=True)
    torch.cuda.synchronize()
    check_stochastic(out.cpu().numpy(), taps.cpu().numpy(), rv, rt, ex)


def _dense(n=64, seed=3):
    vals = synth.dense_density(n=n, seed=seed, period=12.0)
    pts = synth.uniform(3 * 40000, seed + 1).reshape(-1, 3) * np.float32(n + 8) - np.float32(4)
    edge = np.array([[np.nan, 1, 1], [1, 1, -np.inf], [0, 0, 0], [n - 1, n - 1, n - 1],
                     [n - 0.5, 3.25, 7.75], [-1.5, 2, 2], [3e9, 1, 1]], dtype=np.float32)
    return vals, np.concatenate([pts.astype(np.float32), edge])


@pytest.mark.parametrize("fmt", [stf.FMT_F32, stf.FMT_F16])
@pytest.mark.parametrize("filt", FILTERS)
def test_dense_stochastic_and_deterministic(filt, fmt):
    vals, pts = _dense()
    n = vals.shape[0]
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(n, n, n), fmt=fmt)
    ref = textures.Dense3D(quantise(vals, fmt))
    N = pts.shape[0]
    taps = torch.empty((N, 4), dtype=torch.int32, device=dev())
    out = T.lookup(to_dev(pts), taps=taps, filter=filt, seed=123, sample_index=1)
    rv, rt, ex = filters.lookup_3d(ref, pts, filt, stochastic_form=True, seed=123, sample_index=1)
    torch.cuda.synchronize()
    check_stochastic(out.cpu().numpy(), taps.cpu().numpy(), rv, rt, ex)
    det = T.lookup_deterministic(to_dev(pts), filter=filt)
    dv, _, _ = filters.lookup_3d(ref, pts, filt, stochastic_form=False)
    scale = abs_weighted_sum(ref.fetch, [pts[:, 0], pts[:, 1], pts[:, 2]], filt)
    check_deterministic(det.cpu().numpy(), dv, np.nan_to_num(scale))


@pytest.mark.parametrize("filt", FILTERS)
def test_dense_reused_variate(filt):
    vals, pts = _dense(32, seed=7)
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(32, 32, 32), fmt=stf.FMT_F16)
    ref = textures.Dense3D(quantise(vals, stf.FMT_F16))
    N = pts.shape[0]
    taps = torch.empty((N, 4), dtype=torch.int32, device=dev())
    out = T.lookup(to_dev(pts), taps=taps, filter=filt, seed=9, reuse_xi=True)
    rv, rt, ex = filters.lookup_3d(ref, pts, filt, stochastic_form=True, seed=9, reuse=True)
    torch.cuda.synchronize()
    check_stochastic(out.cpu().numpy(), taps.cpu().numpy(), rv, rt, ex)


def test_empty_single_and_chunked_calls():
    vals, pts = _dense(16, seed=4)
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(16, 16, 16), fmt=stf.FMT_F32)
    d = to_dev(pts)
    out = torch.full((pts.shape[0], 1), -7.0, device=dev())
    stf.stf_lookup_batch(T.handle, stf.make_params(), d, None, 0, out)   # no-op
    torch.cuda.synchronize()
    assert torch.all(out == -7.0)
    whole = T.lookup(d, filter="bspline3", seed=4)
    parts = torch.empty_like(whole)
    cuts = [0, 1, 257, 10000, pts.shape[0]]
    for a, b in zip(cuts[:-1], cuts[1:]):
        p = stf.make_params("bspline3", seed=4, query_offset=a)
        stf.stf_lookup_batch(T.handle, p, d[a:], None, b - a, parts[a:])
    torch.cuda.synchronize()
    assert torch.equal(whole, parts)


def test_invalid_arguments_on_gpu():
    vals, pts = _dense(8, seed=2)
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(8, 8, 8))
    d = to_dev(pts)
    out = torch.empty((pts.shape[0], 1), device=dev())
    with pytest.raises(stf.StfError) as e:
        stf.stf_lookup_batch(T.handle, stf.make_params(filter=7), d, None, 10, out)
    assert e.value.status == 1
    with pytest.raises(stf.StfError) as e:
        stf.stf_lookup_batch(T.handle, stf.make_params(), d, d, 10, out)   # lod on a 3D grid
    assert e.value.status == 4
    stf.load().stf_debug_fail_allocation(1)
    with pytest.raises(stf.StfError) as e:
        stf.Texture(stf.KIND_DENSE3D, vals, dims=(8, 8, 8))
    assert e.value.status == 3
    stf.load().stf_debug_fail_allocation(0)
    h = T.handle
    T.close()
    with pytest.raises(stf.StfError) as e:
        stf.stf_lookup_batch(h, stf.make_params(), d, None, 10, out)
    assert e.value.status == 2


@pytest.mark.parametrize("filt", ["linear", "bspline3", "catmull_rom"])
def test_unbiased_over_4096_samples_c1(filt):
    """4096 samples per query, float64 accumulators on the GPU; z-scores against the
    oracle's deterministic filter with the estimator's exact variance (enumerated
    second moment).  Per query the |z| > 3 rate must stay <= 0.5% (0.27% expected);
    the pooled z over all queries must stay within +-3."""
    tex, uv = _c1()
    uv = uv[:65536]
    T = stf.Texture(stf.KIND_TEX2D, tex, dims=(256, 256, 1), channels=4)
    S = 4096
    s, _ = T.accumulate(to_dev(uv), S, filter=filt, seed=31)
    mean = s.cpu().numpy() / S
    ref = textures.Texture2D([tex.astype(np.float64)])
    x = (uv[:, 0] * np.float32(256) - np.float32(0.5)).astype(np.float32)
    y = (uv[:, 1] * np.float32(256) - np.float32(0.5)).astype(np.float32)
    fetch = lambda ix, iy: ref.fetch(np.zeros_like(ix), ix, iy)
    F = filters.expectation_by_enumeration(fetch, [x, y], filt)
    var = np.maximum(filters.expectation_by_enumeration(fetch, [x, y], filt, power=2) - F * F, 0)
    for c in range(4):
        live = var[:, c] > 1e-18
        assert np.all(np.abs(mean[~live, c] - F[~live, c]) <= 1e-6 * (np.abs(F[~live, c]) + 1e-3))
        z = (mean[live, c] - F[live, c]) / np.sqrt(var[live, c] / S)
        assert np.mean(np.abs(z) > 3) <= 0.005, np.mean(np.abs(z) > 3)
        pooled = np.sum(mean[live, c] - F[live, c]) / np.sqrt(np.sum(var[live, c]) / S)
        print("%s channel %d: |z| > 3 rate %.4f, pooled %.3f" % (filt, c, np.mean(np.abs(z) > 3), pooled))
        assert abs(pooled) <= 3.0, pooled


def test_full_size_dense_ray_march_sampled():
    """The benchmark's workload (256^3 FP16, 1920x1080 rays x 16 steps) in the launch
    configuration the benchmark times (no tap output: the 32-bit-index loop), bit-equal
    to the same call with tap output; outputs checked on a seeded sample."""
    vals = synth.dense_density(n=256, seed=3)
    q = synth.camera_queries(**synth.C2_RAYS)
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(256, 256, 256), fmt=stf.FMT_F16)
    d = to_dev(q)
    N = q.shape[0]
    fast = T.lookup(d, filter="bspline3", seed=2024)
    taps = torch.empty((N, 4), dtype=torch.int32, device=dev())
    sto = T.lookup(d, taps=taps, filter="bspline3", seed=2024)
    torch.cuda.synchronize()
    torch.testing.assert_close(fast, sto, rtol=0, atol=0)
    del fast
    det = T.lookup_deterministic(d, filter="bspline3")
    idx = np.sort(np.random.default_rng(0).choice(N, 1 << 20, replace=False))
    ref = textures.Dense3D(quantise(vals, stf.FMT_F16))
    rv, rt, ex = filters.lookup_3d(ref, q[idx], "bspline3", stochastic_form=True, seed=2024,
                                   qid=idx.astype(np.uint64))
    check_stochastic(sto.cpu().numpy()[idx], taps.cpu().numpy()[idx], rv, rt, ex)
    dv, _, _ = filters.lookup_3d(ref, q[idx], "bspline3", stochastic_form=False)
    check_deterministic(det.cpu().numpy()[idx], dv, 0.0)
    stf.stf_synchronize(T.handle)


def test_full_size_tex2d_sampled():
    """The 2D benchmark workload (256^2 RGBA FP32, 16,777,216 uniform uv, B-spline
    bicubic) in the launch configuration the benchmark times (no tap output), bit-equal
    to the same call with tap output, and checked on a seeded sample against the
    oracle."""
    tex = synth.texture2d(256, 256, 4, seed=1)
    T = stf.Texture(stf.KIND_TEX2D, tex, dims=(256, 256, 1), channels=4)
    n = 1 << 24
    uv = synth.uv_queries(n, seed=2)
    d = to_dev(uv)
    fast = T.lookup(d, filter="bspline3", seed=2024)
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    sto = T.lookup(d, taps=taps, filter="bspline3", seed=2024)
    torch.cuda.synchronize()
    torch.testing.assert_close(fast, sto, rtol=0, atol=0)
    idx = np.sort(np.random.default_rng(1).choice(n, 1 << 20, replace=False))
    ref = textures.Texture2D([tex.astype(np.float64)])
    rv, rt, ex = filters.lookup_2d(ref, uv[idx], None, "bspline3", stochastic_form=True, seed=2024,
                                   qid=idx.astype(np.uint64))
    check_stochastic(fast.cpu().numpy()[idx], taps.cpu().numpy()[idx], rv, rt, ex)
    stf.stf_synchronize(T.handle)


@pytest.mark.parametrize("filt", ["linear", "catmull_rom", "catmull_rom_positivized"])
def test_full_size_dense_other_filters_sampled(filt):
    """The dense benchmark workload with the other filters the benchmark times
    (stochastic trilinear, one-tap Catmull-Rom, positivized Catmull-Rom), without tap
    output as timed, bit-equal to the call with tap output, and checked on a seeded
    sample of 2^18 queries against the oracle."""
    vals = synth.dense_density(n=256, seed=3)
    q = synth.camera_queries(**synth.C2_RAYS)
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(256, 256, 256), fmt=stf.FMT_F16)
    d = to_dev(q)
    N = q.shape[0]
    fast = T.lookup(d, filter=filt, seed=2024)
    taps = torch.empty((N, 4), dtype=torch.int32, device=dev())
    sto = T.lookup(d, taps=taps, filter=filt, seed=2024)
    torch.cuda.synchronize()
    torch.testing.assert_close(fast, sto, rtol=0, atol=0)
    idx = np.sort(np.random.default_rng(4).choice(N, 1 << 18, replace=False))
    ref = textures.Dense3D(quantise(vals, stf.FMT_F16))
    rv, rt, ex = filters.lookup_3d(ref, q[idx], filt, stochastic_form=True, seed=2024,
                                   qid=idx.astype(np.uint64))
    gv, gt = sto.cpu().numpy()[idx], taps.cpu().numpy()[idx]
    if filt == "catmull_rom_positivized":
        p = q[idx]
        _check_positivized(gv, gt, rv, rt, ex, positivized_scale([p[:, 0], p[:, 1], p[:, 2]],
                                                                 float(np.max(vals))))
    else:
        check_stochastic(gv, gt, rv, rt, ex)
    stf.stf_synchronize(T.handle)


def _check_positivized(gpu_val, gpu_taps, rv, rt, ex, scale):
    gpu_val = np.asarray(gpu_val, dtype=np.float64).reshape(rv.shape)
    same = np.all(np.asarray(gpu_taps).reshape(-1, 4) == rt, axis=1)
    assert np.all(same | ex), np.nonzero(~(same | ex))[0][:5]
    ok = same & ~ex
    err = np.abs(gpu_val - rv)[ok]
    lim = 2e-6 * (np.abs(rv[ok]) + scale[ok, None])
    assert np.all(err <= lim), np.max(err - lim)


def test_positivized_tex2d_matches_oracle():
    tex, uv = _c1()
    T = stf.Texture(stf.KIND_TEX2D, tex, dims=(256, 256, 1), channels=4)
    n = uv.shape[0]
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    out = T.lookup(to_dev(uv), taps=taps, filter="catmull_rom_positivized", seed=21)
    ref = textures.Texture2D([tex.astype(np.float64)])
    rv, rt, ex = filters.lookup_2d(ref, uv, None, "catmull_rom_positivized", stochastic_form=True, seed=21)
    torch.cuda.synchronize()
    x = (uv[:, 0] * np.float32(256) - np.float32(0.5)).astype(np.float32)
    y = (uv[:, 1] * np.float32(256) - np.float32(0.5)).astype(np.float32)
    _check_positivized(out.cpu().numpy(), taps.cpu().numpy(), rv, rt, ex,
                       positivized_scale([x, y], float(np.max(np.abs(tex)))))
    det = T.lookup_deterministic(to_dev(uv), filter="catmull_rom_positivized")
    det_cr = T.lookup_deterministic(to_dev(uv), filter="catmull_rom")
    assert torch.equal(det, det_cr)


@pytest.mark.parametrize("fmt", [stf.FMT_F32, stf.FMT_F16])
def test_positivized_dense_matches_oracle(fmt):
    vals, pts = _dense()
    n = vals.shape[0]
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(n, n, n), fmt=fmt)
    ref = textures.Dense3D(quantise(vals, fmt))
    N = pts.shape[0]
    taps = torch.empty((N, 4), dtype=torch.int32, device=dev())
    out = T.lookup(to_dev(pts), taps=taps, filter="catmull_rom_positivized", seed=5)
    rv, rt, ex = filters.lookup_3d(ref, pts, "catmull_rom_positivized", stochastic_form=True, seed=5)
    torch.cuda.synchronize()
    _check_positivized(out.cpu().numpy(), taps.cpu().numpy(), rv, rt, ex,
                       positivized_scale([pts[:, 0], pts[:, 1], pts[:, 2]], float(np.max(vals))))


def test_positivized_unbiased_and_lower_variance_c1():
    """4096 samples per query: z-scores of the positivized mean against the
    deterministic filter with its exact variance; its sample variance is below the
    one-tap estimator's on average."""
    tex, uv = _c1()
    uv = uv[:16384]
    T = stf.Texture(stf.KIND_TEX2D, tex, dims=(256, 256, 1), channels=4)
    S = 4096
    s, s2 = T.accumulate(to_dev(uv), S, filter="catmull_rom_positivized", seed=44)
    s_cr, s2_cr = T.accumulate(to_dev(uv), S, filter="catmull_rom", seed=44)
    s, s2, s_cr, s2_cr = s.cpu().numpy(), s2.cpu().numpy(), s_cr.cpu().numpy(), s2_cr.cpu().numpy()
    ref = textures.Texture2D([tex.astype(np.float64)])
    x = (uv[:, 0] * np.float32(256) - np.float32(0.5)).astype(np.float32)
    y = (uv[:, 1] * np.float32(256) - np.float32(0.5)).astype(np.float32)
    F, var = positivized_moments(lambda ix, iy: ref.fetch(np.zeros_like(ix), ix, iy), [x, y])
    mean = s / S
    for c in range(4):
        live = var[:, c] > 1e-18
        z = (mean[live, c] - F[live, c]) / np.sqrt(var[live, c] / S)
        assert np.mean(np.abs(z) > 3) <= 0.005
        pooled = np.sum(mean[live, c] - F[live, c]) / np.sqrt(np.sum(var[live, c]) / S)
        assert abs(pooled) <= 3.0, pooled
    v_pos = np.mean(s2 / S - (s / S) ** 2)
    v_cr = np.mean(s2_cr / S - (s_cr / S) ** 2)
    assert v_pos < v_cr


@pytest.mark.parametrize("offset,seed,sample", [((1 << 32) - 5000, 7, 0),
                                                ((1 << 64) - 5000, 0x123456789ABCDEF0, 3),
                                                (11, 2, (1 << 32) - 1)])
def test_counter_and_key_words(offset, seed, sample):
    """q = query_offset + i crosses into the counter's high word (and wraps at 2^64),
    the seed fills both key words and the sample index reaches 2^32 - 1: taps bit-exact
    against the oracle for 2D (with mip levels) and dense lookups; the call without tap
    output gives the same values."""
    n = 10000
    tex = synth.texture2d(64, 64, 2, seed=3)
    T2 = stf.Texture(stf.KIND_TEX2D, tex, dims=(64, 64, 1), channels=2, mip_levels=7, generate_mips=True)
    uv = synth.uv_queries(n, seed=4)
    lod = synth.lods(n, seed=5, lo=0, hi=6)
    vals, pts = _dense(n=32, seed=6)
    pts = pts[:n]
    T3 = stf.Texture(stf.KIND_DENSE3D, vals, dims=(32, 32, 32))
    qid = (np.arange(n, dtype=np.uint64) + np.uint64(offset % (1 << 64)))
    for T, x, l, ref_fn in (
            (T2, uv, lod, lambda: filters.lookup_2d(textures.Texture2D.box_pyramid(tex.astype(np.float64), 7),
                                                    uv, lod, "bspline3", stochastic_form=True, seed=seed,
                                                    qid=qid, sample_index=sample)),
            (T3, pts, None, lambda: filters.lookup_3d(textures.Dense3D(vals.astype(np.float64)), pts, "bspline3",
                                                      stochastic_form=True, seed=seed, qid=qid,
                                                      sample_index=sample))):
        taps = torch.empty((x.shape[0], 4), dtype=torch.int32, device=dev())
        dl = None if l is None else to_dev(l)
        out = T.lookup(to_dev(x), dl, taps=taps, filter="bspline3", seed=seed, query_offset=offset,
                       sample_index=sample)
        fast = T.lookup(to_dev(x), dl, filter="bspline3", seed=seed, query_offset=offset,
                        sample_index=sample)
        torch.cuda.synchronize()
        torch.testing.assert_close(fast, out, rtol=0, atol=0, equal_nan=True)
        rv, rt, ex = ref_fn()
        gt = taps.cpu().numpy().astype(np.int64)
        same = np.all(gt == rt, axis=1)
        assert np.all(same | ex)
        assert np.mean(same) > 0.99
        gv = out.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(gv - rv)[same] <= 2e-6 * np.abs(rv[same]) + 1e-30)


@pytest.mark.parametrize("filt", ["bspline3", "catmull_rom", "linear"])
def test_degenerate_sizes(filt):
    """One-texel and one-texel-wide 2D textures and 1^3 / 2x1x1 dense grids: every tap
    clamps to the edge (2D) or falls on the background outside the grid (3D); stochastic
    taps and values and deterministic values match the oracle."""
    rng = np.random.default_rng(8)
    uv = rng.uniform(-0.5, 1.5, (3000, 2)).astype(np.float32)
    for W, H in ((1, 1), (1, 16), (16, 1)):
        img = rng.uniform(0, 1, (H, W, 4)).astype(np.float32)
        T = stf.Texture(stf.KIND_TEX2D, img, dims=(W, H, 1), channels=4)
        ref = textures.Texture2D([img.astype(np.float64)])
        taps = torch.empty((uv.shape[0], 4), dtype=torch.int32, device=dev())
        out = T.lookup(to_dev(uv), taps=taps, filter=filt, seed=3)
        rv, rt, ex = filters.lookup_2d(ref, uv, None, filt, stochastic_form=True, seed=3)
        torch.cuda.synchronize()
        check_stochastic(out.cpu().numpy(), taps.cpu().numpy(), rv, rt, ex)
        det = T.lookup_deterministic(to_dev(uv), filter=filt)
        dv, _, _ = filters.lookup_2d(ref, uv, None, filt, stochastic_form=False)
        check_deterministic(det.cpu().numpy(), dv, 4.0)
    pts = rng.uniform(-2.5, 3.5, (3000, 3)).astype(np.float32)
    for dims in ((1, 1, 1), (2, 1, 1)):
        vals = rng.uniform(0.5, 1, dims[::-1]).astype(np.float32)
        T = stf.Texture(stf.KIND_DENSE3D, vals, dims=dims)
        ref = textures.Dense3D(vals.astype(np.float64))
        taps = torch.empty((pts.shape[0], 4), dtype=torch.int32, device=dev())
        out = T.lookup(to_dev(pts), taps=taps, filter=filt, seed=4)
        rv, rt, ex = filters.lookup_3d(ref, pts, filt, stochastic_form=True, seed=4)
        torch.cuda.synchronize()
        check_stochastic(out.cpu().numpy(), taps.cpu().numpy(), rv, rt, ex)
        det = T.lookup_deterministic(to_dev(pts), filter=filt)
        dv, _, _ = filters.lookup_3d(ref, pts, filt, stochastic_form=False)
        check_deterministic(det.cpu().numpy(), dv, 2.0)
