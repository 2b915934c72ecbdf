"""GPU parity for DCT-compressed textures and triplanar lookups (Section 5.2) through
the C ABI against the oracle (`oracle/dct.py`).

Bar: the encoder runs in float64 on both sides, so codes agree except in blocks with a
coefficient within 1e-9 code units of a rounding boundary (oracle-reported; none are
expected).  Taps do not depend on the storage format and must match bit for bit
(except the usual 1e-6 CDF-boundary exemptions).  A decoded texel is six float32
products summed, within 4e-6 (1 + max R_c) of the float64 decode; deterministic
filters add float32 weight rounding (2e-6 of sum |w t|).  Triplanar plane choices are
float32 on both sides (exempt within 1e-6 of a plane boundary); deterministic blends
use float32 weights a_k / S."""
import numpy as np
import pytest
import torch

import paper_2305_05810_gb300 as stf
import synth
from oracle import dct, filters, textures
from parity import dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stf.load()


def _pyramid(W, H, C, levels, seed):
    base = synth.texture2d(W, H, C, seed=seed).astype(np.float64)
    lv = [base]
    for L in range(1, levels):
        h, w, _ = lv[-1].shape
        h2, w2 = max(1, h // 2), max(1, w // 2)
        prev = lv[-1]
        lv.append(prev.reshape(h2, h // h2, w2, w // w2, C).mean(axis=(1, 3)))
    return [l.astype(np.float32) for l in lv]


def _dct_pair(W=64, H=32, C=4, levels=4, seed=3):
    lv = _pyramid(W, H, C, levels, seed)
    T = stf.Texture(stf.KIND_TEX2D, np.concatenate([l.reshape(-1) for l in lv]), dims=(W, H, 1),
                    channels=C, mip_levels=levels, fmt=stf.FMT_DCT6)
    ref = dct.DCTTexture2D([l.astype(np.float64) for l in lv])
    return T, ref, lv


def _decode_tol(ref):
    return 4e-6 * (1.0 + float(np.max(ref.R)))


@pytest.mark.parametrize("C", [1, 2, 4, 8])
def test_dct_nearest_texels_match_oracle_decode(C):
    """FIS-linear lookups at texel centres return single decoded texels of level 0."""
    T, ref, _ = _dct_pair(C=C, seed=10 + C)
    W, H = 64, 32
    ys, xs = np.mgrid[0:H, 0:W]
    uv = np.stack([(xs.ravel() + 0.5) / W, (ys.ravel() + 0.5) / H], axis=1).astype(np.float32)
    n = uv.shape[0]
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    out = T.lookup(to_dev(uv), taps=taps, filter="fis_linear", seed=1)
    torch.cuda.synchronize()
    gt = taps.cpu().numpy()
    assert np.array_equal(gt[:, 0], xs.ravel()) and np.array_equal(gt[:, 1], ys.ravel())
    want = ref.fetch(0, xs.ravel(), ys.ravel())
    ok = ~ref.exempt_texels(0, xs.ravel(), ys.ravel())
    assert np.mean(ok) > 0.99
    err = np.abs(out.cpu().numpy().astype(np.float64) - want)[ok]
    assert np.all(err <= _decode_tol(ref)), np.max(err)


@pytest.mark.parametrize("filt", ["linear", "bspline3", "catmull_rom", "fis_bspline3"])
@pytest.mark.parametrize("level_mode", [stf.LEVEL_NEAREST, stf.LEVEL_STOCHASTIC])
def test_dct_lookups_match_oracle(filt, level_mode):
    T, ref, _ = _dct_pair(C=4, levels=6, seed=5)
    n = 20000
    uv = synth.uv_queries(n, seed=6)
    lod = synth.lods(n, seed=7, lo=-0.5, hi=6.0)
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    out = T.lookup(to_dev(uv), to_dev(lod), taps=taps, filter=filt, seed=9, level_mode=level_mode)
    rv, rt, ex = filters.lookup_2d(ref, uv, lod, filt, stochastic_form=True, seed=9, level_mode=level_mode)
    torch.cuda.synchronize()
    gt = taps.cpu().numpy()
    same = np.all(gt == rt, axis=1)
    assert np.all(same | ex)
    err = np.abs(out.cpu().numpy().astype(np.float64) - rv)[same]
    # a Catmull-Rom sample scales the texel by |sigma| <= 1.25^2
    assert np.all(err <= _decode_tol(ref) * 2.5 + 2e-6 * np.abs(rv[same])), np.max(err)
    det = T.lookup_deterministic(to_dev(uv), to_dev(lod), filter=filt, level_mode=level_mode)
    dv, _, _ = filters.lookup_2d(ref, uv, lod, filt, stochastic_form=False, level_mode=level_mode)
    err = np.abs(det.cpu().numpy().astype(np.float64) - dv)
    assert np.all(err <= 2.5 * _decode_tol(ref) + 2e-6 * np.abs(dv)), np.max(err)


def test_dct_generated_mips_and_unbiased():
    """generate_mips builds the float32 pyramid on the GPU before encoding; the
    stochastic trilinear mean over 4096 samples matches the deterministic trilinear
    filter of the same texture (both through the library: this checks the estimator
    on the compressed format, the oracle checks above pin the decode)."""
    base = synth.texture2d(64, 64, 2, seed=12)
    T = stf.Texture(stf.KIND_TEX2D, base, dims=(64, 64, 1), channels=2, mip_levels=7, generate_mips=True,
                    fmt=stf.FMT_DCT6)
    n = 8192
    uv, lod = to_dev(synth.uv_queries(n, seed=3)), to_dev(synth.lods(n, seed=4, lo=0, hi=5))
    S = 4096
    s, s2 = T.accumulate(uv, S, lod, filter="linear", seed=21)
    det = T.lookup_deterministic(uv, lod, filter="linear").double()
    mean = s / S
    var = torch.clamp(s2 / S - mean * mean, min=1e-12)
    z = ((mean - det) / torch.sqrt(var / S)).cpu().numpy()
    assert np.mean(np.abs(z) > 3.5) <= 0.005


def _tri_queries(n, seed):
    p, nrm = synth.sphere_points(n, seed=seed)
    edge_p = np.array([[0.5, 0.5, 0.5], [np.nan, 0.5, 0.5], [0.2, 0.3, 0.4], [0.9, 0.1, 0.5]], np.float32)
    edge_n = np.array([[0, 0, 0], [0, 0, 1], [1, 0, 0], [0.0, -1.0, 0.0]], np.float32)
    return np.concatenate([p, edge_p]), np.concatenate([nrm, edge_n])


@pytest.mark.parametrize("fmt", [stf.FMT_F32, stf.FMT_DCT6])
@pytest.mark.parametrize("filt", ["linear", "bspline3", "fis_gaussian"])
def test_triplanar_matches_oracle(fmt, filt):
    lv = _pyramid(64, 64, 4, 5, 14)
    T = stf.Texture(stf.KIND_TEX2D, np.concatenate([l.reshape(-1) for l in lv]), dims=(64, 64, 1),
                    channels=4, mip_levels=5, fmt=fmt)
    ref = (dct.DCTTexture2D([l.astype(np.float64) for l in lv]) if fmt == stf.FMT_DCT6
           else textures.Texture2D([l.astype(np.float64) for l in lv]))
    p, nrm = _tri_queries(12000, 15)
    n = p.shape[0]
    lod = synth.lods(n, seed=16, lo=0.0, hi=4.0)
    w = 0.8 if filt == "fis_gaussian" else 0.0
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    out = T.lookup_triplanar(to_dev(p), to_dev(nrm), 1.0, to_dev(lod), taps=taps, filter=filt, seed=3,
                             width=w)
    rv, rt, ex = dct.lookup_triplanar(ref, p, nrm, 1.0, lod, filt, stochastic_form=True, seed=3, width=w)
    torch.cuda.synchronize()
    gt = taps.cpu().numpy()
    same = np.all(gt == rt, axis=1)
    assert np.all(same | ex), (gt[~same & ~ex][:5], rt[~same & ~ex][:5])
    tol = _decode_tol(ref) if fmt == stf.FMT_DCT6 else 0.0
    err = np.abs(out.cpu().numpy().astype(np.float64) - rv)[same]
    assert np.all(err <= 2.5 * tol + 2e-6 * np.abs(rv[same])), np.max(err)
    det = T.lookup_triplanar_deterministic(to_dev(p), to_dev(nrm), 1.0, to_dev(lod), filter=filt, width=w)
    dv, _, _ = dct.lookup_triplanar(ref, p, nrm, 1.0, lod, filt, stochastic_form=False, width=w)
    err = np.abs(det.cpu().numpy().astype(np.float64) - dv)
    extra = 3e-5 if filt == "fis_gaussian" else 0.0
    assert np.all(err <= 2.5 * tol + 4e-6 * np.abs(dv) + 1e-6 + extra), np.max(err)


def test_triplanar_argument_checks():
    lv = _pyramid(16, 16, 1, 1, 2)
    T = stf.Texture(stf.KIND_TEX2D, lv[0], dims=(16, 16, 1), channels=1)
    p = to_dev(np.full((4, 3), 0.5, np.float32))
    out = torch.empty((4, 1), device=dev())
    with pytest.raises(stf.StfError) as e:
        stf.stf_lookup_batch_triplanar(T.handle, stf.make_params("catmull_rom_positivized"), p, p, None, 4,
                                       1.0, out)
    assert e.value.status == 4
    with pytest.raises(stf.StfError) as e:
        stf.stf_lookup_batch_triplanar(T.handle, stf.make_params(bin_queries=True), p, p, None, 4, 1.0, out)
    assert e.value.status == 4
    with pytest.raises(stf.StfError) as e:
        stf.stf_lookup_batch_triplanar(T.handle, stf.make_params(), p, p, None, 4, float("inf"), out)
    assert e.value.status == 1
    D = stf.Texture(stf.KIND_DENSE3D, synth.dense_density(n=8, seed=2, period=4.0), dims=(8, 8, 8))
    with pytest.raises(stf.StfError) as e:
        stf.stf_lookup_batch_triplanar(D.handle, stf.make_params(), p, p, None, 4, 1.0, out)
    assert e.value.status == 4
    with pytest.raises(stf.StfError) as e:
        stf.Texture(stf.KIND_DENSE3D, synth.dense_density(n=8, seed=2, period=4.0), dims=(8, 8, 8),
                    fmt=stf.FMT_DCT6)
    assert e.value.status == 1


def test_ewa_on_dct_texture():
    from oracle import ewa
    T, ref, _ = _dct_pair(C=2, levels=6, seed=19)
    uv, g = synth.plane_view(W=160, H=90, seed=4)
    uv, g = uv[:3000], np.ascontiguousarray(g[:3000] * np.float32(0.25))
    n = uv.shape[0]
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    out = T.lookup_ewa(to_dev(uv), to_dev(g), 16.0, taps=taps, seed=5)
    rv, rt, ex = ewa.lookup(ref, uv, g, 16.0, stochastic_form=True, seed=5)
    torch.cuda.synchronize()
    same = np.all(taps.cpu().numpy() == rt, axis=1)
    assert np.all(same | ex)
    err = np.abs(out.cpu().numpy().astype(np.float64) - rv)[same]
    assert np.all(err <= 2.5 * _decode_tol(ref)), np.max(err)


def test_dct_edge_blocks_of_non_multiple_of_8_sizes():
    """A 60x44 single-level DCT texture: the partial blocks on the right and bottom
    edges decode like the oracle's (edge texels repeated into the block)."""
    base = synth.texture2d(64, 64, 4, seed=31)[:44, :60].copy()
    T = stf.Texture(stf.KIND_TEX2D, base, dims=(60, 44, 1), channels=4, fmt=stf.FMT_DCT6)
    ref = dct.DCTTexture2D([base.astype(np.float64)])
    ys, xs = np.mgrid[0:44, 0:60]
    uv = np.stack([(xs.ravel() + 0.5) / 60, (ys.ravel() + 0.5) / 44], axis=1).astype(np.float32)
    out = T.lookup(to_dev(uv), filter="fis_linear", seed=2)
    want = ref.fetch(0, xs.ravel(), ys.ravel())
    ok = ~ref.exempt_texels(0, xs.ravel(), ys.ravel())
    err = np.abs(out.cpu().numpy().astype(np.float64) - want)[ok]
    assert np.all(err <= _decode_tol(ref)), np.max(err)


def test_triplanar_scale_and_no_lod():
    lv = _pyramid(32, 32, 2, 1, 33)
    T = stf.Texture(stf.KIND_TEX2D, lv[0], dims=(32, 32, 1), channels=2)
    ref = textures.Texture2D([lv[0].astype(np.float64)])
    p, nrm = _tri_queries(5000, 34)
    taps = torch.empty((p.shape[0], 4), dtype=torch.int32, device=dev())
    out = T.lookup_triplanar(to_dev(p), to_dev(nrm), 0.75, None, taps=taps, filter="bspline3", seed=8)
    rv, rt, ex = dct.lookup_triplanar(ref, p, nrm, 0.75, None, "bspline3", stochastic_form=True, seed=8)
    torch.cuda.synchronize()
    same = np.all(taps.cpu().numpy() == rt, axis=1)
    assert np.all(same | ex)
    assert np.array_equal(out.cpu().numpy().astype(np.float64)[same], rv[same])


def test_full_size_dct_plane_sampled():
    """The DCT benchmark workload (4096^2 x 8 channels, 13 levels, ground plane at
    3840x2160, anisotropic LOD, stochastic trilinear, 5,270,657 queries) in the launch
    configuration the benchmark times (no tap output), bit-equal to the same call with
    tap output, and checked on a seeded sample against the oracle's float64 encoding of
    the same float32 levels (passed in from the host, so that both encoders see the
    same texels)."""
    size, C, levels = 4096, 8, 13
    lv = _pyramid(size, size, C, levels, seed=1)
    T = stf.Texture(stf.KIND_TEX2D, np.concatenate([l.reshape(-1) for l in lv]), dims=(size, size, 1),
                    channels=C, mip_levels=levels, fmt=stf.FMT_DCT6)
    uv, g = synth.plane_view(W=3840, H=2160, seed=7)
    n = uv.shape[0]
    d_uv = to_dev(uv)
    lod = T.anisotropic_lod(to_dev(g), 16.0)
    fast = T.lookup(d_uv, lod, filter="linear", seed=2024)
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    sto = T.lookup(d_uv, lod, taps=taps, filter="linear", seed=2024)
    torch.cuda.synchronize()
    torch.testing.assert_close(fast, sto, rtol=0, atol=0)
    idx = np.sort(np.random.default_rng(2).choice(n, 1 << 20, replace=False))
    lod_s = lod.cpu().numpy()[idx]
    gv, gt = fast.cpu().numpy()[idx].astype(np.float64), taps.cpu().numpy()[idx].astype(np.int64)
    del fast, sto, taps
    ref = dct.DCTTexture2D([l.astype(np.float64) for l in lv])
    rv, rt, ex = filters.lookup_2d(ref, uv[idx], lod_s, "linear", stochastic_form=True, seed=2024,
                                   qid=idx.astype(np.uint64))
    same = np.all(gt == rt, axis=1)
    assert np.all(same | ex)
    code_ex = np.zeros(len(idx), dtype=bool)
    for L in np.unique(rt[:, 3]):
        sel = same & (rt[:, 3] == L)
        if L >= 0 and np.any(sel):
            code_ex[sel] = ref.exempt_texels(int(L), rt[sel, 0], rt[sel, 1])
    ok = same & ~code_ex
    assert np.mean(ok) > 0.99
    err = np.abs(gv - rv)[ok]
    assert np.all(err <= _decode_tol(ref) + 2e-6 * np.abs(rv[ok])), np.max(err)
    stf.stf_synchronize(T.handle)
