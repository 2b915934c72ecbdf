"""GPU parity for neural textures: tensor-core decode inside stochastic and
deterministic lookups, forward/backward gradients, and training.

Decode tolerance, from the arithmetic: binary16 operands (latents and weights are
stored in binary16, which the oracle uses too) multiply exactly into float32
accumulators; the only extra rounding is of the hidden activations H1 and H2 to
binary16 between layers (relative 2^-11 each).  An output therefore differs from
the float64 oracle by at most about 2^-11 * (sum_k |W3_kc H2_k| + sum_k |W3_kc|
sum_j |W2_jk H1_j|) plus float32 accumulation; the tests allow twice that plus
1e-6.  Gradients: binary16 activations and back-propagated errors give relative
errors of about 1e-3 on each gradient block; the tests allow 2e-2 of its norm.
"""
import numpy as np
import pytest
import torch

import paper_2305_05810_gb300 as stf
import synth
from oracle import codecs, filters, mlp, neural
from parity import check_stochastic, dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stf.load()


def h16(a):
    return codecs.f16_decode(codecs.f16_encode(np.asarray(a, dtype=np.float64)))


def stored_params(flat):
    """Parameters as the kernels use them: binary16 weights, float32 biases."""
    P = mlp.unflatten(np.asarray(flat, dtype=np.float64))
    for k in ("W1", "W2", "W3"):
        P[k] = h16(P[k])
    for k in ("b1", "b2", "b3"):
        P[k] = np.asarray(P[k], dtype=np.float32).astype(np.float64)
    return P


def split_levels(flat_rows, size, first, count, ch):
    out, o = [], 0
    for L in range(first, first + count):
        n = max(1, size >> L)
        out.append(np.asarray(flat_rows[o:o + n * n]).reshape(n, n, ch))
        o += n * n
    return out


def decode_bound(Z, P):
    """Per-output bound 2 * 2^-11 * (|W3| |H2| + |W3| |W2| |H1|) + 1e-6 (see module doc)."""
    _, (X, A1, H1, A2, H2) = mlp.forward(Z, P)
    s = np.abs(H2) @ np.abs(P["W3"]) + (np.abs(H1) @ np.abs(P["W2"])) @ np.abs(P["W3"])
    return 2.0 * 2.0 ** -11 * s + 1e-6


def make_neural(size=64, latent_levels=3, levels=6, seed=5):
    lat, par = synth.neural_init(size, latent_levels, seed=seed)
    tgt = synth.material(size, seed=seed)
    pyr = synth.box_levels(tgt, levels)
    fb = np.concatenate([p.reshape(-1, 7) for p in pyr[latent_levels:]]) if levels > latent_levels else None
    T = stf.NeuralTexture(size, size, latent_levels, levels, lat, par, fb)
    ref = neural.NeuralTexture2D(split_levels(h16(lat), size, 0, latent_levels, 8), stored_params(par),
                                 [h16(p) for p in pyr[latent_levels:]])
    return T, ref, lat, par, pyr


@pytest.mark.parametrize("level_mode", [stf.LEVEL_NEAREST, stf.LEVEL_STOCHASTIC])
@pytest.mark.parametrize("filt", ["linear", "bspline3", "catmull_rom"])
def test_neural_stochastic_decode_matches_oracle(filt, level_mode):
    T, ref, _, _, _ = make_neural()
    n = 20000
    uv = synth.uv_queries(n, seed=31)
    lod = synth.lods(n, seed=32, lo=-0.5, hi=6.5)
    lod[:3] = [np.nan, 5.9, 0.0]
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    out = T.lookup(to_dev(uv), to_dev(lod), taps=taps, filter=filt, seed=3, level_mode=level_mode)
    torch.cuda.synchronize()
    rv, rt, ex = filters.lookup_2d(ref, uv, lod, filt, stochastic_form=True, seed=3, level_mode=level_mode)
    g_taps = taps.cpu().numpy()
    g_out = out.cpu().numpy().astype(np.float64)
    same = np.all(g_taps == rt, axis=1)
    assert np.all(same | ex)
    # bound per query: decoded texels get the decode bound, fallback texels are exact
    lvl = rt[:, 3]
    bound = np.full(rv.shape, 1e-6)
    dec = same & (lvl >= 0) & (lvl < len(ref.latents))
    for L in np.unique(lvl[dec]):
        m = dec & (lvl == L)
        w, h = ref.size(L)
        Z = ref.latents[L][np.clip(rt[m, 1], 0, h - 1), np.clip(rt[m, 0], 0, w - 1)]
        D = ref.decode(Z)
        c = np.argmax(np.abs(D), axis=1)
        rows = np.arange(D.shape[0])
        sig = np.abs(rv[m][rows, c]) / np.maximum(np.abs(D[rows, c]), 1e-30)   # |sigma| (1 unless Catmull-Rom)
        bound[m] = decode_bound(Z, ref.P) * sig[:, None]
    err = np.abs(g_out - rv)
    assert np.all(err[same] <= bound[same] + 2e-6 * np.abs(rv[same])), np.max(err[same] - bound[same])


@pytest.mark.parametrize("level_mode", [stf.LEVEL_NEAREST, stf.LEVEL_STOCHASTIC])
@pytest.mark.parametrize("filt", ["linear", "bspline3"])
def test_neural_deterministic_decode_matches_oracle(filt, level_mode):
    T, ref, _, _, _ = make_neural()
    n = 4000
    uv = synth.uv_queries(n, seed=41)
    lod = synth.lods(n, seed=42, lo=0.0, hi=5.5)
    out = T.lookup_deterministic(to_dev(uv), to_dev(lod), filter=filt, level_mode=level_mode)
    rv, _, _ = filters.lookup_2d(ref, uv, lod, filt, stochastic_form=False, level_mode=level_mode)
    # bound: every decoded tap contributes at most its weight times the decode bound
    big = max(float(np.max(decode_bound(l.reshape(-1, 8), ref.P))) for l in ref.latents)
    err = np.abs(out.cpu().numpy() - rv)
    assert np.max(err) <= 2 * big + 1e-5, (np.max(err), big)


def test_neural_gradients_match_oracle():
    T, ref, lat, par, pyr = make_neural(size=32, latent_levels=3, levels=3)
    n_lat = lat.shape[0]
    B = 512
    ids = np.random.default_rng(3).choice(n_lat, B, replace=False).astype(np.int64)
    tgt = np.concatenate([p.reshape(-1, 7) for p in pyr[:3]])[ids]
    pg, lg, loss = T.gradients(to_dev(ids), to_dev(tgt.astype(np.float32)))
    P = stored_params(par)
    Z = h16(lat[ids])
    Y, cache = mlp.forward(Z, P)
    g = mlp.backward(cache, P, Y, tgt)
    assert abs(loss.item() - mlp.loss(Y, tgt)) <= 2e-3 * mlp.loss(Y, tgt)
    G = mlp.unflatten(pg.cpu().numpy())
    rels = {}
    for k in mlp.NAMES:
        rels[k] = np.linalg.norm(G[k] - g[k]) / max(np.linalg.norm(g[k]), 1e-12)
    rels["X"] = np.linalg.norm(lg.cpu().numpy() - g["X"]) / np.linalg.norm(g["X"])
    print("relative gradient errors (norm):", {k: "%.2e" % v for k, v in rels.items()})
    assert max(rels.values()) <= 1e-2, rels


def test_training_gains_over_untrained_decoder():
    """Trained on the target, the decoder's texels approach the target far more
    closely than the untrained network's; the neural deterministic lookup then also
    agrees with the stored texture's."""
    size, nlat = 64, 2
    T, ref, lat, par, pyr = make_neural(size=size, latent_levels=nlat, levels=nlat)
    target = to_dev(np.concatenate([p.reshape(-1, 7) for p in pyr[:nlat]]))
    n_lat = lat.shape[0]
    ids = torch.arange(n_lat, device=dev(), dtype=torch.int64)
    _, _, loss0 = T.gradients(ids, target)
    losses = T.train(target, steps=600, batch=1024, lr_latent=3e-2, lr_params=3e-3, seed=11)
    _, _, loss1 = T.gradients(ids, target)
    l0, l1 = loss0.item(), loss1.item()
    assert np.all(np.isfinite(losses.cpu().numpy()))
    assert l1 < 0.05 * l0, (l0, l1)
    # trained parameters read back and decoded by the oracle give the same loss
    p, z = T.read()
    P = stored_params(p.cpu().numpy())
    Y, _ = mlp.forward(h16(z.cpu().numpy()), P)
    assert abs(mlp.loss(Y, target.cpu().numpy()) - l1) <= 5e-2 * l1 + 1e-6
    # neural vs stored texture, deterministic bilinear at level 0
    stored = stf.Texture(stf.KIND_TEX2D, np.concatenate([pyr[0], np.zeros((size, size, 1), np.float32)], axis=2),
                         dims=(size, size, 1), channels=8)
    uv = to_dev(synth.uv_queries(8192, seed=5))
    a = T.lookup_deterministic(uv, filter="linear").cpu().numpy()
    b = stored.lookup_deterministic(uv, filter="linear").cpu().numpy()[:, :7]
    assert np.sqrt(np.mean((a - b) ** 2)) < 0.25 * np.sqrt(l0 / 7)


def test_full_size_neural_sampled():
    """The benchmark's neural workload (4096^2, four 8-channel FP16 latent levels, FP16
    fallback mips, 16,777,216 uv with lod ~ U[0, 4), nearest level, bilinear tap) in the
    benchmark's launch configuration, with the untrained decoder; outputs checked on a
    seeded sample of 2^20 queries against the oracle's decode."""
    size, nlat, nlev = 4096, 4, 13
    lat, par = synth.neural_init(size, nlat, seed=5)
    pyr = synth.box_levels(synth.material(size, seed=5), nlev)
    fb = np.concatenate([p.reshape(-1, 7) for p in pyr[nlat:]])
    T = stf.NeuralTexture(size, size, nlat, nlev, lat, par, fb)
    n = 1 << 24
    uv = synth.uv_queries(n, seed=2)
    lod = synth.lods(n, seed=9)
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    out = T.lookup(to_dev(uv), to_dev(lod), taps=taps, filter="linear", seed=2024,
                   level_mode=stf.LEVEL_NEAREST)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(3).choice(n, 1 << 20, replace=False))
    ref = neural.NeuralTexture2D(split_levels(h16(lat), size, 0, nlat, 8), stored_params(par),
                                 [h16(p) for p in pyr[nlat:]])
    rv, rt, ex = filters.lookup_2d(ref, uv[idx], lod[idx], "linear", stochastic_form=True, seed=2024,
                                   level_mode=stf.LEVEL_NEAREST, qid=idx.astype(np.uint64))
    g_taps = taps.cpu().numpy()[idx]
    g_out = out.cpu().numpy()[idx].astype(np.float64)
    same = np.all(g_taps == rt, axis=1)
    assert np.all(same | ex)
    lvl = rt[:, 3]
    bound = np.full(rv.shape, 1e-6)
    dec = same & (lvl >= 0) & (lvl < nlat)
    for L in np.unique(lvl[dec]):
        m = dec & (lvl == L)
        w, h = ref.size(L)
        Z = ref.latents[L][np.clip(rt[m, 1], 0, h - 1), np.clip(rt[m, 0], 0, w - 1)]
        bound[m] = decode_bound(Z, ref.P)
    err = np.abs(g_out - rv)
    assert np.all(err[same] <= bound[same] + 2e-6 * np.abs(rv[same])), np.max(err[same] - bound[same])

    # the benchmark's call asks for no tap output (the slim decode): the same outputs, every query
    slim = T.lookup(to_dev(uv), to_dev(lod), filter="linear", seed=2024, level_mode=stf.LEVEL_NEAREST)
    torch.cuda.synchronize()
    torch.testing.assert_close(slim, out, rtol=0, atol=0)


@pytest.mark.parametrize("level_mode", [stf.LEVEL_NEAREST, stf.LEVEL_STOCHASTIC])
@pytest.mark.parametrize("filt", ["linear", "bspline3", "catmull_rom"])
def test_neural_slim_decode_equals_tap_output_decode(filt, level_mode):
    """Calls without tap output or permutation take the slim decode (several tiles per
    group of threads); each query's output must equal the tap-output decode's bit for bit,
    on an odd number of tiles with a ragged last one and NaN / infinite coordinates."""
    T, _, _, _, _ = make_neural()
    n = 128 * 37 + 51
    uv = synth.uv_queries(n, seed=13)
    lod = (synth.uniform(n, 14) * np.float32(7.0) - np.float32(0.5)).astype(np.float32)
    uv[5] = [np.nan, 0.5]
    uv[700] = [np.inf, 0.25]
    lod[900] = np.nan
    taps = torch.empty((n, 4), dtype=torch.int32, device=dev())
    ref = T.lookup(to_dev(uv), to_dev(lod), taps=taps, filter=filt, seed=8, level_mode=level_mode)
    slim = T.lookup(to_dev(uv), to_dev(lod), filter=filt, seed=8, level_mode=level_mode)
    torch.cuda.synchronize()
    torch.testing.assert_close(slim, ref, rtol=0, atol=0, equal_nan=True)
