"""Serving loop on the GPU: mixed requests (2D, dense and sparse textures; stochastic
and deterministic; uneven sizes) admitted into overlapping slots under a memory
budget.  Each request's result in the mix must equal the same request run alone
through one direct library call (bit-identical: the variates are keyed on the
request-local query index, whatever the chunking or the mix)."""
import numpy as np
import pytest
import torch

import paper_2305_05810_gb300 as stf
import synth
from paper_2305_05810_gb300 import serving

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def textures():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stf.load()
    tex2d = stf.Texture(stf.KIND_TEX2D, synth.texture2d(256, 256, 4, seed=1), dims=(256, 256, 1),
                        channels=4, mip_levels=9, generate_mips=True)
    dense = stf.Texture(stf.KIND_DENSE3D, synth.dense_density(n=64, seed=3, period=12.0),
                        dims=(64, 64, 64), fmt=stf.FMT_F16)
    origins, values = synth.sparse_cloud(domain=512, seed=4)
    sparse = stf.Texture(stf.KIND_SPARSE3D, values, fmt=stf.FMT_E4M3_SCALED, leaf_origins=origins)
    return {"tex2d": tex2d, "dense": dense, "sparse": sparse}


def _make(textures):
    pools = {
        "tex2d": torch.from_numpy(synth.uv_queries(1 << 20, seed=2)),
        "dense": torch.from_numpy(synth.camera_queries(W=256, H=256, steps=16, centre=(32, 32, 32),
                                                       radius=96, half_span=56, seed=3)),
        "sparse": torch.from_numpy(synth.camera_queries(W=256, H=256, steps=16, centre=(256, 256, 256),
                                                        radius=768, half_span=444, seed=4)),
    }
    lods = torch.from_numpy(synth.lods(1 << 20, seed=9, lo=0, hi=8))
    keys = list(textures)

    def make(i, size, rng):
        key = keys[i % len(keys)]
        pool = pools[key]
        start = int(rng.integers(0, pool.shape[0] - size))
        coords = pool[start:start + size].clone().pin_memory()
        lod = lods[:size].clone().pin_memory() if key == "tex2d" and i % 2 else None
        filt = ("linear", "bspline3", "catmull_rom")[i % 3]
        return serving.Request(i, key, coords, lod, filter=filt, stochastic=(i % 4 != 3), seed=100 + i)
    return make


def test_each_result_is_the_same_alone_and_in_the_mix(textures):
    make = _make(textures)
    reqs = serving.poisson_requests(48, 2000.0, (1000, 1 << 19), make, seed=6)
    backend = serving.TorchBackend(textures, n_slots=6)
    sched = serving.Scheduler(backend, n_slots=6, budget_bytes=64 << 20, chunk_queries=1 << 16)
    done = sched.run(reqs)
    assert len(done) == len(reqs) and sched.peak_active >= 2
    assert sched.peak_in_use <= 64 << 20
    # the slots' device buffers that stay allocated are what the scheduler charges
    held = sum(4 * b.numel() for bufs in backend.slot_bufs for k, b in bufs.items() if k != "h_out")
    assert held == sched.in_use <= 64 << 20
    for r in reqs:
        T = textures[r.texture]
        d = r.coords.cuda()
        lod = None if r.lod is None else r.lod.cuda()
        alone = torch.empty((r.n, T.channels), dtype=torch.float32, device="cuda")
        p = stf.make_params(r.filter, seed=r.seed, level_mode=r.level_mode)
        if r.stochastic:
            stf.stf_lookup_batch(T.handle, p, d, lod, r.n, alone)
        else:
            stf.stf_lookup_batch_deterministic(T.handle, p, d, lod, r.n, alone)
        torch.cuda.synchronize()
        assert torch.equal(alone.cpu(), r.result), r.rid
    s = serving.latency_summary(done)
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_request_over_budget_is_rejected_on_gpu(textures):
    backend = serving.TorchBackend(textures, n_slots=2)
    sched = serving.Scheduler(backend, n_slots=2, budget_bytes=1 << 20)
    big = serving.Request(0, "dense", torch.zeros((1 << 17, 3)))
    with pytest.raises(serving.BudgetError):
        sched.submit(big)


@pytest.mark.parametrize("tail", [1, 5])
def test_host_pipeline_equals_one_device_call(tail):
    """Chunked multi-stream lookups from pinned host memory return the results of one
    device call over the whole batch (variates keyed by the global query index), also
    with the last chunk split into smaller ones."""
    from paper_2305_05810_gb300.pipeline import HostPipeline
    vals = synth.dense_density(n=64, seed=3, period=12.0)
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(64, 64, 64), fmt=stf.FMT_F16)
    q = synth.camera_queries(W=200, H=100, steps=16, centre=(32, 32, 32), radius=96, half_span=56, seed=5)
    n = q.shape[0]
    whole = T.lookup(torch.from_numpy(q).cuda(), filter="bspline3", seed=9, query_offset=123)
    h_q = torch.from_numpy(q).pin_memory()
    h_out = torch.empty((n, 1), dtype=torch.float32).pin_memory()
    pipe = HostPipeline(T, chunk=10007, n_streams=3, tail=tail)
    pipe.lookup(stf.make_params("bspline3", seed=9, query_offset=123), h_q, h_out)
    torch.cuda.synchronize()
    assert torch.equal(whole.cpu(), h_out)
    det = T.lookup_deterministic(torch.from_numpy(q).cuda(), filter="linear")
    pipe.lookup(stf.make_params("linear"), h_q, h_out, stochastic=False)
    torch.cuda.synchronize()
    assert torch.equal(det.cpu(), h_out)


@pytest.mark.parametrize("kind", ["tex2d", "sparse", "neural"])
def test_chunked_calls_equal_one_call(kind):
    """Splitting a batch into calls with advancing query_offset gives the results of one
    call (variates keyed by the global query index), for 2D textures with a level of
    detail, sparse grids and neural textures."""
    if kind == "tex2d":
        T = stf.Texture(stf.KIND_TEX2D, synth.texture2d(64, 64, 4, seed=3), dims=(64, 64, 1), channels=4,
                        mip_levels=7, generate_mips=True)
        q = synth.uv_queries(50000, seed=4)
        lod = torch.from_numpy(synth.lods(50000, seed=5, lo=0, hi=6)).cuda()
        filt = "catmull_rom"
    elif kind == "sparse":
        origins, values = synth.sparse_cloud(domain=256, seed=4)
        T = stf.Texture(stf.KIND_SPARSE3D, values, leaf_origins=origins)
        q = (origins[np.arange(50000) % len(origins)] + synth.uniform(150000, 6).reshape(-1, 3) * 8).astype(np.float32)
        lod, filt = None, "bspline3"
    else:
        lat, par = synth.neural_init(64, 3, seed=5)
        pyr = synth.box_levels(synth.material(64, seed=5), 6)
        fb = np.concatenate([p.reshape(-1, 7) for p in pyr[3:]])
        T = stf.NeuralTexture(64, 64, 3, 6, lat, par, fb)
        q = synth.uv_queries(50000, seed=7)
        lod = torch.from_numpy(synth.lods(50000, seed=8, lo=0, hi=5)).cuda()
        filt = "linear"
    d = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    n = d.shape[0]
    whole = T.lookup(d, lod, filter=filt, seed=12, query_offset=1000)
    parts = torch.empty_like(whole)
    cuts = [0, 1, 129, 4097, 33333, n]
    for a, b in zip(cuts[:-1], cuts[1:]):
        p = stf.make_params(filt, seed=12, query_offset=1000 + a)
        stf.stf_lookup_batch(T.handle, p, d[a:b], None if lod is None else lod[a:b], b - a, parts[a:b])
    torch.cuda.synchronize()
    assert torch.equal(whole, parts)


@pytest.mark.parametrize("kind", ["tex2d", "dense", "sparse", "neural"])
def test_zero_copy_host_buffers_equal_device_buffers(kind):
    """Pinned host buffers passed straight to the lookup (the kernel reads the
    coordinates and writes the results across the host link) give the results of
    device buffers, bit for bit; stf_device_accessible tells the buffers apart."""
    if kind == "tex2d":
        T = stf.Texture(stf.KIND_TEX2D, synth.texture2d(64, 64, 4, seed=3), dims=(64, 64, 1), channels=4,
                        mip_levels=7, generate_mips=True)
        q, lod, filt = synth.uv_queries(70000, seed=4), synth.lods(70000, seed=5, lo=0, hi=6), "bspline3"
    elif kind == "dense":
        T = stf.Texture(stf.KIND_DENSE3D, synth.dense_density(n=32, seed=3, period=8.0), dims=(32, 32, 32),
                        fmt=stf.FMT_F16)
        q = (synth.uniform(3 * 70000, 6).reshape(-1, 3) * np.float32(36) - np.float32(2)).astype(np.float32)
        lod, filt = None, "catmull_rom"
    elif kind == "sparse":
        origins, values = synth.sparse_cloud(domain=256, seed=4)
        T = stf.Texture(stf.KIND_SPARSE3D, values, leaf_origins=origins)
        q = (origins[np.arange(70000) % len(origins)] + synth.uniform(210000, 6).reshape(-1, 3) * 8).astype(np.float32)
        lod, filt = None, "bspline3"
    else:
        lat, par = synth.neural_init(64, 3, seed=5)
        pyr = synth.box_levels(synth.material(64, seed=5), 6)
        fb = np.concatenate([p.reshape(-1, 7) for p in pyr[3:]])
        T = stf.NeuralTexture(64, 64, 3, 6, lat, par, fb)
        q, lod, filt = synth.uv_queries(70000, seed=7), synth.lods(70000, seed=8, lo=0, hi=5), "linear"
    n, C = q.shape[0], T.channels
    h_q = torch.from_numpy(np.ascontiguousarray(q)).pin_memory()
    h_lod = None if lod is None else torch.from_numpy(lod).pin_memory()
    h_out = torch.full((n, C), -1.0).pin_memory()
    pageable = torch.empty(16)
    d_q = h_q.cuda()
    d_lod = None if h_lod is None else h_lod.cuda()
    assert stf.stf_device_accessible(h_q) and stf.stf_device_accessible(h_out) and stf.stf_device_accessible(d_q)
    assert not stf.stf_device_accessible(pageable)
    p = stf.make_params(filt, seed=31, query_offset=77)
    want = torch.empty((n, C), device="cuda")
    stf.stf_lookup_batch(T.handle, p, d_q, d_lod, n, want)
    stf.stf_lookup_batch(T.handle, p, h_q, h_lod, n, h_out)
    torch.cuda.synchronize()
    assert torch.equal(h_out, want.cpu())
