"""The allocation-free binned lookup, stf_lookup_batch_binned_noalloc, against the
regular entry point stf_lookup_batch, through the C ABI.

This entry point exists for callers that must not have the library allocate device
memory (processes that reserve their whole budget up front with their own
allocator, or that cannot accept an allocation's synchronisation); its scratch is a
fixed array inside the library.  Two calls in a row must both agree with the
regular entry point, which also shows that the shared array's leftover contents
from the first call do not leak into the second.  This file is collected last.
"""
import numpy as np
import pytest
import torch

import paper_2305_05810_gb300 as stf
import synth

pytestmark = pytest.mark.gpu
REL = 2e-6   # the stochastic value tolerance used by the parity tests


def _agree(T, coords, lod, params, with_taps=True):
    """Both entry points on the same call; with_taps=False passes no tap output to
    the allocation-free one (the form the benchmark and most callers use)."""
    n = coords.shape[0]
    C = T.channels
    out_ref = torch.empty((n, C), dtype=torch.float32, device=coords.device)
    out_na = torch.full((n, C), float("nan"), dtype=torch.float32, device=coords.device)
    taps_ref = torch.empty((n, 4), dtype=torch.int32, device=coords.device)
    taps_na = torch.full((n, 4), -9, dtype=torch.int32, device=coords.device) if with_taps else None
    stf.stf_lookup_batch(T.handle, params, coords, lod, n, out_ref, taps_ref)
    stf.stf_lookup_batch_binned_noalloc(T.handle, params, coords, lod, n, out_na, taps_na)
    torch.cuda.synchronize()
    if with_taps:
        assert torch.equal(taps_ref, taps_na)
    a, b = out_ref.cpu().numpy(), out_na.cpu().numpy()
    assert np.all(np.abs(a - b) <= REL * np.abs(a))


def test_noalloc_binned_matches_regular_entry_point_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stf.load()
    dev = torch.device("cuda:0")
    vals = synth.dense_density(n=64, seed=3, period=12.0)
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(64, 64, 64), fmt=stf.FMT_F16)
    q = torch.from_numpy(synth.camera_queries(W=160, H=90, steps=16, centre=(32, 32, 32),
                                              radius=96, half_span=56, seed=3)).to(dev)
    for call, filt in enumerate(("bspline3", "catmull_rom")):
        p = stf.make_params(filt, seed=11 + call, query_offset=1000 * call)
        _agree(T, q[: q.shape[0] - 777 * call], None, p)
    _agree(T, q, None, stf.make_params("bspline3", seed=13), with_taps=False)

    img = synth.texture2d(128, 64, 4, seed=2)
    T2 = stf.Texture(stf.KIND_TEX2D, img, dims=(128, 64, 1), channels=4, mip_levels=8,
                     generate_mips=True)
    uv = torch.from_numpy(synth.uv_queries(stf.STF_NOALLOC_MAX_QUERIES, seed=8)).to(dev)
    lod = torch.from_numpy(synth.lods(stf.STF_NOALLOC_MAX_QUERIES, seed=9, lo=0, hi=7)).to(dev)
    for call in range(2):
        _agree(T2, uv, lod if call == 0 else None, stf.make_params("linear", seed=5 + call))

    too_many = torch.empty((stf.STF_NOALLOC_MAX_QUERIES + 1, 2), dtype=torch.float32, device=dev)
    out = torch.empty((too_many.shape[0], 4), dtype=torch.float32, device=dev)
    with pytest.raises(stf.StfError) as e:
        stf.stf_lookup_batch_binned_noalloc(T2.handle, stf.make_params(), too_many, None,
                                            too_many.shape[0], out)
    assert e.value.status == 1 and "limit" in str(e.value)
    T.close()
    T2.close()
