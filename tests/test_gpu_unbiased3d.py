"""GPU unbiasedness of the 3D stochastic lookups (Eq. 3: the expectation of the
single-tap estimate over the tap draw equals the deterministic filter).

Each query runs 4096 stochastic samples (sample indices 0..4095) through
`stf_lookup_accumulate`, which sums the estimates and their squares in float64 on
the GPU.  Each query's mean is scored against the oracle's exact expectation (every
tap combination enumerated, weighted by its probability) with the estimator's exact
variance (the enumerated second moment minus the squared expectation):
z = (mean - F) / sqrt(var / 4096).  The bar is the parity rule's: at most 0.5% of
the queries with |z| > 3 (0.27% expected) and the pooled statistic
sum(mean - F) / sqrt(sum(var) / 4096) within +-3.  Queries whose estimate has no
variance (every drawable tap holds the same value) must return F to float32
rounding.  Grids: a dense FP16 density (the stored half values are the oracle's
texels) and a sparse cloud with FP32 and with E4M3 + per-leaf scale leaves (the
oracle holds the dequantised leaves); trilinear, cubic B-spline and Catmull-Rom
(one tap, sign * sum|w| scale)."""
import numpy as np
import pytest
import torch

import paper_2305_05810_gb300 as stf
import synth
from oracle import codecs, filters, textures
from parity import dev, quantise, to_dev

pytestmark = pytest.mark.gpu
FILTERS = ["linear", "bspline3", "catmull_rom"]
S = 4096


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stf.load()


def _z_test(T, ref, pts, filt, seed):
    s, _ = T.accumulate(to_dev(pts), S, filter=filt, seed=seed)
    mean = s.cpu().numpy()[:, 0] / S
    xs = [pts[:, 0], pts[:, 1], pts[:, 2]]
    F = filters.expectation_by_enumeration(ref.fetch, xs, filt)[:, 0]
    var = np.maximum(filters.expectation_by_enumeration(ref.fetch, xs, filt, power=2)[:, 0] - F * F, 0)
    live = var > 1e-12 * np.maximum(F * F, 1e-12)
    flat = ~live
    assert np.all(np.abs(mean[flat] - F[flat]) <= 4e-7 * np.maximum(np.abs(F[flat]), 1e-6))
    z = (mean[live] - F[live]) / np.sqrt(var[live] / S)
    tail = np.mean(np.abs(z) > 3)
    pooled = np.sum(mean[live] - F[live]) / np.sqrt(np.sum(var[live]) / S)
    print("%s: %d live queries, |z| > 3 rate %.4f, pooled %.3f" % (filt, np.sum(live), tail, pooled))
    assert np.sum(live) > 0.25 * len(pts)       # at least a quarter straddle non-zero texels
    assert tail <= 0.005, tail
    assert abs(pooled) <= 3.0, pooled


@pytest.mark.parametrize("filt", FILTERS)
def test_dense_fp16_unbiased_over_4096_samples(filt):
    n = 64
    vals = synth.dense_density(n=n, seed=3, period=12.0)
    T = stf.Texture(stf.KIND_DENSE3D, vals, dims=(n, n, n), fmt=stf.FMT_F16)
    ref = textures.Dense3D(quantise(vals, stf.FMT_F16).reshape(n, n, n))
    pts = (synth.uniform(3 * 16384, 17).reshape(-1, 3) * np.float32(n + 2) - np.float32(1)).astype(np.float32)
    _z_test(T, ref, pts, filt, seed=41)
    stf.stf_synchronize(T.handle)


@pytest.mark.parametrize("fmt", [stf.FMT_F32, stf.FMT_E4M3_SCALED])
@pytest.mark.parametrize("filt", FILTERS)
def test_sparse_unbiased_over_4096_samples(filt, fmt):
    origins, values = synth.sparse_cloud(domain=256, seed=4)
    T = stf.Texture(stf.KIND_SPARSE3D, values, fmt=fmt, leaf_origins=origins)
    if fmt == stf.FMT_E4M3_SCALED:
        codes, scales = codecs.e4m3_leaf_quantise(values)
        stored = codecs.e4m3_leaf_dequantise(codes, scales)
    else:
        stored = np.asarray(values, dtype=np.float32)
    ref = textures.Sparse3D(origins, stored)
    # queries near active leaves, so that most footprints straddle stored voxels and
    # some straddle a leaf's edge into background
    pts = (origins[np.arange(16384) % len(origins)] +
           synth.uniform(3 * 16384, 23).reshape(-1, 3) * np.float32(10) - np.float32(1)).astype(np.float32)
    _z_test(T, ref, pts, filt, seed=43)
    stf.stf_synchronize(T.handle)
