"""Helpers shared by the GPU parity tests: build matching texture stores for the
library and the oracle, and compare results under the stated tolerances.

Tolerances (from the float32 arithmetic of the kernels):
* tap indices: bit-exact against the oracle's float64 decision, except where a
  variate lies within 1e-6 of a CDF boundary (the oracle reports those as exempt; at
  most 0.2% of a test's queries); an exempt tap may differ by one per axis;
* stochastic values: |gpu - ref| <= 2e-6 |ref| (the texel is exact; only the
  float32 scale sign(w) * sum|w| of Catmull-Rom carries rounding);
* deterministic values: |gpu - ref| <= 2e-6 max(|ref|, sum_i |w_i t_i|), the second
  term covering cancellation between the negative lobes of Catmull-Rom.
"""
import itertools

import numpy as np
import torch

import paper_2305_05810_gb300 as stf
from oracle import codecs, filters, kernels, textures

REL = 2e-6


def dev():
    return torch.device("cuda:0")


def quantise(values, fmt):
    """Values as the library stores them (exact float64)."""
    v = np.asarray(values, dtype=np.float32)
    if fmt == stf.FMT_F16:
        return codecs.f16_decode(codecs.f16_encode(v.astype(np.float64)))
    return v.astype(np.float64)


def abs_weighted_sum(fetch, xs32, filt):
    """sum over taps of |w| |t| (tolerance scale for deterministic filters)."""
    offs, _, _ = kernels.FILTERS[filt]
    frames = [filters.axis_frame(x) for x in xs32]
    weights = [np.abs(filters.axis_weights(f, filt)) for (_, f, _) in frames]
    total = 0.0
    for combo in itertools.product(range(len(offs)), repeat=len(xs32)):
        w = np.prod([weights[a][combo[a]] for a in range(len(xs32))], axis=0)
        total = total + w[:, None] * np.abs(fetch(*[frames[a][0] + offs[combo[a]] for a in range(len(xs32))]))
    return total


def check_stochastic(gpu_val, gpu_taps, ref_val, ref_taps, exempt, dims=3):
    """Assert tap and value parity; returns the number of queries whose taps differ
    (all of them exempt).  The exempt count is printed and must stay below 0.2% of the
    queries (a handful for small cases)."""
    gpu_val = np.asarray(gpu_val, dtype=np.float64).reshape(ref_val.shape)
    gpu_taps = np.asarray(gpu_taps, dtype=np.int64).reshape(-1, 4)
    exempt = np.asarray(exempt, dtype=bool)
    print("exempt %d of %d queries" % (np.sum(exempt), exempt.size))
    assert np.sum(exempt) <= max(4, exempt.size // 500), "exempt %d of %d" % (np.sum(exempt), exempt.size)
    same = np.all(gpu_taps == ref_taps, axis=1)
    bad = ~same & ~exempt
    assert not np.any(bad), "tap mismatch at %s: gpu %s ref %s" % (
        np.nonzero(bad)[0][:5], gpu_taps[bad][:5], ref_taps[bad][:5])
    near = np.all(np.abs(gpu_taps - ref_taps) <= 1, axis=1)
    assert np.all(near[exempt]), "exempt tap more than one texel away"
    err = np.abs(gpu_val - ref_val)[same]
    lim = REL * np.abs(ref_val)[same] + 1e-30
    assert np.all(err <= lim), "value mismatch: max rel %g" % np.max(err / np.maximum(np.abs(ref_val[same]), 1e-30))
    return int(np.sum(~same))


def check_deterministic(gpu_val, ref_val, scale):
    gpu_val = np.asarray(gpu_val, dtype=np.float64).reshape(ref_val.shape)
    err = np.abs(gpu_val - ref_val)
    lim = REL * np.maximum(np.abs(ref_val), scale) + 1e-30
    worst = np.max(err / np.maximum(np.maximum(np.abs(ref_val), scale), 1e-30))
    assert np.all(err <= lim), "deterministic mismatch: worst rel %g" % worst
    return worst


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def positivized_scale(xs32, tmax):
    """(W+ + W-) * max|t| = prod_a sum|w_a| * max|t|: the magnitude the two-tap
    estimate's rounding is relative to."""
    s = 1.0
    for x in xs32:
        _, f, _ = filters.axis_frame(x)
        s = s * np.sum(np.abs(filters.axis_weights(f, "catmull_rom")), axis=0)
    return np.nan_to_num(s) * tmax


def positivized_moments(fetch, xs32):
    """Exact mean and variance of the positivized estimate (two independent draws)."""
    D = len(xs32)
    frames = [filters.axis_frame(x) for x in xs32]
    w64 = [filters.axis_weights(f, "catmull_rom") for (_, f, _) in frames]
    m = filters._block_masses(w64, D)
    res = {}
    for sign in (1, -1):
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
                t = fetch(*idx)
                e1 = e1 + p[:, None] * t
                e2 = e2 + p[:, None] * t * t
        res[sign] = (W[:, None], e1, e2)
    (Wp, p1, p2), (Wn, n1, n2) = res[1], res[-1]
    return Wp * p1 - Wn * n1, Wp ** 2 * (p2 - p1 ** 2) + Wn ** 2 * (n2 - n1 ** 2)
