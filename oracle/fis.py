"""Filter importance sampling, float64 (test infrastructure only).

Section 4.4, "Filter Importance Sampling (FIS)": instead of drawing one of the
discrete taps, FIS draws a continuous offset s from the filter's own density and
returns the texel nearest to x + s, the texel with index floor(x + s + 1/2) in
raster coordinates (texel i centred at i).  Taking the nearest texel reconstructs
the texels with a unit box, so the filter that is actually applied is the sampled
density convolved with that box:

* B-splines.  The B-spline of degree n is the box convolved with the B-spline of
  degree n - 1 (Cox-de Boor).  Sampling s as the sum of n independent uniforms on
  [-1/2, 1/2) (the density of the degree n - 1 B-spline) therefore applies the
  degree-n B-spline: n = 1 (uniform jitter) is stochastic linear interpolation,
  n = 3 the cubic B-spline of Eq. 9.
* Gaussian.  s = sigma * z with z normal (Box-Muller); the applied filter is the
  Gaussian convolved with the box, tap i carrying
  Phi((i + 1/2 - x) / sigma) - Phi((i - 1/2 - x) / sigma).

Variates are the query's 24-bit Philox words (philox.query_variates):

* B-spline of degree n: uniform j of axis a is word a of stream j (j < n).
* Gaussian: the Box-Muller pair (u0, u1) of stream 0 gives the x and y offsets
  sigma * sqrt(-2 ln(1 - u0)) * (cos 2 pi u1, sin 2 pi u1); a third axis takes
  sigma * sqrt(-2 ln(1 - u2)) * cos(2 pi u3).  1 - u keeps the logarithm finite
  (u = 0 occurs, u = 1 does not); the largest radius is therefore
  sigma * sqrt(-2 ln 2^-24) = 5.77 sigma.

Readings: the paper's example samples "a triangular PDF over [-1.5, 1.5]" for the
quadratic B-spline; the triangle (sum of two uniforms) has support [-1, 1] and the
applied quadratic B-spline, after the box, spans [-1.5, 1.5].  Sampling by a sum of
uniforms is one of the two methods the section names (the other is CDF
inversion); the sum is exact in the arithmetic used here.
"""
import math

import numpy as np
from scipy import special

IDX_LIMIT = 1 << 24
SCALE = 2.0 ** 24
# Largest offset a 24-bit Box-Muller draw can make, in units of sigma.
GAUSS_REACH = math.sqrt(-2.0 * math.log(2.0 ** -24))
# Decisions near a texel boundary that float32 Box-Muller arithmetic may take the
# other way: relative half-width of the exempt band around each boundary.
GAUSS_EXEMPT = 4e-6


def _coord(x32):
    x = np.asarray(x32, dtype=np.float32).astype(np.float64)
    finite = np.isfinite(x)
    return np.clip(np.where(finite, x, 0.0), -IDX_LIMIT, IDX_LIMIT), finite


def bspline_nearest(x32, us):
    """Index of the texel nearest to x + s, s = sum_j (u_j - 1/2) over the n
    variates in `us` (each a multiple of 2^-24 in [0, 1)).

    floor(x + s + 1/2) = floor(x + sum u - (n - 1)/2).  Every term is a multiple of
    2^-24 except x, so the value is formed exactly as floor((floor(x 2^24) + sum u 2^24
    - (n - 1) 2^23) / 2^24): the floor of a real y over the integer 2^24 equals the
    floor of floor(y) over it."""
    n = len(us)
    x, finite = _coord(x32)
    X = np.floor(x * SCALE)                           # exact: x is a float32, |x| <= 2^24
    K = np.zeros_like(X)
    for u in us:
        K = K + np.round(np.asarray(u, dtype=np.float64) * SCALE)
    idx = np.floor((X + K - (n - 1) * SCALE / 2) / SCALE)   # |numerator| < 2^50: exact
    return idx.astype(np.int64), finite


def box_muller(u0, u1, sigma):
    """sigma * sqrt(-2 ln(1 - u0)) * (cos 2 pi u1, sin 2 pi u1), float64."""
    r = sigma * np.sqrt(-2.0 * np.log1p(-np.asarray(u0, dtype=np.float64)))
    t = 2.0 * np.pi * np.asarray(u1, dtype=np.float64)
    return r * np.cos(t), r * np.sin(t)


def gaussian_offsets(words0, dims, sigma):
    """Per-axis offsets of one query from the four words of its stream 0."""
    ox, oy = box_muller(words0[0], words0[1], sigma)
    if dims == 2:
        return [ox, oy]
    oz, _ = box_muller(words0[2], words0[3], sigma)
    return [ox, oy, oz]


def gaussian_nearest(x32, off):
    """floor(x + off + 1/2) and whether float32 evaluation may round across the
    boundary (distance below GAUSS_EXEMPT * (1 + |off|))."""
    x, finite = _coord(x32)
    y = x + off + 0.5
    idx = np.floor(y)
    d = np.minimum(y - idx, idx + 1 - y)
    return idx.astype(np.int64), finite, d < GAUSS_EXEMPT * (1.0 + np.abs(off))


def gaussian_reach(sigma):
    """Largest offset of a 24-bit Box-Muller draw: 5.77 sigma."""
    return GAUSS_REACH * sigma


def gaussian_window(x32, sigma):
    """First and last tap index a 24-bit draw can reach from x (nearest texel of
    x +- reach), per query."""
    x, _ = _coord(x32)
    R = gaussian_reach(sigma)
    return np.floor(x - R + 0.5).astype(np.int64), np.floor(x + R + 0.5).astype(np.int64)


def gaussian_tap_weight(i, x, sigma):
    """Phi((i + 1/2 - x)/sigma) - Phi((i - 1/2 - x)/sigma): the box-convolved
    Gaussian at tap i (the probability that x + s rounds to i)."""
    s = sigma * math.sqrt(2.0)
    return 0.5 * (special.erf((i + 0.5 - x) / s) - special.erf((i - 0.5 - x) / s))


def deterministic_gaussian(fetch, xs32, sigma, background=0.0):
    """sum over the reachable window of prod_a w_a(i_a) * t(i): the expectation of the
    Gaussian FIS lookup, up to the mass beyond 5.77 sigma (below 1e-8 per axis)."""
    D = len(xs32)
    frames = [_coord(x) for x in xs32]
    finite = np.logical_and.reduce([fin for (_, fin) in frames])
    lo_hi = [gaussian_window(x, sigma) for x in xs32]
    span = int(max(np.max(hi - lo) for lo, hi in lo_hi)) + 1
    total = None
    for combo in np.ndindex(*([span] * D)):
        w = 1.0
        idx = []
        for a in range(D):
            lo, hi = lo_hi[a]
            i = lo + combo[a]
            inside = i <= hi
            w = w * np.where(inside, gaussian_tap_weight(i, frames[a][0], sigma), 0.0)
            idx.append(np.minimum(i, hi))
        t = fetch(*idx)
        total = w[:, None] * t if total is None else total + w[:, None] * t
    total[~finite] = background
    return total


def stochastic(fetch, xs32, filt, streams, sigma=None, background=0.0):
    """One FIS lookup per query.  streams[j] = the four words of Philox stream j.
    Returns (value (N, C), indices, exempt, finite)."""
    D = len(xs32)
    if filt == "fis_gaussian":
        off = gaussian_offsets(streams[0], D, sigma)
        res = [gaussian_nearest(x, o) for x, o in zip(xs32, off)]
        idx = [r[0] for r in res]
        finite = np.logical_and.reduce([r[1] for r in res])
        exempt = np.logical_or.reduce([r[2] for r in res]) & finite
    else:
        n = FIS_DEGREE[filt]
        res = [bspline_nearest(x, [streams[j][a] for j in range(n)]) for a, x in enumerate(xs32)]
        idx = [r[0] for r in res]
        finite = np.logical_and.reduce([r[1] for r in res])
        exempt = np.zeros_like(finite)
    val = fetch(*idx)
    val[~finite] = background
    return val, idx, exempt, finite


# Degree of the B-spline each FIS filter applies, i.e. the number of uniforms summed.
FIS_DEGREE = {"fis_linear": 1, "fis_bspline3": 3}
# Deterministic twin of each FIS filter (the filter it applies).
FIS_TWIN = {"fis_linear": "linear", "fis_bspline3": "bspline3", "fis_gaussian": "gaussian"}
STREAMS = {"fis_linear": 1, "fis_bspline3": 3, "fis_gaussian": 1}
