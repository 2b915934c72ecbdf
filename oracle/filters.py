"""Stochastic and deterministic filtered lookups, float64 (test infrastructure only).

What is computed, per query, with the paper's definitions:

* Deterministic filter: the discrete weighted sum F = sum_i w_i t_i (Eq. 2) over
  the separable tap window; for B-splines this is the 4x4 (4x4x4) sum of Eq. 9,
  read as K_bs(s - (floor(s) + i)) since the printed equation drops the "- s".
* Stochastic filter: one tap per axis is drawn with probability |w| / sum |w|
  (sampling arrays, Section 2.2; separable functions, Section 2.2 and 4.2) and the
  single texel is returned, times sign(w) * sum |w| per axis when the kernel has
  negative lobes (the absolute-value rule noted under "Positivization",
  Section 2.2).  For the non-negative kernels the factor is exactly 1 (Eq. 3).
* Exact expectation: every tap combination weighted by its selection probability
  (Eq. 3), which must reproduce the deterministic filter.

Readings where the paper is silent or inconsistent (all stated in the design notes):

* 2D raster coordinate: x = u * W_L - 1/2 (texel centres at i + 1/2, as in the
  discrete Gaussian listing of Appendix B); 3D index coordinates are used as is.
* Taps are ordered from low to high coordinate and tap k is the smallest k with
  u * S < C_k, C_k = sum_{j<=k} |w_j|, S = C_last (sampling arrays, Section 2.2).
  If rounding leaves no such k, the last tap with |w| > 0 is taken.
* Every decision is taken in float64 from the definition: the weights are evaluated
  at the exact fraction x - floor(x), C_k and S are float64 sums of |w|, and the
  product u * S is float64.  A float32 implementation (the paper's listings are
  float32) can decide otherwise only where u lies within its rounding error of a
  boundary C_k / S; `boundary_distance` reports that distance so that callers can
  exempt queries within 1e-6 of a boundary.  Values, sums and expectations are
  float64.
* Variates: independent per axis by default.  With reuse, one variate is carried
  from axis to axis through the remapping of Eq. 4, generalised to several taps:
  u' = (u * S - C_{k-1}) / |w_k|.
* A NaN or infinite coordinate returns the background value and fetches nothing.
* MIP level (2D): lod is clamped to [0, levels - 1]; the stochastic level is
  floor(lod + u_L) (the +/- 1/2 jitter of the anisotropic-LOD listing, Appendix B,
  followed by rounding), so the upper level is taken with probability frac(lod);
  its deterministic twin blends floor(lod) and the next level by frac(lod).  The
  "nearest" level mode uses floor(lod + 1/2) in both forms.
"""
import itertools
import numpy as np

from . import fis
from .kernels import FILTERS
from .philox import query_variates

IDX_LIMIT = 1 << 24          # floor(x) is clamped to +-2^24 before it becomes an index
EXEMPT = 1e-6                # boundary distance under which a tap index may differ
LEVEL_NEAREST, LEVEL_STOCHASTIC = 0, 1


def axis_frame(x32):
    """floor(x) as an index and the fraction x - floor(x) of a float32 coordinate,
    exact in float64."""
    x = np.asarray(x32, dtype=np.float32).astype(np.float64)
    finite = np.isfinite(x)
    xs = np.where(finite, x, 0.0)
    fl = np.floor(xs)
    f = xs - fl
    i0 = np.clip(fl, -IDX_LIMIT, IDX_LIMIT).astype(np.int64)
    return i0, f, finite


def axis_weights(f, filt):
    """float64 weights K(f - o) for the filter's tap offsets o, shape (T, N)."""
    offs, K, _ = FILTERS[filt]
    f = np.asarray(f, dtype=np.float64)
    return np.stack([K(f - o) for o in offs])


def select_tap(u, w64):
    """Inverse-CDF tap choice in float64 (sampling arrays, Section 2.2): the smallest
    k with u * S < C_k, C_k = sum_{j<=k} |w_j|, S = C_last.  Returns (k, the variate
    remapped into the chosen tap's interval by Eq. 4, u' = (u S - C_{k-1}) / |w_k|)."""
    a = np.abs(np.asarray(w64, dtype=np.float64))
    C = np.cumsum(a, axis=0)
    S = C[-1]
    us = np.asarray(u, dtype=np.float64) * S
    below = us[None, :] < C
    T = C.shape[0]
    k = np.argmax(below, axis=0)
    last_pos = T - 1 - np.argmax((a > 0)[::-1], axis=0)
    k = np.where(below.any(axis=0), k, last_pos)      # only if every weight is zero
    cols = np.arange(k.shape[0])
    c_prev = np.where(k > 0, C[np.maximum(k - 1, 0), cols], 0.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        u2 = (us - c_prev) / a[k, cols]
    u2 = np.clip(np.nan_to_num(u2), 0.0, np.nextafter(1.0, 0.0))
    return k, u2


def boundary_distance(u, w64):
    """float64 distance of u to the nearest interior CDF boundary C_k / S."""
    a = np.abs(w64)
    C = np.cumsum(a, axis=0)
    S = C[-1]
    interior = C[:-1] / S
    return np.min(np.abs(np.asarray(u)[None, :] - interior), axis=0)


def stochastic(fetch, xs32, filt, us, reuse=False, background=0.0):
    """One stochastic lookup per query.

    fetch(*idx) -> (N, C) texel values; xs32: list of D float32 raster coordinates;
    us: list of D variates.  Returns (value (N, C), indices list of D int arrays,
    exempt (N,) bool, finite (N,) bool).
    """
    offs, _, nonneg = FILTERS[filt]
    offs = np.asarray(offs)
    N = np.asarray(xs32[0]).shape[0]
    sigma = np.ones(N)
    exempt = np.zeros(N, dtype=bool)
    finite = np.ones(N, dtype=bool)
    amp = np.ones(N)
    u_carry = np.asarray(us[0], dtype=np.float64)
    idx = []
    for a, x in enumerate(xs32):
        i0, f, fin = axis_frame(x)
        finite &= fin
        w64 = axis_weights(f, filt)
        u = u_carry if reuse else np.asarray(us[a], dtype=np.float64)
        k, u2 = select_tap(u, w64)
        exempt |= boundary_distance(u, w64) < EXEMPT * amp
        wk = w64[k, np.arange(N)]
        S = np.sum(np.abs(w64), axis=0)
        if reuse:
            amp = amp * S / np.abs(wk)
            u_carry = u2
        if not nonneg:
            sigma = sigma * np.sign(wk) * S
        idx.append(i0 + offs[k])
    val = sigma[:, None] * fetch(*idx)
    val[~finite] = background
    return val, idx, exempt, finite


def deterministic(fetch, xs32, filt, background=0.0):
    """Full-footprint weighted sum (Eq. 2 / Eq. 9) over every tap combination."""
    offs, _, _ = FILTERS[filt]
    frames = [axis_frame(x) for x in xs32]
    weights = [axis_weights(f, filt) for (_, f, _) in frames]
    finite = np.logical_and.reduce([fin for (_, _, fin) in frames])
    total = None
    for combo in itertools.product(range(len(offs)), repeat=len(xs32)):
        w = np.prod([weights[a][combo[a]] for a in range(len(xs32))], axis=0)
        t = fetch(*[frames[a][0] + offs[combo[a]] for a in range(len(xs32))])
        total = w[:, None] * t if total is None else total + w[:, None] * t
    total[~finite] = background
    return total


def expectation_by_enumeration(fetch, xs32, filt, power=1):
    """E[<F>^power] = sum over tap combinations of p(combo) * estimate(combo)^power,
    with p = prod |w| / S and estimate = prod(sign(w) S) * t (or t for non-negative
    kernels).  power=1 gives the expectation (Eq. 3), power=2 the second moment from
    which the exact variance of one stochastic lookup follows."""
    offs, _, nonneg = FILTERS[filt]
    frames = [axis_frame(x) for x in xs32]
    weights = [axis_weights(f, filt) for (_, f, _) in frames]
    sums = [np.sum(np.abs(w), axis=0) for w in weights]
    total = None
    for combo in itertools.product(range(len(offs)), repeat=len(xs32)):
        p = np.ones(weights[0].shape[1])
        sig = np.ones_like(p)
        for a in range(len(xs32)):
            wk = weights[a][combo[a]]
            p = p * np.abs(wk) / sums[a]
            if not nonneg:
                sig = sig * np.sign(wk) * sums[a]
        t = fetch(*[frames[a][0] + offs[combo[a]] for a in range(len(xs32))])
        term = p[:, None] * (sig[:, None] * t) ** power
        total = term if total is None else total + term
    return total


# ---------------------------------------------------------------- positivization

def _block_masses(weights, dims):
    """Per-axis inner (taps 1, 2) and outer (taps 0, 3) |w| sums, and the masses of the
    2^D blocks (bit a of the block set = axis a takes an outer tap)."""
    ain = [np.abs(w[1]) + np.abs(w[2]) for w in weights]
    aout = [np.abs(w[0]) + np.abs(w[3]) for w in weights]
    masses = []
    for b in range(1 << dims):
        m = np.ones_like(ain[0])
        for a in range(dims):
            m = m * (aout[a] if (b >> a) & 1 else ain[a])
        masses.append(m)
    return masses


def _blocks_of_sign(dims, sign):
    """Blocks whose taps carry that sign: (-1)^(number of outer axes)."""
    return [b for b in range(1 << dims) if (-1) ** bin(b).count("1") == sign]


def positivized(fetch, xs32, u_pos, u_neg, background=0.0):
    """Two-tap positivized estimate of the Catmull-Rom filter (Section 2.2,
    "Positivization"; Appendix B): <F> = W+ t(j+) - W- t(j-), where W+ and W- are the
    sums of the positive and of the absolute negative weights and j+ / j- are drawn
    from each set with probability proportional to |w|.

    Reading for separable cubic weights with signs (-, +, +, -) on each axis: the
    2^D blocks "inner (taps 1, 2) or outer (taps 0, 3) on each axis" partition the
    taps by sign (an even number of outer axes is positive).  A set is sampled by
    choosing one of its blocks with probability proportional to its mass (variate
    u[D]), then on each axis a tap of the block's pair with probability proportional
    to |w| (variate u[a]).  Decisions in float64 as for `stochastic`; the negative
    sample is skipped when W- is zero.  u_pos / u_neg: lists of D + 1 variates.
    Returns (value, positive tap indices, negative tap indices, exempt, finite)."""
    D = len(xs32)
    N = np.asarray(xs32[0]).shape[0]
    frames = [axis_frame(x) for x in xs32]
    finite = np.logical_and.reduce([fin for (_, _, fin) in frames])
    w64 = [axis_weights(f, "catmull_rom") for (_, f, _) in frames]
    m64 = _block_masses(w64, D)
    exempt = np.zeros(N, dtype=bool)
    out = {}
    with np.errstate(invalid="ignore", divide="ignore"):   # empty sets (W = 0) are unused
        for sign, u in ((1, u_pos), (-1, u_neg)):
            out[sign] = _sample_set(D, sign, u, w64, m64, frames, exempt)
    Wp, ip = out[1]
    Wn, ineg = out[-1]
    val = Wp[:, None] * fetch(*ip)
    neg = Wn > 0
    if np.any(neg):
        tn = fetch(*ineg)
        val = val - np.where(neg, Wn, 0.0)[:, None] * tn
    val[~finite] = background
    return val, ip, ineg, exempt & finite, finite


def _sample_set(D, sign, u, w64, m64, frames, exempt):
    """One sign's block and per-axis taps (see `positivized`); updates exempt."""
    blocks = _blocks_of_sign(D, sign)
    Wb = np.stack([m64[b] for b in blocks])
    W = np.sum(Wb, axis=0)
    # block choice: inverse CDF over the set's blocks in increasing order, float64
    C = np.cumsum(Wb, axis=0)
    us = np.asarray(u[D], dtype=np.float64) * C[-1]
    kb = np.sum(us[None, :] >= C[:-1], axis=0)
    chosen = np.asarray(blocks)[kb]
    interior = C[:-1] / np.where(W > 0, W, 1)
    exempt |= (W > 0) & (np.min(np.abs(np.asarray(u[D])[None, :] - interior), axis=0) < EXEMPT)
    idx = []
    for a in range(D):
        outer = (chosen >> a) & 1
        pair = np.where(outer[None, :] == 1, w64[a][[0, 3]], w64[a][[1, 2]])
        k, _ = select_tap(u[a], pair)
        exempt |= (W > 0) & (boundary_distance(u[a], pair) < EXEMPT)
        tap = np.where(outer == 1, np.where(k == 0, 0, 3), np.where(k == 0, 1, 2))
        idx.append(frames[a][0] - 1 + tap)
    return W, idx


def positivized_expectation(fetch, xs32):
    """Exact expectation of `positivized` by enumerating both sets' blocks and taps:
    sum over positive (block, taps) of p * W+ t  minus  the same over negative ones."""
    D = len(xs32)
    frames = [axis_frame(x) for x in xs32]
    w64 = [axis_weights(f, "catmull_rom") for (_, f, _) in frames]
    m64 = _block_masses(w64, D)
    total = 0.0
    for sign in (1, -1):
        blocks = _blocks_of_sign(D, sign)
        W = np.sum([m64[b] for b in blocks], axis=0)
        for b in blocks:
            pb = np.where(W > 0, m64[b] / np.where(W > 0, W, 1), 0.0)
            pairs = [((0, 3) if (b >> a) & 1 else (1, 2)) for a in range(D)]
            for combo in itertools.product((0, 1), repeat=D):
                p = pb.copy()
                idx = []
                for a in range(D):
                    t0, t1 = pairs[a]
                    tap = (t0, t1)[combo[a]]
                    s = np.abs(w64[a][t0]) + np.abs(w64[a][t1])
                    p = p * np.where(s > 0, np.abs(w64[a][tap]) / np.where(s > 0, s, 1), 0.0)
                    idx.append(frames[a][0] - 1 + tap)
                total = total + (sign * p * W)[:, None] * fetch(*idx)
    return total


# ---------------------------------------------------------------- texture wrappers

def _level_choice(lod32, nlev, level_mode, u_level, stochastic_form):
    """Per-query level(s): returns (L0, L1, frac weight of L1, exempt)."""
    N = lod32.shape[0]
    zero = np.zeros(N, dtype=np.int64)
    if lod32 is None or nlev == 1:
        return zero, zero, np.zeros(N), np.zeros(N, dtype=bool)
    lod = np.clip(np.nan_to_num(lod32.astype(np.float32), nan=0.0),
                  np.float32(0), np.float32(nlev - 1)).astype(np.float32)
    lod = lod.astype(np.float64)
    if level_mode == LEVEL_NEAREST:
        h = lod + 0.5                                   # exact in float64
        L = np.minimum(np.floor(h).astype(np.int64), nlev - 1)
        exempt = np.abs(h - np.round(h)) < EXEMPT
        return L, L, np.zeros(N), exempt
    L0 = np.floor(lod).astype(np.int64)
    a = lod - np.floor(lod)
    if stochastic_form:
        s = lod + np.asarray(u_level, dtype=np.float64)  # exact: both are short binary fractions
        L = np.minimum(np.floor(s).astype(np.int64), nlev - 1)
        frac_to_boundary = np.abs(a - (1.0 - u_level))
        exempt = (frac_to_boundary < EXEMPT) & (L0 < nlev - 1)
        return L, L, np.zeros(N), exempt
    L1 = np.minimum(L0 + 1, nlev - 1)
    return L0, L1, a, np.zeros(N, dtype=bool)


def _raster(uv32, tex, L):
    W = np.array([tex.size(l)[0] for l in range(len(tex.levels))], dtype=np.float32)[L]
    H = np.array([tex.size(l)[1] for l in range(len(tex.levels))], dtype=np.float32)[L]
    x = ((uv32[:, 0] * W).astype(np.float32) - np.float32(0.5)).astype(np.float32)
    y = ((uv32[:, 1] * H).astype(np.float32) - np.float32(0.5)).astype(np.float32)
    return x, y


def _fis_streams(qid, sample_index, seed, filt):
    return [query_variates(qid, sample_index, seed, stream=j) for j in range(fis.STREAMS[filt])]


def lookup_2d(tex, uv, lod, filt, *, stochastic_form, level_mode=LEVEL_STOCHASTIC,
              qid=None, sample_index=0, seed=0, reuse=False, width=None):
    """2D (MIP-mapped) lookup.  Returns (values (N, C), taps (N, 4) int, exempt).
    width: the Gaussian's sigma in texels of the chosen level (fis_gaussian)."""
    uv32 = np.asarray(uv, dtype=np.float32).reshape(-1, 2)
    N = uv32.shape[0]
    lod32 = None if lod is None else np.asarray(lod, dtype=np.float32)
    nlev = len(tex.levels)
    if qid is None:
        qid = np.arange(N, dtype=np.uint64)
    u = query_variates(qid, sample_index, seed)
    bad_lod = np.zeros(N, dtype=bool) if lod32 is None else ~np.isfinite(lod32)
    lod_in = np.zeros(N, dtype=np.float32) if lod32 is None else lod32
    L0, L1, a, exempt = _level_choice(lod_in, nlev if lod32 is not None else 1,
                                      level_mode, u[3], stochastic_form)
    taps = np.zeros((N, 4), dtype=np.int64)
    if stochastic_form and filt == "catmull_rom_positivized":
        x, y = _raster(uv32, tex, L0)
        u1 = query_variates(qid, sample_index, seed, stream=1)
        val, idx, _, ex, fin = positivized(lambda ix, iy: tex.fetch(L0, ix, iy), [x, y],
                                           [u[0], u[1], u[2]], [u1[0], u1[1], u1[2]])
        fin &= ~bad_lod
        val[~fin] = 0.0
        taps[:, 0], taps[:, 1], taps[:, 3] = idx[0], idx[1], L0
        taps[~fin] = (0, 0, 0, -1)
        return val, taps, (exempt | ex) & fin
    if stochastic_form and filt.startswith("fis_"):
        x, y = _raster(uv32, tex, L0)
        val, idx, ex, fin = fis.stochastic(lambda ix, iy: tex.fetch(L0, ix, iy), [x, y], filt,
                                           _fis_streams(qid, sample_index, seed, filt), width)
        fin &= ~bad_lod
        val[~fin] = 0.0
        taps[:, 0], taps[:, 1], taps[:, 3] = idx[0], idx[1], L0
        taps[~fin] = (0, 0, 0, -1)
        return val, taps, (exempt | ex) & fin
    if filt == "catmull_rom_positivized":
        filt = "catmull_rom"          # the deterministic twin is the Catmull-Rom filter
    if filt.startswith("fis_"):
        filt = fis.FIS_TWIN[filt]     # the filter that FIS applies
    if filt == "gaussian":
        det = lambda L, xs: fis.deterministic_gaussian(lambda ix, iy: tex.fetch(L, ix, iy), xs, width)
    else:
        det = lambda L, xs: deterministic(lambda ix, iy: tex.fetch(L, ix, iy), xs, filt)
    if stochastic_form:
        x, y = _raster(uv32, tex, L0)
        val, idx, ex, fin = stochastic(lambda ix, iy: tex.fetch(L0, ix, iy), [x, y], filt,
                                       [u[0], u[1]], reuse)
        fin &= ~bad_lod
        val[~fin] = 0.0
        taps[:, 0], taps[:, 1], taps[:, 3] = idx[0], idx[1], L0
        taps[~fin] = (0, 0, 0, -1)
        return val, taps, (exempt | ex) & fin
    x0, y0 = _raster(uv32, tex, L0)
    v0 = det(L0, [x0, y0])
    x1, y1 = _raster(uv32, tex, L1)
    v1 = det(L1, [x1, y1])
    val = (1.0 - a)[:, None] * v0 + a[:, None] * v1
    val[bad_lod] = 0.0
    return val, None, None


def lookup_3d(grid, p, filt, *, stochastic_form, qid=None, sample_index=0, seed=0,
              reuse=False, width=None):
    """3D lookup in index space (dense or sparse grid)."""
    p32 = np.asarray(p, dtype=np.float32).reshape(-1, 3)
    N = p32.shape[0]
    xs = [p32[:, 0], p32[:, 1], p32[:, 2]]
    if filt.startswith("fis_"):
        if not stochastic_form:
            twin = fis.FIS_TWIN[filt]
            if twin == "gaussian":
                return fis.deterministic_gaussian(grid.fetch, xs, width, grid.background), None, None
            return deterministic(grid.fetch, xs, twin, grid.background), None, None
        if qid is None:
            qid = np.arange(N, dtype=np.uint64)
        val, idx, ex, fin = fis.stochastic(grid.fetch, xs, filt,
                                           _fis_streams(qid, sample_index, seed, filt), width,
                                           grid.background)
        taps = np.zeros((N, 4), dtype=np.int64)
        taps[:, 0], taps[:, 1], taps[:, 2] = idx
        taps[~fin] = (0, 0, 0, -1)
        return val, taps, ex & fin
    if filt == "catmull_rom_positivized":
        if not stochastic_form:
            return deterministic(grid.fetch, xs, "catmull_rom", grid.background), None, None
        if qid is None:
            qid = np.arange(N, dtype=np.uint64)
        u0 = query_variates(qid, sample_index, seed, stream=0)
        u1 = query_variates(qid, sample_index, seed, stream=1)
        val, idx, _, ex, fin = positivized(grid.fetch, xs, [u0[0], u0[1], u0[2], u0[3]],
                                           [u1[0], u1[1], u1[2], u1[3]], grid.background)
        taps = np.zeros((N, 4), dtype=np.int64)
        taps[:, 0], taps[:, 1], taps[:, 2] = idx
        taps[~fin] = (0, 0, 0, -1)
        return val, taps, ex & fin
    if not stochastic_form:
        return deterministic(grid.fetch, xs, filt, grid.background), None, None
    if qid is None:
        qid = np.arange(N, dtype=np.uint64)
    u = query_variates(qid, sample_index, seed)
    val, idx, ex, fin = stochastic(grid.fetch, xs, filt, [u[0], u[1], u[2]], reuse,
                                   grid.background)
    taps = np.zeros((N, 4), dtype=np.int64)
    taps[:, 0], taps[:, 1], taps[:, 2] = idx
    taps[~fin] = (0, 0, 0, -1)
    return val, taps, ex & fin
