"""Anisotropic level of detail and stochastic EWA filtering, float64 (test
infrastructure only).

* Anisotropic level of detail (Section 5.2, "Anisotropic filtering and
  minification"; the anisotropic LOD listing of Appendix B).  A lookup's footprint
  is the ellipse spanned by the texture-coordinate derivatives along the two screen
  axes.  In level-0 texels the axes are d_x = (du/dx W, dv/dx H) and
  d_y = (du/dy W, dv/dy H); the longer one is the major axis.  When the minor axis is
  more than max_anisotropy times shorter than the major one it is lengthened to
  major / max_anisotropy, and lod = log2(minor length).  The lookup then picks one
  level around lod (stochastic: floor(lod + u); deterministic: blend of floor(lod)
  and the next level), as the other 2D lookups do.

* EWA (Greene and Heckbert; Section 4.2 and the stochastic EWA listing of
  Appendix B, which samples pbrt's EWA filter).  At level L with axes d0, d1 in
  that level's texels, the filter is a Gaussian over the ellipse
  Q(s, t) = A s^2 + B s t + C t^2 < 1 around the lookup's raster position, where
  (A, B, C) / F is the inverse of the covariance d0 d0^T + d1 d1^T + I (the identity
  adds a one-texel reconstruction filter):
      A = d0.v^2 + d1.v^2 + 1,  B = -2 (d0.u d0.v + d1.u d1.v),  C = d0.u^2 + d1.u^2 + 1,
      F = A C - B^2 / 4.
  Texel (s, t) carries weight LUT(Q): the table of exp(-alpha r) - exp(-alpha),
  alpha = 2, on r = i / (LUT_SIZE - 1), indexed by min(floor(Q LUT_SIZE),
  LUT_SIZE - 1) (the paper's EWA filter reads pbrt's Gaussian table; the paper does
  not print it, and this is the table's documented definition).  The deterministic
  filter is sum(w t) / sum(w) over the texels of the ellipse's bounding box; the
  stochastic one returns one texel drawn with probability w / sum(w).

Precision.  Every quantity and decision here is float64, from the definitions above:
the footprint, the level, the ellipse, Q, the table index and weight, the running
sums and the inverse-CDF choice.  Beside each float64 quantity the oracle carries a
bound on how far any float32 evaluation of the same formula can be from it (running
error analysis: one correctly rounded operation adds at most 2^-24 of its result,
plus an absolute 2^-149 for subnormal results; a sum or product of a few terms is
bounded for every evaluation order and with or without fused multiply-adds).  A
decision that such a float32 evaluation could take otherwise is reported: the
level when the bounded lod reaches a level boundary, a texel's weight when its
bounded Q reaches a table boundary, and the stochastic texel when some weights
within their bounds, plus float32 rounding of the running sums, could move the
inverse-CDF choice.  The stochastic lookup marks those queries exempt; the
deterministic one returns a tolerance that covers them.

The 2D raster position u W_L - 1/2 is taken as float32 (two correctly rounded
operations, exact for power-of-two sizes except below half a texel): it is the
query's coordinate in the level's raster, the input from which every decision
starts.

Readings: (i) the stochastic draw is the inverse CDF over the texels in row-major
order (rows t ascending, then s ascending), smallest k with u S < C_k, rather than the
listing's one-pass reservoir update; the two give the same distribution, and the
inverse CDF keeps the chosen texel a pure function of u.  (ii) A footprint larger
than the coarsest level (lod above the top level) is shrunk at the chosen level so
that its minor axis is 2 texels, which keeps the ellipse bounded; the coarsest level
then covers the footprint.  (iii) Variates: word 0 of stream 0 picks the texel,
word 3 the level.
"""
import math
from collections import namedtuple

import numpy as np

LUT_SIZE = 128
ALPHA = 2.0
F32 = np.float32
EXEMPT = 1e-6                 # the parity rule's band around every CDF boundary

U = 2.0 ** -24                # float32 unit roundoff
SUB = 2.0 ** -149             # absolute allowance per operation (subnormal results)
REF = 2.0 ** -50              # relative allowance for float64's own rounding
LOG2_ULPS = 2.0               # twice the documented maximum error of CUDA's log2f
FLT_MAX = float(np.finfo(np.float32).max)


def weight_lut():
    """exp(-alpha r) - exp(-alpha) at r = i / (LUT_SIZE - 1), float64."""
    r = np.arange(LUT_SIZE, dtype=np.float64) / (LUT_SIZE - 1)
    return np.exp(-ALPHA * r) - np.exp(-ALPHA)


# --------------------------------------------------------------- bounded arithmetic
# A bounded number is (v, e): v the float64 value of the exact formula, e a bound on
# |x32 - v| for a float32 evaluation x32 of the same formula.

def _rounded(v, prop):
    a = np.abs(v)
    return prop + U * (a + prop) + SUB + REF * a


def exact(v):
    v = np.asarray(v, dtype=np.float64)
    return v, np.zeros_like(v)


def bmul(x, y):
    (xv, xe), (yv, ye) = x, y
    v = xv * yv
    return v, _rounded(v, np.abs(xv) * ye + np.abs(yv) * xe + xe * ye)


def badd(x, y):
    v = x[0] + y[0]
    return v, _rounded(v, x[1] + y[1])


def bneg(x):
    return -x[0], x[1]


def bpow2(x, c):
    """Multiplication by a power of two (exact in float32 barring range limits)."""
    return x[0] * c, x[1] * abs(c) + SUB


def bdiv(x, y):
    (xv, xe), (yv, ye) = x, y
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        v = xv / yv
        den = np.abs(yv) - ye
        prop = np.where(den > 0, (xe + np.abs(v) * ye) / np.where(den > 0, den, 1.0), np.inf)
    return v, _rounded(v, prop)


def bsqrt(x):
    xv, xe = x
    v = np.sqrt(np.maximum(xv, 0.0))
    lo = np.sqrt(np.maximum(xv - xe, 0.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        prop = np.minimum(np.where(v + lo > 0, xe / np.where(v + lo > 0, v + lo, 1.0), np.inf),
                          np.sqrt(xe))
    return v, _rounded(v, prop)


def bselect(cond, amb, x_true, x_false):
    """A float64 branch: the taken side's value; where a float32 evaluation could take
    the other side (amb), the bound also covers that side's value."""
    v = np.where(cond, x_true[0], x_false[0])
    e = np.where(cond, x_true[1], x_false[1])
    other = np.where(cond, x_false[0], x_true[0])
    oe = np.where(cond, x_false[1], x_true[1])
    return v, np.where(amb, np.maximum(e, np.abs(other - v) + oe), e)


def _less_amb(x, y):
    """x < y in float64, and whether float32 evaluations could order them otherwise."""
    return x[0] < y[0], np.abs(x[0] - y[0]) <= x[1] + y[1]


def blog2(x):
    """log2 with its bound as an interval (lo, hi); -inf allowed below."""
    xv, xe = x
    with np.errstate(divide="ignore", invalid="ignore"):
        v = np.log2(xv)
        lo = np.log2(np.maximum(xv - xe, 0.0))
        hi = np.log2(xv + xe)
    slack = lambda z: LOG2_ULPS * U * 2 * np.where(np.isfinite(z), np.abs(z), 0.0) + 2.0 ** -60
    return v, lo - slack(lo), hi + slack(hi)


# --------------------------------------------------------------- footprint and LOD

Footprint = namedtuple("Footprint", "major minor lod lod_lo lod_hi finite ambiguous")


def footprint(W, H, grad, max_anisotropy):
    """Per query (float64, arrays of N): the major axis (Mx, My) and the minor axis
    after the anisotropy limit (mx, my), in uv units, each a bounded pair (v, e); lod =
    log2(minor length in level-0 texels) with the interval [lod_lo, lod_hi] a float32
    evaluation stays in; `finite` (input derivatives finite and squared lengths within
    float32 range); `ambiguous` (float32 evaluations could disagree on which clamped
    axis the footprint has, which the bounds do not cover)."""
    g = np.asarray(grad, dtype=np.float32).astype(np.float64).reshape(-1, 4)
    with np.errstate(over="ignore", invalid="ignore"):
        ax = bmul(exact(g[:, 0]), exact(float(W)))
        ay = bmul(exact(g[:, 1]), exact(float(H)))
        bx = bmul(exact(g[:, 2]), exact(float(W)))
        by = bmul(exact(g[:, 3]), exact(float(H)))
        la = badd(bmul(ax, ax), bmul(ay, ay))
        lb = badd(bmul(bx, bx), bmul(by, by))
    finite = np.all(np.isfinite(g), axis=1) & (la[0] + la[1] < FLT_MAX) & (lb[0] + lb[1] < FLT_MAX)
    over_amb = np.all(np.isfinite(g), axis=1) & ~finite & \
        ((la[0] - la[1] < FLT_MAX * (1 - 4 * U)) & (lb[0] - lb[1] < FLT_MAX * (1 - 4 * U)))
    swap, swap_amb = _less_amb(la, lb)
    lmaj = (np.where(swap, lb[0], la[0]), np.where(swap, lb[1], la[1]))
    lmin = (np.where(swap, la[0], lb[0]), np.where(swap, la[1], lb[1]))
    major = bsqrt(lmaj)
    minor = bsqrt(lmin)
    Mx, My = exact(np.where(swap, g[:, 2], g[:, 0])), exact(np.where(swap, g[:, 3], g[:, 1]))
    mx, my = exact(np.where(swap, g[:, 0], g[:, 2])), exact(np.where(swap, g[:, 1], g[:, 3]))
    ma = exact(float(np.float32(max_anisotropy)))
    mm = bmul(minor, ma)
    lt, lt_amb = _less_amb(mm, major)
    pos = minor[0] > 0
    pos_amb = minor[0] <= minor[1]
    clamp = pos & lt
    clamp_amb = (pos & lt_amb) | (pos_amb & lt)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        scale = bdiv(major, mm)
        scale = (np.where(clamp | clamp_amb, scale[0], 1.0), np.where(clamp | clamp_amb, scale[1], 0.0))
        mx = bselect(clamp, clamp_amb, bmul(mx, scale), mx)
        my = bselect(clamp, clamp_amb, bmul(my, scale), my)
        minor = bselect(clamp, clamp_amb, bmul(minor, scale), minor)
    # Swapped labels give the same ellipse (it is symmetric in d0 and d1); they matter
    # only through the anisotropy limit, which then must not apply either way.
    ambiguous = (swap_amb & (clamp | clamp_amb)) | over_amb
    lod, lod_lo, lod_hi = blog2(minor)
    return Footprint((Mx, My), (mx, my), lod, lod_lo, lod_hi, finite & ~ambiguous, ambiguous)


def footprint_finite(W, H, grad):
    """Derivatives finite, with squared lengths in texels within float32 range (others
    are treated like non-finite input: background)."""
    fp = footprint(W, H, grad, 1.0)
    return fp.finite | fp.ambiguous


# --------------------------------------------------------------- ellipse at a level

def level_axes(WL, HL, fp, q):
    """Axes of query q at a level of WL x HL texels, in that level's texels, with the
    oversize shrink (reading ii): bounded (d0u, d0v, d1u, d1v)."""
    (Mx, My), (mx, my) = fp.major, fp.minor
    sel = lambda p: (p[0][q], p[1][q])
    d0u, d0v = bmul(sel(Mx), exact(float(WL))), bmul(sel(My), exact(float(HL)))
    d1u, d1v = bmul(sel(mx), exact(float(WL))), bmul(sel(my), exact(float(HL)))
    m = bsqrt(badd(bmul(d1u, d1u), bmul(d1v, d1v)))
    big, big_amb = _less_amb(exact(2.0), m)
    k = bdiv(exact(2.0), m) if m[0] > 0 else exact(1.0)
    return tuple(bselect(big, big_amb, bmul(d, k), d) for d in (d0u, d0v, d1u, d1v))


def ellipse(d0u, d0v, d1u, d1v):
    """Normalised (A, B, C) and the bounding-box half extents (hs, ht), each a
    bounded pair.  Arguments are bounded pairs or plain numbers (taken as exact)."""
    d0u, d0v, d1u, d1v = (d if isinstance(d, tuple) else exact(float(d)) for d in (d0u, d0v, d1u, d1v))
    one = exact(1.0)
    A = badd(badd(bmul(d0v, d0v), bmul(d1v, d1v)), one)
    B = bpow2(badd(bmul(d0u, d0v), bmul(d1u, d1v)), -2.0)
    C = badd(badd(bmul(d0u, d0u), bmul(d1u, d1u)), one)
    F = badd(bmul(A, C), bneg(bpow2(bmul(B, B), 0.25)))
    inv = bdiv(one, F)
    A, B, C = bmul(A, inv), bmul(B, inv), bmul(C, inv)
    det = badd(bpow2(bmul(A, C), 4.0), bneg(bmul(B, B)))
    inv_det = bdiv(one, det)
    hs = bmul(bpow2(inv_det, 2.0), bsqrt(bmul(det, C)))
    ht = bmul(bpow2(inv_det, 2.0), bsqrt(bmul(A, det)))
    return A, B, C, hs, ht


def raster(uv, WL, HL):
    """Raster position u W_L - 1/2 as float32, clamped to +-2^24 texels as in the other
    2D lookups."""
    lim = F32(1 << 24)
    st_s = np.clip(F32(F32(F32(uv[0]) * F32(WL)) - F32(0.5)), -lim, lim)
    st_t = np.clip(F32(F32(F32(uv[1]) * F32(HL)) - F32(0.5)), -lim, lim)
    return float(st_s), float(st_t)


def _box_range(c, h):
    """Integer range [ceil(c - h), floor(c + h)] in float64, and the wider range a
    float32 evaluation of the two ends could produce."""
    lo, hi = c - h[0], c + h[0]
    dlo = h[1] + U * (abs(lo) + h[1]) + SUB
    dhi = h[1] + U * (abs(hi) + h[1]) + SUB
    nominal = (math.ceil(lo), math.floor(hi))
    widest = (math.ceil(lo - dlo), math.floor(hi + dhi))
    surest = (math.ceil(lo + dlo), math.floor(hi - dhi))
    return nominal, widest, surest


def texels_and_weights(st_s, st_t, ell):
    """The texels a float32 evaluation may visit (row-major: t, then s) with their
    float64 weights w (0 outside the float64 box or ellipse) and bounds [lo, hi] on
    the weight a float32 evaluation gives them (its table entries rounded to float32,
    its Q within the derived bound, its box ends possibly one texel off)."""
    A, B, C, hs, ht = ell
    (s_nom, s_wide, s_sure), (t_nom, t_wide, t_sure) = _box_range(st_s, hs), _box_range(st_t, ht)
    assert s_wide[1] - s_wide[0] < 4096 and t_wide[1] - t_wide[0] < 4096
    si = np.arange(s_wide[0], s_wide[1] + 1)
    ti = np.arange(t_wide[0], t_wide[1] + 1)
    tt, ss = np.meshgrid(ti - st_t, si - st_s, indexing="ij")        # (rows t, cols s)
    Q = A[0] * ss * ss + B[0] * ss * tt + C[0] * tt * tt
    T = abs(A[0]) * ss * ss + abs(B[0]) * np.abs(ss * tt) + abs(C[0]) * tt * tt
    # coefficient errors, the float32 differences ss = s - st_s and tt = t - st_t
    # (2 U relative each, entering squared or as a product), and at most four roundings
    # along any evaluation order of the three-term form
    eQ = A[1] * ss * ss + B[1] * np.abs(ss * tt) + C[1] * tt * tt + (2 * U + 4 * U / (1 - 4 * U)) * T
    # a texel index beyond 2^24 is not a float32 number: its conversion adds up to
    # U |i| to ss or tt before the subtraction (raster positions clamped near +-2^24)
    es = np.where(np.abs(si) > (1 << 24), U * np.abs(si), 0.0)[None, :]
    et = np.where(np.abs(ti) > (1 << 24), U * np.abs(ti), 0.0)[:, None]
    aA, aB, aC = abs(A[0]), abs(B[0]), abs(C[0])
    eQ = eQ + (2 * aA * np.abs(ss) + aB * np.abs(tt)) * es + (aB * np.abs(ss) + 2 * aC * np.abs(tt)) * et \
        + aA * es * es + aB * es * et + aC * et * et
    eQ = eQ * (1 + 1e-6) + 4 * SUB
    lut = weight_lut()

    def weight(q):
        idx = np.clip(np.floor(q * LUT_SIZE), 0, LUT_SIZE - 1).astype(np.int64)
        return np.where(q < 1.0, lut[idx], 0.0)

    w = weight(Q)
    lo = weight(Q + eQ) * (1 - 2 * U)    # the table decreases with Q; float32 entries
    hi = weight(np.maximum(Q - eQ, 0.0)) * (1 + 2 * U)
    in_s = (si >= s_nom[0]) & (si <= s_nom[1])
    in_t = (ti >= t_nom[0]) & (ti <= t_nom[1])
    sure_s = (si >= s_sure[0]) & (si <= s_sure[1])
    sure_t = (ti >= t_sure[0]) & (ti <= t_sure[1])
    w = np.where(in_t[:, None] & in_s[None, :], w, 0.0)
    lo = np.where(sure_t[:, None] & sure_s[None, :], lo, 0.0)
    S, Tm = np.meshgrid(si, ti)
    return S.reshape(-1), Tm.reshape(-1), w.reshape(-1), lo.reshape(-1), hi.reshape(-1)


def select(w, u):
    """Smallest k with u S < C_k over the float64 running sums of w, and the float64
    distance of u to the nearest interior boundary C_k / S."""
    Cs = np.cumsum(w)
    S = Cs[-1]
    us = u * S
    k = int(np.argmax(us < Cs))
    interior = Cs[:-1][w[:-1] > 0] / S
    d = float(np.min(np.abs(u - interior))) if interior.size else 1.0
    return k, d


def choice_uncertain(w, lo, hi, u, k):
    """Whether a float32 evaluation, its weights anywhere in [lo, hi] and its running
    sums and u S rounded in float32, could choose another texel than k.  The kernel
    keeps k iff u S' < C'_k and u S' >= C'_{k-1}; both sides are linear in the
    weights, so their extremes over the box are taken term by term."""
    n = len(w)
    g = n * U / (1 - n * U)
    margin = (2 * g + 2 * U) * np.sum(hi) + 2 * SUB * n
    j = np.arange(n)
    upper = np.sum(np.where(j <= k, (u - 1.0) * lo, u * hi))        # max of u S' - C'_k
    if upper + margin >= 0:
        return True
    if k > 0:
        lower = np.sum(np.where(j <= k - 1, (u - 1.0) * hi, u * lo))  # min of u S' - C'_{k-1}
        if lower - margin < 0:
            return True
    return False


def deterministic_bound(w, lo, hi, tv, R):
    """Bound on |R' - R| for a float32 evaluation of sum(w t) / sum(w): weights within
    [lo, hi], and float32 running sums of w and w t."""
    n = max(int(np.sum(hi > 0)), 1)
    g = n * U / (1 - n * U)
    d = np.maximum(hi - w, w - lo)
    S_lo = np.sum(lo) * (1 - g)
    if S_lo <= 0:
        return np.full(tv.shape[1], np.inf)
    tmax = np.max(np.abs(tv), axis=0) if len(tv) else np.zeros(tv.shape[1])
    weights = np.sum(d[:, None] * (np.abs(tv) + np.abs(R)[None, :]), axis=0) / S_lo
    sums = (2 * g + 3 * U) * (tmax + np.abs(R)) * (1 + g)
    return weights + sums


# --------------------------------------------------------------- level choice

def _levels(fp, q, nlev, level_mode, u_level, stochastic_form):
    """Level(s) of query q: (L0, L1, frac of L1, e_frac, ambiguous)."""
    if nlev == 1:
        return 0, 0, 0.0, 0.0, False
    clampl = lambda z: min(max(float(z), 0.0), float(nlev - 1))
    lc, lc_lo, lc_hi = clampl(fp.lod[q]), clampl(fp.lod_lo[q]), clampl(fp.lod_hi[q])
    if stochastic_form or level_mode == 0:
        off = 0.5 if level_mode == 0 else float(u_level)
        s, s_lo, s_hi = lc + off, lc_lo + off, lc_hi + off
        s_lo -= U * abs(s_lo)
        s_hi += U * abs(s_hi)
        pick = lambda z: min(int(math.floor(z)), nlev - 1)
        L = pick(s)
        return L, L, 0.0, 0.0, pick(s_lo) != pick(s_hi)
    L0 = int(math.floor(lc))
    amb = int(math.floor(lc_lo)) != int(math.floor(lc_hi))
    return L0, min(L0 + 1, nlev - 1), lc - L0, (lc_hi - lc_lo) + U, amb


# --------------------------------------------------------------- lookups

def lookup(tex, uv, grad, max_anisotropy, *, stochastic_form, level_mode=1, qid=None,
           sample_index=0, seed=0):
    """EWA lookups.  Stochastic form: (values (N, C) float64, taps (N, 4) int64
    (s, t, 0, level), exempt (N,) bool).  Deterministic form: (values, None, tol (N,)
    float64: the derived bound on a float32 evaluation's deviation, inf where a level
    boundary is within reach)."""
    from .philox import query_variates
    uv32 = np.asarray(uv, dtype=np.float32).reshape(-1, 2)
    g32 = np.asarray(grad, dtype=np.float32).reshape(-1, 4)
    N = uv32.shape[0]
    nlev = len(tex.levels)
    C = tex.levels[0].shape[2]
    W0, H0 = tex.size(0)
    if qid is None:
        qid = np.arange(N, dtype=np.uint64)
    u = query_variates(qid, sample_index, seed)
    fp = footprint(W0, H0, g32, max_anisotropy)
    val = np.zeros((N, C))
    taps = np.zeros((N, 4), dtype=np.int64)
    exempt = np.zeros(N, dtype=bool)
    tol = np.zeros(N)
    ok = np.all(np.isfinite(uv32), axis=1) & fp.finite
    for q in range(N):
        if not ok[q]:
            taps[q] = (0, 0, 0, -1)
            exempt[q] = fp.ambiguous[q]
            tol[q] = np.inf if fp.ambiguous[q] else 0.0
            continue
        L0, L1, frac, e_frac, amb = _levels(fp, q, nlev, level_mode, u[3][q], stochastic_form)
        if stochastic_form:
            ell, st = _ellipse_at(tex, L0, fp, q, uv32[q])
            s, t, w, lo, hi = texels_and_weights(st[0], st[1], ell)
            k, d = select(w, u[0][q])
            exempt[q] = amb or d < EXEMPT or choice_uncertain(w, lo, hi, u[0][q], k)
            taps[q] = (s[k], t[k], 0, L0)
            val[q] = tex.fetch(np.array([L0]), np.array([s[k]]), np.array([t[k]]))[0]
            continue
        parts = [(L0, 1.0 - frac)] if frac == 0.0 else [(L0, 1.0 - frac), (L1, frac)]
        Rs = []
        for L, wl in parts:
            ell, st = _ellipse_at(tex, L, fp, q, uv32[q])
            s, t, w, lo, hi = texels_and_weights(st[0], st[1], ell)
            texv = tex.fetch(np.full(len(s), L), s, t)
            R = (w[:, None] * texv).sum(axis=0) / w.sum()
            Rs.append(R)
            val[q] += wl * R
            tol[q] += wl * np.max(deterministic_bound(w, lo, hi, texv, R))
        if len(Rs) == 2:
            tol[q] += e_frac * np.max(np.abs(Rs[1] - Rs[0]))
        tol[q] = 2 * tol[q] + U * np.max(np.abs(val[q]))
        if amb:
            tol[q] = np.inf
    if not stochastic_form:
        return val, None, tol
    return val, taps, exempt & ok


def _ellipse_at(tex, L, fp, q, uvq):
    WL, HL = tex.size(L)
    return ellipse(*level_axes(WL, HL, fp, q)), raster(uvq, WL, HL)


def expectation(tex, uv, grad, max_anisotropy, level_mode=1, seed=0, sample_index=0):
    """Exact expectation of the stochastic EWA lookup over the texel draw (the level
    fixed by the query's level variate): sum_k (w_k / S) t_k."""
    from .philox import query_variates
    uv32 = np.asarray(uv, dtype=np.float32).reshape(-1, 2)
    g32 = np.asarray(grad, dtype=np.float32).reshape(-1, 4)
    N = uv32.shape[0]
    nlev = len(tex.levels)
    W0, H0 = tex.size(0)
    u = query_variates(np.arange(N, dtype=np.uint64), sample_index, seed)
    fp = footprint(W0, H0, g32, max_anisotropy)
    out = np.zeros((N, tex.levels[0].shape[2]))
    for q in range(N):
        L, _, _, _, _ = _levels(fp, q, nlev, level_mode, u[3][q], True)
        ell, st = _ellipse_at(tex, L, fp, q, uv32[q])
        s, t, w, _, _ = texels_and_weights(st[0], st[1], ell)
        out[q] = ((w / w.sum())[:, None] * tex.fetch(np.full(len(s), L), s, t)).sum(axis=0)
    return out


def texel_count(tex, uv, grad, max_anisotropy, level_mode=1):
    """Weighted texels per query at the levels the deterministic filter visits (the
    largest of its two levels)."""
    uv32 = np.asarray(uv, dtype=np.float32).reshape(-1, 2)
    g32 = np.asarray(grad, dtype=np.float32).reshape(-1, 4)
    W0, H0 = tex.size(0)
    fp = footprint(W0, H0, g32, max_anisotropy)
    ok = np.all(np.isfinite(uv32), axis=1) & fp.finite
    out = np.zeros(uv32.shape[0], dtype=np.int64)
    for q in np.nonzero(ok)[0]:
        L0, L1, frac, _, _ = _levels(fp, q, len(tex.levels), level_mode, 0.0, False)
        for L in ({L0, L1} if frac > 0 else {L0}):
            ell, st = _ellipse_at(tex, L, fp, q, uv32[q])
            out[q] = max(out[q], int(np.sum(texels_and_weights(st[0], st[1], ell)[2] > 0)))
    return out
