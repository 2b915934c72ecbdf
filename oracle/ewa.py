"""Anisotropic level of detail and stochastic EWA filtering (test infrastructure
only).

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

Precision.  pbrt computes this in float (float32), and the tap decision here is
taken in float32 as for the other filters: every step from the derivatives to the
table index and the running weight sum is a float32 operation in a fixed order, so
the choice is reproducible exactly by any float32 implementation of the same steps.
Expectations and deterministic sums are float64 over those float32 weights.

Readings: (i) the stochastic draw is the inverse CDF over the texels in row-major
order (rows t ascending, then s ascending), smallest k with u S < C_k, rather than the
listing's one-pass reservoir update; the two give the same distribution, and the
inverse CDF keeps the chosen texel a pure function of u.  (ii) A footprint larger
than the coarsest level (lod above the top level) is shrunk at the chosen level so
that its minor axis is 2 texels, which keeps the ellipse bounded; the coarsest level
then covers the footprint.  (iii) Variates: word 0 of stream 0 picks the texel,
word 3 the level.
"""
import numpy as np

LUT_SIZE = 128
ALPHA = 2.0
F32 = np.float32


def weight_lut():
    """exp(-alpha r) - exp(-alpha) at r = i / (LUT_SIZE - 1), rounded to float32."""
    r = np.arange(LUT_SIZE, dtype=np.float64) / (LUT_SIZE - 1)
    return (np.exp(-ALPHA * r) - np.exp(-ALPHA)).astype(np.float32)


def _f(x):
    return np.asarray(x, dtype=np.float32)


def _dot(ax, ay, bx, by):
    return _f(_f(ax * bx) + _f(ay * by))


def footprint(W, H, grad, max_anisotropy):
    """Per query: (major uv vector, minor uv vector after the anisotropy clamp, lod),
    float32.  grad: (N, 4) du/dx, dv/dx, du/dy, dv/dy in uv units."""
    with np.errstate(over="ignore", invalid="ignore"):
        return _footprint(W, H, grad, max_anisotropy)


def _footprint(W, H, grad, max_anisotropy):
    g = _f(grad)
    Wf, Hf = F32(W), F32(H)
    ax, ay = _f(g[:, 0]), _f(g[:, 1])         # d_x in uv
    bx, by = _f(g[:, 2]), _f(g[:, 3])         # d_y in uv
    la = _dot(_f(ax * Wf), _f(ay * Hf), _f(ax * Wf), _f(ay * Hf))
    lb = _dot(_f(bx * Wf), _f(by * Hf), _f(bx * Wf), _f(by * Hf))
    swap = la < lb                              # the longer axis is the major one
    Mx, My = np.where(swap, bx, ax), np.where(swap, by, ay)
    mx, my = np.where(swap, ax, bx), np.where(swap, ay, by)
    major = np.sqrt(np.where(swap, lb, la)).astype(np.float32)
    minor = np.sqrt(np.where(swap, la, lb)).astype(np.float32)
    ma = F32(max_anisotropy)
    clamp = (minor > 0) & (_f(minor * ma) < major)
    with np.errstate(divide="ignore", invalid="ignore"):
        scale = np.where(clamp, _f(major / _f(minor * ma)), F32(1))
    mx, my, minor = _f(mx * scale), _f(my * scale), _f(minor * scale)
    with np.errstate(divide="ignore"):
        lod = np.log2(minor).astype(np.float32)   # -inf for a zero footprint
    return (Mx, My), (mx, my), lod


def footprint_finite(W, H, grad):
    """Derivatives whose squared lengths in texels stay finite in float32 (others are
    treated like non-finite input: background)."""
    g = _f(grad)
    out = np.all(np.isfinite(g), axis=1)
    for a, b in ((0, 1), (2, 3)):
        with np.errstate(over="ignore", invalid="ignore"):
            l2 = _dot(_f(g[:, a] * F32(W)), _f(g[:, b] * F32(H)), _f(g[:, a] * F32(W)), _f(g[:, b] * F32(H)))
        out &= np.isfinite(l2)
    return out


def ellipse(d0u, d0v, d1u, d1v):
    """Normalised (A, B, C) and the bounding-box half extents, float32 steps."""
    A = _f(_f(_f(d0v * d0v) + _f(d1v * d1v)) + F32(1))
    B = _f(F32(-2) * _f(_f(d0u * d0v) + _f(d1u * d1v)))
    C = _f(_f(_f(d0u * d0u) + _f(d1u * d1u)) + F32(1))
    Fv = _f(_f(A * C) - _f(_f(B * B) * F32(0.25)))
    inv = _f(F32(1) / Fv)
    A, B, C = _f(A * inv), _f(B * inv), _f(C * inv)
    det = _f(_f(_f(F32(4) * A) * C) - _f(B * B))
    inv_det = _f(F32(1) / det)
    hs = _f(_f(F32(2) * inv_det) * np.sqrt(_f(det * C)).astype(np.float32))
    ht = _f(_f(F32(2) * inv_det) * np.sqrt(_f(A * det)).astype(np.float32))
    return A, B, C, hs, ht


def level_axes(tex, L, major, minor):
    """Axes at level L in that level's texels, with the oversize shrink (reading ii)."""
    WL = F32(tex.size(L)[0])
    HL = F32(tex.size(L)[1])
    d0u, d0v = _f(major[0] * WL), _f(major[1] * HL)
    d1u, d1v = _f(minor[0] * WL), _f(minor[1] * HL)
    m = np.sqrt(_dot(d1u, d1v, d1u, d1v)).astype(np.float32)
    big = m > F32(2)
    with np.errstate(divide="ignore", invalid="ignore"):
        k = np.where(big, _f(F32(2) / m), F32(1))
    return _f(d0u * k), _f(d0v * k), _f(d1u * k), _f(d1v * k)


def texels_and_weights(st_s, st_t, A, B, C, hs, ht):
    """For one query (scalars): the texels (s, t) of the bounding box in row-major
    order that carry positive weight, their float32 weights, and the float32 running
    sums."""
    lut = weight_lut()
    s0 = int(np.ceil(_f(st_s - hs)))
    assert np.ceil(_f(st_s + hs)) - s0 < 4096 and np.ceil(_f(st_t + ht)) - np.ceil(_f(st_t - ht)) < 4096
    s1 = int(np.floor(_f(st_s + hs)))
    t0 = int(np.ceil(_f(st_t - ht)))
    t1 = int(np.floor(_f(st_t + ht)))
    ss = _f(np.arange(s0, s1 + 1, dtype=np.float32) - st_s)
    out_s, out_t, out_w = [], [], []
    for it in range(t0, t1 + 1):
        tt = _f(F32(it) - st_t)
        # Q = (A ss + B tt) ss + C tt^2, each product and sum rounded to float32 in
        # this order; Q < 1 bounds the table index by LUT_SIZE - 1
        r2 = _f(_f(_f(_f(A * ss) + _f(B * tt)) * ss) + _f(C * _f(tt * tt)))
        inside = r2 < F32(1)
        idx = _f(r2 * F32(LUT_SIZE)).astype(np.int64)
        w = lut[np.clip(idx, 0, LUT_SIZE - 1)]
        keep = inside & (w > 0)
        out_s.append(np.arange(s0, s1 + 1)[keep])
        out_t.append(np.full(int(np.sum(keep)), it))
        out_w.append(w[keep])
    s = np.concatenate(out_s) if out_s else np.zeros(0, np.int64)
    t = np.concatenate(out_t) if out_t else np.zeros(0, np.int64)
    w = np.concatenate(out_w) if out_w else np.zeros(0, np.float32)
    csum = np.cumsum(w, dtype=np.float32)
    return s, t, w, csum


def select(w, csum, u):
    """Smallest k with fl(u S) < C_k (float32), and the float64 distance of u to the
    nearest interior boundary C_k / S."""
    S = csum[-1]
    us = _f(F32(u) * S)
    k = int(np.sum(csum[:-1] <= us))
    exact = np.cumsum(w.astype(np.float64))
    d = np.min(np.abs(u - exact[:-1] / exact[-1])) if len(w) > 1 else 1.0
    return k, d


def raster(uv, WL, HL):
    """Raster position u W_L - 1/2, clamped to +-2^24 texels as in the other 2D lookups."""
    lim = F32(1 << 24)
    st_s = np.clip(_f(_f(uv[0] * F32(WL)) - F32(0.5)), -lim, lim)
    st_t = np.clip(_f(_f(uv[1] * F32(HL)) - F32(0.5)), -lim, lim)
    return F32(st_s), F32(st_t)


EXEMPT_LEVEL = 4e-6     # log2 may differ by an ulp between float32 implementations


def _levels(lod, nlev, level_mode, u_level, stochastic_form):
    """Level(s) of one query from its float32 lod (as the other 2D lookups)."""
    lc = F32(min(max(float(lod), 0.0), float(nlev - 1)))     # lod is never NaN here
    if nlev == 1:
        return 0, 0, 0.0, False
    if level_mode == 0:                                  # nearest
        L = min(int(np.floor(_f(lc + F32(0.5)))), nlev - 1)
        return L, L, 0.0, abs((float(lc) + 0.5) - round(float(lc) + 0.5)) < EXEMPT_LEVEL
    L0 = int(np.floor(lc))
    frac = float(lc) - L0
    if stochastic_form:
        L = min(int(np.floor(_f(lc + F32(u_level)))), nlev - 1)
        ex = (L0 < nlev - 1) and abs(frac - (1.0 - u_level)) < EXEMPT_LEVEL
        return L, L, 0.0, ex
    return L0, min(L0 + 1, nlev - 1), frac, False


def lookup(tex, uv, grad, max_anisotropy, *, stochastic_form, level_mode=1, qid=None,
           sample_index=0, seed=0):
    """EWA lookups.  Returns (values (N, C) float64, taps (N, 4) int64 (s, t, 0, level),
    exempt (N,) bool); taps and exempt are None for the deterministic form."""
    from .philox import query_variates
    uv32 = _f(np.asarray(uv).reshape(-1, 2))
    g32 = _f(np.asarray(grad).reshape(-1, 4))
    N = uv32.shape[0]
    nlev = len(tex.levels)
    C = tex.levels[0].shape[2]
    W0, H0 = tex.size(0)
    if qid is None:
        qid = np.arange(N, dtype=np.uint64)
    u = query_variates(qid, sample_index, seed)
    major, minor, lod = footprint(W0, H0, g32, max_anisotropy)
    val = np.zeros((N, C))
    taps = np.zeros((N, 4), dtype=np.int64)
    exempt = np.zeros(N, dtype=bool)
    ok = np.all(np.isfinite(uv32), axis=1) & footprint_finite(W0, H0, g32)
    for q in range(N):
        if not ok[q]:
            taps[q] = (0, 0, 0, -1)
            continue
        L0, L1, frac, ex = _levels(lod[q], nlev, level_mode, u[3][q], stochastic_form)
        exempt[q] = ex
        parts = [(L0, 1.0 - frac)] if (stochastic_form or frac == 0.0) else [(L0, 1.0 - frac), (L1, frac)]
        for L, wl in parts:
            WL, HL = tex.size(L)
            st_s, st_t = raster(uv32[q], WL, HL)
            d0u, d0v, d1u, d1v = level_axes(tex, L, (major[0][q:q + 1], major[1][q:q + 1]),
                                            (minor[0][q:q + 1], minor[1][q:q + 1]))
            A, B, Cc, hs, ht = ellipse(d0u[0], d0v[0], d1u[0], d1v[0])
            s, t, w, csum = texels_and_weights(st_s, st_t, A, B, Cc, hs, ht)
            if stochastic_form:
                k, _ = select(w, csum, u[0][q])
                taps[q] = (s[k], t[k], 0, L)
                val[q] = tex.fetch(np.array([L]), np.array([s[k]]), np.array([t[k]]))[0]
            else:
                texv = tex.fetch(np.full(len(s), L), s, t)
                w64 = w.astype(np.float64)
                val[q] += wl * (w64[:, None] * texv).sum(axis=0) / w64.sum()
    if not stochastic_form:
        return val, None, None
    return val, taps, exempt & ok


def expectation(tex, uv, grad, max_anisotropy, level_mode=1, seed=0, sample_index=0):
    """Exact expectation of the stochastic EWA lookup over the texel draw (the level
    fixed by the query's level variate): sum_k (w_k / S) t_k."""
    from .philox import query_variates
    uv32 = _f(np.asarray(uv).reshape(-1, 2))
    g32 = _f(np.asarray(grad).reshape(-1, 4))
    N = uv32.shape[0]
    nlev = len(tex.levels)
    W0, H0 = tex.size(0)
    u = query_variates(np.arange(N, dtype=np.uint64), sample_index, seed)
    major, minor, lod = footprint(W0, H0, g32, max_anisotropy)
    out = np.zeros((N, tex.levels[0].shape[2]))
    for q in range(N):
        L, _, _, _ = _levels(lod[q], nlev, level_mode, u[3][q], True)
        WL, HL = tex.size(L)
        st_s, st_t = raster(uv32[q], WL, HL)
        d0u, d0v, d1u, d1v = level_axes(tex, L, (major[0][q:q + 1], major[1][q:q + 1]),
                                        (minor[0][q:q + 1], minor[1][q:q + 1]))
        A, B, Cc, hs, ht = ellipse(d0u[0], d0v[0], d1u[0], d1v[0])
        s, t, w, _ = texels_and_weights(st_s, st_t, A, B, Cc, hs, ht)
        w64 = w.astype(np.float64)
        out[q] = ((w64 / w64.sum())[:, None] * tex.fetch(np.full(len(s), L), s, t)).sum(axis=0)
    return out
