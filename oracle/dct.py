"""DCT-compressed 2D textures and stochastic triplanar mapping, float64 (test
infrastructure only).

Section 5.2, "Texture compression": each 8x8 block of texels stores, per channel, the
six lowest-frequency coefficients of its 2D DCT in 32 bits: 7 bits for the DC
coefficient and 5 bits for each of the other five (16x compression of 8-bit
texels).  Stochastic filtering decodes one texel per lookup instead of every tap.

Readings (the paper gives the bit budget and nothing else):

* Transform: the orthonormal 8-point DCT-II per axis,
  F(u, v) = a(u) a(v) sum_{x,y} f(x, y) cos((2x+1) u pi / 16) cos((2y+1) v pi / 16),
  a(0) = sqrt(1/8), a(k > 0) = 1/2, u along x.  The kept coefficients are those with
  u + v <= 2 (the first six of the zig-zag order), stored in the order
  (0,0), (1,0), (0,1), (2,0), (1,1), (0,2).
* Texel values lie in [0, 1] (8-bit data).  DC = 8 * block mean lies in [0, 8]: code
  round(DC * 127 / 8) clamped to [0, 127], decoded as code * 8 / 127.
* AC: symmetric codes in [-15, 15] on [-R_c, R_c], R_c = the largest |AC| of channel
  c over all blocks of all levels (one float per channel kept with the texture):
  code round(AC * 15 / R_c), decoded as code * R_c / 15.  R_c below 2^-20 (a channel
  without detail, whose AC values are rounding noise) is taken as 0: all AC codes 0.
  Rounding is half away from zero.
* Packing: bits 0-6 the DC code, bits 7+5j .. 11+5j AC code j (j = 0..4) as a 5-bit
  two's complement.  Storage [level][block y][block x][channel], one uint32 each.
* Blocks of a level of W_L x H_L texels: ceil(W_L / 8) x ceil(H_L / 8); texels beyond
  the level's edge are copies of the nearest edge texel (clamp) before the
  transform.  Levels: the 2x2 box pyramid of the uncompressed level 0, each level
  compressed on its own.
* Decoding texel (x, y) of a block: f = sum_k F_k a(u_k) cos((2x+1) u_k pi/16)
  a(v_k) cos((2y+1) v_k pi/16) over the six kept coefficients.

Triplanar mapping (Section 5.2, "Triplanar mapping"; Eq. 3): a query at position p
with unit normal n blends three lookups of one texture at uv = s (p_y, p_z),
s (p_x, p_z), s (p_x, p_y) (planes YZ, XZ, XY) with weights |n_x|, |n_y|, |n_z| divided
by their sum.  The stochastic form draws one plane with probability equal to its
weight (inverse CDF in float64 over the planes in that order, word 2 of the
query's stream 0) and filters that plane's lookup stochastically; the
deterministic form blends the three deterministic lookups.
"""
import math

import numpy as np

KEPT = ((0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2))
DC_STEPS = 127
AC_STEPS = 15


def basis_1d():
    """c[u][x] = a(u) cos((2x+1) u pi / 16), u = 0..2, x = 0..7 (float64)."""
    c = np.zeros((3, 8))
    for u in range(3):
        a = math.sqrt(1 / 8) if u == 0 else 0.5
        for x in range(8):
            c[u, x] = a * math.cos((2 * x + 1) * u * math.pi / 16)
    return c


def forward(block):
    """The six kept coefficients of an (8, 8, C) block indexed [y][x][c], float64."""
    c = basis_1d()
    b = np.asarray(block, dtype=np.float64)
    return np.stack([np.einsum("yxc,x,y->c", b, c[u], c[v]) for (u, v) in KEPT])   # (6, C)


def _round_half_away(x):
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def blocks_of(level):
    """(BH, BW, 8, 8, C) blocks of an (H, W, C) level, edge texels repeated."""
    H, W, C = level.shape
    BH, BW = -(-H // 8), -(-W // 8)
    ys = np.minimum(np.arange(BH * 8), H - 1)
    xs = np.minimum(np.arange(BW * 8), W - 1)
    full = np.asarray(level, dtype=np.float64)[ys][:, xs]
    return full.reshape(BH, 8, BW, 8, C).transpose(0, 2, 1, 3, 4)


def coefficients(levels):
    """Per level: (BH, BW, 6, C) float64 coefficients."""
    out = []
    for lv in levels:
        bl = blocks_of(lv)
        BH, BW = bl.shape[:2]
        co = np.zeros((BH, BW, 6, lv.shape[2]))
        c = basis_1d()
        for k, (u, v) in enumerate(KEPT):
            co[:, :, k, :] = np.einsum("abyxc,x,y->abc", bl, c[u], c[v])
        out.append(co)
    return out


def encode(levels):
    """Codes (list of (BH, BW, C) uint32 arrays), AC ranges R (C,), and the distance
    (in code units) of every quantised value to a rounding boundary (list of
    (BH, BW, C) arrays: the smallest over the block's six coefficients)."""
    co = coefficients(levels)
    C = levels[0].shape[2]
    R = np.zeros(C)
    for cl in co:
        R = np.maximum(R, np.max(np.abs(cl[:, :, 1:, :]), axis=(0, 1, 2)))
    R = np.where(R < 2.0 ** -20, 0.0, R)
    codes, margins = [], []
    for cl in co:
        dc = cl[:, :, 0, :] * DC_STEPS / 8.0
        q_dc = np.clip(_round_half_away(dc), 0, DC_STEPS)
        with np.errstate(divide="ignore", invalid="ignore"):
            ac = np.where(R > 0, cl[:, :, 1:, :] * AC_STEPS / np.where(R > 0, R, 1), 0.0)
        q_ac = np.clip(_round_half_away(ac), -AC_STEPS, AC_STEPS)
        word = q_dc.astype(np.uint64)
        for j in range(5):
            word |= ((q_ac[:, :, j, :].astype(np.int64) & 31).astype(np.uint64) << np.uint64(7 + 5 * j))
        codes.append(word.astype(np.uint32))
        dist = lambda v: np.abs(np.abs(v - np.floor(v)) - 0.5)
        m = np.minimum(dist(dc), np.min(dist(ac), axis=2))
        margins.append(m)
    return codes, R, margins


def unpack(word):
    """(6,) + shape integer codes of packed words."""
    w = np.asarray(word, dtype=np.int64)
    dc = w & 127
    acs = []
    for j in range(5):
        a = (w >> (7 + 5 * j)) & 31
        acs.append(np.where(a >= 16, a - 32, a))
    return np.stack([dc] + acs)


def dequantise(word, R):
    """Coefficient values of packed words; R broadcasts over the channel axis."""
    q = unpack(word).astype(np.float64)
    out = np.empty_like(q)
    out[0] = q[0] * 8.0 / DC_STEPS
    out[1:] = q[1:] * (np.asarray(R, dtype=np.float64) / AC_STEPS)
    return out


class DCTTexture2D:
    """Compressed texel store with the same fetch interface as textures.Texture2D."""

    def __init__(self, levels_f64):
        self.sizes = [(lv.shape[1], lv.shape[0]) for lv in levels_f64]
        self.C = levels_f64[0].shape[2]
        self.codes, self.R, self.margins = encode(levels_f64)
        self.levels = [np.zeros((1, 1, self.C))] * len(levels_f64)   # shape info only
        self.c = basis_1d()

    def size(self, level):
        """(width, height) of a level."""
        return self.sizes[level]

    def fetch(self, level, ix, iy):
        """Decoded texels (N, C) at clamped (ix, iy) of level(s)."""
        level = np.broadcast_to(np.asarray(level), np.shape(ix))
        out = np.zeros((np.size(ix), self.C))
        ix = np.asarray(ix).ravel()
        iy = np.asarray(iy).ravel()
        level = np.asarray(level).ravel()
        for L in np.unique(level):
            sel = level == L
            W, H = self.sizes[L]
            x = np.clip(ix[sel], 0, W - 1)
            y = np.clip(iy[sel], 0, H - 1)
            words = self.codes[L][y >> 3, x >> 3]                    # (n, C)
            F = dequantise(words, self.R)                            # (6, n, C)
            val = np.zeros((len(x), self.C))
            for k, (u, v) in enumerate(KEPT):
                val += F[k] * (self.c[u, x & 7] * self.c[v, y & 7])[:, None]
            out[sel] = val
        return out

    def exempt_texels(self, level, ix, iy, tol=1e-9):
        """Texels whose block holds a coefficient within tol (code units) of a
        rounding boundary: an independent float64 encoder may round it the other way."""
        W, H = self.sizes[level]
        x = np.clip(ix, 0, W - 1)
        y = np.clip(iy, 0, H - 1)
        return np.min(self.margins[level][y >> 3, x >> 3], axis=-1) < tol


def triplanar_planes(p, n, scale):
    """uv of the three planes (YZ, XZ, XY) and their weights, float32 uv and float64
    weights; returns (uvs list of (N, 2) float32, w (3, N) float64, w32 (3, N) float32)."""
    p32 = np.asarray(p, dtype=np.float32)
    s = np.float32(scale)
    uvs = [np.stack([(p32[:, 1] * s), (p32[:, 2] * s)], axis=1).astype(np.float32),
           np.stack([(p32[:, 0] * s), (p32[:, 2] * s)], axis=1).astype(np.float32),
           np.stack([(p32[:, 0] * s), (p32[:, 1] * s)], axis=1).astype(np.float32)]
    a = np.abs(np.asarray(n, dtype=np.float32)).T                   # (3, N) float32
    return uvs, a.astype(np.float64), a


def choose_plane(a32, u):
    """Inverse CDF over |n_x|, |n_y|, |n_z| in float64: the number of the first two
    running sums that are <= u * S.  Returns (plane, exempt: u within 1e-6 of a
    boundary, where a float32 evaluation may decide otherwise)."""
    A = np.asarray(a32, dtype=np.float64)
    c0 = A[0]
    c1 = A[0] + A[1]
    S = c1 + A[2]
    us = np.asarray(u, dtype=np.float64) * S
    k = (us >= c0).astype(np.int64) + (us >= c1).astype(np.int64)
    with np.errstate(divide="ignore", invalid="ignore"):
        d = np.minimum(np.abs(u - c0 / S), np.abs(u - c1 / S))
    return k, d < 1e-6


def lookup_triplanar(tex, p, n, scale, lod, filt, *, stochastic_form, level_mode=1, seed=0,
                     sample_index=0, qid=None, width=None):
    """Triplanar lookups of a 2D texture (plain or DCT).  Returns (values (N, C),
    taps (N, 4) with the plane in the z slot, exempt) or (values, None, None)."""
    from . import filters
    from .philox import query_variates
    N = np.asarray(p).shape[0]
    if qid is None:
        qid = np.arange(N, dtype=np.uint64)
    uvs, A, a32 = triplanar_planes(p, n, scale)
    finite = np.all(np.isfinite(np.asarray(p, dtype=np.float32)), axis=1) & \
        np.all(np.isfinite(np.asarray(n, dtype=np.float32)), axis=1) & (np.sum(A, axis=0) > 0)
    if not stochastic_form:
        S = np.sum(A, axis=0)
        val = 0.0
        for k in range(3):
            v, _, _ = filters.lookup_2d(tex, uvs[k], lod, filt, stochastic_form=False,
                                        level_mode=level_mode, width=width)
            with np.errstate(invalid="ignore", divide="ignore"):
                val = val + (A[k] / S)[:, None] * v
        val = np.where(finite[:, None], val, 0.0)
        return val, None, None
    u = query_variates(qid, sample_index, seed)
    k, ex_plane = choose_plane(a32, u[2])
    k = np.where(finite, k, 0)
    uv = np.take_along_axis(np.stack(uvs), k[None, :, None].repeat(2, axis=2), axis=0)[0]
    val, taps, ex = filters.lookup_2d(tex, uv, lod, filt, stochastic_form=True, level_mode=level_mode,
                                      qid=qid, sample_index=sample_index, seed=seed, width=width)
    taps[:, 2] = np.where(taps[:, 3] >= 0, k, taps[:, 2])
    val[~finite] = 0.0
    taps[~finite] = (0, 0, 0, -1)
    return val, taps, (ex | ex_plane) & finite
