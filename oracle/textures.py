"""Texel stores for the oracle (test infrastructure only).

The paper's texture function t is non-zero only at the discrete texel locations
(Section 2.1, Eq. 1); a filtered lookup reads t at integer raster positions.  The
paper fixes no addressing rule, so the readings used throughout are:

* 2D textures: clamp-to-edge addressing; MIP level L has size max(1, W >> L) by
  max(1, H >> L) and each of its texels is the mean of the level-0 texels it covers
  (a box-filtered pyramid, Section 2.1 "Minification").
* dense 3D grids: a voxel value sits at each integer index coordinate; positions
  outside the grid read the background value.
* sparse 3D grids: only active leaves (8x8x8 voxel blocks) store values; everything
  else reads the background value.  The oracle keeps the leaves in a plain
  key -> leaf map, deliberately not a tree.

All stored values are held as exact float64 copies of what the texture stores.
"""
import numpy as np


class Texture2D:
    """Levels: list of float64 arrays of shape (H_L, W_L, C)."""

    def __init__(self, levels):
        self.levels = [np.asarray(l, dtype=np.float64) for l in levels]
        self.channels = self.levels[0].shape[2]

    @staticmethod
    def box_pyramid(level0, num_levels):
        """Pyramid whose level L texel (x, y) is the mean of the level-0 block it
        covers; power-of-two sizes."""
        base = np.asarray(level0, dtype=np.float64)
        H, W, C = base.shape
        levels = [base]
        for L in range(1, num_levels):
            wl, hl = max(1, W >> L), max(1, H >> L)
            bx, by = W // wl, H // hl
            levels.append(base.reshape(hl, by, wl, bx, C).mean(axis=(1, 3)))
        return Texture2D(levels)

    def size(self, level):
        """(width, height) of a level."""
        h, w, _ = self.levels[level].shape
        return w, h

    def fetch(self, level, ix, iy):
        """Texel values (N, C) at integer positions, clamp-to-edge, per-query level."""
        level = np.asarray(level, dtype=np.int64)
        ix = np.asarray(ix, dtype=np.int64)
        iy = np.asarray(iy, dtype=np.int64)
        out = np.zeros((ix.shape[0], self.channels))
        for L in np.unique(level):
            m = level == L
            h, w, _ = self.levels[L].shape
            out[m] = self.levels[L][np.clip(iy[m], 0, h - 1), np.clip(ix[m], 0, w - 1)]
        return out


class Dense3D:
    """values: float64 array (Z, Y, X); value at integer (x, y, z)."""

    def __init__(self, values, background=0.0):
        self.values = np.asarray(values, dtype=np.float64)
        self.background = float(background)
        self.channels = 1

    def fetch(self, ix, iy, iz):
        """Values (N, 1) at integer voxel positions; the background outside."""
        Z, Y, X = self.values.shape
        ix, iy, iz = (np.asarray(a, dtype=np.int64) for a in (ix, iy, iz))
        inside = (ix >= 0) & (ix < X) & (iy >= 0) & (iy < Y) & (iz >= 0) & (iz < Z)
        out = np.full(ix.shape[0], self.background)
        out[inside] = self.values[iz[inside], iy[inside], ix[inside]]
        return out[:, None]


class Sparse3D:
    """Leaves: origins (L, 3) int (multiples of 8) and values (L, 8, 8, 8) indexed
    [x & 7, y & 7, z & 7] (float32 or float64, read exactly).  Lookup goes through a
    sorted key map."""

    OFF = 1 << 20

    def __init__(self, origins, leaf_values, background=0.0):
        origins = np.asarray(origins, dtype=np.int64).reshape(-1, 3)
        lv = np.asarray(leaf_values)
        if lv.dtype not in (np.float32, np.float64):
            lv = lv.astype(np.float64)
        self.values = lv.reshape(-1, 8, 8, 8)       # float32 leaves are kept as is (exact)
        keys = self._key(origins[:, 0] >> 3, origins[:, 1] >> 3, origins[:, 2] >> 3)
        order = np.argsort(keys, kind="stable")
        self.keys = keys[order]
        self.slot = order
        if len(self.keys) > 1 and np.any(np.diff(self.keys) == 0):
            raise ValueError("duplicate leaf origin")
        self.background = float(background)
        self.channels = 1

    def _key(self, kx, ky, kz):
        o = self.OFF
        return ((kx + o) << 42) | ((ky + o) << 21) | (kz + o)

    def fetch(self, ix, iy, iz):
        """Values (N, 1) at integer voxel positions; the background outside."""
        ix, iy, iz = (np.asarray(a, dtype=np.int64) for a in (ix, iy, iz))
        lim = self.OFF - 1
        ok = (np.abs(ix >> 3) < lim) & (np.abs(iy >> 3) < lim) & (np.abs(iz >> 3) < lim)
        key = self._key(np.where(ok, ix >> 3, 0), np.where(ok, iy >> 3, 0), np.where(ok, iz >> 3, 0))
        pos = np.searchsorted(self.keys, key)
        pos_c = np.minimum(pos, max(len(self.keys) - 1, 0))
        hit = ok & (len(self.keys) > 0) & (self.keys[pos_c] == key) if len(self.keys) else np.zeros_like(ok)
        out = np.full(ix.shape[0], self.background)
        if np.any(hit):
            leaf = self.slot[pos_c[hit]]
            out[hit] = self.values[leaf, ix[hit] & 7, iy[hit] & 7, iz[hit] & 7].astype(np.float64)
        return out[:, None]
