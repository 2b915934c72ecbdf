"""Neural texture for the oracle (test infrastructure only): a pyramid whose first
levels hold latent texels decoded by the MLP of ``oracle.mlp`` and whose remaining
levels hold stored texels (the fallback).  It exposes the same ``levels`` /
``size`` / ``fetch`` interface as ``textures.Texture2D``, so ``filters.lookup_2d``
filters it unchanged: the stochastic form decodes the one latent texel it picks
(Eq. 3), the deterministic form decodes every tap and weights the decoded values
(filtering after decoding, as Section 5.2 describes for compressed textures).
"""
import numpy as np

from . import mlp


class NeuralTexture2D:
    """Neural texture: latent levels decoded by the MLP, then stored fallback levels.
    `fetch` returns decoded texels for latent levels and stored texels above them."""

    def __init__(self, latents, params, fallback=()):
        self.latents = [np.asarray(l, dtype=np.float64) for l in latents]
        self.fallback = [np.asarray(f, dtype=np.float64) for f in fallback]
        self.P = {k: np.asarray(v, dtype=np.float64) for k, v in params.items()}
        self.levels = self.latents + self.fallback
        self.channels = self.P["W3"].shape[1]

    def size(self, level):
        """(width, height) of a level."""
        h, w = self.levels[level].shape[:2]
        return w, h

    def decode(self, Z):
        """Decoder output for latent rows Z."""
        return mlp.forward(Z, self.P)[0]

    def fetch(self, level, ix, iy):
        """Texels (N, 7) at clamped (ix, iy) of level(s)."""
        level = np.asarray(level, dtype=np.int64)
        ix = np.asarray(ix, dtype=np.int64)
        iy = np.asarray(iy, dtype=np.int64)
        out = np.zeros((ix.shape[0], self.channels))
        nl = len(self.latents)
        for L in np.unique(level):
            m = level == L
            h, w = self.levels[L].shape[:2]
            cx, cy = np.clip(ix[m], 0, w - 1), np.clip(iy[m], 0, h - 1)
            if L < nl:
                out[m] = self.decode(self.latents[L][cy, cx])
            else:
                out[m] = self.fallback[L - nl][cy, cx][:, :self.channels]
        return out
