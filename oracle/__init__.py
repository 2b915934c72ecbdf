"""Plain float64 CPU oracle for stochastic texture filtering.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or link
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA library.

Modules (each cites the passage of the paper it follows):

* ``philox``   -- counter-based generator for the variates xi (Section 2.2).
* ``kernels``  -- the 1D filter kernels of Appendix A.
* ``codecs``   -- binary16 and E4M3 storage formats.
* ``textures`` -- texel stores: 2D MIP pyramids, dense and sparse 3D grids.
* ``filters``  -- deterministic (Eq. 2, Eq. 9) and stochastic (Eq. 3, sampling
  arrays of Section 2.2) lookups, positivization, and the exact expectation by
  enumeration.
* ``fis``      -- filter importance sampling (Section 4.4): B-splines by sums of
  uniforms, the Gaussian by Box-Muller, nearest-texel lookup.
* ``ewa``      -- anisotropic level of detail and (stochastic) EWA filtering
  (Sections 4.2, 5.2; Appendix B).
* ``dct``      -- DCT-compressed textures and stochastic triplanar mapping
  (Section 5.2).
* ``mlp``      -- float64 forward and backward of the neural-texture decoder.
* ``neural``   -- neural-texture lookups (latent fetch + decoder).

Every function is pinned by a test in ``tests/test_oracle_*.py`` against something
other than itself (closed forms, brute force, an independent library, or a value
the paper prints).
"""
from . import philox, kernels, codecs, textures, fis, filters, ewa, dct  # noqa: F401
