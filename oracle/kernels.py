"""1D filter kernels of Appendix A ("Filter Kernels"), written from their piecewise
definitions in float64 (test infrastructure only).

* K0, the unit box (nearest neighbour).
* K1, the unit tent (linear interpolation).
* K3, the cubic family with free parameter a (Keys); a = -1/2 is Catmull-Rom.
  The paper leaves |t| = 1 and |t| = 2 unassigned; both pieces are zero there, so
  the first piece is taken on |t| <= 1 and the second on 1 < |t| < 2.
* Kbs, the cubic B-spline (Appendix A, "Convolutional").

Every function accepts scalars or arrays; the arithmetic runs in the dtype of ``t``
(float64 for values, float32 when the oracle takes a tap decision in the precision
of the paper's listings).
"""
import numpy as np


def k0_box(t):
    """Unit box K0 (Appendix A): 1 on |t| < 1/2, else 0."""
    t = np.asarray(t)
    return np.where(np.abs(t) < 0.5, t.dtype.type(1), t.dtype.type(0))


def k1_tent(t):
    """Unit tent K1 (Appendix A): 1 - |t| on |t| < 1, else 0."""
    t = np.asarray(t)
    a = np.abs(t)
    return np.where(a < 1, 1 - a, t.dtype.type(0))


def k3_cubic(t, a=-0.5):
    """Cubic K3 (Appendix A): (a+2)|t|^3 - (a+3)|t|^2 + 1 on |t| <= 1,
    a|t|^3 - 5a|t|^2 + 8a|t| - 4a on 1 < |t| < 2, else 0."""
    t = np.asarray(t)
    x = np.abs(t)
    a = t.dtype.type(a)
    inner = (a + 2) * x * x * x - (a + 3) * x * x + 1
    outer = a * x * x * x - 5 * a * x * x + 8 * a * x - 4 * a
    return np.where(x <= 1, inner, np.where(x < 2, outer, t.dtype.type(0)))


def k_bspline3(t):
    """Cubic B-spline K_bs (Appendix A, "Convolutional"): (4 - 6|t|^2 + 3|t|^3)/6
    on |t| <= 1, (2 - |t|)^3 / 6 on 1 < |t| <= 2, else 0."""
    t = np.asarray(t)
    x = np.abs(t)
    sixth = t.dtype.type(1) / 6
    inner = sixth * (4 - 3 * x * x * (2 - x))
    y = 2 - x
    outer = sixth * (y * y * y)
    return np.where(x <= 1, inner, np.where(x <= 2, outer, t.dtype.type(0)))


# Filter name -> (tap offsets relative to floor(x), kernel, kernel is non-negative)
FILTERS = {
    "linear": ((0, 1), k1_tent, True),
    "bspline3": ((-1, 0, 1, 2), k_bspline3, True),
    "catmull_rom": ((-1, 0, 1, 2), lambda t: k3_cubic(t, -0.5), False),
}
FILTER_IDS = {"linear": 0, "bspline3": 1, "catmull_rom": 2}
