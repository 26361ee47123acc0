"""Comparison helpers shared by the GPU parity tests (no arithmetic of the method lives here)."""
import numpy as np

# FP64 gate: per output component array, max_x |y - y_ref| <= TOL_F64 * max_x |y_ref|
# (pointwise relative error with the array's own maximum as the floor: Gamma and nabla beta cancel to
# ~0 at some points, where only an absolute error relative to the component's scale is meaningful).
TOL_F64 = 1e-12

OUT_NAMES = (["ginv%d" % p for p in range(6)] + ["gamma%d_%d" % (i, p) for i in range(3) for p in range(6)] +
             ["dbcov%d%d" % (i, j) for i in range(3) for j in range(3)] + ["dtg%d" % p for p in range(6)])
IN_NAMES = (["g%d" % p for p in range(6)] + ["dg%d_%d" % (p, k) for p in range(6) for k in range(3)] +
            ["K%d" % p for p in range(6)] + ["alpha"] + ["beta%d" % i for i in range(3)] +
            ["dbeta%d%d" % (i, j) for i in range(3) for j in range(3)])


def component_errors(y, y_ref):
    """Per-row normwise relative error max|y - y_ref| / max|y_ref| (absolute error where the row of
    y_ref is identically zero)."""
    y = np.asarray(y, dtype=np.float64)
    y_ref = np.asarray(y_ref, dtype=np.float64)
    assert y.shape == y_ref.shape
    if y.shape[-1] == 0:
        return np.zeros(y.shape[0])
    diff = np.abs(y - y_ref).max(axis=1)
    scale = np.abs(y_ref).max(axis=1)
    return np.where(scale > 0, diff / np.where(scale > 0, scale, 1.0), diff)


def pointwise_floor_errors(y, y_ref, floor_frac):
    """max_x |y - y_ref| / max(|y_ref(x)|, floor_frac * max|y_ref|) per row (a stricter view)."""
    y = np.asarray(y, dtype=np.float64)
    y_ref = np.asarray(y_ref, dtype=np.float64)
    scale = np.abs(y_ref).max(axis=1, keepdims=True)
    den = np.maximum(np.abs(y_ref), floor_frac * scale)
    den = np.where(den > 0, den, 1.0)
    return (np.abs(y - y_ref) / den).max(axis=1)


# Pointwise view: |y(x) - y_ref(x)| / max(|y_ref(x)|, POINTWISE_FLOOR * max|y_ref|) per component.  At
# points where a component cancels to below the floor only an error relative to the component's scale
# is attainable (the summands that cancel are of that scale, and each carries its own rounding), so
# the bound is the relative error allowed at the floor: binary64 results carry errors of a few units in
# the last place of the summands (~1e-16 of the scale), i.e. ~1e-10 at the floor; float-float pairs
# (48 significant bits) ~1e-14 of the scale, i.e. ~1e-8.  The bounds below leave a factor ~10-100.
POINTWISE_FLOOR = 1e-6
POINTWISE_F64 = 1e-8
POINTWISE_FF = 1e-6


def assert_pointwise(y, y_ref, bound, names=OUT_NAMES, what=""):
    errs = pointwise_floor_errors(y, y_ref, POINTWISE_FLOOR)
    bad = [(names[c], float(errs[c])) for c in range(len(errs)) if not errs[c] <= bound]
    assert not bad, "%s pointwise (floor %.0e of the component maximum) over %.1e: %s" % (
        what, POINTWISE_FLOOR, bound, bad[:8])
    return errs


def assert_components(y, y_ref, tol, names=OUT_NAMES, what=""):
    errs = component_errors(y, y_ref)
    bad = [(names[c], float(errs[c])) for c in range(len(errs)) if not errs[c] <= tol]
    assert not bad, "%s components over %.1e: %s" % (what, tol, bad[:8])
    return errs
