"""Per-layer error checks shared by the GPU parity tests.

Two per-layer figures are asserted beside the overall relative L2 error:

* the layer's error relative to the RMS of the whole output, <= tol;
* the layer's error relative to its OWN RMS, <= tol * min(OWN_CAP, max(1,
  RMS_all / RMS_l)).  A layer's spectrum b_l = sum_g B_lg d_g carries the
  rounding of the shared star spectra d_g, whose size is set by the strong
  layers, so a weak layer may see up to RMS_all / RMS_l times the relative
  rounding of a strong one.  The cap (10) keeps the bound tight enough that a
  weak layer computed wrongly (an error of the order of its own RMS) fails.
  Layers whose RMS is below OWN_FLOOR * RMS_all (values at rounding level,
  e.g. in degenerate plans) are not checked on their own.
"""
import numpy as np

OWN_CAP = 10.0
OWN_FLOOR = 1e-6


def rel_errors(got, ref):
    """(overall, per layer relative to the whole RMS, per layer relative to its own RMS)."""
    diff = got - ref
    overall = np.linalg.norm(diff) / np.linalg.norm(ref)
    scale = np.sqrt(np.mean(ref ** 2))
    rms_l = np.sqrt(np.mean(ref ** 2, axis=(1, 2)))
    err_l = np.sqrt(np.mean(diff ** 2, axis=(1, 2)))
    per_layer = err_l / scale
    own = err_l / np.where(rms_l > 0, rms_l, 1.0)
    return overall, per_layer, own


def own_bounds(ref, tol):
    """Bound on each layer's error relative to its own RMS, and the mask of the
    layers strong enough to be checked on their own."""
    scale = np.sqrt(np.mean(ref ** 2))
    rms_l = np.sqrt(np.mean(ref ** 2, axis=(1, 2)))
    checked = rms_l > OWN_FLOOR * scale
    ratio = np.where(checked, scale / np.where(rms_l > 0, rms_l, 1.0), 1.0)
    return tol * np.minimum(OWN_CAP, np.maximum(1.0, ratio)), checked


def assert_layers(got, ref, tol, what=""):
    overall, per_layer, own = rel_errors(got, ref)
    bound, checked = own_bounds(ref, tol)
    assert overall <= tol, (what, overall, per_layer)
    assert np.all(per_layer <= tol), (what, per_layer)
    bad = checked & (own > bound)
    assert not np.any(bad), (what, {"layers": np.nonzero(bad)[0].tolist(), "own": own[bad].tolist(),
                                    "bound": bound[bad].tolist()})
    return overall, per_layer, own
