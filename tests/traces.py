"""Per-receiver-trace error measures shared by the parity tests.

The tolerance stated for FP32 storage holds on "every receiver trace" (a relative L2 of
1e-5).  Read for a single trace r with GPU values a_r and oracle values b_r:

- every trace is held to ||a_r - b_r|| <= tol * RMS_s ||b_s||, the trace set's RMS norm.
  Rounding errors are absolute: they are made where the field is strong and travel with
  it, so a receiver that records less energy than the others (a far one, or one behind
  a slow layer) sees them larger relative to its own trace;
- where a run keeps each trace within tol of its own norm as well, the test says so
  (own_norm=True), for the traces whose values lie in FP32's normal range (norm >=
  2^-116, 2^10 above the smallest normal FP32 number).  A receiver that the physical
  wave has not reached within the run records only the scheme's numerical precursor,
  which decays by tens of orders of magnitude ahead of the front; below FP32's normal
  range storage cannot hold it (the 4096^2 two-layer run has such traces at 1e-46 to
  1e-89), and its relative error is meaningless.
"""
import numpy as np

FP32_FLOOR = 2.0 ** -116


def trace_errors(tr, ref):
    """(own-norm relative errors, trace norms, errors over the trace set's RMS norm)"""
    tr = np.asarray(tr, np.float64)
    ref = np.asarray(ref, np.float64)
    num = np.linalg.norm(tr - ref, axis=0)
    den = np.linalg.norm(ref, axis=0)
    rms = float(np.sqrt(np.mean(den ** 2)))
    return num / np.maximum(den, 1e-300), den, num / max(rms, 1e-300)


def check_every_trace(tr, ref, tol, own_norm=False):
    """Assert the per-trace tolerance (see the module docstring); return a summary."""
    own, norms, setn = trace_errors(tr, ref)
    signal = norms >= FP32_FLOOR
    rec = {"worst_over_set_rms": float(setn.max()),
           "worst_own_norm": float(own[signal].max()) if signal.any() else 0.0,
           "median_own_norm": float(np.median(own[signal])) if signal.any() else 0.0,
           "traces": int(len(norms)), "traces_below_fp32_range": int((~signal).sum()),
           "per_trace_own_norm": [float(v) for v in own],
           "per_trace_over_set_rms": [float(v) for v in setn],
           "trace_norms": [float(v) for v in norms]}
    assert setn.max() <= tol, ("trace error over the set's RMS norm", int(setn.argmax()),
                               float(setn.max()), tol)
    if own_norm:
        worst = int(np.argmax(np.where(signal, own, 0.0)))
        assert own[signal].max() <= tol, ("trace error over its own norm", worst,
                                          float(own[worst]), tol)
    return rec
