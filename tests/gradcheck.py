"""Error metric of the adjoint tests: each gradient on its own scale.

For one instance, output k of (gq, gqd, gqdd) is measured as
    max_i |g_k,i - g*_k,i| / max(max_i |g*_k,i|, FLOOR * max_k,i |g*_k,i|)
and the error is the largest over the three outputs and the batch. A small
output is held to its own size, down to FLOOR of the instance's largest
gradient. The floor exists because one output can vanish identically. For
example, d tau / d qd of a single revolute joint is zero, and its computed
value is rounding noise of terms as large as the other outputs.
"""
import numpy as np

# An output smaller than 0.1% of the instance's largest gradient is measured
# against that 0.1%: at the FP32 bar it must then be right to 1e-6 of the
# largest gradient. Measured on each output's own scale, the FP32 errors stay
# below 2e-5 for chains of up to 128 links; the one output that vanishes
# identically (d tau / d qd of one joint) comes out zero to 1e-15 of the
# largest gradient.
FLOOR = 1e-3


def per_output_errors(g, ref, floor=FLOOR):
    """Per instance, the error of each output on its own floored scale.
    Returns an array [3, B]."""
    g = [np.asarray(x, dtype=np.float64) for x in g]
    ref = [np.asarray(x, dtype=np.float64) for x in ref]
    allmax = np.max(np.stack([np.max(np.abs(r), axis=1) for r in ref]), axis=0)
    errs = []
    for a, r in zip(g, ref):
        num = np.max(np.abs(a - r), axis=1)
        den = np.maximum(np.max(np.abs(r), axis=1), floor * allmax)
        errs.append(num / np.maximum(den, 1e-300))
    return np.stack(errs)


def grad_err(g, ref, floor=FLOOR):
    """Largest per-output error over the outputs and the batch."""
    return float(np.max(per_output_errors(g, ref, floor)))
