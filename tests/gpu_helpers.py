"""Helpers shared by the GPU parity tests: run the CUDA path through its C ABI
and compare with the oracle field by field.  Every comparison is also
recorded (test, what, achieved per-field errors, bound) in MARGINS, which the
session writes out as JSON when DGFV_PARITY_MARGINS names a file."""
import os

import numpy as np

from paper_2502_19342_gb300 import workloads as W

# Tolerance of R(U) and of RK states against the FP64 oracle, relative to the
# largest magnitude of each conserved field.
RTOL = 1e-12


def per_field(prob, x):
    off, _ = W.offsets(prob)
    V = W.n_vars(prob)
    n = W.points_per_dir(prob)
    out = [[] for _ in range(V)]
    for e in range(len(off)):
        m3 = int(n[e]) ** 3
        blk = x[off[e]:off[e] + V * m3].reshape(V, m3)
        for v in range(V):
            out[v].append(blk[v])
    return [np.concatenate(o) for o in out]


# A field's scale is the largest |R| of that field, but at least FLOOR times the
# largest |R| over all fields: the terms summed into every field are of the
# common flux-divergence magnitude, so a field whose R cancels to a small value
# (a momentum component in a nearly uniform flow) keeps the rounding error of
# those terms, not one relative to its own small result.
FLOOR = 1e-2


MARGINS = []


def record(what, errs, bound):
    """Keep one comparison's achieved errors and bound for the margin report."""
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    errs = [float(e) for e in np.atleast_1d(errs)]
    MARGINS.append(dict(test=test, what=what, max_err=max(errs), errs=errs, bound=float(bound)))


def field_errors(prob, got, ref):
    """max |got - ref| / scale for every conserved field (see FLOOR)."""
    g, r = per_field(prob, got), per_field(prob, ref)
    top = max(np.abs(b).max() for b in r)
    return [float(np.abs(a - b).max() / max(np.abs(b).max(), FLOOR * top, 1e-300)) for a, b in zip(g, r)]


def assert_fields_close(prob, got, ref, rtol=RTOL, what="R"):
    errs = field_errors(prob, got, ref)
    record(what, errs, rtol)
    assert np.isfinite(ref).all(), f"{what}: the reference is not finite"
    assert all(e <= rtol for e in errs), f"{what}: per-field relative errors {errs}"  # NaN fails too
    return errs


def assert_rhs_close(oracle, prob, U, got, factor=3.0):
    """R(U) of the CUDA path against the oracle evaluated in extended precision.

    Per field the bound is max(RTOL, factor * e), where e is the FP64 oracle's
    own largest per-field deviation from the extended-precision value on the
    same input: a high-order operator sums terms much larger than R, so 1e-12
    relative is at the FP64 rounding floor and a correct FP64 evaluation (the
    FP64 oracle itself) can sit above it.  The CUDA path must be as accurate
    as the FP64 oracle within `factor`."""
    ref = oracle.eval_rhs_extended(prob, U)
    assert np.isfinite(ref).all(), "the oracle's R is not finite on this input"
    own = field_errors(prob, oracle.eval_rhs(prob, U), ref)
    errs = field_errors(prob, got, ref)
    bound = [max(RTOL, factor * max(own))] * len(own)
    record("R", errs, bound[0])
    assert all(e <= b for e, b in zip(errs, bound)), f"R: per-field errors {errs}, bounds {bound}"
    return errs, own


def assert_adjoint_close(oracle, prob, U, Rbar, got, factor=3.0):
    """U_bar = R'(U)^T R_bar of the CUDA path against the oracle's adjoint by
    columns (one exact tangent per unit vector; tiny meshes), with the bar of
    R(U): per field max(RTOL, factor * e), e the FP64 oracle's own largest
    per-field deviation from its long-double evaluation."""
    ref = oracle.adjoint_columns(prob, U, Rbar, extended=True)
    assert np.isfinite(ref).all(), "the oracle's adjoint is not finite on this input"
    own = field_errors(prob, oracle.adjoint_columns(prob, U, Rbar), ref)
    errs = field_errors(prob, got, ref)
    bound = max(RTOL, factor * max(own))
    record("U_bar", errs, bound)
    assert all(e <= bound for e in errs), f"U_bar: per-field errors {errs}, bound {bound} (oracle's own {own})"
    return errs, own


def ctx_for(prob, opts=None, N_min=None, N_max=None):
    from paper_2502_19342_gb300 import dgfv
    return dgfv.Context(prob, N_min=N_min, N_max=N_max, opts=opts)


def to_dev(U):
    import torch
    return torch.from_numpy(np.ascontiguousarray(U, np.float64)).cuda()


def gpu_rhs(prob, U, **kw):
    ctx = ctx_for(prob, **kw)
    R = ctx.eval_rhs(to_dev(U)).cpu().numpy()
    ctx.close()
    return R
