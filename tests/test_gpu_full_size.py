"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times (one launch per kernel over all degrees, autotuned volume
tiles, fused face values): the 48^3 turbulence case after one adaptation (the
decisions, the remapped state, R(U) and the time step), the 256 batched
domains, the 16^3 mixing layer and the 16^3 hp shock case; the adjoint on the
mixing layer and on a hybrid DG/FV hp shock pattern.

The FP64 oracle runs on the whole mesh (a few seconds on the host cores).  For
the two large cases the long-double evaluation that fixes the small cases'
bound is too slow on hosts whose long double is software quad precision, so
their bound comes from samples (see each test); for the turbulence case: on an 8^3-element mesh
with the same degree/FV distribution e = the FP64 oracle's own deviation from
its long-double evaluation; the CUDA path and the FP64 oracle may each sit 3e
(CUDA) and e (oracle) from the exact value, so they may differ by 4e, and never
by less than 2e-12."""
import numpy as np
import pytest

from paper_2502_19342_gb300 import workloads as W
from tests.gpu_helpers import RTOL, field_errors, record, to_dev

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _sample(prob, nel_s=8, seed=5):
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, len(prob["N"]), nel_s ** 3)
    L = prob["hi"][0] - prob["lo"][0]
    s = dict(prob)
    s["dims"] = np.array([[nel_s] * 3], np.int32)
    s["lo"] = prob["lo"][:1].copy()
    s["hi"] = (prob["lo"][0] + L * nel_s / prob["dims"][0]).reshape(1, 3)
    s["N"] = prob["N"][idx].copy()
    s["fv"] = prob["fv"][idx].copy()
    return s, W.smooth_random_state(s, seed, amp=0.05)


def _bound(oracle, prob):
    s, Us = _sample(prob)
    e = max(field_errors(s, oracle.eval_rhs(s, Us), oracle.eval_rhs_extended(s, Us)))
    return max(2 * RTOL, 4 * e)


def _rhs_parity(oracle, prob, U, ctx):
    R = ctx.eval_rhs(to_dev(U)).cpu().numpy()
    Ro = oracle.eval_rhs(prob, U)
    assert np.isfinite(Ro).all()
    errs = field_errors(prob, R, Ro)
    bound = _bound(oracle, prob)
    record("R full size", errs, bound)
    assert all(e <= bound for e in errs), f"R: per-field errors {errs}, bound {bound}"
    return errs


def test_turbulence_48_adapt_remap_rhs_dt(oracle):
    from paper_2502_19342_gb300 import dgfv
    thr = W.THRESHOLDS
    prob, U = W.turbulence(seed=0, nel=(48, 48, 48), N0=4)
    ctx = dgfv.Context(prob, N_min=1, N_max=7, opts=dict(cfl_c=0.5, cfl_v=0.5, thresholds=thr))
    ctx.set_state(to_dev(U))
    # the first adaptation of the benchmark: decisions and remap
    oIp, oIh = oracle.indicator(prob, U)
    Nn, fn = oracle.adapt_decide(prob, oIp, oIh, thr, 1, 7)
    near = np.zeros(len(Nn), bool)
    for T in thr:
        near |= (np.abs(oIp - T) < 1e-10) | (np.abs(oIh - T) < 1e-10)
    st = ctx.adapt()
    N, fv = ctx.get_degrees()
    differ = ((N != Nn) | (fv != fn)) & ~near
    assert not differ.any(), f"{differ.sum()} decisions differ outside the 1e-10 band"
    assert st["n_near"] == int(near.sum())
    assert (N != prob["N"]).sum() + (fv != prob["fv"]).sum() > 1000  # the step really adapts
    new = dict(prob, N=N, fv=fv)
    U1 = ctx.get_state().cpu().numpy()
    np.testing.assert_allclose(U1, oracle.remap(prob, N, fv, U), atol=1e-13, rtol=0)
    # R(U) and the time step in the benchmark's launch configuration
    ctx.autotune()
    _rhs_parity(oracle, new, U1, ctx)
    dt, dtc, dtv = ctx.compute_dt(to_dev(U1))
    rdt, rdtc, rdtv = oracle.dt(new, U1, 0.5, 0.5)
    assert abs(dtc - rdtc) <= 1e-14 * rdtc and abs(dtv - rdtv) <= 1e-14 * rdtv
    ctx.close()


def test_batched_domains_full(oracle):
    """The domains share no faces, so R of a domain alone is R of the batch
    restricted to it: on 12 sampled domains (every degree, up to 40k DOFs each)
    the batch's R from the CUDA path meets the small-case bar against the
    long-double oracle (3x the FP64 oracle's own error); on the whole batch it
    is within 4x the largest such own error of the FP64 oracle."""
    from paper_2502_19342_gb300 import dgfv
    prob, U = W.batched_domains()
    ctx = dgfv.Context(prob, N_min=1, N_max=7)
    ctx.set_state(to_dev(U))
    ctx.autotune()
    R = ctx.eval_rhs(to_dev(U)).cpu().numpy()
    ctx.close()
    rng = np.random.default_rng(7)
    doms = W.domain_slices(prob)
    picked, own = [], []
    for i in rng.permutation(len(doms)):
        sub, sl = doms[i]
        if sl.stop - sl.start > 40000 * W.n_vars(prob):
            continue
        Us = U[sl]
        ext = oracle.eval_rhs_extended(sub, Us)
        e = max(field_errors(sub, oracle.eval_rhs(sub, Us), ext))
        got = field_errors(sub, R[sl], ext)
        record(f"R domain {i}", got, max(RTOL, 3 * e))
        assert max(got) <= max(RTOL, 3 * e), (i, got, e)
        own.append(e)
        picked.append(int(sub["N"][0]))
        if len(picked) >= 12 and len(set(picked)) >= 7:
            break
    assert len(set(picked)) == 7
    Ro = oracle.eval_rhs(prob, U)
    errs = field_errors(prob, R, Ro)
    bound = max(2 * RTOL, 4 * max(own))
    record("R whole batch", errs, bound)
    assert all(e <= bound for e in errs), f"R: per-field errors {errs}, bound {bound}"


@pytest.mark.parametrize("case", ["mixing_layer", "hp_shock"])
def test_mixing_layer_and_hp_shock_full(oracle, case):
    """0.5e6 and 0.6e6 DOFs: small enough for the long-double oracle on the
    whole mesh, so the small-case bar applies unchanged."""
    from paper_2502_19342_gb300 import dgfv
    from tests.gpu_helpers import assert_rhs_close
    prob, U = W.mixing_layer() if case == "mixing_layer" else W.hp_shock(0)
    ctx = dgfv.Context(prob)
    ctx.set_state(to_dev(U))
    ctx.autotune()
    assert_rhs_close(oracle, prob, U, ctx.eval_rhs(to_dev(U)).cpu().numpy())
    ctx.close()


def test_mortar_half_refined_cube_full(oracle):
    """The benchmark's non-conforming workload (62k elements, 8M DOFs, type-3
    mortars on both x interfaces, N in 2..5, 5 % FV): R(U) of the whole mesh and
    the time step against the FP64 oracle.  Bound as for the turbulence case
    (4e, at least 2e-12), e the FP64 oracle's own error on the same generator at
    k = 8, scaled by the ratio of element sizes 24/8: for the same smooth field R
    stays O(1) while the summed terms grow like 1/h, and so does the rounding
    relative to R (the oracle's own error at k = 4, 8, 12: 2.0e-13, 6.8e-13,
    1.1e-12)."""
    from paper_2502_19342_gb300 import dgfv
    prob, U = W.half_refined_wave(24)
    ctx = dgfv.Context(prob, N_min=1, N_max=7, opts=dict(cfl_c=0.5, cfl_v=0.5))
    ctx.set_state(to_dev(U))
    R = ctx.eval_rhs(to_dev(U)).cpu().numpy()
    Ro = oracle.eval_rhs(prob, U)
    assert np.isfinite(Ro).all()
    s, Us = W.half_refined_wave(8)
    e = max(field_errors(s, oracle.eval_rhs(s, Us), oracle.eval_rhs_extended(s, Us)))
    bound = max(2 * RTOL, 4 * e * 24 / 8)
    errs = field_errors(prob, R, Ro)
    record("R full size", errs, bound)
    assert all(x <= bound for x in errs), f"R: per-field errors {errs}, bound {bound}"
    dt = ctx.compute_dt(to_dev(U))
    dto = oracle.dt(prob, U, 0.5, 0.5)
    assert abs(dt[0] - dto[0]) <= 1e-13 * dto[0]
    ctx.close()


def _hybrid_hp_shock(perturb=1e-4):
    """The hp shock case with the elements on the shock (|x - 0.4| < 0.13) and
    on the bubble's interface (|r - 0.2| < 0.07) switched to FV sub-cells by
    the oracle's V^{DG->FV} (668 FV elements of 4,096).  The flow carries
    smooth perturbations of relative size 1e-4: on the unperturbed state the
    sub-cell means of the uniform regions differ by rounding only, so the
    minmod branches there, and with them the tangent, are decided by rounding
    (a relative change of 1e-15 in U moves the oracle's own <R_bar, J v> by
    up to 40 %).  Larger perturbations raise the part of the tangent that the
    LLF wave-speed maximum switches on near-equal sides (spread 3e-13 at
    1e-4, 2e-11 at 1e-2, relative to the sum of the absolute terms)."""
    import oracle as O
    prob, U = W.hp_shock(0, perturb=perturb)
    _, _, corner, h = W.element_index(prob)
    xc = corner + 0.5 * h
    r = np.sqrt(((xc - np.array([0.8, 0.5, 0.5])) ** 2).sum(1))
    fv = ((np.abs(xc[:, 0] - 0.4) < 0.13) | (np.abs(r - 0.2) < 0.07)).astype(np.uint8)
    return dict(prob, fv=fv), O.remap(prob, prob["N"], fv, U)


@pytest.mark.parametrize("case", ["mixing_layer", "hp_shock_hybrid"])
def test_rhs_vjp_full_size(oracle, case):
    """The adjoint at full size: the mixing layer (4,096 elements, N = 4, 3
    species; the adjoint workload) and the hp shock case with FV elements.
    (a) <R_bar, J v> of the oracle's exact tangent = <U_bar, v> along two
    random directions; (b) 16 sampled entries U_bar_j against the oracle's
    column sum_i R_bar_i (J e_j)_i.  Bar: 1e-12 relative to the sum of the
    absolute terms of the oracle's dot product, or 4 times the oracle's own
    spread, whichever is larger: the change of its value when U moves by a
    relative 1e-15 (the minmod and wave-speed branches make the Jacobian
    piecewise, and a branch decided within rounding may go either way on
    either side).  The oracle's own tangent sits ~1e-16 (same measure) from
    its long-double value here."""
    import math
    from paper_2502_19342_gb300 import dgfv
    prob, U = W.mixing_layer() if case == "mixing_layer" else _hybrid_hp_shock()
    rng = np.random.default_rng(11)
    Rbar = rng.standard_normal(U.size)
    Up = U * (1 + 1e-15 * rng.standard_normal(U.size))
    ctx = dgfv.Context(prob)
    ctx.set_state(to_dev(U))
    Ub = ctx.rhs_vjp(to_dev(U), to_dev(Rbar)).cpu().numpy()
    ctx.close()
    assert np.isfinite(Ub).all()

    def bar(t, tp):
        return max(1e-12 * np.abs(t).sum(), 4 * abs(math.fsum(t) - math.fsum(tp)))

    for _ in range(2):
        v = rng.standard_normal(U.size) * 1e-2 * np.abs(U).mean()
        t = Rbar * oracle.eval_rhs_jvp(prob, U, v)[1]
        tp = Rbar * oracle.eval_rhs_jvp(prob, Up, v)[1]
        lhs, rhs = math.fsum(t), math.fsum(Ub * v)
        assert abs(lhs - rhs) <= bar(t, tp), (lhs, rhs, bar(t, tp))
    for j in rng.choice(U.size, 16, replace=False):
        e = np.zeros(U.size)
        e[j] = 1.0
        t = Rbar * oracle.eval_rhs_jvp(prob, U, e)[1]
        tp = Rbar * oracle.eval_rhs_jvp(prob, Up, e)[1]
        ref = math.fsum(t)
        assert abs(Ub[j] - ref) <= bar(t, tp), (int(j), Ub[j], ref, bar(t, tp))
