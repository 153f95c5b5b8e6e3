"""GPU parity of the per-element sub-cell variant (N_fv = 0 in the mesh
descriptor): an FV element of degree N has N+1 sub-cells per direction, the
common-DOF scheme the paper contrasts with its own in Sec. 1.  DG/FV faces
couple on the FV side's grid (V^{FV->DG} the L2 projection where that grid is
coarser than N+1), FV/FV faces of unequal counts on the finer grid by sub-cell
overlaps.  Compared with the oracle's implementation of the same reading,
the adjoint with the oracle's exact dual-number tangent."""
import numpy as np
import pytest

from paper_2502_19342_gb300 import workloads as W
from tests.gpu_helpers import assert_adjoint_close, assert_fields_close, assert_rhs_close, ctx_for, to_dev

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _own(seed, nk=2, dims=(3, 4, 3), Nlo=1, Nhi=6, fv_frac=0.4, riemann=0, mu=2e-3, nodes=0):
    sp = W.species_set([W.AIR, W.HELIUM, W.CO2][:nk], mu=mu)
    n = int(np.prod(dims))
    prob = W.make_problem([(dims, (0, 0, 0), (1.0, 1.1, 0.9))], sp, n_fv=2, N=W.random_degrees(n, Nlo, Nhi, seed),
                          fv=W.random_fv(n, fv_frac, seed), riemann=riemann, nodes=nodes, fv_own_n=1)
    return prob, W.smooth_random_state(prob, seed, amp=0.15)


@pytest.mark.parametrize("seed,nk,riemann,mu,nodes", [(1, 2, 0, 2e-3, 0), (2, 3, 1, 2e-3, 0), (3, 2, 2, 0.0, 0),
                                                      (4, 1, 0, 1e-3, 0), (5, 3, 2, 3e-3, 1)])
def test_rhs_per_element_sub_cells(oracle, seed, nk, riemann, mu, nodes):
    """R(U) at the bar of R on random degrees 1..6 with 40 % FV elements: FV
    elements coarser and finer than their DG neighbours, FV/FV faces of unequal
    counts; LG and LGL nodes."""
    prob, U = _own(seed, nk=nk, riemann=riemann, mu=mu, nodes=nodes)
    ctx = ctx_for(prob, N_min=1, N_max=6)
    assert ctx.state_size == U.size
    R = ctx.eval_rhs(to_dev(U)).cpu().numpy()
    ctx.close()
    assert_rhs_close(oracle, prob, U, R)


def test_bank_maps_per_element(oracle):
    """V^{DG->FV} to every count, V^{FV->DG} from every count (the L2
    projection below N+1) and the sub-cell overlaps, against the oracle."""
    prob, _ = _own(1)
    ctx = ctx_for(prob, N_min=1, N_max=6)
    for N in range(1, 7):
        for m in range(2, 8):
            np.testing.assert_allclose(ctx.bank_entry(6, N, m), oracle.dg2fv(N, m).ravel(), atol=1e-14)
            np.testing.assert_allclose(ctx.bank_entry(7, N, m), oracle.fv2dg(N, m).ravel(), atol=1e-12)
            np.testing.assert_allclose(ctx.bank_entry(14, N, m), oracle.fv_overlap(N + 1, m).ravel(), atol=1e-15)
    ctx.close()


def test_time_step_and_adaptation_per_element(oracle):
    """CFL step (FV spacing h/(N+1) per element), indicator decisions, and the
    remap of an adaptation: switching DG <-> FV keeps the state size."""
    prob, U = _own(7, nk=2, Nlo=2, Nhi=5, fv_frac=0.3)
    thr = (1.0, 1.6, 3.0, 7.0)
    ctx = ctx_for(prob, opts=dict(thresholds=thr, cfl_c=0.5, cfl_v=0.4), N_min=1, N_max=6)
    Ud = to_dev(U)
    dt = ctx.compute_dt(Ud)
    rdt = oracle.dt(prob, U, 0.5, 0.4)
    np.testing.assert_allclose(dt, rdt, rtol=1e-14)
    ctx.set_state(Ud)
    ctx.adapt()
    N_new, fv_new = ctx.get_degrees()
    oIp, oIh = oracle.indicator(prob, U)
    near = np.zeros(len(oIp), bool)
    for T in thr:
        near |= (np.abs(oIp - T) < 1e-10) | (np.abs(oIh - T) < 1e-10)
    assert not near.any()
    oN, ofv = oracle.adapt_decide(prob, oIp, oIh, thr, 1, 6)
    np.testing.assert_array_equal(N_new, oN)
    np.testing.assert_array_equal(fv_new, ofv)
    new = dict(prob, N=oN, fv=ofv)
    Ug = ctx.get_state().cpu().numpy()
    Uo = oracle.remap(prob, oN, ofv, U)
    assert_fields_close(new, Ug, Uo, what="remapped state", rtol=1e-13)
    # every element that only switched DG <-> FV keeps its DOFs
    same_N = oN == prob["N"]
    n_old = W.points_per_dir(prob)[same_N]
    n_new = W.points_per_dir(new)[same_N]
    np.testing.assert_array_equal(n_old, n_new)
    ctx.close()


def test_rk_steps_and_free_stream_per_element(oracle):
    """Three SSP-RK3 steps at a fixed step against the oracle's rollout, and a
    constant state that stays constant."""
    prob, U = _own(9, nk=2, fv_frac=0.35)
    ctx = ctx_for(prob, N_min=1, N_max=6)
    dt = 0.5 * ctx.compute_dt(to_dev(U))[0]
    ctx.set_state(to_dev(U))
    for _ in range(3):
        ctx.rk_step(dt, want_dt=False)
    Uo, _ = oracle.rk3(prob, U, 3, dt_fixed=dt)
    assert_fields_close(prob, ctx.get_state().cpu().numpy(), Uo, what="U(3 steps, per-element sub-cells)")
    U0 = W.constant_state(prob, [0.6, 0.4], (0.5, -0.3, 0.2), 1.2)
    R = ctx.eval_rhs(to_dev(U0)).cpu().numpy()
    assert np.abs(R).max() < 1e-11
    ctx.close()


@pytest.mark.parametrize("seed,nk,riemann,mu,nodes", [(11, 2, 0, 2e-3, 0), (12, 3, 1, 2e-3, 0), (13, 2, 2, 0.0, 0),
                                                      (14, 1, 0, 1e-3, 0), (15, 3, 2, 3e-3, 1)])
def test_rhs_vjp_per_element_sub_cells_dot_product(oracle, seed, nk, riemann, mu, nodes):
    """The adjoint with per-element sub-cell counts: the FV element reverse on
    each element's own grid, the neighbour layers' transposes (overlap maps
    between FV elements of different counts, V^{DG->FV} to DG neighbours), the
    DG/FV and FV/FV face reverses on the finer or FV grid; <R_bar, J v> with the
    oracle's exact dual-number JVP against <J^T R_bar, v>."""
    prob, U = _own(seed, nk=nk, riemann=riemann, mu=mu, nodes=nodes)
    rng = np.random.default_rng(seed)
    Rbar = rng.standard_normal(U.size)
    ctx = ctx_for(prob, N_min=1, N_max=6)
    Ubar = ctx.rhs_vjp(to_dev(U), to_dev(Rbar)).cpu().numpy()
    ctx.close()
    for _ in range(3):
        v = rng.standard_normal(U.size) * 1e-2 * np.abs(U).mean()
        _, Jv = oracle.eval_rhs_jvp(prob, U, v)
        lhs, rhs = float(np.dot(Rbar, Jv)), float(np.dot(Ubar, v))
        scale = float(np.abs(Rbar * Jv).sum())
        assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs, scale)


def test_rhs_vjp_per_element_sub_cells_columns(oracle):
    """A 2x2x1 mesh with FV elements of 3 and 4 sub-cells side by side and DG
    neighbours of degree 1 and 2: the whole J^T R_bar, field by field, against
    the oracle's adjoint by columns, at the bar of R."""
    sp = W.species_set([W.AIR, W.HELIUM], mu=2e-3)
    prob = W.make_problem([((2, 2, 1), (0, 0, 0), (1.0, 0.8, 0.5))], sp, n_fv=2, N=np.array([2, 1, 3, 2], np.int8),
                          fv=np.array([1, 0, 1, 0], np.uint8), fv_own_n=1)
    U = W.smooth_random_state(prob, 5, amp=0.1)
    Rbar = np.random.default_rng(5).standard_normal(U.size)
    ctx = ctx_for(prob, N_min=1, N_max=3)
    Ubar = ctx.rhs_vjp(to_dev(U), to_dev(Rbar)).cpu().numpy()
    ctx.close()
    assert_adjoint_close(oracle, prob, U, Rbar, Ubar)


def test_rk_step_vjp_per_element_sub_cells(oracle):
    """One SSP-RK3 step's adjoint (stages recomputed) with per-element sub-cell
    counts, against the stage-by-stage tangent built from the oracle's JVP."""
    prob, U = _own(16, nk=2, fv_frac=0.35)
    ctx = ctx_for(prob, N_min=1, N_max=6)
    Ud = to_dev(U)
    dt = 0.5 * ctx.compute_dt(Ud)[0]
    rng = np.random.default_rng(16)
    lam = rng.standard_normal(U.size)
    Ubar = ctx.rk_step_vjp(Ud, dt, to_dev(lam)).cpu().numpy()
    ctx.close()
    v = rng.standard_normal(U.size) * 1e-2 * np.abs(U).mean()
    R0, J0 = oracle.eval_rhs_jvp(prob, U, v)
    U1 = U + dt * R0
    V1 = v + dt * J0
    R1, J1 = oracle.eval_rhs_jvp(prob, U1, V1)
    U2 = 0.75 * U + 0.25 * (U1 + dt * R1)
    V2 = 0.75 * v + 0.25 * (V1 + dt * J1)
    _, J2 = oracle.eval_rhs_jvp(prob, U2, V2)
    V3 = v / 3.0 + 2.0 / 3.0 * (V2 + dt * J2)
    lhs, rhs = float(np.dot(lam, V3)), float(np.dot(Ubar, v))
    scale = float(np.abs(lam * V3).sum())
    assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs, scale)
