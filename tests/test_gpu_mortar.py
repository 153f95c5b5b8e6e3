"""Parity of the CUDA path with the FP64 oracle on non-conforming meshes
(mortar interfaces of types 1-3, Sec. 3.2.3): the mortar matrices of the
operator bank, R(U) with random hp/FV patterns (LG, LGL and the split form,
every flux choice), SSP-RK3 steps on the half-refined cube of Sec. 4.1 with a
pattern redrawn between steps, free-stream preservation, adaptation, the
adjoint through the mortars, and the refusal of malformed chains."""
import numpy as np
import pytest

from paper_2502_19342_gb300 import workloads as W
from tests.gpu_helpers import assert_adjoint_close, assert_fields_close, assert_rhs_close, ctx_for, gpu_rhs, to_dev

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _all_types(seed, nk=2, Nlo=1, Nhi=7, fv_frac=0.3, n_fv=8, riemann=0, mu=2e-3, nodes=0, split=0):
    """Chain with mortars of type 1 (y halved, big side left), type 2 (z halved),
    type 3 (both, big side right) and a conforming interface between different
    x spacings; several tiles per element kind."""
    specs = [W.AIR, W.HELIUM, W.CO2][:nk]
    sp = W.species_set(specs, mu=mu)
    doms = W.chain_domains([(3, 2, 2, 0.5), (2, 4, 2, 0.25), (1, 4, 4, 0.25), (2, 2, 2, 0.5)])
    ne = sum(int(np.prod(d[0])) for d in doms)
    prob = W.make_problem(doms, sp, n_fv=n_fv, N=W.random_degrees(ne, Nlo, Nhi, seed),
                          fv=W.random_fv(ne, fv_frac, seed), riemann=riemann, nodes=nodes, split=split, chain=1)
    return prob, W.smooth_random_state(prob, seed, amp=0.1)


def _half_refined(seed, k=2, Nlo=2, Nhi=5, fv_frac=0.3, n_fv=8, riemann=0, mu=2e-3, nk=2):
    specs = [W.AIR, W.HELIUM, W.CO2][:nk]
    sp = W.species_set(specs, mu=mu)
    doms = W.chain_domains([(k, 2 * k, 2 * k, 1.0), (k // 2, k, k, 1.0)], L=(2.0, 2.0))
    ne = sum(int(np.prod(d[0])) for d in doms)
    prob = W.make_problem(doms, sp, n_fv=n_fv, N=W.random_degrees(ne, Nlo, Nhi, seed),
                          fv=W.random_fv(ne, fv_frac, seed), riemann=riemann, chain=1)
    return prob, W.smooth_random_state(prob, seed, amp=0.1)


@pytest.mark.parametrize("nodes", [0, 1])
def test_mortar_bank_matches_oracle(oracle, nodes):
    prob, _ = _all_types(0, nodes=nodes)
    ctx = ctx_for(prob, N_min=1, N_max=7)
    for N in range(1, 8):
        for h in (0, 1):
            np.testing.assert_allclose(ctx.bank_entry(10, N, h), oracle.mortar(N, h, nodes=nodes).ravel(), atol=1e-14)
            np.testing.assert_allclose(ctx.bank_entry(11, N, h), oracle.mortar(N, h, proj=True, nodes=nodes).ravel(),
                                       atol=1e-13)
    for h in (0, 1):
        np.testing.assert_array_equal(ctx.bank_entry(12, 1, h), oracle.mortar(8, h, fv=True).ravel())
        np.testing.assert_array_equal(ctx.bank_entry(13, 1, h), oracle.mortar(8, h, proj=True, fv=True).ravel())
    ctx.close()


@pytest.mark.parametrize("nk,riemann,mu,seed,nodes,split,fv_frac", [
    (2, 0, 2e-3, 1, 0, 0, 0.3), (3, 1, 2e-3, 2, 0, 0, 0.3), (3, 2, 0.0, 3, 0, 0, 0.4), (2, 0, 2e-3, 4, 0, 0, 0.0),
    (2, 0, 2e-3, 5, 0, 0, 1.0), (3, 0, 2e-3, 6, 1, 0, 0.3), (3, 2, 1e-3, 7, 1, 1, 0.3), (1, 1, 2e-3, 8, 0, 0, 0.5)])
def test_rhs_on_mortar_chain(oracle, nk, riemann, mu, seed, nodes, split, fv_frac):
    """Random degrees 1..7 and FV elements on both sides of every mortar type:
    R(U) of the CUDA path within the oracle's own rounding level (pure DG and
    pure FV meshes included)."""
    prob, U = _all_types(seed, nk=nk, riemann=riemann, mu=mu, nodes=nodes, split=split, fv_frac=fv_frac)
    assert_rhs_close(oracle, prob, U, gpu_rhs(prob, U))


@pytest.mark.parametrize("riemann,seed", [(0, 21), (2, 22)])
def test_rhs_on_mortar_chain_odd_fv_count(oracle, riemann, seed):
    """N_FV = 7: the middle sub-cell of a big FV side straddles the two halves
    of the face, so the FV mortar maps split it (half of it on each virtual
    side); degrees 1..6 and 40 % FV elements."""
    prob, U = _all_types(seed, n_fv=7, Nhi=6, fv_frac=0.4, riemann=riemann)
    assert_rhs_close(oracle, prob, U, gpu_rhs(prob, U))


def test_rhs_free_stream_on_mortar_chain(oracle):
    """A uniform state gives R = 0 to rounding: on this chain (elements down to
    h = 1/8, degrees up to 7) the FP64 oracle itself reaches ~1e-11, so the
    bound is 3x the oracle's own level (and 5e-12 at least)."""
    prob, _ = _all_types(9, riemann=1)
    U = W.constant_state(prob, [0.6, 0.4], (0.8, -0.3, 0.2), 1.0)
    R = gpu_rhs(prob, U)
    own = np.abs(oracle.eval_rhs(prob, U)).max()
    assert own < 1e-10
    assert np.abs(R).max() < max(5e-12, 3 * own)


def test_rk3_steps_on_half_refined_cube_with_changing_pattern(oracle):
    """Sec. 4.1 layout: three SSP-RK3 steps, new random degrees and FV flags
    (with the remap of the state), three more; the state against the oracle's."""
    prob, U = _half_refined(10, riemann=2)
    ctx = ctx_for(prob, N_min=1, N_max=7)
    ctx.set_state(to_dev(U))
    dt = 2e-4
    for _ in range(3):
        ctx.rk_step(dt)
    Uo, _ = oracle.rk3(prob, U, 3, dt_fixed=dt)
    assert_fields_close(prob, ctx.get_state().cpu().numpy(), Uo, what="U(3 steps)")
    ne = W.n_elements(prob)
    N2, fv2 = W.random_degrees(ne, 2, 5, 77), W.random_fv(ne, 0.3, 77)
    ctx.set_degrees(N2, fv2, remap=True)
    prob2 = dict(prob, N=N2, fv=fv2)
    Uo2 = oracle.remap(prob, N2, fv2, Uo)
    for _ in range(3):
        ctx.rk_step(dt)
    Uo2, _ = oracle.rk3(prob2, Uo2, 3, dt_fixed=dt)
    assert_fields_close(prob2, ctx.get_state().cpu().numpy(), Uo2, what="U(3 + 3 steps)")
    ctx.close()


def test_lsrk4_and_positivity_limiter_on_half_refined_cube(oracle):
    """The low-storage RK4 (Sec. 3.3) and the Zhang-Shu limiter after every
    stage (Sec. 3.5) on the mortar mesh: three steps each against the oracle."""
    prob, U = _half_refined(17, fv_frac=0.2, riemann=2)
    ctx = ctx_for(prob, N_min=1, N_max=7, opts={"integrator": 1})
    ctx.set_state(to_dev(U))
    for _ in range(3):
        ctx.rk_step(2e-4)
    Uo, _ = oracle.lsrk4(prob, U, 3, dt_fixed=2e-4)
    assert_fields_close(prob, ctx.get_state().cpu().numpy(), Uo, what="U(3 LSRK4 steps)")
    ctx.close()
    pp = dict(prob, pp_limiter=1, pp_eps=1e-10)
    ctx = ctx_for(pp, N_min=1, N_max=7)
    ctx.set_state(to_dev(U))
    for _ in range(3):
        ctx.rk_step(2e-4)
    Uo, _ = oracle.rk3(pp, U, 3, dt_fixed=2e-4)
    assert_fields_close(pp, ctx.get_state().cpu().numpy(), Uo, what="U(3 limited SSP-RK3 steps)")
    ctx.close()


def test_time_step_and_graph_on_mortar_chain(oracle):
    """CFL time step with the element sizes of both halves, and an RK step replayed
    from a captured graph equals the direct launches."""
    prob, U = _half_refined(11, fv_frac=0.2)
    ctx = ctx_for(prob)
    ctx.set_state(to_dev(U))
    dt_g = ctx.compute_dt(to_dev(U))
    dt_o = oracle.dt(prob, U, 0.5, 0.5)
    assert abs(dt_g[0] - dt_o[0]) <= 1e-13 * dt_o[0]
    ctx.rk_steps(2, dt=1e-4)
    A = ctx.get_state().cpu().numpy()
    ctx.set_state(to_dev(U))
    for _ in range(2):
        ctx.rk_step(1e-4)
    B = ctx.get_state().cpu().numpy()
    np.testing.assert_array_equal(A, B)
    ctx.close()


def test_adapt_on_mortar_chain_matches_oracle(oracle):
    """The indicator and the remap are per element, mortars or not; after the
    adaptation R(U) on the new pattern matches the oracle."""
    prob, U = _all_types(12, Nlo=2, Nhi=6, fv_frac=0.2)
    thr = (1.0, 1.6, 3.0, 7.0)
    ctx = ctx_for(prob, N_min=1, N_max=7, opts={"thresholds": thr})
    ctx.set_state(to_dev(U))
    ctx.adapt()
    N_new, fv_new = ctx.get_degrees()
    oIp, oIh = oracle.indicator(prob, U)
    oN, ofv = oracle.adapt_decide(prob, oIp, oIh, thr, 1, 7)
    np.testing.assert_array_equal(N_new, oN)
    np.testing.assert_array_equal(fv_new, ofv)
    new = dict(prob, N=oN, fv=ofv)
    Un = oracle.remap(prob, oN, ofv, U)
    R = ctx.eval_rhs(to_dev(Un)).cpu().numpy()
    assert_rhs_close(oracle, new, Un, R)
    ctx.close()


def test_bad_chains_are_refused():
    """Neighbouring domains whose ny or nz differ by other than 1:1 or 2:1, or
    that are finer in y on one side and in z on the other, are refused."""
    from paper_2502_19342_gb300 import dgfv
    prob, U = _all_types(13, fv_frac=0.0, Nhi=4)
    for dims in ([[2, 2, 2], [2, 6, 2]], [[2, 4, 2], [2, 2, 4]]):
        dd = np.array(dims, np.int32)
        ne = int(np.prod(dd, axis=1).sum())
        bad = dict(prob, dims=dd, lo=prob["lo"][:2], hi=prob["hi"][:2], N=prob["N"][:ne], fv=prob["fv"][:ne])
        with pytest.raises(dgfv.DgfvError):
            ctx_for(bad)


@pytest.mark.parametrize("seed,mu,nodes", [(14, 2e-3, 0), (15, 0.0, 0), (16, 3e-3, 1)])
def test_rhs_vjp_on_mortar_chain_dot_product(oracle, seed, mu, nodes):
    """The adjoint through the mortars (the interpolation to the virtual sides
    and the projection back, transposed): <R_bar, J v> with the oracle's exact
    dual-number JVP equals <J^T R_bar, v> of the CUDA path, DG elements of
    degrees 1..6 on every mortar type."""
    prob, U = _all_types(seed, fv_frac=0.0, Nhi=6, mu=mu, nodes=nodes)
    rng = np.random.default_rng(seed)
    Rbar = rng.standard_normal(U.size)
    ctx = ctx_for(prob, N_min=1, N_max=7)
    Ubar = ctx.rhs_vjp(to_dev(U), to_dev(Rbar)).cpu().numpy()
    for _ in range(3):
        v = rng.standard_normal(U.size) * 1e-2 * np.abs(U).mean()
        _, Jv = oracle.eval_rhs_jvp(prob, U, v)
        lhs, rhs = float(np.dot(Rbar, Jv)), float(np.dot(Ubar, v))
        scale = float(np.abs(Rbar * Jv).sum())
        assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs, scale)
    ctx.close()


@pytest.mark.parametrize("seed,mu,riemann,n_fv", [(24, 2e-3, 0, 6), (25, 0.0, 2, 7), (26, 3e-3, 1, 6),
                                                (27, 2e-3, 1, 8)])
def test_rhs_vjp_on_mortar_chain_with_fv_elements(oracle, seed, mu, riemann, n_fv):
    """Hybrid DG/FV patterns on every mortar type: the FV big and small sides'
    maps (M^FV), the neighbour values gathered across mortars, transposed;
    <R_bar, J v> with the oracle's JVP against <J^T R_bar, v>."""
    prob, U = _all_types(seed, fv_frac=0.35, Nhi=n_fv - 1, n_fv=n_fv, mu=mu, riemann=riemann)
    rng = np.random.default_rng(seed)
    Rbar = rng.standard_normal(U.size)
    ctx = ctx_for(prob, N_min=1, N_max=n_fv - 1)
    Ubar = ctx.rhs_vjp(to_dev(U), to_dev(Rbar)).cpu().numpy()
    for _ in range(3):
        v = rng.standard_normal(U.size) * 1e-2 * np.abs(U).mean()
        _, Jv = oracle.eval_rhs_jvp(prob, U, v)
        lhs, rhs = float(np.dot(Rbar, Jv)), float(np.dot(Ubar, v))
        scale = float(np.abs(Rbar * Jv).sum())
        assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs, scale)
    ctx.close()


@pytest.mark.parametrize("fv", [None, [0, 1, 0, 0, 1]])
def test_rhs_vjp_on_mortar_chain_columns(oracle, fv):
    """A tiny chain (a type-3 mortar each way, 5 elements of degree 1-2; with
    FV elements (N_FV = 3) on both the small and the big side): the whole
    J^T R_bar entry by entry against the oracle's JVP columns."""
    sp = W.species_set([W.AIR, W.HELIUM], mu=2e-3)
    doms = W.chain_domains([(1, 2, 2, 0.5), (1, 1, 1, 0.5)])
    prob = W.make_problem(doms, sp, n_fv=3, N=W.random_degrees(5, 1, 2, 3), fv=fv, chain=1)
    U = W.smooth_random_state(prob, 3, amp=0.1)
    rng = np.random.default_rng(3)
    Rbar = rng.standard_normal(U.size)
    ctx = ctx_for(prob, N_min=1, N_max=2)
    Ubar = ctx.rhs_vjp(to_dev(U), to_dev(Rbar)).cpu().numpy()
    assert_adjoint_close(oracle, prob, U, Rbar, Ubar)
    ctx.close()
