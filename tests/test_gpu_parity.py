"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded
inputs: R(U), the time step, SSP-RK3 steps, the modal indicator's decisions
and the remap, on small cases that span several tiles and ragged tails, the
paper-shaped workloads and edge cases."""
import numpy as np
import pytest

from paper_2502_19342_gb300 import workloads as W
from tests.gpu_helpers import RTOL, assert_fields_close, assert_rhs_close, ctx_for, gpu_rhs, record, to_dev

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _mixed(seed, nk=2, nel=(3, 4, 5), Nlo=1, Nhi=7, fv_frac=0.25, n_fv=8, riemann=0, mu=2e-3, box=(1.0, 1.3, 0.9),
           nodes=0, split=0):
    specs = [W.AIR, W.HELIUM, W.CO2][:nk]
    sp = W.species_set(specs, mu=mu)
    n = nel[0] * nel[1] * nel[2]
    prob = W.make_problem([(nel, (0, 0, 0), box)], sp, n_fv=n_fv, N=W.random_degrees(n, Nlo, Nhi, seed),
                          fv=W.random_fv(n, fv_frac, seed), riemann=riemann, nodes=nodes, split=split)
    return prob, W.smooth_random_state(prob, seed, amp=0.1)


@pytest.mark.parametrize("nodes", [0, 1])
def test_operator_bank_matches_oracle(oracle, nodes):
    prob, _ = _mixed(0, nodes=nodes)
    ctx = ctx_for(prob, N_min=1, N_max=7)
    for N in range(1, 8):
        b = oracle.basis(N, nodes)
        np.testing.assert_allclose(ctx.bank_entry(0, N), b["x"], atol=1e-15)
        np.testing.assert_allclose(ctx.bank_entry(1, N), b["w"], atol=1e-15)
        np.testing.assert_allclose(ctx.bank_entry(2, N), b["Dhat"].ravel(), atol=1e-12)
        np.testing.assert_allclose(ctx.bank_entry(9, N), b["D"].ravel(), atol=1e-12)
        np.testing.assert_allclose(ctx.bank_entry(3, N), b["lm"], atol=1e-14)
        np.testing.assert_allclose(ctx.bank_entry(4, N), b["lp"], atol=1e-14)
        np.testing.assert_allclose(ctx.bank_entry(6, N), oracle.dg2fv(N, 8, nodes).ravel(), atol=1e-14)
        np.testing.assert_allclose(ctx.bank_entry(7, N), oracle.fv2dg(N, 8, nodes).ravel(), atol=1e-12)
        np.testing.assert_allclose(ctx.bank_entry(8, N), np.linalg.inv(oracle.leg_vandermonde(N, nodes)).ravel(),
                                   atol=1e-13)
        for M in range(1, 8):
            np.testing.assert_allclose(ctx.bank_entry(5, N, M), oracle.vmap(N, M, nodes).ravel(), atol=1e-13)
    ctx.close()


def test_rhs_plain_tiny(oracle):
    """4x4x4 elements, N = 3, two species, viscous: R(U) per field within
    1e-12 of the extended-precision oracle, or within 3x the FP64 oracle's own
    rounding error where that is larger."""
    prob, U = W.plain_tiny(0)
    assert_rhs_close(oracle, prob, U, gpu_rhs(prob, U))


@pytest.mark.parametrize("nk,riemann,mu,seed,nodes,split", [
    (2, 0, 2e-3, 1, 0, 0), (3, 0, 2e-3, 2, 0, 0), (2, 1, 2e-3, 3, 0, 0), (3, 1, 0.0, 4, 0, 0),
    (1, 0, 1e-3, 5, 0, 0), (3, 1, 5e-3, 6, 0, 0), (3, 2, 2e-3, 7, 0, 0), (2, 2, 0.0, 8, 0, 0),
    (3, 0, 2e-3, 9, 1, 0), (3, 1, 2e-3, 10, 1, 1), (2, 0, 0.0, 11, 1, 1), (3, 2, 1e-3, 12, 1, 1)])
def test_rhs_mixed_hp_fv(oracle, nk, riemann, mu, seed, nodes, split):
    """Random degrees 1..7 and FV elements (N_FV = 8) on a 3x4x5 box: every
    face type (equal and unequal degree, DG/FV, FV/FV) and ragged tiles; LG
    nodes, LGL nodes, and the split form on LGL nodes."""
    prob, U = _mixed(seed, nk=nk, riemann=riemann, mu=mu, nodes=nodes, split=split)
    assert_rhs_close(oracle, prob, U, gpu_rhs(prob, U))


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("nk,n_fv,riemann,mu", [(2, 7, 0, 2e-3), (3, 8, 2, 2e-3), (2, 9, 0, 1e-3),
                                                 (3, 5, 1, 3e-3), (1, 8, 0, 0.0), (2, 2, 0, 2e-3), (3, 3, 1, 1e-3)])
def test_fv_kernel_layouts_match_oracle(oracle, variant, nk, n_fv, riemann, mu):
    """The shared-memory layouts of the FV sub-cell kernel (gradients
    recomputed at each face / kept per sub-cell / kept, with the z faces in a
    second pass where two CTAs then fit per SM) on a hybrid mesh with 40 % FV
    elements, N_FV = 2, 3, 5, 7, 8, 9 (two sub-cells: one interior face per
    line, every cell a boundary cell): R(U) against the oracle at the bar of
    R."""
    sp = W.species_set([W.AIR, W.HELIUM, W.CO2][:nk], mu=mu)
    n = 3 * 3 * 4
    N = W.random_degrees(n, 1, min(6, n_fv - 1), 40 + n_fv)
    prob = W.make_problem([((3, 3, 4), (0, 0, 0), (1.0, 0.9, 1.2))], sp, n_fv=n_fv, N=N,
                          fv=W.random_fv(n, 0.4, 40 + n_fv), riemann=riemann)
    U = W.smooth_random_state(prob, 40 + n_fv, amp=0.15)
    from paper_2502_19342_gb300 import dgfv
    ctx = dgfv.Context(prob)
    ctx.set_fv_variant(variant)
    R = ctx.eval_rhs(to_dev(U)).cpu().numpy()
    ctx.close()
    assert_rhs_close(oracle, prob, U, R)


@pytest.mark.parametrize("nk,n_fv", [(2, 7), (3, 5), (1, 6)])
def test_fv_two_pass_layout_is_the_kept_gradient_layout_bit_for_bit(nk, n_fv):
    """The z faces in a second pass, the first pass's flux differences kept in
    the cell's row: the same sums in the same order as one pass, so R(U) and
    an SSP-RK3 step are bitwise those of the one-pass layout."""
    sp = W.species_set([W.AIR, W.HELIUM, W.CO2][:nk], mu=2e-3)
    n = 3 * 3 * 4
    N = W.random_degrees(n, 1, n_fv - 1, 60 + n_fv)
    prob = W.make_problem([((3, 3, 4), (0, 0, 0), (1.0, 0.9, 1.2))], sp, n_fv=n_fv, N=N,
                          fv=W.random_fv(n, 0.5, 60 + n_fv))
    U = to_dev(W.smooth_random_state(prob, 60 + n_fv, amp=0.15))
    from paper_2502_19342_gb300 import dgfv
    out = []
    for variant in (2, 3):
        ctx = dgfv.Context(prob)
        ctx.set_fv_variant(variant)
        R = ctx.eval_rhs(U)
        ctx.set_state(U)
        dt = 0.5 * ctx.compute_dt(U)[0]
        ctx.rk_step(dt, want_dt=False)
        out.append((R, ctx.get_state()))
        ctx.close()
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])


def test_rhs_batched_domains(oracle):
    """Several independent periodic domains of uneven size and degree in one context."""
    sp = W.species_set([W.AIR, W.HELIUM, W.CO2], mu=1e-3)
    rng = np.random.default_rng(11)
    doms, N = [], []
    for d in range(6):
        dims = tuple(int(x) for x in rng.integers(1, 4, 3))
        lo = tuple(float(x) for x in rng.uniform(-1, 1, 3))
        doms.append((dims, lo, tuple(l + float(s) for l, s in zip(lo, rng.uniform(0.5, 2.0, 3)))))
        N += [int(rng.integers(1, 8))] * int(np.prod(dims))
    prob = W.make_problem(doms, sp, n_fv=8, N=np.array(N, np.int8), fv=W.random_fv(len(N), 0.2, 3))
    U = W.smooth_random_state(prob, 3, amp=0.05)
    assert_rhs_close(oracle, prob, U, gpu_rhs(prob, U))


def test_rhs_free_stream(oracle):
    prob, _ = _mixed(7, nk=3, riemann=1)
    U = W.constant_state(prob, [0.5, 0.3, 0.2], (1.0, -0.5, 0.25), 1.0)
    R = gpu_rhs(prob, U)
    assert np.abs(R).max() < 1e-11


@pytest.mark.parametrize("riemann,nodes,split", [(1, 0, 0), (2, 1, 1)])
def test_free_stream_stays_constant_for_180_steps(riemann, nodes, split):
    """Free-stream preservation over time (Sec. 4.1: a constant state on a
    random hp/FV pattern stays constant through 180 time steps, the errors at
    round-off): 180 SSP-RK3 steps at CFL 0.5 on random degrees 1..7 with FV
    elements; Roe-HH on LG nodes, and the hybrid flux with the split form on
    LGL nodes."""
    from paper_2502_19342_gb300 import dgfv
    prob, _ = _mixed(8, nk=3, riemann=riemann, nodes=nodes, split=split)
    U = W.constant_state(prob, [0.5, 0.3, 0.2], (1.0, -0.5, 0.25), 1.0)
    ctx = dgfv.Context(prob, N_min=1, N_max=7, opts=dict(cfl_c=0.5, cfl_v=0.5))
    U0 = to_dev(U)
    ctx.set_state(U0)
    ctx.rk_steps(180, -1.0, want_dt=False)
    Uf = ctx.get_state()
    ctx.close()
    err = (Uf - U0).abs() / U0.abs().max()
    record("U(180 steps) - U(0)", float(err.max()), 1e-12)
    assert float(err.max()) < 1e-12
    assert float(err.pow(2).mean().sqrt()) < 1e-13


def test_rhs_edge_degrees_and_single_element_domains(oracle):
    """Degree extremes N = 1 and 7, FV with N_FV = N_max + 1, and 1-element-wide
    periodic directions (an element is its own neighbour)."""
    sp = W.species_set([W.AIR, W.HELIUM], mu=2e-3)
    doms = [((1, 1, 1), (0, 0, 0), (1, 1, 1)), ((2, 1, 3), (0, 0, 0), (1, 0.5, 1.5)), ((1, 4, 1), (0, 0, 0), (0.3, 1, 0.3))]
    n = 1 + 6 + 4
    N = np.array([7, 1, 7, 1, 7, 1, 7, 1, 2, 7, 3], np.int8)
    fv = np.array([0, 0, 1, 0, 0, 1, 0, 0, 1, 0, 0], np.uint8)
    prob = W.make_problem(doms, sp, n_fv=8, N=N, fv=fv, riemann=1)
    assert n == len(N)
    U = W.smooth_random_state(prob, 9, amp=0.05)
    assert_rhs_close(oracle, prob, U, gpu_rhs(prob, U))


def test_time_step(oracle):
    prob, U = _mixed(12, nk=3)
    ctx = ctx_for(prob, opts=dict(cfl_c=0.5, cfl_v=0.4))
    dt, dtc, dtv = ctx.compute_dt(to_dev(U))
    rdt, rdtc, rdtv = oracle.dt(prob, U, 0.5, 0.4)
    assert abs(dtc - rdtc) <= 1e-14 * rdtc
    assert abs(dtv - rdtv) <= 1e-14 * rdtv
    assert abs(dt - rdt) <= 1e-14 * rdt


def test_rk3_ten_steps_plain_tiny(oracle):
    """The plain tiny case advanced 10 SSP-RK3 steps at CFL 0.5: the final state
    per field within 1e-12 of the oracle's."""
    prob, U = W.plain_tiny(0)
    ctx = ctx_for(prob, opts=dict(cfl_c=0.5, cfl_v=0.5))
    ctx.set_state(to_dev(U))
    dts = [ctx.rk_step(-1.0) for _ in range(10)]
    Ug = ctx.get_state().cpu().numpy()
    Uo, odts = oracle.rk3(prob, U, 10, cfl_c=0.5, cfl_v=0.5)
    np.testing.assert_allclose(dts, odts, rtol=1e-13)
    assert_fields_close(prob, Ug - U, Uo - U, what="U(t10) - U(0)", rtol=1e-10)
    assert_fields_close(prob, Ug, Uo, what="U(t10)")


def test_rk_steps_graph_matches_single_steps(oracle):
    prob, U = _mixed(13, nk=2, Nhi=5)
    a = ctx_for(prob)
    b = ctx_for(prob)
    a.set_state(to_dev(U))
    b.set_state(to_dev(U))
    for _ in range(4):
        a.rk_step(-1.0)
    b.rk_steps(4, -1.0)
    np.testing.assert_array_equal(a.get_state().cpu().numpy(), b.get_state().cpu().numpy())


def test_rk3_mixed_fixed_dt(oracle):
    prob, U = _mixed(14, nk=3, riemann=1, Nhi=6)
    ctx = ctx_for(prob)
    ctx.set_state(to_dev(U))
    dt = 2e-4
    for _ in range(3):
        ctx.rk_step(dt)
    Uo, _ = oracle.rk3(prob, U, 3, dt_fixed=dt)
    assert_fields_close(prob, ctx.get_state().cpu().numpy(), Uo, what="U(3 steps)")


def _decisions_match(oracle, prob, U, thr, N_min, N_max):
    ctx = ctx_for(prob, opts=dict(thresholds=thr), N_min=N_min, N_max=N_max)
    Ip, Ih, dec = ctx.indicator(to_dev(U))
    Ip, Ih, dec = Ip.cpu().numpy(), Ih.cpu().numpy(), dec.cpu().numpy()
    oIp, oIh = oracle.indicator(prob, U)
    # Indicator values agree to the rounding of the logarithm of small modal
    # energies (an energy fraction w carries a relative error of about
    # 1e-16/sqrt(w), so fractions near the 1e-24 floor move I by up to ~1e-6);
    # the contract is on the decisions: bit-exact outside a 1e-10 band.
    np.testing.assert_allclose(Ip, oIp, rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(Ih, oIh, rtol=1e-6, atol=1e-9)
    Nn, fn = oracle.adapt_decide(prob, oIp, oIh, thr, N_min, N_max)
    code = np.zeros(len(Nn), np.uint8)
    code[(fn == 1) & (prob["fv"] == 0)] = 1
    code[(fn == 0) & (prob["fv"] == 1)] = 2
    code[(Nn > prob["N"]) & (code == 0)] = 3
    code[(Nn < prob["N"]) & (code == 0)] = 4
    near = np.zeros(len(Nn), bool)
    for T in thr:
        near |= (np.abs(oIp - T) < 1e-10) | (np.abs(oIh - T) < 1e-10)
    mism = (code != dec) & ~near
    assert not mism.any(), f"{mism.sum()} decisions differ outside the 1e-10 band"
    return ctx, code, near.sum()


def test_indicator_decisions_hp_shock(oracle):
    """Decisions on the hp-mixed shock workload (reduced to 8x8x8 elements, with
    random FV elements): bit-exact except for elements whose indicator lies
    within 1e-10 of a threshold."""
    prob, U = W.hp_shock(0, nel=(8, 8, 8))
    prob["fv"] = W.random_fv(W.n_elements(prob), 0.2, 1)
    U = W.build_state(prob, lambda x, y, z: (
        [2.3 + 0.2 * np.tanh((x - 0.5) / 0.05), 0.2 + 0.1 * np.sin(6 * y)], (0.1 + 0 * x, 0 * x, 0 * x),
        1.6 + 0.5 * np.tanh((x - 1.0) / 0.03)))
    ctx, code, near = _decisions_match(oracle, prob, U, W.THRESHOLDS, 2, 6)
    assert (code != 0).sum() > 10  # the case exercises the rules
    ctx.close()


def test_adapt_remaps_like_the_oracle(oracle):
    prob, U = _mixed(21, nk=2, Nlo=2, Nhi=6, fv_frac=0.2, n_fv=8)
    thr = (1.0, 1.6, 3.0, 7.0)
    ctx, code, near = _decisions_match(oracle, prob, U, thr, 1, 7)
    assert near == 0
    ctx.set_state(to_dev(U))
    stats = ctx.adapt()
    N_new, fv_new = ctx.get_degrees()
    oIp, oIh = oracle.indicator(prob, U)
    oN, ofv = oracle.adapt_decide(prob, oIp, oIh, thr, 1, 7)
    np.testing.assert_array_equal(N_new, oN)
    np.testing.assert_array_equal(fv_new, ofv)
    assert stats["n_changed"] == int((code != 0).sum())
    Ug = ctx.get_state().cpu().numpy()
    Uo = oracle.remap(prob, oN, ofv, U)
    new = dict(prob, N=oN, fv=ofv)
    assert_fields_close(new, Ug, Uo, what="remapped state", rtol=1e-13)
    ctx.close()


def test_set_degrees_remap_round_trip(oracle):
    prob, U = _mixed(22, nk=3, Nlo=1, Nhi=6, fv_frac=0.0)
    ctx = ctx_for(prob, N_min=1, N_max=7)
    ctx.set_state(to_dev(U))
    up = (prob["N"] + 1).astype(np.int8)
    ctx.set_degrees(up, None, remap=True)
    ctx.set_degrees(prob["N"], None, remap=True)
    np.testing.assert_allclose(ctx.get_state().cpu().numpy(), U, atol=1e-12)
    ctx.set_degrees(prob["N"], np.ones(len(up), np.uint8), remap=True)
    ctx.set_degrees(prob["N"], None, remap=True)
    np.testing.assert_allclose(ctx.get_state().cpu().numpy(), U, atol=1e-11)


def test_rejects_bad_arguments():
    from paper_2502_19342_gb300 import dgfv
    prob, U = _mixed(0)
    ctx = ctx_for(prob, N_min=1, N_max=7)
    with pytest.raises(dgfv.DgfvError):
        ctx.set_degrees(np.full(ctx.n_elem, 9, np.int8))
    with pytest.raises(ValueError):
        ctx.eval_rhs(to_dev(U[:-1]))
    with pytest.raises(dgfv.DgfvError):
        ctx.rk_step(-1.0)  # no state yet
    ctx.close()
    with pytest.raises(dgfv.DgfvError):
        ctx_for(dict(prob, riemann=3))  # no such flux


def test_launch_modes_and_autotuned_tiles_give_identical_results(oracle):
    """One launch per kernel, one launch per degree bin, and autotuned volume
    tiles run the same per-element arithmetic: bitwise equal results."""
    sp = W.species_set([W.AIR, W.HELIUM, W.CO2], mu=1e-3)
    rng = np.random.default_rng(31)
    doms, N = [], []
    for _ in range(12):
        nd = int(rng.integers(1, 4))
        doms.append(((nd, nd, nd), (0, 0, 0), (1, 1, 1)))
        N += [int(rng.integers(1, 8))] * nd ** 3
    prob = W.make_problem(doms, sp, n_fv=8, N=np.array(N, np.int8))
    U = W.smooth_random_state(prob, 31, amp=0.05)
    ctx = ctx_for(prob, N_min=1, N_max=7)
    Ud = to_dev(U)
    R0 = ctx.eval_rhs(Ud).cpu().numpy()
    ctx.set_launch_mode(True)
    R1 = ctx.eval_rhs(Ud).cpu().numpy()
    ctx.set_launch_mode(False)
    ctx.set_state(Ud)
    tuned = ctx.autotune()
    assert tuned.pop("variant") in range(4)
    assert set(tuned) == set(int(x) for x in np.unique(prob["N"]))
    R2 = ctx.eval_rhs(Ud).cpu().numpy()
    # persistent volume kernel (work queue over the tiles of every degree), with
    # the tuned tiles and with many more tiles than resident CTAs
    ctx.set_launch_mode(2)
    R3 = ctx.eval_rhs(Ud).cpu().numpy()
    ctx.set_state(Ud)
    ctx.rk_steps(2, 1e-4, want_dt=False)  # graph capture of the persistent launch (queue reset inside)
    S3 = ctx.get_state().cpu().numpy()
    ctx.set_launch_mode(0)
    ctx.set_state(Ud)
    ctx.rk_steps(2, 1e-4, want_dt=False)
    S0 = ctx.get_state().cpu().numpy()
    np.testing.assert_array_equal(R1, R0)
    np.testing.assert_array_equal(R2, R0)
    # the persistent kernel is the same tile body compiled into another kernel:
    # the compiler may contract multiply-adds differently, so it agrees to rounding
    np.testing.assert_allclose(R3, R0, rtol=1e-12, atol=1e-12 * np.abs(R0).max())
    np.testing.assert_allclose(S3, S0, rtol=1e-13, atol=0)
    assert_rhs_close(oracle, prob, U, R0)
    ctx.close()


def test_split_form_rk3_steps(oracle):
    """Split form on LGL nodes, mixed degrees and FV elements, 3 species,
    viscous, Roe-HH between DG elements: 5 SSP-RK3 steps at a fixed step."""
    prob, U = _mixed(21, nk=3, riemann=2, Nhi=6, nodes=1, split=1)
    ctx = ctx_for(prob)
    ctx.set_state(to_dev(U))
    dt = 2e-4
    for _ in range(5):
        ctx.rk_step(dt)
    Uo, _ = oracle.rk3(prob, U, 5, dt_fixed=dt)
    assert_fields_close(prob, ctx.get_state().cpu().numpy(), Uo, what="U(5 steps, split form)")


def test_split_form_indicator_and_remap_on_lgl(oracle):
    """Indicator decisions and the remap on LGL nodes (their Vandermonde and
    projection matrices differ from the LG ones)."""
    prob, U = _mixed(22, nk=3, nodes=1, split=1, fv_frac=0.2)
    ctx = ctx_for(prob, N_min=1, N_max=7)
    Ip, Ih, _ = ctx.indicator(to_dev(U))
    oIp, oIh = oracle.indicator(prob, U)
    np.testing.assert_allclose(Ip.cpu().numpy(), oIp, rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(Ih.cpu().numpy(), oIh, rtol=1e-6, atol=1e-9)
    ctx.set_state(to_dev(U))
    N2 = np.clip(prob["N"] + np.where(np.arange(len(prob["N"])) % 2 == 0, 1, -1), 1, 7).astype(np.int8)
    fv2 = prob["fv"].copy()
    fv2[::5] ^= 1
    ctx.set_degrees(N2, fv2, remap=True)
    ref = oracle.remap(prob, N2, fv2, U)
    np.testing.assert_allclose(ctx.get_state().cpu().numpy(), ref, atol=1e-13)
    ctx.close()


def test_lsrk4_steps_match_oracle(oracle):
    """Five-stage low-storage RK4 (Sec. 3.3): 4 steps at a fixed step on a mixed
    hp/FV pattern (Roe-HH), and 3 CFL steps on the plain tiny case."""
    prob, U = _mixed(23, nk=3, riemann=1, Nhi=6)
    ctx = ctx_for(prob, opts=dict(integrator=1))
    ctx.set_state(to_dev(U))
    for _ in range(4):
        ctx.rk_step(2e-4)
    Uo, _ = oracle.lsrk4(prob, U, 4, dt_fixed=2e-4)
    assert_fields_close(prob, ctx.get_state().cpu().numpy(), Uo, what="U(4 LSRK4 steps)")
    ctx.close()
    prob, U = W.plain_tiny(0)
    ctx = ctx_for(prob, opts=dict(cfl_c=0.5, cfl_v=0.5, integrator=1))
    ctx.set_state(to_dev(U))
    dts = [ctx.rk_step(-1.0) for _ in range(3)]
    Uo, odts = oracle.lsrk4(prob, U, 3, cfl_c=0.5, cfl_v=0.5)
    np.testing.assert_allclose(dts, odts, rtol=1e-13)
    assert_fields_close(prob, ctx.get_state().cpu().numpy(), Uo, what="U(3 LSRK4 CFL steps)")
    ctx.close()


def test_lsrk4_graph_equals_steps_and_stage_adjoint_is_rejected():
    from paper_2502_19342_gb300 import dgfv
    prob, U = _mixed(24, nk=2)
    ctx = ctx_for(prob, opts=dict(integrator=1))
    ctx.set_state(to_dev(U))
    for _ in range(3):
        ctx.rk_step(1e-4, want_dt=False)
    a = ctx.get_state()
    ctx.set_state(to_dev(U))
    ctx.rk_steps(3, 1e-4, want_dt=False)
    assert torch.equal(ctx.get_state(), a)
    s1, s2 = torch.empty_like(a), torch.empty_like(a)
    with pytest.raises(dgfv.DgfvError):
        ctx.rk_step_save(1e-4, s1, s2)
    ctx.close()


@pytest.mark.parametrize("nk,fv_frac,riemann", [(1, 0.4, 0), (2, 0.3, 2), (2, 1.0, 1)])
def test_nine_sub_cells_per_direction(oracle, nk, fv_frac, riemann):
    """N_FV = 9 (the paper's TGV set-up): FV elements of 729 sub-cells next to DG
    elements of degrees 1..7 (the state tiles of such an element exceed the
    512-node tiling, the sub-cell kernel runs at its generic size), R(U) and
    three SSP-RK3 steps against the oracle."""
    prob, U = _mixed(40 + nk, nk=nk, nel=(3, 3, 2), Nlo=1, Nhi=7, fv_frac=fv_frac, n_fv=9, riemann=riemann)
    assert_rhs_close(oracle, prob, U, gpu_rhs(prob, U))
    ctx = ctx_for(prob)
    ctx.set_state(to_dev(U))
    for _ in range(3):
        ctx.rk_step(1e-4)
    Uo, _ = oracle.rk3(prob, U, 3, dt_fixed=1e-4)
    assert_fields_close(prob, ctx.get_state().cpu().numpy(), Uo, what="U(3 steps)")
    ctx.close()


def test_nine_sub_cells_with_three_species_is_refused():
    """One FV element of 9^3 sub-cells and 7 variables needs more shared memory
    than one CTA has: dgfv_init_mesh refuses the context."""
    from paper_2502_19342_gb300 import dgfv
    prob, _ = _mixed(44, nk=3, nel=(2, 2, 2), n_fv=9)
    with pytest.raises(dgfv.DgfvError):
        ctx_for(prob)


def test_tgv_sutherland_indicator_choice_and_lsrk4(oracle):
    """The supersonic TGV set-up (Sec. 4.3) on 6^3 elements with degrees 2..4 and
    FV elements: R(U) with Sutherland's viscosity, the indicator with
    p-refinement on the pressure and FV on the density, and 3 low-storage RK4
    CFL steps.  (On 4^3 elements the p-coupling of N = 2 faces to N = 4 gives
    negative pressures at face points, in the oracle and the CUDA path alike.)"""
    n = 216
    prob, U = W.tgv(nel=6, N0=W.random_degrees(n, 2, 4, 31), fv=W.random_fv(n, 0.2, 31))
    assert_rhs_close(oracle, prob, U, gpu_rhs(prob, U))
    ctx = ctx_for(prob, opts=dict(integrator=1, cfl_c=0.5, cfl_v=0.5), N_min=2, N_max=4)
    Ip, Ih, _ = ctx.indicator(to_dev(U))
    oIp, oIh = oracle.indicator(prob, U)
    np.testing.assert_allclose(Ip.cpu().numpy(), oIp, rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(Ih.cpu().numpy(), oIh, rtol=1e-6, atol=1e-9)
    ctx.set_state(to_dev(U))
    dts = [ctx.rk_step(-1.0) for _ in range(3)]
    Uo, odts = oracle.lsrk4(prob, U, 3, cfl_c=0.5, cfl_v=0.5)
    np.testing.assert_allclose(dts, odts, rtol=1e-13)
    assert_fields_close(prob, ctx.get_state().cpu().numpy(), Uo, what="TGV U(3 LSRK4 steps)")
    ctx.close()


def _amplified_rarefaction(oracle, nodes=0):
    """The limiter pins' rarefaction after 46 (LGL: 30) SSP-RK3 steps with every
    element's deviation from its mean amplified sixfold (negative partial
    densities and internal energies at some points, positive means)."""
    sp = W.species_set([W.AIR, W.HELIUM], mu=0.0)
    prob = W.make_problem([((16, 1, 1), (0, 0, 0), (1, 1.0 / 16, 1.0 / 16))], sp, n_fv=6, N=3, nodes=nodes)

    def fn(x, y, z):
        v = 12.0 * np.tanh((x - 0.5) / 0.05) * np.sin(2 * np.pi * x) ** 2
        return [0.5 + 0 * x, 0.5 + 0 * x], (v, 0 * x, 0 * x), 0.4 + 0 * x
    U = W.build_state(prob, fn)
    X, _ = oracle.rk3(prob, U, 46 if nodes == 0 else 30, cfl_c=0.3, cfl_v=0.3)  # LGL breaks down earlier
    assert np.isfinite(X).all()
    w = np.polynomial.legendre.leggauss(4)[1] if nodes == 0 else np.array([1 / 6, 5 / 6, 5 / 6, 1 / 6])
    w3 = np.einsum("k,j,i->kji", w, w, w).ravel() / 8.0
    for e in range(16):
        blk = X[e * 384:(e + 1) * 384].reshape(6, 64)
        m = blk @ w3
        blk[:] = m[:, None] + 6.0 * (blk - m[:, None])
    return prob, U, X


@pytest.mark.parametrize("nodes", [0, 1])
def test_pp_limiter_once_matches_oracle(oracle, nodes):
    prob, _, X = _amplified_rarefaction(oracle, nodes)
    ref, n_ref = oracle.pp_limit(prob, X, 1e-10)
    assert n_ref > 0
    ctx = ctx_for(prob, opts=dict(pp_eps=1e-10))
    Xd = to_dev(X)
    n = ctx.pp_limit(Xd)
    assert n == n_ref
    assert_fields_close(prob, Xd.cpu().numpy(), ref, rtol=1e-12, what="limited state")
    ctx.close()


def test_pp_limiter_in_the_stages_matches_oracle(oracle):
    """SSP-RK3 with the limiter after every stage through the breakdown point of
    the unlimited rarefaction (step 47).  Near vacuum the limited dynamics
    amplify rounding: the oracle started from U (1 + 1e-15 noise) drifts from
    itself by ~1e-10 after 48 steps and ~1e-5 after 52.  The bound is 10x that
    drift of the oracle against itself (at least 1e-10)."""
    from tests.gpu_helpers import field_errors
    prob, U, _ = _amplified_rarefaction(oracle)
    p = dict(prob, pp_limiter=1, pp_eps=1e-10)
    steps = 48
    Uo, dto = oracle.rk3(p, U, steps, cfl_c=0.3, cfl_v=0.3)
    noise = 1e-15 * np.random.default_rng(0).standard_normal(U.size)
    Up, _ = oracle.rk3(p, U * (1 + noise), steps, cfl_c=0.3, cfl_v=0.3)
    bound = max(1e-10, 10 * max(field_errors(prob, Up, Uo)))
    ctx = ctx_for(p, opts=dict(cfl_c=0.3, cfl_v=0.3))
    ctx.set_state(to_dev(U))
    dts = [ctx.rk_step(-1.0) for _ in range(steps)]
    assert ctx.pp_count() > 0
    np.testing.assert_allclose(dts, dto, rtol=1e-10)
    assert_fields_close(prob, ctx.get_state().cpu().numpy(), Uo, rtol=bound, what=f"U({steps} limited steps)")
    ctx.close()


@pytest.mark.parametrize("riemann", [0, 1, 2])
def test_all_fv_mesh_and_uniform_max_degree(oracle, riemann):
    """Degenerate patterns: every element FV (no DG work at all: empty volume,
    lifting and mixed-face launches) and every element at the maximum degree
    N = 7 (no FV, no mixed faces); R and two RK steps."""
    sp = W.species_set([W.AIR, W.HELIUM, W.CO2], mu=1e-3)
    for N, fv in ((3, 1), (7, 0)):
        prob = W.make_problem([((3, 3, 2), (0, 0, 0), (1, 1, 0.7))], sp, n_fv=8, N=N, fv=fv, riemann=riemann)
        U = W.smooth_random_state(prob, 40 + N, amp=0.1)
        assert_rhs_close(oracle, prob, U, gpu_rhs(prob, U))
        ctx = ctx_for(prob, N_min=1, N_max=7)
        ctx.set_state(to_dev(U))
        for _ in range(2):
            ctx.rk_step(1e-4)
        Uo, _ = oracle.rk3(prob, U, 2, dt_fixed=1e-4)
        assert_fields_close(prob, ctx.get_state().cpu().numpy(), Uo, what=f"U(N={N}, fv={fv})")
        ctx.close()


def test_degenerate_calls_leave_the_state_alone():
    """Zero RK steps, an adaptation whose thresholds can never fire, and the
    adjoint of a zero R_bar: the state and the pattern stay bitwise as they
    were and U_bar is exactly zero; a host state of the wrong size is refused."""
    from paper_2502_19342_gb300 import dgfv
    prob, U = _mixed(3)
    ctx = ctx_for(prob, N_min=1, N_max=7, opts=dict(thresholds=(-1e300, 1e300, -1e300, 1e300)))
    ctx.set_state(to_dev(U))
    ctx.rk_steps(0, -1.0, want_dt=False)
    np.testing.assert_array_equal(ctx.get_state().cpu().numpy(), U)
    N0, f0 = ctx.get_degrees()
    st = ctx.adapt()
    assert st["n_changed"] == 0 and st["n_near"] == 0
    N1, f1 = ctx.get_degrees()
    assert (N0 == N1).all() and (f0 == f1).all()
    np.testing.assert_array_equal(ctx.get_state().cpu().numpy(), U)
    Ub = ctx.rhs_vjp(to_dev(U), torch.zeros(U.size, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.isfinite(Ub).all() and not Ub.any()
    with pytest.raises(dgfv.DgfvError):
        ctx.set_state_host(np.zeros(U.size - 1))
    ctx.close()


def test_checkpoint_and_resume_is_bitwise():
    """Checkpoint/resume: the state with its degrees and FV flags, saved after
    two adaptation cycles and loaded into a new context of the same mesh,
    continues bit for bit like the context that kept running (adaptation, CFL
    time steps and stages included)."""
    from paper_2502_19342_gb300 import dgfv
    prob, U = _mixed(21, nk=3, fv_frac=0.3)
    opts = dict(thresholds=W.THRESHOLDS, cfl_c=0.5, cfl_v=0.5)
    a = dgfv.Context(prob, N_min=1, N_max=7, opts=opts)
    a.set_state(to_dev(U))
    for _ in range(2):
        a.adapt()
        a.rk_steps(3, -1.0, want_dt=False)
    N, fv = a.get_degrees()
    saved = a.get_state()
    for _ in range(2):
        a.adapt()
        a.rk_steps(3, -1.0, want_dt=False)
    b = dgfv.Context(prob, N_min=1, N_max=7, opts=opts)
    b.set_degrees(N, fv, remap=False)
    b.set_state(saved)
    for _ in range(2):
        b.adapt()
        b.rk_steps(3, -1.0, want_dt=False)
    Na, fva = a.get_degrees()
    Nb, fvb = b.get_degrees()
    np.testing.assert_array_equal(Na, Nb)
    np.testing.assert_array_equal(fva, fvb)
    assert torch.equal(a.get_state(), b.get_state())
    a.close()
    b.close()
